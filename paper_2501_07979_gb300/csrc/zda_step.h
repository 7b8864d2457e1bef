// Parameters of the fused leap-frog step kernel (zda_step.cu).
#pragma once
#include "zda_internal.h"

namespace zda {

struct FusedParams {
    int nr, nphi, nz, nzs;                     // nzs: z stride of the field arrays
    int pr_in, pr_out, pz;
    int tj, i_range;                           // phi rows per CTA, radii per CTA
    float dt, inv_dr, inv_dz, inv_dphi;
    float2 bloch, bloch_inv;
    const float2 *Er, *Ep, *Ez, *Hr, *Hp, *Hz;          // E^n, H^{n-1/2}
    float2 *oEr, *oEp, *oEz, *oHr, *oHp, *oHz;          // E^{n+1}, H^{n+1/2}
    const float2 *psH_hr_z, *psH_hp_z, *psH_hp_r, *psH_hz_r;     // H-side CPML (read)
    float2 *opsH_hr_z, *opsH_hp_z, *opsH_hp_r, *opsH_hz_r;       // H-side CPML (write)
    float2 *psE_er_z, *psE_ep_z, *psE_ep_r, *psE_ez_r;           // E-side CPML (in place)
    Tables t;
    const float *rb_r, *rb_p, *rb_z;
    int src_mode, src_k;
    float src_scale;
    const float2 *beta_r, *beta_p;
    int nq;
    int mon_k;
    float2 *mon;
    int des_k0, des_nk;
    float2 *des;
    float2 *src_rad;                           // adjoint runs: per-step radial source [2][n_r] (r, phi)
    int *err;                                  // device error word (bounded waits that gave up)
    int wait_limit;                            // polls of an mbarrier before giving up
    int inject_timeout;                        // test only: also wait on a barrier nobody arrives on
};

// One time step = launch_fused_pre (adjoint runs: per-step radial source),
// launch_fused_stream (the streaming E/H kernel; needs an even n_z for its
// 16-byte bulk copies), launch_fused_post (the running DFTs, if requested).
cudaError_t launch_fused_pre(const FusedParams &p, int n, cudaStream_t s);
cudaError_t launch_fused_stream(const FusedParams &p, int n, cudaStream_t s);
cudaError_t launch_fused_post(const FusedParams &p, int n, cudaStream_t s);
int fused_launches_per_step(const FusedParams &p);
int fused_blocks_per_sm(int tj, int nz, int pz);
int fused_max_nz();

}  // namespace zda
