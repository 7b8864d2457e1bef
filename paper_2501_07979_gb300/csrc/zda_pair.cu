// Split step kernels, two z-cells per thread (sm_103a).
//
// Same scheme and arithmetic as k_update_h / k_update_e (one thread per Yee
// cell), but each thread owns the z-cells (2 kp, 2 kp + 1) and moves every
// field component as one aligned 16-byte float4: half the load/store
// instructions and twice the bytes in flight per instruction, which is what
// the one-cell kernels lack (they are latency-bound at 48-59 % of DRAM
// bandwidth with traffic equal to the algorithmic bytes).  The z-neighbour
// outside the pair comes from one extra 8-byte load (an L1 hit).  Needs an
// even n_z and an even z-PML width, so that a pair never straddles a CPML
// slab boundary; otherwise the one-cell kernels run.  Stretched-coordinate
// r-PML columns (rpml_metric = 1, uniform per block since blockIdx.z = i)
// take the split radial curl and the 1/r~ recursion of k_update_h / k_update_e;
// that code is compiled only into the RM = true instances (the H kernel at
// 3 blocks per SM, 80 registers), so the default form keeps its budget of
// 64 registers at 4 blocks per SM without spilling.
#include "zda_internal.h"

namespace zda {

// Thread block: PY phi rows x (256 / PY) z-pairs.  PY is a template
// parameter (4, 8, 16 or 32) chosen per zone by the tile tuner: zones with
// few phi cells waste no rows with PY = 4 or 8, long z-columns coalesce
// better with more z-pairs per block.

struct C2 { float2 a, b; };                      // the pair (k, k+1)

__device__ __forceinline__ C2 ld4(const float2 *p)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return C2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ C2 ld4rw(const float2 *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return C2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void st4(float2 *p, C2 c)
{
    *reinterpret_cast<float4 *>(p) = make_float4(c.a.x, c.a.y, c.b.x, c.b.y);
}
__device__ __forceinline__ C2 cmul2(float2 s, C2 c) { return C2{c_mul(s, c.a), c_mul(s, c.b)}; }
// Inverse permittivity of a site: the hardware reciprocal (rcp.approx, about
// 1 ulp) instead of an IEEE division; the E update was issue-bound with the
// division sequence (4 % faster without it), and 1 ulp is far below the
// single-precision time stepping's own rounding.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <bool RM, int PY>
__global__ void __launch_bounds__(256, RM ? 3 : 4) k_update_h_pair(const StepParams p)
{
    constexpr int PX = 256 / PY;
    const int kp = blockIdx.x * PX + threadIdx.x;
    const int j = blockIdx.y * PY + threadIdx.y;
    const int i = blockIdx.z;
    const int nz = p.nz, nphi = p.nphi;
    const int k = 2 * kp;
    if (k >= nz || j >= nphi) return;
    const size_t sj = (size_t)nz, si = (size_t)nphi * nz;
    const size_t c = (size_t)i * si + (size_t)j * sj + k;
    const float2 zero = make_float2(0.f, 0.f);

    const C2 er = ld4(p.f.Er + c), ep = ld4(p.f.Ep + c), ez = ld4(p.f.Ez + c);
    C2 ez_jp, er_jp;
    if (j + 1 < nphi) {
        ez_jp = ld4(p.f.Ez + c + sj);
        er_jp = ld4(p.f.Er + c + sj);
    } else {
        const size_t c0 = c - (size_t)(nphi - 1) * sj;
        ez_jp = cmul2(p.bloch, ld4(p.f.Ez + c0));
        er_jp = cmul2(p.bloch, ld4(p.f.Er + c0));
    }
    const bool kin2 = k + 2 < nz, iin = i + 1 < p.nr;
    const float2 ep_k2 = kin2 ? __ldg(p.f.Ep + c + 2) : zero;     // z-neighbour of the second cell
    const float2 er_k2 = kin2 ? __ldg(p.f.Er + c + 2) : zero;
    const C2 ez_ip = iin ? ld4(p.f.Ez + c + si) : C2{zero, zero};
    const C2 ep_ip = iin ? ld4(p.f.Ep + c + si) : C2{zero, zero};
    const float irn = __ldg(p.t.inv_r_n + i), irh = __ldg(p.t.inv_r_h + i);
    const int kz = (k < p.pz) ? k : ((k >= nz - p.pz) ? k - (nz - 2 * p.pz) : -1);
    const int ir = (i < p.pr_in) ? i : ((i >= p.nr - p.pr_out) ? i - (p.nr - p.pr_in - p.pr_out) : -1);
    const float dt = p.dt;
    const size_t zx = ((size_t)i * nphi + j) * (2 * p.pz) + (kz >= 0 ? kz : 0);
    const size_t rx = ((size_t)(ir >= 0 ? ir : 0) * nphi + j) * nz + k;
    float bzh[2] = {0.f, 0.f}, czh[2] = {0.f, 0.f};
    if (kz >= 0) {
        bzh[0] = __ldg(p.t.bz_h + k); bzh[1] = __ldg(p.t.bz_h + k + 1);
        czh[0] = __ldg(p.t.cz_h + k); czh[1] = __ldg(p.t.cz_h + k + 1);
    }
    const float brh = ir >= 0 ? __ldg(p.t.br_h + i) : 0.f, crh = ir >= 0 ? __ldg(p.t.cr_h + i) : 0.f;

    const float2 EP[3] = {ep.a, ep.b, ep_k2}, ER[3] = {er.a, er.b, er_k2};
    const float2 EZ[2] = {ez.a, ez.b}, EZJ[2] = {ez_jp.a, ez_jp.b}, ERJ[2] = {er_jp.a, er_jp.b};
    const float2 EZI[2] = {ez_ip.a, ez_ip.b}, EPI[2] = {ep_ip.a, ep_ip.b};
    C2 hr = ld4rw(p.f.Hr + c), hp = ld4rw(p.f.Hp + c), hz = ld4rw(p.f.Hz + c);
    float2 *HR[2] = {&hr.a, &hr.b}, *HP[2] = {&hp.a, &hp.b}, *HZ[2] = {&hz.a, &hz.b};
    C2 ps_r = C2{zero, zero}, ps_p = C2{zero, zero}, ps_pr = C2{zero, zero}, ps_zr = C2{zero, zero};
    if (kz >= 0) { ps_r = ld4rw(p.psi.hr_z + zx); ps_p = ld4rw(p.psi.hp_z + zx); }
    if (ir >= 0) { ps_pr = ld4rw(p.psi.hp_r + rx); ps_zr = ld4rw(p.psi.hz_r + rx); }
    float2 *PR[2] = {&ps_r.a, &ps_r.b}, *PP[2] = {&ps_p.a, &ps_p.b};
    float2 *PPR[2] = {&ps_pr.a, &ps_pr.b}, *PZR[2] = {&ps_zr.a, &ps_zr.b};
    const bool sr = RM && ir >= 0;
    if (sr) {                                   // stretched-coordinate r-PML column
        C2 pm_r = ld4rw(p.rm.hr + rx), pm_z = ld4rw(p.rm.hz + rx);
        float2 *MR[2] = {&pm_r.a, &pm_r.b}, *MZ[2] = {&pm_z.a, &pm_z.b};
        const float bmn = __ldg(p.rm.bm_n + i), cmn = __ldg(p.rm.cm_n + i);
        const float bmh = __ldg(p.rm.bm_h + i), cmh = __ldg(p.rm.cm_h + i);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            {                                   // H_r
                const float2 X = c_scale(c_sub(EZJ[u], EZ[u]), p.inv_dphi);
                *MR[u] = c_add(c_scale(*MR[u], bmn), c_scale(X, cmn));
                const float2 dph = c_scale(c_add(X, *MR[u]), irn);
                float2 dz = c_scale(c_sub(EP[u + 1], EP[u]), p.inv_dz);
                if (kz >= 0) {
                    *PR[u] = c_add(c_scale(*PR[u], bzh[u]), c_scale(dz, czh[u]));
                    dz = c_add(dz, *PR[u]);
                }
                *HR[u] = c_sub(*HR[u], c_scale(c_sub(dph, dz), dt));
            }
            {                                   // H_phi
                float2 dz = c_scale(c_sub(ER[u + 1], ER[u]), p.inv_dz);
                float2 drr = c_scale(c_sub(EZI[u], EZ[u]), p.inv_dr);
                if (kz >= 0) {
                    *PP[u] = c_add(c_scale(*PP[u], bzh[u]), c_scale(dz, czh[u]));
                    dz = c_add(dz, *PP[u]);
                }
                *PPR[u] = c_add(c_scale(*PPR[u], brh), c_scale(drr, crh));
                drr = c_add(drr, *PPR[u]);
                *HP[u] = c_sub(*HP[u], c_scale(c_sub(dz, drr), dt));
            }
            {                                   // H_z: stretched derivative + metric part / r~
                float2 drr = c_scale(c_sub(EPI[u], EP[u]), p.inv_dr);
                *PZR[u] = c_add(c_scale(*PZR[u], brh), c_scale(drr, crh));
                drr = c_add(drr, *PZR[u]);
                const float2 X = c_sub(c_scale(c_add(EPI[u], EP[u]), 0.5f), c_scale(c_sub(ERJ[u], ER[u]), p.inv_dphi));
                *MZ[u] = c_add(c_scale(*MZ[u], bmh), c_scale(X, cmh));
                *HZ[u] = c_sub(*HZ[u], c_scale(c_add(drr, c_scale(c_add(X, *MZ[u]), irh)), dt));
            }
        }
        st4(p.rm.hr + rx, pm_r);
        st4(p.rm.hz + rx, pm_z);
    } else {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        // H_r
        {
            const float2 dph = c_scale(c_sub(EZJ[u], EZ[u]), irn * p.inv_dphi);
            float2 dz = c_scale(c_sub(EP[u + 1], EP[u]), p.inv_dz);
            if (kz >= 0) {
                *PR[u] = c_add(c_scale(*PR[u], bzh[u]), c_scale(dz, czh[u]));
                dz = c_add(dz, *PR[u]);
            }
            *HR[u] = c_sub(*HR[u], c_scale(c_sub(dph, dz), dt));
        }
        // H_phi
        {
            float2 dz = c_scale(c_sub(ER[u + 1], ER[u]), p.inv_dz);
            float2 drr = c_scale(c_sub(EZI[u], EZ[u]), p.inv_dr);
            if (kz >= 0) {
                *PP[u] = c_add(c_scale(*PP[u], bzh[u]), c_scale(dz, czh[u]));
                dz = c_add(dz, *PP[u]);
            }
            if (ir >= 0) {
                *PPR[u] = c_add(c_scale(*PPR[u], brh), c_scale(drr, crh));
                drr = c_add(drr, *PPR[u]);
            }
            *HP[u] = c_sub(*HP[u], c_scale(c_sub(dz, drr), dt));
        }
        // H_z
        {
            float2 drr = c_add(c_scale(c_sub(EPI[u], EP[u]), p.inv_dr), c_scale(c_add(EPI[u], EP[u]), 0.5f * irh));
            const float2 dph = c_scale(c_sub(ERJ[u], ER[u]), irh * p.inv_dphi);
            if (ir >= 0) {
                *PZR[u] = c_add(c_scale(*PZR[u], brh), c_scale(drr, crh));
                drr = c_add(drr, *PZR[u]);
            }
            *HZ[u] = c_sub(*HZ[u], c_scale(c_sub(drr, dph), dt));
        }
    }
    }
    st4(p.f.Hr + c, hr);
    st4(p.f.Hp + c, hp);
    st4(p.f.Hz + c, hz);
    if (kz >= 0) { st4(p.psi.hr_z + zx, ps_r); st4(p.psi.hp_z + zx, ps_p); }
    if (ir >= 0) { st4(p.psi.hp_r + rx, ps_pr); st4(p.psi.hz_r + rx, ps_zr); }
}

template <bool RM, int PY, int MINB>
__global__ void __launch_bounds__(256, MINB) k_update_e_pair(const StepParams p, const int n)
{
    constexpr int PX = 256 / PY;
    const int kp = blockIdx.x * PX + threadIdx.x;
    const int j = blockIdx.y * PY + threadIdx.y;
    const int i = blockIdx.z;
    const int nz = p.nz, nphi = p.nphi, nr = p.nr;
    const int k = 2 * kp;
    if (k >= nz || j >= nphi) return;
    const size_t sj = (size_t)nz, si = (size_t)nphi * nz;
    const size_t c = (size_t)i * si + (size_t)j * sj + k;
    const float2 zero = make_float2(0.f, 0.f);

    const C2 hr = ld4(p.f.Hr + c), hp = ld4(p.f.Hp + c), hz = ld4(p.f.Hz + c);
    C2 hz_jm, hr_jm;
    if (j > 0) {
        hz_jm = ld4(p.f.Hz + c - sj);
        hr_jm = ld4(p.f.Hr + c - sj);
    } else {
        const size_t c1 = c + (size_t)(nphi - 1) * sj;
        hz_jm = cmul2(p.bloch_inv, ld4(p.f.Hz + c1));
        hr_jm = cmul2(p.bloch_inv, ld4(p.f.Hr + c1));
    }
    const float2 hp_km = (k > 0) ? __ldg(p.f.Hp + c - 1) : zero;     // z-neighbour of the first cell
    const float2 hr_km = (k > 0) ? __ldg(p.f.Hr + c - 1) : zero;
    const C2 hz_im = (i > 0) ? ld4(p.f.Hz + c - si) : C2{zero, zero};
    const C2 hp_im = (i > 0) ? ld4(p.f.Hp + c - si) : C2{zero, zero};
    const float irn = __ldg(p.t.inv_r_n + i), irh = __ldg(p.t.inv_r_h + i);
    const int kz = (k < p.pz) ? k : ((k >= nz - p.pz) ? k - (nz - 2 * p.pz) : -1);
    const int ir = (i < p.pr_in) ? i : ((i >= nr - p.pr_out) ? i - (nr - p.pr_in - p.pr_out) : -1);
    const float dt = p.dt;
    const size_t ij = (size_t)i * nphi + j;
    const size_t zx = ij * (2 * p.pz) + (kz >= 0 ? kz : 0);
    const size_t rx = ((size_t)(ir >= 0 ? ir : 0) * nphi + j) * nz + k;

    const float2 HP[3] = {hp_km, hp.a, hp.b}, HRk[3] = {hr_km, hr.a, hr.b};   // index u+1 = cell u
    const float2 HZ[2] = {hz.a, hz.b}, HZJ[2] = {hz_jm.a, hz_jm.b}, HRJ[2] = {hr_jm.a, hr_jm.b};
    const float2 HZI[2] = {hz_im.a, hz_im.b}, HPI[2] = {hp_im.a, hp_im.b};
    C2 er = ld4rw(p.f.Er + c), ep = ld4rw(p.f.Ep + c), ez = ld4rw(p.f.Ez + c);
    float2 *ER[2] = {&er.a, &er.b}, *EP[2] = {&ep.a, &ep.b}, *EZ[2] = {&ez.a, &ez.b};
    C2 ps_r = C2{zero, zero}, ps_p = C2{zero, zero}, ps_pr = C2{zero, zero}, ps_zr = C2{zero, zero};
    if (kz >= 0) { ps_r = ld4rw(p.psi.er_z + zx); ps_p = ld4rw(p.psi.ep_z + zx); }
    if (ir >= 0) { ps_pr = ld4rw(p.psi.ep_r + rx); ps_zr = ld4rw(p.psi.ez_r + rx); }
    float2 *PR[2] = {&ps_r.a, &ps_r.b}, *PP[2] = {&ps_p.a, &ps_p.b};
    float2 *PPR[2] = {&ps_pr.a, &ps_pr.b}, *PZR[2] = {&ps_zr.a, &ps_zr.b};
    const float rbr = __ldg(p.rb_r + ij), rbp = __ldg(p.rb_p + ij), rbz = __ldg(p.rb_z + ij);
    const float brn = ir >= 0 ? __ldg(p.t.br_n + i) : 0.f, crn = ir >= 0 ? __ldg(p.t.cr_n + i) : 0.f;
    const bool sr = RM && ir >= 0;                     // stretched-coordinate r-PML column
    C2 pm_r = C2{zero, zero}, pm_z = C2{zero, zero};
    float bmn = 0.f, cmn = 0.f, bmh = 0.f, cmh = 0.f;
    if (sr) {
        pm_r = ld4rw(p.rm.er + rx);
        pm_z = ld4rw(p.rm.ez + rx);
        bmn = __ldg(p.rm.bm_n + i); cmn = __ldg(p.rm.cm_n + i);
        bmh = __ldg(p.rm.bm_h + i); cmh = __ldg(p.rm.cm_h + i);
    }
    float2 *MER[2] = {&pm_r.a, &pm_r.b}, *MEZ[2] = {&pm_z.a, &pm_z.b};

#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int kk = k + u;
        float2 jr = zero, jp = zero;
        if (kk == p.src_k) {
            if (p.src_mode == SRC_PLANE_WAVE) {
                const float a = __ldg(p.t.pulse + n) * p.src_scale;
                const float2 pn = p.t.ph_n[j], ph = p.t.ph_h[j];
                jr = c_scale(pn, a);
                jp = make_float2(-ph.y * a, ph.x * a);
            } else if (p.src_mode == SRC_ADJOINT) {       // radial profile of this step (k_adjoint_source_rad)
                jr = c_mul(p.t.ph_n[j], p.src_rad[i]);
                jp = c_mul(p.t.ph_h[j], p.src_rad[nr + i]);
            }
        }
        const float bzn = kz >= 0 ? __ldg(p.t.bz_n + kk) : 0.f, czn = kz >= 0 ? __ldg(p.t.cz_n + kk) : 0.f;
        if (kk > 0) {                                       // E_r
            float2 dph;
            if (sr) {
                const float2 X = c_scale(c_sub(HZ[u], HZJ[u]), p.inv_dphi);
                *MER[u] = c_add(c_scale(*MER[u], bmh), c_scale(X, cmh));
                dph = c_scale(c_add(X, *MER[u]), irh);
            } else {
                dph = c_scale(c_sub(HZ[u], HZJ[u]), irh * p.inv_dphi);
            }
            float2 dz = c_scale(c_sub(HP[u + 1], HP[u]), p.inv_dz);
            if (kz >= 0) {
                *PR[u] = c_add(c_scale(*PR[u], bzn), c_scale(dz, czn));
                dz = c_add(dz, *PR[u]);
            }
            const float ie = rcp_approx(__ldg(p.t.a_n + kk) + __ldg(p.t.d_n + kk) * rbr);
            *ER[u] = c_add(*ER[u], c_scale(c_sub(c_sub(dph, dz), jr), dt * ie));
        }
        if (i > 0 && kk > 0) {                              // E_phi
            float2 dz = c_scale(c_sub(HRk[u + 1], HRk[u]), p.inv_dz);
            float2 drr = c_scale(c_sub(HZ[u], HZI[u]), p.inv_dr);
            if (kz >= 0) {
                *PP[u] = c_add(c_scale(*PP[u], bzn), c_scale(dz, czn));
                dz = c_add(dz, *PP[u]);
            }
            if (ir >= 0) {
                *PPR[u] = c_add(c_scale(*PPR[u], brn), c_scale(drr, crn));
                drr = c_add(drr, *PPR[u]);
            }
            const float ie = rcp_approx(__ldg(p.t.a_n + kk) + __ldg(p.t.d_n + kk) * rbp);
            *EP[u] = c_add(*EP[u], c_scale(c_sub(c_sub(dz, drr), jp), dt * ie));
        }
        if (i > 0 && sr) {                                  // E_z, stretched r-PML column
            float2 drr = c_scale(c_sub(HP[u + 1], HPI[u]), p.inv_dr);
            *PZR[u] = c_add(c_scale(*PZR[u], brn), c_scale(drr, crn));
            drr = c_add(drr, *PZR[u]);
            const float2 X = c_sub(c_scale(c_add(HP[u + 1], HPI[u]), 0.5f), c_scale(c_sub(HRk[u + 1], HRJ[u]), p.inv_dphi));
            *MEZ[u] = c_add(c_scale(*MEZ[u], bmn), c_scale(X, cmn));
            const float ie = rcp_approx(__ldg(p.t.a_c + kk) + __ldg(p.t.d_c + kk) * rbz);
            *EZ[u] = c_add(*EZ[u], c_scale(c_add(drr, c_scale(c_add(X, *MEZ[u]), irn)), dt * ie));
        } else if (i > 0) {                                 // E_z
            float2 drr = c_add(c_scale(c_sub(HP[u + 1], HPI[u]), p.inv_dr),
                               c_scale(c_add(HP[u + 1], HPI[u]), 0.5f * irn));
            const float2 dph = c_scale(c_sub(HRk[u + 1], HRJ[u]), irn * p.inv_dphi);
            if (ir >= 0) {
                *PZR[u] = c_add(c_scale(*PZR[u], brn), c_scale(drr, crn));
                drr = c_add(drr, *PZR[u]);
            }
            const float ie = rcp_approx(__ldg(p.t.a_c + kk) + __ldg(p.t.d_c + kk) * rbz);
            *EZ[u] = c_add(*EZ[u], c_scale(c_sub(drr, dph), dt * ie));
        }
    }
    st4(p.f.Er + c, er);
    st4(p.f.Ep + c, ep);
    st4(p.f.Ez + c, ez);
    if (kz >= 0) { st4(p.psi.er_z + zx, ps_r); st4(p.psi.ep_z + zx, ps_p); }
    if (ir >= 0) { st4(p.psi.ep_r + rx, ps_pr); st4(p.psi.ez_r + rx, ps_zr); }
    if (sr) { st4(p.rm.er + rx, pm_r); st4(p.rm.ez + rx, pm_z); }

    // history slot of the time-blocked DFT (entries as in dft_site)
    if (p.dft_hist && (p.des || p.mon)) {
        const size_t plane = (size_t)nr * nphi, ndes = p.des ? plane * p.des_nk : 0;
        float2 *hs = p.dft_hist + (size_t)(n % DFT_BLOCK) * p.dft_ne;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int dk = k + u - p.des_k0;
            if (p.des && dk >= 0 && dk < p.des_nk) {
                const size_t t = ij * p.des_nk + dk;
                hs[t] = *ER[u];
                hs[ndes + t] = *EP[u];
                hs[2 * ndes + t] = *EZ[u];
            }
            if (p.mon && k + u == p.mon_k) {
                hs[3 * ndes + ij] = *ER[u];
                hs[3 * ndes + plane + ij] = *EP[u];
            }
        }
    }
}

// Running DFTs of E^{n+1}, blocked over time.  Each step the E update writes
// E at the DFT sites (design volume: 3 components x n_r n_phi design_nk;
// monitor plane: E_r, E_phi x n_r n_phi) into slot n mod DFT_BLOCK of a
// history buffer; every DFT_BLOCK steps (and after the last step)
// k_dft_flush adds sum_l E_l e^{i w_q (n0 + l) dt} dt to each accumulator,
// which it reads and writes once per block instead of once per step.
// Entry e: design e = c ndes + (ij nk + kk) (c < 3), then monitor
// 3 ndes + c plane + ij (c < 2).
// One thread per DFT site (design: 3 components, monitor: E_r, E_phi); the
// block's twiddles for the flushed steps sit in shared memory; frequencies
// in chunks of 8.
__global__ void k_dft_flush(const StepParams p, int nslots, int n0)
{
    __shared__ float2 tws[DFT_BLOCK * ZDA_DFT_MAXQ];
    const int nq = p.nq;
    for (int i = threadIdx.x; i < nslots * nq; i += blockDim.x) tws[i] = p.t.twiddle[(size_t)n0 * nq + i];
    __syncthreads();
    const size_t plane = (size_t)p.nr * p.nphi, ndes = p.des ? plane * p.des_nk : 0;
    const size_t nsites = ndes + (p.mon ? plane : 0), ne = p.dft_ne;
    const size_t site = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= nsites) return;
    const bool des = site < ndes;
    const int ncomp = des ? 3 : 2;
    const size_t u = des ? site : site - ndes;
    const size_t e0 = des ? site : 3 * ndes + u, estride = des ? ndes : plane;   // history entries
    float2 *d = des ? p.des + site : p.mon + u;
    const size_t cstride = des ? ndes : plane, qstride = des ? 3 * ndes : 2 * plane;
    for (int q0 = 0; q0 < nq; q0 += 8) {
        float2 acc[3][8];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[c][q] = make_float2(0.f, 0.f);
        for (int l = 0; l < nslots; ++l) {
            const float2 *h = p.dft_hist + (size_t)l * ne + e0;
            float2 x[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) x[c] = c < ncomp ? h[c * estride] : make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q0 + q >= nq) break;
                const float2 w = tws[l * nq + q0 + q];
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[c][q] = c_fma(x[c], w, acc[c][q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q0 + q >= nq) break;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (c >= ncomp) break;
                float2 *dd = d + (size_t)(q0 + q) * qstride + c * cstride;
                const float2 v = *dd;
                *dd = make_float2(v.x + acc[c][q].x, v.y + acc[c][q].y);
            }
        }
    }
}

size_t dft_entries(const StepParams &p)
{
    const size_t plane = (size_t)p.nr * p.nphi;
    return (p.des ? 3 * plane * p.des_nk : 0) + (p.mon ? 2 * plane : 0);
}

bool dft_flush_due(const StepParams &p, int n, int n_steps)
{
    return dft_entries(p) > 0 && ((n % DFT_BLOCK) == DFT_BLOCK - 1 || n == n_steps - 1);
}

void launch_dft_flush(const StepParams &p, int n, cudaStream_t s)
{
    const size_t plane = (size_t)p.nr * p.nphi;
    const size_t nsites = (p.des ? plane * p.des_nk : 0) + (p.mon ? plane : 0);
    const int nslots = n % DFT_BLOCK + 1;
    k_dft_flush<<<(unsigned)((nsites + 255) / 256), 256, 0, s>>>(p, nslots, n - (nslots - 1));
}

// Adjoint source of step n per radius: sum_q beta_q(r) k_q(t_{n+1/2}) for the
// E_r and E_phi sites (the e^{i phi} factor is applied per row).
__global__ void k_adjoint_source_rad(const StepParams p, const int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.nr) return;
    const float2 *kt = p.t.adj_time + (size_t)n * p.nq;
    float2 sr = make_float2(0.f, 0.f), sp = make_float2(0.f, 0.f);
    for (int q = 0; q < p.nq; ++q) {
        sr = c_fma(p.beta_r[(size_t)q * p.nr + i], kt[q], sr);
        sp = c_fma(p.beta_p[(size_t)q * p.nr + i], kt[q], sp);
    }
    p.src_rad[i] = sr;
    p.src_rad[p.nr + i] = sp;
}

void launch_adjoint_source_rad(const StepParams &p, int n, cudaStream_t s)
{
    k_adjoint_source_rad<<<(p.nr + 127) / 128, 128, 0, s>>>(p, n);
}

bool pair_kernels_apply(const StepParams &p) { return p.nz % 2 == 0 && p.pz % 2 == 0 && !p.bor; }

template <int PY>
static void launch_h_py(const StepParams &p, cudaStream_t s)
{
    constexpr int PX = 256 / PY;
    dim3 b(PX, PY), g((p.nz / 2 + PX - 1) / PX, (p.nphi + PY - 1) / PY, p.nr);
    if (p.rpml_metric) k_update_h_pair<true, PY><<<g, b, 0, s>>>(p);
    else k_update_h_pair<false, PY><<<g, b, 0, s>>>(p);
}

// E update: 2 blocks per SM (120 registers, no spills) or 3 (80 registers, a
// few spilled to local memory), chosen by the tuner
template <int PY>
static void launch_e_py(const StepParams &p, int n, cudaStream_t s)
{
    constexpr int PX = 256 / PY;
    dim3 b(PX, PY), g((p.nz / 2 + PX - 1) / PX, (p.nphi + PY - 1) / PY, p.nr);
    if (p.e_blocks == 3) {
        if (p.rpml_metric) k_update_e_pair<true, PY, 3><<<g, b, 0, s>>>(p, n);
        else k_update_e_pair<false, PY, 3><<<g, b, 0, s>>>(p, n);
    } else {
        if (p.rpml_metric) k_update_e_pair<true, PY, 2><<<g, b, 0, s>>>(p, n);
        else k_update_e_pair<false, PY, 2><<<g, b, 0, s>>>(p, n);
    }
}

bool pair_rows_ok(int rows) { return rows == 4 || rows == 8 || rows == 16 || rows == 32; }

void launch_update_h_pair(const StepParams &p, cudaStream_t s)
{
    switch (p.pair_rows) {
    case 4: launch_h_py<4>(p, s); break;
    case 8: launch_h_py<8>(p, s); break;
    case 32: launch_h_py<32>(p, s); break;
    default: launch_h_py<16>(p, s); break;
    }
}

void launch_update_e_pair(const StepParams &p, int n, cudaStream_t s)
{
    switch (p.pair_rows) {
    case 4: launch_e_py<4>(p, n, s); break;
    case 8: launch_e_py<8>(p, n, s); break;
    case 32: launch_e_py<32>(p, n, s); break;
    default: launch_e_py<16>(p, n, s); break;
    }
}

}  // namespace zda
