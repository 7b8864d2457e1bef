// Internal declarations shared by the libzda translation units.
// Device layout (all complex values are float2 = (re, im)):
//   fields       E_r, E_phi, E_z, H_r, H_phi, H_z: [n_r][n_phi][n_z], z fastest
//   z-CPML psi   [n_r][n_phi][2 pml_z]        (lower slab, then upper slab)
//   r-CPML psi   [pml_r_in + pml_r_out][n_phi][n_z]
//   metric psi   [pml_r_in + pml_r_out][n_phi][n_z]   (stretched-radius r-PML, H_r H_z E_r E_z)
//   monitor DFT  [Q][2][n_r][n_phi]
//   design DFT   [Q][3][n_r][n_phi][nk]      (nk design planes fastest)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace zda {

__host__ __device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 c_fma(float2 a, float2 b, float2 acc) {   // acc + a b
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__host__ __device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }

#ifdef __CUDACC__
// Running-DFT update X_q += E_c w_q for nc components at stride `comp`,
// frequencies at stride `qstride`: each chunk of frequencies loads all its
// accumulators before any store, so the read-modify-writes overlap instead
// of serialising on possible aliasing.
template <int NC, int CH = 4>
__device__ __forceinline__ void dft_update(float2 *d, size_t qstride, size_t comp, const float2 *tw, int nq,
                                           const float2 (&e)[NC])
{
    for (int q0 = 0; q0 < nq; q0 += CH) {
        float2 v[CH][NC], w[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            if (q0 + u < nq) {
                w[u] = tw[q0 + u];
#pragma unroll
                for (int c = 0; c < NC; ++c) v[u][c] = d[(size_t)(q0 + u) * qstride + c * comp];
            }
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            if (q0 + u < nq) {
#pragma unroll
                for (int c = 0; c < NC; ++c) d[(size_t)(q0 + u) * qstride + c * comp] = c_fma(e[c], w[u], v[u][c]);
            }
        }
    }
}
#endif

// Per-position coefficient tables (device pointers into the workspace).
struct Tables {
    const float *inv_r_n, *inv_r_h;            // 1/r_i (n_r+1), 1/r_{i+1/2} (n_r)
    const float *br_n, *cr_n, *br_h, *cr_h;    // CPML b, c at r nodes / half nodes
    const float *bz_n, *cz_n, *bz_h, *cz_h;    // CPML b, c at z nodes / half nodes
    const float *a_n, *d_n, *a_c, *d_c;        // eps = a[k] + d[k] rhobar at node / cell planes
    const float2 *ph_n, *ph_h;                 // e^{i m phi_j}, e^{i m phi_{j+1/2}}
    const float *pulse;                        // g(t_{n+1/2})          [T]
    const float2 *twiddle;                     // e^{i w_q t_{n+1}} dt  [T][Q]
    const float2 *adj_time;                    // adjoint profiles k_q  [T][Q]
};

struct Fields { float2 *Er, *Ep, *Ez, *Hr, *Hp, *Hz; };
struct Psi { float2 *hr_z, *hp_z, *hp_r, *hz_r, *er_z, *ep_z, *ep_r, *ez_r; };
// Stretched-coordinate r-PML: 1/r~ recursion tables and metric auxiliaries.
struct Metric {
    const float *bm_n, *cm_n, *bm_h, *cm_h;    // at r nodes / half nodes (0: r~ = r)
    float2 *hr, *hz, *er, *ez;                 // [pml_r_in + pml_r_out][n_phi][n_z]
};

enum { SRC_NONE = 0, SRC_PLANE_WAVE = 1, SRC_ADJOINT = 2 };

struct StepParams {
    int nr, nphi, nz;
    int pr_in, pr_out, pz;
    int bor;                                   // continuous axisymmetry: (1/r) d/dphi -> i m / r
    float m;
    float dt, inv_dr, inv_dz, inv_dphi;
    float2 bloch, bloch_inv;                   // e^{+-i m tau}
    Fields f;
    Psi psi;
    Tables t;
    const float *rb_r, *rb_p, *rb_z;           // transverse density averages [n_r][n_phi]
    int src_mode, src_k;
    float src_scale;                           // 1/(2 dz) for the plane wave
    const float2 *beta_r, *beta_p;             // adjoint radial profiles [Q][n_r]
    float2 *src_rad;                           // adjoint source of the current step [2][n_r]
    float2 *dft_hist;                          // DFT_BLOCK slots of E at the DFT sites (time-blocked DFT)
    size_t dft_ne;                             // entries per slot
    int nq;
    int mon_k;                                 // < 0: no monitor DFT
    float2 *mon;
    int des_k0, des_nk;                        // des_nk == 0: no design DFT
    float2 *des;
    // r-PML form: 0 = CPML on the whole (1/r) d/dr (r .) term, real-radius
    // metric; 1 = stretched coordinates: inside the r-PML only the derivative
    // part is stretched and the metric parts are divided by r~ (rm tables)
    int rpml_metric;
    Metric rm;
    int pair_rows;                             // two-z-cell split kernels: phi rows per thread block (4, 8, 16, 32)
    int e_blocks;                              // ... E update's thread blocks per SM (2 or 3)
};

// kernels (zda_kernels.cu)
void launch_update_h(const StepParams &p, cudaStream_t s);
void launch_update_e(const StepParams &p, int n, cudaStream_t s);
// two z-cells per thread (zda_pair.cu): even n_z, even pml_z, wedge zones
bool pair_kernels_apply(const StepParams &p);
bool pair_rows_ok(int rows);
void launch_update_h_pair(const StepParams &p, cudaStream_t s);
void launch_update_e_pair(const StepParams &p, int n, cudaStream_t s);   // writes the DFT history; see launch_dft_flush
// Time-blocked running DFT of the split step (two z-cells per thread).
constexpr int DFT_BLOCK = 32;
#define ZDA_DFT_MAXQ 16
size_t dft_entries(const StepParams &p);
bool dft_flush_due(const StepParams &p, int n, int n_steps);
void launch_dft_flush(const StepParams &p, int n, cudaStream_t s);
void launch_adjoint_source_rad(const StepParams &p, int n, cudaStream_t s);

struct FilterParams {
    int nrd, nphi, di_max, dj_max;
    float dr, dphi, R, r_c0;                   // r_c(i) = r_c0 + i dr
    float beta, eta;                           // beta <= 0: no projection
    int filter_on;
};
void launch_filter_norm(const FilterParams &fp, float *norm, cudaStream_t s);
void launch_filter_project(const FilterParams &fp, const float *rho, const float *norm, float *rho_bar,
                           float *rho_t, cudaStream_t s);
void launch_filter_project_backward(const FilterParams &fp, const float *rho_bar, const float *norm,
                                    const float *g_t, float *g_rho, cudaStream_t s);
void launch_rho_bar(const float *rho_t, int nr, int nphi, int i_d0, int i_d1, float *rb_r, float *rb_p,
                    float *rb_z, cudaStream_t s);

void launch_focal_partial(const float2 *mon, const double2 *Gr, const double2 *Gp, const double2 *emph_n,
                          const double2 *emph_h, int nq, int nr, int nphi, double2 *partial, cudaStream_t s);
void launch_focal_nn(const float *y, int n, int nq, int i_d0, int nrd, int nphi, int nr, float scale,
                     const double2 *Gr, const double2 *Gp, const double2 *emph_n, const double2 *emph_h, double2 *S,
                     cudaStream_t s);
void launch_focal_nn_T(const double2 *G, int n, int nq, int i_d0, int nrd, int nphi, int nr, float scale,
                       const double2 *Gr, const double2 *Gp, const double2 *emph_n, const double2 *emph_h, float *dy,
                       cudaStream_t s);
void launch_focal_sum(const double2 *partial, int nq, int nr, double2 *S, int *status, cudaStream_t s);
void launch_adjoint_profiles(const double2 *g, const double2 *Gr, const double2 *Gp, const float *wt, int nq,
                             int nr, double r_lo, double dr, double vol_scale, float2 *beta_r, float2 *beta_p,
                             cudaStream_t s);
void launch_site_gradient(const float2 *des_f, const float2 *des_a, const float *wt, int nq, int nr, int nphi,
                          int nk, double r_lo, double dr, double vol_scale, float *site_grad, cudaStream_t s);
void launch_cell_gradient(const float *site_grad, int nr, int nphi, int nk, int i_d0, int nrd, float deps,
                          float *g_t, cudaStream_t s);
// decay probe: field energy of the state cur and of cur - prev
void launch_field_energy(const StepParams &p, const Fields &cur, const Fields &prev, double r_lo, double dr,
                         double vol_dphi_dz, double *partial, double *w_out, double *wdot_out, cudaStream_t s);
void launch_fill_status_check(const float *x, size_t n, int *status, cudaStream_t s);
void launch_lens_sum(const double2 *const *S, int nzones, int nq, double2 *out, int *status, cudaStream_t s);
// cross != 0 (n_fold 1 or 2): the transmitted intensity keeps the +-1 cross term
// focal-spot evaluation (zda_eval.cu); n_lambda <= ZDA_EVAL_MAX_LAMBDA
#define ZDA_EVAL_MAX_LAMBDA 8
struct EvalScalars {
    double incident[ZDA_EVAL_MAX_LAMBDA], p_trans[ZDA_EVAL_MAX_LAMBDA], lambda[ZDA_EVAL_MAX_LAMBDA];
    double area, focal, n_top;
};
void launch_eval_line_points(double *pts, int n_line, double x_max, cudaStream_t s);
void launch_eval_fwhm(const double2 *field, int nl, int n_line, double x_max, double n_top, double *line, double *fw,
                      double *i0, cudaStream_t s);
void launch_eval_disc_points(const double *fw, int nl, int n_rad, int n_ang, double *pts, cudaStream_t s);
void launch_eval_finish(const double2 *field, int nl, int n_rad, int n_ang, const double *fw, const double *i0,
                        const EvalScalars &sc, double *out, cudaStream_t s);
void launch_incident_intensity(const float2 *mon, int nl, int nr, int nphi, int i0, int i1, double dphi, double n_sub,
                               double *out, cudaStream_t s);
void launch_field_intensity(const double2 *field, int nl, int n, double n_top, double *out, cudaStream_t s);
void launch_encircled_power(const double *r, const double *I, int n_prof, int n, double *out, cudaStream_t s);
void launch_phi_means(const float2 *mon, const double2 *emph_n, const double2 *emph_h, int nq, int nr, int nphi,
                      int cross, double2 *umean, double *pt_row, cudaStream_t s);
void launch_focal_plane(const double2 *umean, const double *rr, const double *wr, const double *rp, const double *wp,
                        int nr, int nl, const double *pts, int pstride, int npts, double zf, const double *kk, int ns,
                        double2 *ex, double2 *ey, cudaStream_t s);

}  // namespace zda

// Sets the calling thread's message returned by zda_last_error().
void zda_internal_set_error(const char *msg);
