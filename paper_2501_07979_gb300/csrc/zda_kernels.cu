// CUDA kernels of libzda (sm_103a).
//
// Time loop (section "Differentiable FDTD in cylindrical coordinates",
// Eqs. 3-5): fields are stored in Bloch-periodic form psi = u e^{i m phi},
// so Eq. 5's im/r terms are plain phi-differences and the wedge wraps with
// e^{+-i m tau}.  Yee sites: E_r(i+1/2,j,k) E_phi(i,j+1/2,k) E_z(i,j,k+1/2),
// H_r(i,j+1/2,k+1/2) H_phi(i+1/2,j,k+1/2) H_z(i+1/2,j+1/2,k); PEC behind the
// CPMLs.  The update kernels map one thread to one Yee cell with lanes along
// z (coalesced 256-byte rows per component); the j, k neighbours come from
// L1 and the i neighbours from L2.  CPML auxiliaries live only in the PML
// slabs; the plane-wave / adjoint sources and the running DFTs are fused
// into the E update.
//
// Stretched-coordinate r-PML (rpml_metric = 1): inside the r-PML the z-curls'
// (1/r) d/dr (r F) = (F(i+1) - F(i))/dr + (F(i+1) + F(i))/(2 r) is split; only
// the derivative carries the CPML stretch, and the metric part
// X = (F(i+1) + F(i))/2 -+ dF/dphi (and the phi-derivative of the r-curls) is
// divided by the stretched radius through 1/r~ = (1/r)(X + psi_m),
// psi_m <- bm psi_m + cm X (bm = cm = 0 where r~ = r, the inner slab).
//
// Continuous axisymmetry (the axis zone, one phi cell): every (1/r) d/dphi
// is i m / r times the local value.  On the axis (r_lo = 0) the table entry
// 1/r_0 is 0, so H_r(0) keeps its value 0; E_z(0) and E_phi(0) are not
// updated (E_z vanishes on the axis for |m| = 1 and E_phi(0), H_r(0) enter the
// other updates multiplied by r = 0).
#include "zda_internal.h"

namespace zda {

#define ZDA_BX 32
#define ZDA_BY 8

__device__ __forceinline__ int zslab(int k, int nz, int pz) {
    if (k < pz) return k;
    if (k >= nz - pz) return k - (nz - 2 * pz);
    return -1;
}
__device__ __forceinline__ int rslab(int i, int nr, int pin, int pout) {
    if (i < pin) return i;
    if (i >= nr - pout) return i - (nr - pin - pout);
    return -1;
}

// ------------------------------------------------------------------ H update
// H^{n+1/2} = H^{n-1/2} - dt curl E^n  (Eq. 3 with mu = 1)
__global__ void __launch_bounds__(ZDA_BX * ZDA_BY) k_update_h(const StepParams p)
{
    const int k = blockIdx.x * ZDA_BX + threadIdx.x;
    const int j = blockIdx.y * ZDA_BY + threadIdx.y;
    const int i = blockIdx.z;
    if (k >= p.nz || j >= p.nphi) return;
    const int nz = p.nz, nphi = p.nphi;
    const size_t sj = (size_t)nz, si = (size_t)nphi * nz;
    const size_t c = (size_t)i * si + (size_t)j * sj + k;
    const float2 zero = make_float2(0.f, 0.f);

    const float2 er = p.f.Er[c], ep = p.f.Ep[c], ez = p.f.Ez[c];
    float2 ez_jp, er_jp;
    if (j + 1 < nphi) {
        ez_jp = p.f.Ez[c + sj];
        er_jp = p.f.Er[c + sj];
    } else {                                   // wrap: psi(phi + tau) = e^{i m tau} psi(phi)
        const size_t c0 = c - (size_t)(nphi - 1) * sj;
        ez_jp = c_mul(p.bloch, p.f.Ez[c0]);
        er_jp = c_mul(p.bloch, p.f.Er[c0]);
    }
    const bool kin = k + 1 < nz, iin = i + 1 < p.nr;
    const float2 ep_kp = kin ? p.f.Ep[c + 1] : zero;
    const float2 er_kp = kin ? p.f.Er[c + 1] : zero;
    const float2 ez_ip = iin ? p.f.Ez[c + si] : zero;
    const float2 ep_ip = iin ? p.f.Ep[c + si] : zero;
    const float irn = __ldg(p.t.inv_r_n + i), irh = __ldg(p.t.inv_r_h + i);
    const int kz = zslab(k, nz, p.pz);
    const int ir = rslab(i, p.nr, p.pr_in, p.pr_out);
    const float dt = p.dt;
    const bool sr = p.rpml_metric && ir >= 0;          // stretched r-PML column (uniform per block)
    const size_t rx = ((size_t)(ir >= 0 ? ir : 0) * nphi + j) * nz + k;

    // H_r(i, j+1/2, k+1/2): (1/r) dE_z/dphi - dE_phi/dz
    {
        float2 dph;
        if (sr) {
            const float2 X = p.bor ? c_scale(make_float2(-ez.y, ez.x), p.m) : c_scale(c_sub(ez_jp, ez), p.inv_dphi);
            const float2 pm = c_add(c_scale(p.rm.hr[rx], __ldg(p.rm.bm_n + i)), c_scale(X, __ldg(p.rm.cm_n + i)));
            p.rm.hr[rx] = pm;
            dph = c_scale(c_add(X, pm), irn);
        } else {
            dph = p.bor ? c_scale(make_float2(-ez.y, ez.x), p.m * irn) : c_scale(c_sub(ez_jp, ez), irn * p.inv_dphi);
        }
        float2 dz = c_scale(c_sub(ep_kp, ep), p.inv_dz);
        if (kz >= 0) {
            const size_t ix = ((size_t)i * nphi + j) * (2 * p.pz) + kz;
            float2 ps = c_add(c_scale(p.psi.hr_z[ix], __ldg(p.t.bz_h + k)), c_scale(dz, __ldg(p.t.cz_h + k)));
            p.psi.hr_z[ix] = ps;
            dz = c_add(dz, ps);
        }
        const float2 h = p.f.Hr[c];
        p.f.Hr[c] = c_sub(h, c_scale(c_sub(dph, dz), dt));
    }
    // H_phi(i+1/2, j, k+1/2): dE_r/dz - dE_z/dr
    {
        float2 dz = c_scale(c_sub(er_kp, er), p.inv_dz);
        float2 drr = c_scale(c_sub(ez_ip, ez), p.inv_dr);
        if (kz >= 0) {
            const size_t ix = ((size_t)i * nphi + j) * (2 * p.pz) + kz;
            float2 ps = c_add(c_scale(p.psi.hp_z[ix], __ldg(p.t.bz_h + k)), c_scale(dz, __ldg(p.t.cz_h + k)));
            p.psi.hp_z[ix] = ps;
            dz = c_add(dz, ps);
        }
        if (ir >= 0) {
            const size_t ix = ((size_t)ir * nphi + j) * nz + k;
            float2 ps = c_add(c_scale(p.psi.hp_r[ix], __ldg(p.t.br_h + i)), c_scale(drr, __ldg(p.t.cr_h + i)));
            p.psi.hp_r[ix] = ps;
            drr = c_add(drr, ps);
        }
        const float2 h = p.f.Hp[c];
        p.f.Hp[c] = c_sub(h, c_scale(c_sub(dz, drr), dt));
    }
    // H_z(i+1/2, j+1/2, k): (1/r) d(r E_phi)/dr - (1/r) dE_r/dphi
    //   (r_{i+1} E(i+1) - r_i E(i)) / (r_{i+1/2} dr) = (E(i+1)-E(i))/dr + (E(i+1)+E(i)) / (2 r_{i+1/2})
    if (sr) {
        float2 drr = c_scale(c_sub(ep_ip, ep), p.inv_dr);
        const float2 ps = c_add(c_scale(p.psi.hz_r[rx], __ldg(p.t.br_h + i)), c_scale(drr, __ldg(p.t.cr_h + i)));
        p.psi.hz_r[rx] = ps;
        drr = c_add(drr, ps);
        const float2 X = c_sub(c_scale(c_add(ep_ip, ep), 0.5f),
                               p.bor ? c_scale(make_float2(-er.y, er.x), p.m) : c_scale(c_sub(er_jp, er), p.inv_dphi));
        const float2 pm = c_add(c_scale(p.rm.hz[rx], __ldg(p.rm.bm_h + i)), c_scale(X, __ldg(p.rm.cm_h + i)));
        p.rm.hz[rx] = pm;
        const float2 h = p.f.Hz[c];
        p.f.Hz[c] = c_sub(h, c_scale(c_add(drr, c_scale(c_add(X, pm), irh)), dt));
    } else {
        float2 drr = c_add(c_scale(c_sub(ep_ip, ep), p.inv_dr), c_scale(c_add(ep_ip, ep), 0.5f * irh));
        const float2 dph = p.bor ? c_scale(make_float2(-er.y, er.x), p.m * irh)
                                 : c_scale(c_sub(er_jp, er), irh * p.inv_dphi);
        if (ir >= 0) {
            const size_t ix = ((size_t)ir * nphi + j) * nz + k;
            float2 ps = c_add(c_scale(p.psi.hz_r[ix], __ldg(p.t.br_h + i)), c_scale(drr, __ldg(p.t.cr_h + i)));
            p.psi.hz_r[ix] = ps;
            drr = c_add(drr, ps);
        }
        const float2 h = p.f.Hz[c];
        p.f.Hz[c] = c_sub(h, c_scale(c_sub(drr, dph), dt));
    }
}

// ------------------------------------------------------------------ E update
// E^{n+1} = E^n + dt/eps (curl H^{n+1/2} - J^{n+1/2})  (Eq. 4), then the
// running DFT X_q += E^{n+1} e^{i w_q t_{n+1}} dt.
__global__ void __launch_bounds__(ZDA_BX * ZDA_BY) k_update_e(const StepParams p, const int n)
{
    const int k = blockIdx.x * ZDA_BX + threadIdx.x;
    const int j = blockIdx.y * ZDA_BY + threadIdx.y;
    const int i = blockIdx.z;
    if (k >= p.nz || j >= p.nphi) return;
    const int nz = p.nz, nphi = p.nphi, nr = p.nr;
    const size_t sj = (size_t)nz, si = (size_t)nphi * nz;
    const size_t c = (size_t)i * si + (size_t)j * sj + k;
    const float2 zero = make_float2(0.f, 0.f);

    const float2 hr = p.f.Hr[c], hp = p.f.Hp[c], hz = p.f.Hz[c];
    float2 hz_jm, hr_jm;
    if (j > 0) {
        hz_jm = p.f.Hz[c - sj];
        hr_jm = p.f.Hr[c - sj];
    } else {                                   // psi(phi - tau) = e^{-i m tau} psi(phi)
        const size_t c1 = c + (size_t)(nphi - 1) * sj;
        hz_jm = c_mul(p.bloch_inv, p.f.Hz[c1]);
        hr_jm = c_mul(p.bloch_inv, p.f.Hr[c1]);
    }
    const float2 hp_km = (k > 0) ? p.f.Hp[c - 1] : zero;
    const float2 hr_km = (k > 0) ? p.f.Hr[c - 1] : zero;
    const float2 hz_im = (i > 0) ? p.f.Hz[c - si] : zero;
    const float2 hp_im = (i > 0) ? p.f.Hp[c - si] : zero;
    const float irn = __ldg(p.t.inv_r_n + i), irh = __ldg(p.t.inv_r_h + i);
    const int kz = zslab(k, nz, p.pz);
    const int ir = rslab(i, nr, p.pr_in, p.pr_out);
    const float dt = p.dt;
    const size_t ij = (size_t)i * nphi + j;
    const bool sr = p.rpml_metric && ir >= 0;          // stretched r-PML column (uniform per block)
    const size_t rx = ((size_t)(ir >= 0 ? ir : 0) * nphi + j) * nz + k;

    float2 jr = zero, jp = zero;
    if (k == p.src_k) {
        if (p.src_mode == SRC_PLANE_WAVE) {
            // m = +1 part of an x-polarised sheet: (1/2, i/2) e^{i m phi} g(t) / dz
            const float a = __ldg(p.t.pulse + n) * p.src_scale;
            const float2 pn = p.t.ph_n[j], ph = p.t.ph_h[j];
            jr = c_scale(pn, a);
            jp = make_float2(-ph.y * a, ph.x * a);
        } else if (p.src_mode == SRC_ADJOINT) {
            float2 sr = zero, sp = zero;
            const float2 *kt = p.t.adj_time + (size_t)n * p.nq;
            for (int q = 0; q < p.nq; ++q) {
                const float2 kq = kt[q];
                sr = c_fma(p.beta_r[(size_t)q * nr + i], kq, sr);
                sp = c_fma(p.beta_p[(size_t)q * nr + i], kq, sp);
            }
            jr = c_mul(p.t.ph_n[j], sr);
            jp = c_mul(p.t.ph_h[j], sp);
        }
    }

    float2 er = p.f.Er[c], ep = p.f.Ep[c], ez = p.f.Ez[c];
    // E_r(i+1/2, j, k): (1/r) dH_z/dphi - dH_phi/dz ; PEC at k = 0
    if (k > 0) {
        float2 dph;
        if (sr) {
            const float2 X = p.bor ? c_scale(make_float2(-hz.y, hz.x), p.m) : c_scale(c_sub(hz, hz_jm), p.inv_dphi);
            const float2 pm = c_add(c_scale(p.rm.er[rx], __ldg(p.rm.bm_h + i)), c_scale(X, __ldg(p.rm.cm_h + i)));
            p.rm.er[rx] = pm;
            dph = c_scale(c_add(X, pm), irh);
        } else {
            dph = p.bor ? c_scale(make_float2(-hz.y, hz.x), p.m * irh) : c_scale(c_sub(hz, hz_jm), irh * p.inv_dphi);
        }
        float2 dz = c_scale(c_sub(hp, hp_km), p.inv_dz);
        if (kz >= 0) {
            const size_t ix = ij * (2 * p.pz) + kz;
            float2 ps = c_add(c_scale(p.psi.er_z[ix], __ldg(p.t.bz_n + k)), c_scale(dz, __ldg(p.t.cz_n + k)));
            p.psi.er_z[ix] = ps;
            dz = c_add(dz, ps);
        }
        const float ie = 1.0f / (__ldg(p.t.a_n + k) + __ldg(p.t.d_n + k) * __ldg(p.rb_r + ij));
        er = c_add(er, c_scale(c_sub(c_sub(dph, dz), jr), dt * ie));
        p.f.Er[c] = er;
    }
    // E_phi(i, j+1/2, k): dH_r/dz - dH_z/dr ; PEC at i = 0 and k = 0
    if (i > 0 && k > 0) {
        float2 dz = c_scale(c_sub(hr, hr_km), p.inv_dz);
        float2 drr = c_scale(c_sub(hz, hz_im), p.inv_dr);
        if (kz >= 0) {
            const size_t ix = ij * (2 * p.pz) + kz;
            float2 ps = c_add(c_scale(p.psi.ep_z[ix], __ldg(p.t.bz_n + k)), c_scale(dz, __ldg(p.t.cz_n + k)));
            p.psi.ep_z[ix] = ps;
            dz = c_add(dz, ps);
        }
        if (ir >= 0) {
            const size_t ix = ((size_t)ir * nphi + j) * nz + k;
            float2 ps = c_add(c_scale(p.psi.ep_r[ix], __ldg(p.t.br_n + i)), c_scale(drr, __ldg(p.t.cr_n + i)));
            p.psi.ep_r[ix] = ps;
            drr = c_add(drr, ps);
        }
        const float ie = 1.0f / (__ldg(p.t.a_n + k) + __ldg(p.t.d_n + k) * __ldg(p.rb_p + ij));
        ep = c_add(ep, c_scale(c_sub(c_sub(dz, drr), jp), dt * ie));
        p.f.Ep[c] = ep;
    }
    // E_z(i, j, k+1/2): (1/r) d(r H_phi)/dr - (1/r) dH_r/dphi ; PEC at i = 0
    //   (r_{i+1/2} H(i+1/2) - r_{i-1/2} H(i-1/2)) / (r_i dr) = (H - H_im)/dr + (H + H_im) / (2 r_i)
    if (i > 0 && sr) {
        float2 drr = c_scale(c_sub(hp, hp_im), p.inv_dr);
        const float2 ps = c_add(c_scale(p.psi.ez_r[rx], __ldg(p.t.br_n + i)), c_scale(drr, __ldg(p.t.cr_n + i)));
        p.psi.ez_r[rx] = ps;
        drr = c_add(drr, ps);
        const float2 X = c_sub(c_scale(c_add(hp, hp_im), 0.5f),
                               p.bor ? c_scale(make_float2(-hr.y, hr.x), p.m) : c_scale(c_sub(hr, hr_jm), p.inv_dphi));
        const float2 pm = c_add(c_scale(p.rm.ez[rx], __ldg(p.rm.bm_n + i)), c_scale(X, __ldg(p.rm.cm_n + i)));
        p.rm.ez[rx] = pm;
        const float ie = 1.0f / (__ldg(p.t.a_c + k) + __ldg(p.t.d_c + k) * __ldg(p.rb_z + ij));
        ez = c_add(ez, c_scale(c_add(drr, c_scale(c_add(X, pm), irn)), dt * ie));
        p.f.Ez[c] = ez;
    } else if (i > 0) {
        float2 drr = c_add(c_scale(c_sub(hp, hp_im), p.inv_dr), c_scale(c_add(hp, hp_im), 0.5f * irn));
        const float2 dph = p.bor ? c_scale(make_float2(-hr.y, hr.x), p.m * irn)
                                 : c_scale(c_sub(hr, hr_jm), irn * p.inv_dphi);
        if (ir >= 0) {
            const size_t ix = ((size_t)ir * nphi + j) * nz + k;
            float2 ps = c_add(c_scale(p.psi.ez_r[ix], __ldg(p.t.br_n + i)), c_scale(drr, __ldg(p.t.cr_n + i)));
            p.psi.ez_r[ix] = ps;
            drr = c_add(drr, ps);
        }
        const float ie = 1.0f / (__ldg(p.t.a_c + k) + __ldg(p.t.d_c + k) * __ldg(p.rb_z + ij));
        ez = c_add(ez, c_scale(c_sub(drr, dph), dt * ie));
        p.f.Ez[c] = ez;
    }

    // running DFTs of E^{n+1}
    if (p.mon && k == p.mon_k) {
        const size_t plane = (size_t)nr * nphi;
        const float2 e2[2] = {er, ep};
        dft_update<2>(p.mon + ij, 2 * plane, plane, p.t.twiddle + (size_t)n * p.nq, p.nq, e2);
    }
    if (p.des) {
        const int kk = k - p.des_k0;
        if (kk >= 0 && kk < p.des_nk) {
            const size_t comp = (size_t)nr * nphi * p.des_nk;
            const float2 e3[3] = {er, ep, ez};
            dft_update<3>(p.des + ij * p.des_nk + kk, 3 * comp, comp, p.t.twiddle + (size_t)n * p.nq, p.nq, e3);
        }
    }
}

void launch_update_h(const StepParams &p, cudaStream_t s)
{
    dim3 b(ZDA_BX, ZDA_BY), g((p.nz + ZDA_BX - 1) / ZDA_BX, (p.nphi + ZDA_BY - 1) / ZDA_BY, p.nr);
    k_update_h<<<g, b, 0, s>>>(p);
}

void launch_update_e(const StepParams &p, int n, cudaStream_t s)
{
    dim3 b(ZDA_BX, ZDA_BY), g((p.nz + ZDA_BX - 1) / ZDA_BX, (p.nphi + ZDA_BY - 1) / ZDA_BY, p.nr);
    k_update_e<<<g, b, 0, s>>>(p, n);
}

// ------------------------------------------------ density -> rho~ (conic + tanh)
// Conic filter on the curvilinear wedge: weight max(0, 1 - d/R),
// d^2 = (di dr)^2 + (r_c dj dphi)^2 with r_c the output pixel's radius; phi
// wraps (the density repeats every wedge); taps beyond the design's r-edges
// are dropped and the weights renormalised.  Then the tanh projection.
__device__ __forceinline__ float cone_w(const FilterParams &fp, int i, int di, int dj)
{
    const float rc = fp.r_c0 + i * fp.dr;
    const float a = di * fp.dr, b = rc * dj * fp.dphi;
    return fmaxf(0.f, 1.f - sqrtf(a * a + b * b) / fp.R);
}

__device__ __forceinline__ float proj(const FilterParams &fp, float x)
{
    if (fp.beta <= 0.f) return x;
    const float te = tanhf(fp.beta * fp.eta);
    return (te + tanhf(fp.beta * (x - fp.eta))) / (te + tanhf(fp.beta * (1.f - fp.eta)));
}

__device__ __forceinline__ float proj_grad(const FilterParams &fp, float x)
{
    if (fp.beta <= 0.f) return 1.f;
    const float te = tanhf(fp.beta * fp.eta);
    const float ch = coshf(fp.beta * (x - fp.eta));
    return fp.beta / (ch * ch) / (te + tanhf(fp.beta * (1.f - fp.eta)));
}

__global__ void k_filter_norm(const FilterParams fp, float *norm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= fp.nrd) return;
    float s = 0.f;
    for (int di = -fp.di_max; di <= fp.di_max; ++di) {
        if (i + di < 0 || i + di >= fp.nrd) continue;
        for (int dj = -fp.dj_max; dj <= fp.dj_max; ++dj) s += cone_w(fp, i, di, dj);
    }
    norm[i] = s;
}

__global__ void k_filter_project(const FilterParams fp, const float *__restrict__ rho,
                                 const float *__restrict__ norm, float *rho_bar, float *rho_t)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= fp.nphi || i >= fp.nrd) return;
    const int nphi = fp.nphi;
    float v;
    if (fp.filter_on) {
        float s = 0.f;
        for (int di = -fp.di_max; di <= fp.di_max; ++di) {
            const int ii = i + di;
            if (ii < 0 || ii >= fp.nrd) continue;
            const float *row = rho + (size_t)ii * nphi;
            for (int dj = -fp.dj_max; dj <= fp.dj_max; ++dj) {
                const float w = cone_w(fp, i, di, dj);
                if (w == 0.f) continue;
                int jj = (j + dj) % nphi;
                if (jj < 0) jj += nphi;
                s = fmaf(w, __ldg(row + jj), s);
            }
        }
        v = s / norm[i];
    } else {
        v = rho[(size_t)i * nphi + j];
    }
    rho_bar[(size_t)i * nphi + j] = v;
    rho_t[(size_t)i * nphi + j] = proj(fp, v);
}

// dI/drho[i'][j'] = sum_{di,dj} w(i'-di; di, dj) / norm(i'-di) * P'(rho_bar) g_t  at (i'-di, j'-dj)
__global__ void k_filter_project_bwd(const FilterParams fp, const float *__restrict__ rho_bar,
                                     const float *__restrict__ norm, const float *__restrict__ g_t,
                                     float *g_rho)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= fp.nphi || i >= fp.nrd) return;
    const int nphi = fp.nphi;
    if (!fp.filter_on) {
        const size_t ix = (size_t)i * nphi + j;
        g_rho[ix] = g_t[ix] * proj_grad(fp, rho_bar[ix]);
        return;
    }
    float s = 0.f;
    for (int di = -fp.di_max; di <= fp.di_max; ++di) {
        const int io = i - di;                  // output pixel row that read this input with offset di
        if (io < 0 || io >= fp.nrd) continue;
        const float inv_n = 1.f / norm[io];
        for (int dj = -fp.dj_max; dj <= fp.dj_max; ++dj) {
            const float w = cone_w(fp, io, di, dj);
            if (w == 0.f) continue;
            int jo = (j - dj) % nphi;
            if (jo < 0) jo += nphi;
            const size_t ox = (size_t)io * nphi + jo;
            s = fmaf(w * inv_n, g_t[ox] * proj_grad(fp, rho_bar[ox]), s);
        }
    }
    g_rho[(size_t)i * nphi + j] = s;
}

void launch_filter_norm(const FilterParams &fp, float *norm, cudaStream_t s)
{
    k_filter_norm<<<(fp.nrd + 127) / 128, 128, 0, s>>>(fp, norm);
}
void launch_filter_project(const FilterParams &fp, const float *rho, const float *norm, float *rho_bar,
                           float *rho_t, cudaStream_t s)
{
    dim3 g((fp.nphi + 127) / 128, fp.nrd);
    k_filter_project<<<g, 128, 0, s>>>(fp, rho, norm, rho_bar, rho_t);
}
void launch_filter_project_backward(const FilterParams &fp, const float *rho_bar, const float *norm,
                                    const float *g_t, float *g_rho, cudaStream_t s)
{
    dim3 g((fp.nphi + 127) / 128, fp.nrd);
    k_filter_project_bwd<<<g, 128, 0, s>>>(fp, rho_bar, norm, g_t, g_rho);
}

// Transverse averages of the cell density (0 in the r-PML columns, where the
// design layer holds eps_lo): E_r sites average the two phi-neighbour cells,
// E_phi sites the two r-neighbours, E_z sites four; phi wraps, r clamps.
__global__ void k_rho_bar(const float *__restrict__ rho_t, int nr, int nphi, int i_d0, int i_d1,
                          float *rb_r, float *rb_p, float *rb_z)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= nphi || i >= nr) return;
    auto cell = [&](int ii, int jj) -> float {
        if (ii < 0) ii = 0;
        if (jj < 0) jj += nphi;
        return (ii >= i_d0 && ii < i_d1) ? rho_t[(size_t)(ii - i_d0) * nphi + jj] : 0.f;
    };
    const float c00 = cell(i, j), c0m = cell(i, j - 1), cm0 = cell(i - 1, j), cmm = cell(i - 1, j - 1);
    const size_t ix = (size_t)i * nphi + j;
    rb_r[ix] = 0.5f * (c0m + c00);
    rb_p[ix] = 0.5f * (cm0 + c00);
    rb_z[ix] = 0.25f * (cmm + cm0 + c0m + c00);
}

// Field energy of the current state and of its one-step difference (decay
// probe): per radius i (one block), sum over the sites of eps |E|^2 V and
// |H|^2 V, V = r dr dphi dz with r the site's radius (E_r, H_phi, H_z at
// r_{i+1/2}; E_phi, E_z, H_r at r_i), for cur and for cur - prev; FP64
// block sums into partial[2 i], partial[2 i + 1].
__global__ void k_field_energy(const StepParams p, const Fields fc, const Fields fp, double r_lo, double dr,
                               double vol_dphi_dz, double *partial)
{
    const float2 *cur[6] = {fc.Er, fc.Ep, fc.Ez, fc.Hr, fc.Hp, fc.Hz};
    const float2 *prev[6] = {fp.Er, fp.Ep, fp.Ez, fp.Hr, fp.Hp, fp.Hz};
    const int i = blockIdx.x;
    const int nphi = p.nphi, nz = p.nz;
    const size_t base = (size_t)i * nphi * nz;
    const double rn = r_lo + i * dr, rh = r_lo + (i + 0.5) * dr;
    double w = 0.0, wd = 0.0;
    for (int t = threadIdx.x; t < nphi * nz; t += blockDim.x) {
        const int j = t / nz, k = t % nz;
        const size_t c = base + t, ij = (size_t)i * nphi + j;
        const float er = p.t.a_n[k] + p.t.d_n[k] * p.rb_r[ij];
        const float ep = p.t.a_n[k] + p.t.d_n[k] * p.rb_p[ij];
        const float ez = p.t.a_c[k] + p.t.d_c[k] * p.rb_z[ij];
        const double wgt[6] = {er * rh, ep * rn, ez * rn, rn, rh, rh};
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const float2 a = cur[f][c], b = prev[f][c];
            const float dx = a.x - b.x, dy = a.y - b.y;
            w += wgt[f] * ((double)a.x * a.x + (double)a.y * a.y);
            wd += wgt[f] * ((double)dx * dx + (double)dy * dy);
        }
    }
    __shared__ double sw[256], sd[256];
    sw[threadIdx.x] = w;
    sd[threadIdx.x] = wd;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sw[threadIdx.x] += sw[threadIdx.x + o];
            sd[threadIdx.x] += sd[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * i] = sw[0] * dr * vol_dphi_dz;
        partial[2 * i + 1] = sd[0] * dr * vol_dphi_dz;
    }
}

__global__ void k_field_energy_sum(const double *partial, int nr, double *w_out, double *wdot_out)
{
    __shared__ double sw[256], sd[256];
    double w = 0.0, wd = 0.0;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        w += partial[2 * i];
        wd += partial[2 * i + 1];
    }
    sw[threadIdx.x] = w;
    sd[threadIdx.x] = wd;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sw[threadIdx.x] += sw[threadIdx.x + o];
            sd[threadIdx.x] += sd[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *w_out = sw[0];
        *wdot_out = sd[0];
    }
}

void launch_field_energy(const StepParams &p, const Fields &cur, const Fields &prev, double r_lo, double dr,
                         double vol_dphi_dz, double *partial, double *w_out, double *wdot_out, cudaStream_t s)
{
    k_field_energy<<<p.nr, 256, 0, s>>>(p, cur, prev, r_lo, dr, vol_dphi_dz, partial);
    k_field_energy_sum<<<1, 256, 0, s>>>(partial, p.nr, w_out, wdot_out);
}

void launch_rho_bar(const float *rho_t, int nr, int nphi, int i_d0, int i_d1, float *rb_r, float *rb_p,
                    float *rb_z, cudaStream_t s)
{
    dim3 g((nphi + 127) / 128, nr);
    k_rho_bar<<<g, 128, 0, s>>>(rho_t, nr, nphi, i_d0, i_d1, rb_r, rb_p, rb_z);
}

// ------------------------------------------------ near-to-far focal transform
// S_q = sum_i Gr[q][i] sum_j e^{-i phi_j} E_r(q,i,j) + Gp[q][i] sum_j e^{-i phi_{j+1/2}} E_phi(q,i,j)
// (Rayleigh-Sommerfeld weights with quadrature, the -i of the E_phi term and
// the conjugation of the -w entries are in the radial tables).  Warp-shuffle
// block reductions in FP64; one partial per (q, i), then a per-q sum:
// deterministic, no atomics.
__device__ __forceinline__ double2 d_cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 block_sum2(double2 v)
{
    __shared__ double2 red[32];
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    v = (threadIdx.x < nw) ? red[threadIdx.x] : make_double2(0.0, 0.0);
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, o);
            v.y += __shfl_down_sync(0xffffffffu, v.y, o);
        }
    return v;
}

__global__ void k_focal_partial(const float2 *__restrict__ mon, const double2 *__restrict__ Gr,
                                const double2 *__restrict__ Gp, const double2 *__restrict__ emph_n,
                                const double2 *__restrict__ emph_h, int nr, int nphi, double2 *partial)
{
    const int i = blockIdx.x, q = blockIdx.y;
    const size_t plane = (size_t)nr * nphi;
    const float2 *er = mon + (size_t)q * 2 * plane + (size_t)i * nphi;
    const float2 *ep = er + plane;
    double2 sr = make_double2(0, 0), sp = make_double2(0, 0);
    for (int j = threadIdx.x; j < nphi; j += blockDim.x) {
        const float2 a = er[j], b = ep[j];
        const double2 pa = d_cmul(emph_n[j], make_double2(a.x, a.y));
        const double2 pb = d_cmul(emph_h[j], make_double2(b.x, b.y));
        sr.x += pa.x; sr.y += pa.y;
        sp.x += pb.x; sp.y += pb.y;
    }
    const double2 gr = Gr[(size_t)q * nr + i], gp = Gp[(size_t)q * nr + i];
    const double2 tr = d_cmul(gr, sr), tp = d_cmul(gp, sp);
    double2 v = block_sum2(make_double2(tr.x + tp.x, tr.y + tp.y));
    if (threadIdx.x == 0) partial[(size_t)q * nr + i] = v;
}

__global__ void k_focal_sum(const double2 *__restrict__ partial, int nr, double2 *S, int *status)
{
    const int q = blockIdx.x;
    double2 v = make_double2(0, 0);
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
        const double2 a = partial[(size_t)q * nr + i];
        v.x += a.x; v.y += a.y;
    }
    v = block_sum2(v);
    if (threadIdx.x == 0) {
        S[q] = v;
        if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(status, 1);
    }
}

void launch_focal_partial(const float2 *mon, const double2 *Gr, const double2 *Gp, const double2 *emph_n,
                          const double2 *emph_h, int nq, int nr, int nphi, double2 *partial, cudaStream_t s)
{
    dim3 g(nr, nq);
    k_focal_partial<<<g, 256, 0, s>>>(mon, Gr, Gp, emph_n, emph_h, nr, nphi, partial);
}
void launch_focal_sum(const double2 *partial, int nq, int nr, double2 *S, int *status, cudaStream_t s)
{
    k_focal_sum<<<nq, 256, 0, s>>>(partial, nr, S, status);
}

// ------------------------------------------------ focal transform on surrogate outputs
// The surrogate's output y[b][id][j][ch] holds the monitor DFT of design row
// i = i_d0 + id in channels ch = (q 2 + comp) 2 + part (part 0 real, 1
// imaginary), divided by `scale`.  S[b][q] = sum_i Gr_q(i) sum_j emph_n(j) E_r
// + Gp_q(i) sum_j emph_h(j) E_phi over those rows (the outer edge node of
// E_phi, i = i_d1, is not among them).
__global__ void k_focal_nn(const float *__restrict__ y, int nq, int i_d0, int nrd, int nphi, int nr, float scale,
                           const double2 *__restrict__ Gr, const double2 *__restrict__ Gp,
                           const double2 *__restrict__ emph_n, const double2 *__restrict__ emph_h, double2 *S)
{
    const int q = blockIdx.x, b = blockIdx.y;
    const int nch = 4 * nq;
    double2 acc = make_double2(0, 0);
    for (int t = threadIdx.x; t < nrd * nphi; t += blockDim.x) {
        const int id = t / nphi, j = t % nphi, i = i_d0 + id;
        const float *v = y + (((size_t)b * nrd + id) * nphi + j) * nch + q * 4;
        const double2 er = make_double2((double)v[0] * scale, (double)v[1] * scale);
        const double2 ep = make_double2((double)v[2] * scale, (double)v[3] * scale);
        const double2 a = d_cmul(Gr[(size_t)q * nr + i], d_cmul(emph_n[j], er));
        const double2 c = d_cmul(Gp[(size_t)q * nr + i], d_cmul(emph_h[j], ep));
        acc.x += a.x + c.x;
        acc.y += a.y + c.y;
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0) S[(size_t)b * nq + q] = acc;
}

// Transpose: dy = d obj / d y for G = dobj/dRe S + i dobj/dIm S per (b, q):
// with w the site weight, d/dRe m = Re(conj(G) w), d/dIm m = Im(G conj(w)), times scale.
__global__ void k_focal_nn_T(const double2 *__restrict__ G, int nq, int i_d0, int nrd, int nphi, int nr, int n,
                             float scale, const double2 *__restrict__ Gr, const double2 *__restrict__ Gp,
                             const double2 *__restrict__ emph_n, const double2 *__restrict__ emph_h, float *dy)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long tot = (long)n * nrd * nphi * nq * 2;
    if (t >= tot) return;
    const int comp = (int)(t % 2), q = (int)((t / 2) % nq);
    const long pix = t / (2 * nq);
    const int j = (int)(pix % nphi), id = (int)((pix / nphi) % nrd);
    const int b = (int)(pix / ((long)nphi * nrd)), i = i_d0 + id;
    const double2 w = comp == 0 ? d_cmul(Gr[(size_t)q * nr + i], emph_n[j]) : d_cmul(Gp[(size_t)q * nr + i], emph_h[j]);
    const double2 g = G[(size_t)b * nq + q];
    const double dre = g.x * w.x + g.y * w.y;      // Re(conj(G) w)
    const double dim = g.y * w.x - g.x * w.y;      // Im(G conj(w))
    float *o = dy + pix * (4 * nq) + (q * 2 + comp) * 2;
    o[0] = (float)(dre * scale);
    o[1] = (float)(dim * scale);
}

void launch_focal_nn(const float *y, int n, int nq, int i_d0, int nrd, int nphi, int nr, float scale,
                     const double2 *Gr, const double2 *Gp, const double2 *emph_n, const double2 *emph_h, double2 *S,
                     cudaStream_t s)
{
    k_focal_nn<<<dim3(nq, n), 256, 0, s>>>(y, nq, i_d0, nrd, nphi, nr, scale, Gr, Gp, emph_n, emph_h, S);
}

void launch_focal_nn_T(const double2 *G, int n, int nq, int i_d0, int nrd, int nphi, int nr, float scale,
                       const double2 *Gr, const double2 *Gp, const double2 *emph_n, const double2 *emph_h, float *dy,
                       cudaStream_t s)
{
    const long tot = (long)n * nrd * nphi * nq * 2;
    k_focal_nn_T<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, nq, i_d0, nrd, nphi, nr, n, scale, Gr, Gp, emph_n,
                                                              emph_h, dy);
}

// ------------------------------------------------ adjoint source profiles
// The transpose of the focal transform gives the sensitivity
// a_q = conj(g_q) w_q on the monitor sites; the adjoint (+m) run is driven by
// b_q = i conj(a_q) / (wt_q V) = [i g_q conj(G_q(r)) / (wt_q V(r))] e^{i phi}.
__global__ void k_adjoint_profiles(const double2 *__restrict__ g, const double2 *__restrict__ Gr,
                                   const double2 *__restrict__ Gp, const float *__restrict__ wt, int nr,
                                   double r_lo, double dr, double vol_scale, float2 *beta_r, float2 *beta_p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
    if (i >= nr) return;
    const double2 gq = g[q];
    const double w = (double)wt[q];
    const double Vr = (r_lo + (i + 0.5) * dr) * vol_scale;   // r dr dphi dz
    const double Vp = (r_lo + i * dr) * vol_scale;
    const double2 ig = make_double2(-gq.y, gq.x);              // i g
    const double2 cr = d_cmul(ig, make_double2(Gr[(size_t)q * nr + i].x, -Gr[(size_t)q * nr + i].y));
    const double2 cp = d_cmul(ig, make_double2(Gp[(size_t)q * nr + i].x, -Gp[(size_t)q * nr + i].y));
    beta_r[(size_t)q * nr + i] = make_float2((float)(cr.x / (w * Vr)), (float)(cr.y / (w * Vr)));
    beta_p[(size_t)q * nr + i] = (Vp > 0) ? make_float2((float)(cp.x / (w * Vp)), (float)(cp.y / (w * Vp)))
                                          : make_float2(0.f, 0.f);
}

void launch_adjoint_profiles(const double2 *g, const double2 *Gr, const double2 *Gp, const float *wt, int nq,
                             int nr, double r_lo, double dr, double vol_scale, float2 *beta_r, float2 *beta_p,
                             cudaStream_t s)
{
    dim3 gr((nr + 127) / 128, nq);
    k_adjoint_profiles<<<gr, 128, 0, s>>>(g, Gr, Gp, wt, nr, r_lo, dr, vol_scale, beta_r, beta_p);
}

// ------------------------------------------------ gradient overlap
// dI/deps_s = Re sum_q wt_q^2 V_s E_q(s) conj(A_{qbar}(s)), qbar the index of
// -w_q (the adjoint +m run carries the Bloch -m adjoint field as its
// conjugate at the opposite frequency).
__global__ void k_site_gradient(const float2 *__restrict__ des_f, const float2 *__restrict__ des_a,
                                const float *__restrict__ wt, int nq, int nr, int nphi, int nk, double r_lo,
                                double dr, double vol_scale, float *site_grad)
{
    const size_t comp = (size_t)nr * nphi * nk;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * comp) return;
    const int c = (int)(t / comp);
    const size_t s = t - (size_t)c * comp;
    const int i = (int)(s / ((size_t)nphi * nk));
    const int nl = nq / 2;
    float acc = 0.f;
    for (int q = 0; q < nq; ++q) {
        const int qb = (q + nl) % nq;
        const float2 e = des_f[((size_t)q * 3 + c) * comp + s];
        const float2 a = des_a[((size_t)qb * 3 + c) * comp + s];
        const float w2 = wt[q] * wt[q];
        acc = fmaf(w2, e.x * a.x + e.y * a.y, acc);           // Re(e conj(a))
    }
    const double r = (c == 0) ? r_lo + (i + 0.5) * dr : r_lo + i * dr;
    site_grad[t] = acc * (float)(r * vol_scale);
}

// Transpose of the site averaging: each design cell (i, j, k) collects a
// quarter of the gradient of every E site whose permittivity averages it,
// summed over the design layer's z-cells, times (eps_hi - eps_lo).
__global__ void k_cell_gradient(const float *__restrict__ sg, int nr, int nphi, int nk, int i_d0, int nrd,
                                float deps, float *g_t)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int ic = blockIdx.y;
    if (j >= nphi || ic >= nrd) return;
    const int i = i_d0 + ic;
    const size_t comp = (size_t)nr * nphi * nk;
    const int jp = (j + 1 < nphi) ? j + 1 : 0;
    const bool ip_ok = i + 1 < nr;
    auto G = [&](int c, int ii, int jj, int kk) -> float {
        return sg[(size_t)c * comp + ((size_t)ii * nphi + jj) * nk + kk];
    };
    float acc = 0.f;
    for (int kk = 0; kk + 1 < nk; ++kk) {      // design cells k0 .. k1-1 ; E planes k0 .. k1
        float s = G(0, i, j, kk) + G(0, i, jp, kk) + G(0, i, j, kk + 1) + G(0, i, jp, kk + 1);
        s += G(1, i, j, kk) + G(1, i, j, kk + 1);
        s += G(2, i, j, kk) + G(2, i, jp, kk);
        if (ip_ok) {
            s += G(1, i + 1, j, kk) + G(1, i + 1, j, kk + 1);
            s += G(2, i + 1, j, kk) + G(2, i + 1, jp, kk);
        }
        acc += 0.25f * s;
    }
    g_t[(size_t)ic * nphi + j] = acc * deps;
}

void launch_site_gradient(const float2 *des_f, const float2 *des_a, const float *wt, int nq, int nr, int nphi,
                          int nk, double r_lo, double dr, double vol_scale, float *site_grad, cudaStream_t s)
{
    const size_t n = (size_t)3 * nr * nphi * nk;
    k_site_gradient<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(des_f, des_a, wt, nq, nr, nphi, nk, r_lo, dr,
                                                               vol_scale, site_grad);
}
void launch_cell_gradient(const float *site_grad, int nr, int nphi, int nk, int i_d0, int nrd, float deps,
                          float *g_t, cudaStream_t s)
{
    dim3 g((nphi + 127) / 128, nrd);
    k_cell_gradient<<<g, 128, 0, s>>>(site_grad, nr, nphi, nk, i_d0, nrd, deps, g_t);
}

// Lens focal phasors: the sum over zones of each zone's S (the only
// cross-zone coupling of a lens), with a non-finite flag.
__global__ void k_lens_sum(const double2 *const *S, int nzones, int nq, double2 *out, int *status)
{
    const int q = threadIdx.x;
    if (q >= nq) return;
    double2 v = make_double2(0.0, 0.0);
    for (int z = 0; z < nzones; ++z) {
        const double2 a = S[z][q];
        v.x += a.x;
        v.y += a.y;
    }
    out[q] = v;
    if (!isfinite(v.x) || !isfinite(v.y)) atomicOr(status, 1);
}

void launch_lens_sum(const double2 *const *S, int nzones, int nq, double2 *out, int *status, cudaStream_t s)
{
    k_lens_sum<<<1, 32, 0, s>>>(S, nzones, nq, out, status);
}

// ------------------------------------------------ focal-plane evaluation
// Per zone: phi-means of the m = +1 run's monitor DFT, u_c(q, i) =
// (1/n_phi) sum_j Psi_c(q, i, j) e^{-i phi} (E_r at phi_j, E_phi at
// phi_{j+1/2}; no phase in the axis zone), and the transmitted-power density
// sum over the row of |E_r|^2 + |E_phi|^2 of the physical phasor at +w_l,
// Psi(+w) + conj(Psi(-w)).
// Per radius and frequency: the phi-means of the monitor DFT (times the
// e^{-i m phi} phases) and, per wavelength, sum_j of the transmitted
// intensity.  The physical +w field is E+ + E- (E+ = psi(+w), E- =
// conj(psi(-w))); over the n wedge copies the cross term 2 Re(E+ conj(E-))
// turns by e^{2 i tau} per copy and cancels for n >= 3 (and for continuous
// axisymmetry), so only abs(E+)^2 + abs(E-)^2 is summed; with cross != 0
// (n = 1, 2) abs(E+ + E-)^2.
__global__ void k_phi_means(const float2 *__restrict__ mon, const double2 *__restrict__ emph_n,
                            const double2 *__restrict__ emph_h, int nq, int nr, int nphi, int cross, double2 *umean,
                            double *pt_row)
{
    const int i = blockIdx.x, q = blockIdx.y;
    const size_t plane = (size_t)nr * nphi;
    const int nl = nq / 2;
    const float2 *er = mon + (size_t)q * 2 * plane + (size_t)i * nphi;
    const float2 *ep = er + plane;
    double2 sr = make_double2(0, 0), sp = make_double2(0, 0);
    double pw = 0.0;
    for (int j = threadIdx.x; j < nphi; j += blockDim.x) {
        const float2 a = er[j], b = ep[j];
        const double2 pa = d_cmul(emph_n[j], make_double2(a.x, a.y));
        const double2 pb = d_cmul(emph_h[j], make_double2(b.x, b.y));
        sr.x += pa.x; sr.y += pa.y;
        sp.x += pb.x; sp.y += pb.y;
        if (q < nl) {                                   // physical phasor at +w_q
            const float2 *er2 = mon + (size_t)(q + nl) * 2 * plane + (size_t)i * nphi;
            const float2 *ep2 = er2 + plane;
            if (cross) {
                const double xr = (double)a.x + er2[j].x, yr = (double)a.y - er2[j].y;
                const double xp = (double)b.x + ep2[j].x, yp = (double)b.y - ep2[j].y;
                pw += xr * xr + yr * yr + xp * xp + yp * yp;
            } else {
                const double c0 = er2[j].x, c1 = er2[j].y, c2 = ep2[j].x, c3 = ep2[j].y;
                pw += (double)a.x * a.x + (double)a.y * a.y + (double)b.x * b.x + (double)b.y * b.y +
                      c0 * c0 + c1 * c1 + c2 * c2 + c3 * c3;
            }
        }
    }
    const double2 tr = block_sum2(sr);
    __syncthreads();
    const double2 tp = block_sum2(sp);
    __syncthreads();
    const double2 tw = block_sum2(make_double2(pw, 0.0));
    if (threadIdx.x == 0) {
        umean[((size_t)q * 2 + 0) * nr + i] = make_double2(tr.x / nphi, tr.y / nphi);
        umean[((size_t)q * 2 + 1) * nr + i] = make_double2(tp.x / nphi, tp.y / nphi);
        if (q < nl) pt_row[(size_t)q * nr + i] = tw.x;
    }
}

void launch_phi_means(const float2 *mon, const double2 *emph_n, const double2 *emph_h, int nq, int nr, int nphi,
                      int cross, double2 *umean, double *pt_row, cudaStream_t s)
{
    dim3 g(nr, nq);
    k_phi_means<<<g, 256, 0, s>>>(mon, emph_n, emph_h, nq, nr, nphi, cross, umean, pt_row);
}

// Focal-plane field of one zone at points P = (x, y, z_f) above the monitor
// plane: Rayleigh-Sommerfeld (first kind) over the zone's annulus with the
// azimuthal orders +-1 of its near field,
//   E_x(Q) = e^{i phi}(u+_r cos - u+_phi sin) + e^{-i phi}(u-_r cos - u-_phi sin)
//   E_y(Q) = e^{i phi}(u+_r sin + u+_phi cos) + e^{-i phi}(u-_r sin + u-_phi cos)
// with u+ = u(+w), u- = conj(u(-w)); each component integrated on its own
// radial grid (weights wr, wp include r dr) and n_s phi samples.
// Accumulates (E_x, E_y) into ex, ey [n_lambda][n_pts].
__global__ void k_focal_plane(const double2 *__restrict__ umean, const double *__restrict__ rr,
                              const double *__restrict__ wr, const double *__restrict__ rp,
                              const double *__restrict__ wp, int nr, int nl, const double *__restrict__ pts,
                              int pstride, int npts, double zf0, const double *__restrict__ kk, int ns, double2 *ex,
                              double2 *ey)
{
    const int pidx = blockIdx.x, l = blockIdx.y;
    const double px = pts[pstride * pidx], py = pts[pstride * pidx + 1];
    const double zf = zf0 + (pstride == 3 ? pts[3 * pidx + 2] : 0.0);      // height above the focal plane
    const double k = kk[l];
    const double2 *upr = umean + ((size_t)l * 2 + 0) * nr, *upp = umean + ((size_t)l * 2 + 1) * nr;
    const double2 *umr = umean + ((size_t)(l + nl) * 2 + 0) * nr, *ump = umean + ((size_t)(l + nl) * 2 + 1) * nr;
    double2 ax = make_double2(0, 0), ay = make_double2(0, 0);
    const double dphi = 2.0 * M_PI / ns;
    const size_t total = (size_t)2 * nr * ns;
    for (size_t t = threadIdx.x; t < total; t += blockDim.x) {
        const int comp = (int)(t / ((size_t)nr * ns));
        const size_t rem = t - (size_t)comp * nr * ns;
        const int i = (int)(rem / ns), s = (int)(rem % ns);
        const double w = comp == 0 ? wr[i] : wp[i];
        if (w == 0.0) continue;
        const double r = comp == 0 ? rr[i] : rp[i];
        double sn, cs;
        sincos(s * dphi, &sn, &cs);
        const double dx = px - r * cs, dy = py - r * sn;
        const double R = sqrt(zf * zf + dx * dx + dy * dy);
        double sk, ck;
        sincos(k * R, &sk, &ck);
        // K = (1/2pi)(z/R)(1/R - ik) e^{ikR}/R, times the quadrature weight
        const double f = w * dphi * zf / (2.0 * M_PI * R * R);
        const double2 K = d_cmul(make_double2(f / R, -f * k), make_double2(ck, sk));
        const double2 ep = make_double2(cs, sn), em = make_double2(cs, -sn);     // e^{+-i phi}
        double2 ux, uy;
        if (comp == 0) {        // u_r terms: cos / sin
            const double2 a = d_cmul(ep, upr[i]);
            const double2 umc = make_double2(umr[i].x, -umr[i].y);
            const double2 b = d_cmul(em, umc);
            ux = make_double2((a.x + b.x) * cs, (a.y + b.y) * cs);
            uy = make_double2((a.x + b.x) * sn, (a.y + b.y) * sn);
        } else {                // u_phi terms: -sin / cos
            const double2 a = d_cmul(ep, upp[i]);
            const double2 umc = make_double2(ump[i].x, -ump[i].y);
            const double2 b = d_cmul(em, umc);
            ux = make_double2(-(a.x + b.x) * sn, -(a.y + b.y) * sn);
            uy = make_double2((a.x + b.x) * cs, (a.y + b.y) * cs);
        }
        const double2 cx = d_cmul(K, ux), cy = d_cmul(K, uy);
        ax.x += cx.x; ax.y += cx.y;
        ay.x += cy.x; ay.y += cy.y;
    }
    const double2 sx = block_sum2(ax);
    __syncthreads();
    const double2 sy = block_sum2(ay);
    if (threadIdx.x == 0) {
        double2 *ox = ex + (size_t)l * npts + pidx, *oy = ey + (size_t)l * npts + pidx;
        ox->x += sx.x; ox->y += sx.y;
        oy->x += sy.x; oy->y += sy.y;
    }
}

void launch_focal_plane(const double2 *umean, const double *rr, const double *wr, const double *rp, const double *wp,
                        int nr, int nl, const double *pts, int pstride, int npts, double zf, const double *kk, int ns,
                        double2 *ex, double2 *ey, cudaStream_t s)
{
    dim3 g(npts, nl);
    k_focal_plane<<<g, 256, 0, s>>>(umean, rr, wr, rp, wp, nr, nl, pts, pstride, npts, zf, kk, ns, ex, ey);
}

__global__ void k_status_check(const float *x, size_t n, int *status)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; t < n; t += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(x[t])) { atomicOr(status, 1); return; }
}
void launch_fill_status_check(const float *x, size_t n, int *status, cudaStream_t s)
{
    k_status_check<<<152, 256, 0, s>>>(x, n, status);
}

}  // namespace zda
