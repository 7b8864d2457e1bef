// Host side of the libzda C ABI (declared in include/zda.h).
//
// The library computes its coefficient tables in FP64 on the host (radii,
// CPML profiles, layer permittivities, source phases, pulse samples, DFT
// twiddles e^{i w t} dt, the broadband adjoint pulse matrix, the
// Rayleigh-Sommerfeld radial weights) and uploads them into the caller's
// workspace; every per-cell and per-step operation runs in the kernels of
// zda_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "zda.h"
#include "zda_internal.h"
#include "zda_step.h"
#include "zda_tile.h"

using cd = std::complex<double>;

static thread_local std::string g_err;

static zda_status fail(zda_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

void zda_internal_set_error(const char *msg) { g_err = msg ? msg : ""; }

#define CUDA_TRY(expr)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ZDA_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));     \
    } while (0)

static_assert(ZDA_DFT_MAXQ == ZDA_MAX_FREQ, "the blocked DFT keeps one accumulator per signed frequency");

struct zda_ctx {
    int device;
};

namespace {

struct Layout {           // byte offsets inside the workspace
    size_t fields, psi_z, psi_r, psi_m, fields2, psi_h2, mon, des_f, des_a, rho_in, rho_bar, rho_t, rb, site_grad, g_t, g_rho,
        norm, src_rad, dft_hist, inv_r_n, inv_r_h, br_n, cr_n, br_h, cr_h, bm_n, cm_n, bm_h, cm_h, bz_n, cz_n, bz_h, cz_h, a_n, d_n, a_c, d_c, ph_n,
        ph_h, pulse, twiddle, adj_time, Gr, Gp, emph_n, emph_h, wt, beta_r, beta_p, g_in, partial, S,
        umean, pt_row, qr, qw, qp, qwp, kk, energy, energy_part, status, total;
};

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct zda_zone {
    zda_ctx *ctx = nullptr;
    zda_zone_desc d{};
    double dt = 0, dphi = 0, tau = 0;
    int nq = 2, nrd = 0, nk = 0, i_d0 = 0, i_d1 = 0, di_max = 0, dj_max = 0;
    std::vector<double> lambda{1.0};
    double f0 = 1.0, sigma = 0.5, t0 = 2.0;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    Layout L{};
    bool tables_dirty = true;
    bool have_forward = false;
    bool adjoint_ok = false;        // the broadband adjoint pulse matrix was invertible
    long long launches = 0;
    // time-step kernel: 0 = split H/E launches (default), 1 = fused single launch
    // streaming along r (bulk-copy ring), 3 = fused single launch on TMA-staged
    // tiles (tile_phi rows x 32 z-cells, streaming over i_ranges radius ranges), 4 = split
    // step with the E half on TMA-staged tiles (tile_phi rows, i_ranges radius ranges), 5 = split
    // step with both halves on those tiles
    int variant = 0, tile_phi = 2, i_ranges = 0;
    zda::TileMaps tmaps[2];         // tensor maps of the two field buffers (variant 3)
    const char *tmaps_ws = nullptr; // the workspace and tile shape they were encoded for
    int tmaps_tj = 0;
    bool kernel_default = true;     // the creation-time choice, not one made by zda_zone_set_kernel
    zda::TileEMaps emaps;           // tensor maps of the field buffer (variants 4, 5)
    const char *emaps_ws = nullptr;
    int emaps_tj = 0;
    zda::TileHMaps hmaps;           // tensor maps of the field buffer for the H half (variant 5)
    const char *hmaps_ws = nullptr;
    int hmaps_tj = 0;
    int wait_limit = 1 << 22, inject_timeout = 0;   // bounded mbarrier waits of the fused step
    bool pair_kernels = true;       // split step: two z-cells per thread where the grid allows
    int rpml = 0;                   // r-PML form (zda_zone_set_radial_pml)
    int last_parity = 0;            // fused runs: which buffer holds the final fields
    int probe_every = 0, probe_n = 0;   // decay probe of forward runs: sampling period, samples of the last run
    // optional CUDA-event timing of every `time_every`-th H/E launch pair
    int time_every = 0;
    std::vector<cudaEvent_t> ev;    // ring of 4 events per sample: launches 1 | 2 | 3 of a step
    std::vector<char> ev_pending;
    int ev_next = 0;
    double t_h_ms = 0, t_e_ms = 0, t_x_ms = 0;
    long long t_count = 0;
    ~zda_zone();
};

static void timing_drain_slot(zda_zone &z, int slot)
{
    if (!z.ev_pending[slot]) return;
    cudaEventSynchronize(z.ev[4 * slot + 3]);
    float a = 0, b = 0, c = 0;
    cudaEventElapsedTime(&a, z.ev[4 * slot], z.ev[4 * slot + 1]);
    cudaEventElapsedTime(&b, z.ev[4 * slot + 1], z.ev[4 * slot + 2]);
    cudaEventElapsedTime(&c, z.ev[4 * slot + 2], z.ev[4 * slot + 3]);
    z.t_h_ms += a;
    z.t_e_ms += b;
    z.t_x_ms += c;
    z.t_count++;
    z.ev_pending[slot] = 0;
}

static void timing_release(zda_zone &z)
{
    for (size_t s = 0; s < z.ev_pending.size(); ++s) timing_drain_slot(z, (int)s);
    for (cudaEvent_t e : z.ev) cudaEventDestroy(e);
    z.ev.clear();
    z.ev_pending.clear();
    z.time_every = 0;
}

zda_zone::~zda_zone() { timing_release(*this); }

// ------------------------------------------------------------------ tables
static double layer_eps_at(const zda_zone_desc &d, int k)
{
    double e = d.layer_eps[0];
    for (int l = 0; l < d.n_layers; ++l)
        if (k >= d.layer_k0[l]) e = d.layer_eps[l];
    return e;
}

// Convolutional PML (kappa = 1): sigma = sigma_max x^3 with
// sigma_max = -4 ln(1e-8) / (2 d), alpha = 0.05 (2 pi f0) (1 - x);
// b = exp(-(sigma + alpha) dt), c = sigma / (sigma + alpha) (b - 1);
// x = depth into the PML / its thickness.
//
// Stretched-radius form of the r-PML (metric != 0; section "Differentiable
// FDTD": the stretched coordinate r~ enters the equations themselves): in
// the outer slab r~ = r + Omega(r) / (alpha_max - i w) with
// Omega = int sigma dr' = sigma_max d x^4 / 4, and s_r takes the same
// constant alpha_max so that dr~/dr = s_r; 1/r~ = (1/r) / (1 + sigma_m /
// (alpha_max - i w)), sigma_m = Omega / r, is the same recursion with
// sigma_m (the `metric` tables).  The inner slab keeps the real radius (a
// stretched inner radius has Im r~ < 0, under which the wedge's
// non-propagating azimuthal orders grow) and its graded alpha.
static void cpml_table(const zda_zone &z, double lo, double hi, int n_in, int n_out, double h,
                       const std::vector<double> &pos, std::vector<float> &b, std::vector<float> &c,
                       int stretched_outer = 0, std::vector<float> *bm = nullptr, std::vector<float> *cm = nullptr)
{
    const double a_max = 0.05 * 2.0 * M_PI * z.f0;
    b.assign(pos.size(), 0.f);
    c.assign(pos.size(), 0.f);
    if (bm) bm->assign(pos.size(), 0.f);
    if (cm) cm->assign(pos.size(), 0.f);
    auto recursion = [&](double sg, double al, float &bo, float &co) {
        const double bb = std::exp(-(sg + al) * z.dt);
        bo = (float)bb;
        co = (float)(sg / (sg + al) * (bb - 1.0));
    };
    for (size_t t = 0; t < pos.size(); ++t) {
        const double x0 = pos[t];
        double x = 0.0, thick = h;
        bool outer = false;
        if (n_in > 0 && x0 < lo + n_in * h) { thick = n_in * h; x = (lo + thick - x0) / thick; }
        if (n_out > 0 && x0 > hi - n_out * h) { thick = n_out * h; x = (x0 - (hi - thick)) / thick; outer = true; }
        x = std::min(std::max(x, 0.0), 1.0);
        if (x <= 0.0) continue;
        const double smax = -4.0 * std::log(1e-8) / (2.0 * thick);
        const double sg = smax * x * x * x;
        if (stretched_outer && outer) {
            recursion(sg, a_max, b[t], c[t]);
            const double sm = smax * thick * x * x * x * x / 4.0 / x0;
            if (bm && cm) recursion(sm, a_max, (*bm)[t], (*cm)[t]);
        } else {
            recursion(sg, a_max * (1.0 - x), b[t], c[t]);
        }
    }
}

// Complex Gauss-Jordan inverse with partial pivoting (n <= ZDA_MAX_FREQ).
static bool invert(std::vector<cd> &A, int n, double tiny)
{
    std::vector<cd> inv(n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::abs(A[r * n + col]) > std::abs(A[piv * n + col])) piv = r;
        if (std::abs(A[piv * n + col]) <= tiny) return false;
        for (int t = 0; t < n; ++t) {
            std::swap(A[col * n + t], A[piv * n + t]);
            std::swap(inv[col * n + t], inv[piv * n + t]);
        }
        const cd p = A[col * n + col];
        for (int t = 0; t < n; ++t) { A[col * n + t] /= p; inv[col * n + t] /= p; }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const cd f = A[r * n + col];
            if (f == 0.0) continue;
            for (int t = 0; t < n; ++t) {
                A[r * n + t] -= f * A[col * n + t];
                inv[r * n + t] -= f * inv[col * n + t];
            }
        }
    }
    A = inv;
    return true;
}

static double omega_q(const zda_zone &z, int q)
{
    const int nl = (int)z.lambda.size();
    const double w = 2.0 * M_PI / z.lambda[q % nl];
    return q < nl ? w : -w;
}

static void compute_layout(zda_zone &z)
{
    const zda_zone_desc &d = z.d;
    const size_t nr = d.n_r, np = d.n_phi, nz = d.n_z, Q = z.nq, T = d.n_steps;
    const size_t ncell = nr * np * nz, plane = nr * np;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + std::max<size_t>(bytes, 1)); return o; };
    Layout &L = z.L;
    L.fields = take(6 * ncell * sizeof(float2));
    L.psi_z = take(4 * plane * 2 * d.pml_z * sizeof(float2));
    L.psi_r = take(4 * (size_t)(d.pml_r_in + d.pml_r_out) * np * nz * sizeof(float2));
    L.psi_m = take(4 * (size_t)(d.pml_r_in + d.pml_r_out) * np * nz * sizeof(float2));   // zeroed with psi_r
    // second field buffer and H-side CPML set for the fused (ping-pong) step
    L.fields2 = take(6 * ncell * sizeof(float2));
    L.psi_h2 = take((2 * plane * 2 * d.pml_z + 2 * (size_t)(d.pml_r_in + d.pml_r_out) * np * nz) * sizeof(float2));
    L.mon = take(Q * 2 * plane * sizeof(float2));
    L.des_f = take(Q * 3 * plane * z.nk * sizeof(float2));
    L.des_a = take(Q * 3 * plane * z.nk * sizeof(float2));
    L.rho_in = take((size_t)z.nrd * np * sizeof(float));
    L.rho_bar = take((size_t)z.nrd * np * sizeof(float));
    L.rho_t = take((size_t)z.nrd * np * sizeof(float));
    L.rb = take(3 * plane * sizeof(float));
    L.site_grad = take(3 * plane * z.nk * sizeof(float));
    L.g_t = take((size_t)z.nrd * np * sizeof(float));
    L.g_rho = take((size_t)z.nrd * np * sizeof(float));
    L.norm = take((size_t)z.nrd * sizeof(float));
    L.src_rad = take(2 * nr * sizeof(float2));
    // history of the time-blocked DFT: design (3 components) + monitor (2) sites per slot
    L.dft_hist = take((size_t)zda::DFT_BLOCK * (3 * plane * z.nk + 2 * plane) * sizeof(float2));
    L.inv_r_n = take((nr + 1) * sizeof(float));
    L.inv_r_h = take(nr * sizeof(float));
    L.br_n = take((nr + 1) * sizeof(float));
    L.cr_n = take((nr + 1) * sizeof(float));
    L.br_h = take(nr * sizeof(float));
    L.cr_h = take(nr * sizeof(float));
    L.bm_n = take((nr + 1) * sizeof(float));
    L.cm_n = take((nr + 1) * sizeof(float));
    L.bm_h = take(nr * sizeof(float));
    L.cm_h = take(nr * sizeof(float));
    L.bz_n = take((nz + 1) * sizeof(float));
    L.cz_n = take((nz + 1) * sizeof(float));
    L.bz_h = take(nz * sizeof(float));
    L.cz_h = take(nz * sizeof(float));
    L.a_n = take(nz * sizeof(float));
    L.d_n = take(nz * sizeof(float));
    L.a_c = take(nz * sizeof(float));
    L.d_c = take(nz * sizeof(float));
    L.ph_n = take(np * sizeof(float2));
    L.ph_h = take(np * sizeof(float2));
    L.pulse = take(T * sizeof(float));
    L.twiddle = take(T * Q * sizeof(float2));
    L.adj_time = take(T * Q * sizeof(float2));
    L.Gr = take(Q * nr * sizeof(double2));
    L.Gp = take(Q * nr * sizeof(double2));
    L.emph_n = take(np * sizeof(double2));
    L.emph_h = take(np * sizeof(double2));
    L.wt = take(Q * sizeof(float));
    L.beta_r = take(Q * nr * sizeof(float2));
    L.beta_p = take(Q * nr * sizeof(float2));
    L.g_in = take(Q * sizeof(double2));
    L.partial = take(Q * nr * sizeof(double2));
    L.S = take(Q * sizeof(double2));
    L.umean = take(Q * 2 * nr * sizeof(double2));
    L.pt_row = take(Q * nr * sizeof(double));
    L.qr = take(nr * sizeof(double));
    L.qw = take(nr * sizeof(double));
    L.qp = take(nr * sizeof(double));
    L.qwp = take(nr * sizeof(double));
    L.kk = take(Q * sizeof(double));
    L.energy = take(2 * T * sizeof(double));            // decay probe: W, Wdot per sample
    L.energy_part = take(2 * nr * sizeof(double));
    L.status = take(sizeof(int) * 4);
    L.total = off;
}

template <class T> static T *P(const zda_zone &z, size_t off) { return (T *)(z.ws + off); }

static zda_status upload(zda_zone &z)
{
    const zda_zone_desc &d = z.d;
    const int nr = d.n_r, np = d.n_phi, nz = d.n_z, Q = z.nq, T = d.n_steps;
    std::vector<float> f;
    auto put = [&](size_t off, const void *src, size_t bytes) -> cudaError_t {
        return cudaMemcpy(z.ws + off, src, bytes, cudaMemcpyHostToDevice);
    };
    // radii
    std::vector<float> irn(nr + 1), irh(nr);
    for (int i = 0; i <= nr; ++i) {
        const double r = d.r_lo + i * d.dr;
        irn[i] = r > 0 ? (float)(1.0 / r) : 0.f;        // axis: the 1/r terms vanish there
    }
    for (int i = 0; i < nr; ++i) irh[i] = (float)(1.0 / (d.r_lo + (i + 0.5) * d.dr));
    CUDA_TRY(put(z.L.inv_r_n, irn.data(), irn.size() * 4));
    CUDA_TRY(put(z.L.inv_r_h, irh.data(), irh.size() * 4));
    // CPML
    {
        std::vector<double> rn(nr + 1), rh(nr), zn(nz + 1), zh(nz);
        for (int i = 0; i <= nr; ++i) rn[i] = d.r_lo + i * d.dr;
        for (int i = 0; i < nr; ++i) rh[i] = d.r_lo + (i + 0.5) * d.dr;
        for (int k = 0; k <= nz; ++k) zn[k] = k * d.dz;
        for (int k = 0; k < nz; ++k) zh[k] = (k + 0.5) * d.dz;
        const double rhi = d.r_lo + nr * d.dr, zhi = nz * d.dz;
        std::vector<float> b, c, bm, cm;
        cpml_table(z, d.r_lo, rhi, d.pml_r_in, d.pml_r_out, d.dr, rn, b, c, z.rpml, &bm, &cm);
        CUDA_TRY(put(z.L.br_n, b.data(), b.size() * 4));
        CUDA_TRY(put(z.L.cr_n, c.data(), c.size() * 4));
        CUDA_TRY(put(z.L.bm_n, bm.data(), bm.size() * 4));
        CUDA_TRY(put(z.L.cm_n, cm.data(), cm.size() * 4));
        cpml_table(z, d.r_lo, rhi, d.pml_r_in, d.pml_r_out, d.dr, rh, b, c, z.rpml, &bm, &cm);
        CUDA_TRY(put(z.L.br_h, b.data(), b.size() * 4));
        CUDA_TRY(put(z.L.cr_h, c.data(), c.size() * 4));
        CUDA_TRY(put(z.L.bm_h, bm.data(), bm.size() * 4));
        CUDA_TRY(put(z.L.cm_h, cm.data(), cm.size() * 4));
        cpml_table(z, 0.0, zhi, d.pml_z, d.pml_z, d.dz, zn, b, c);
        CUDA_TRY(put(z.L.bz_n, b.data(), b.size() * 4));
        CUDA_TRY(put(z.L.cz_n, c.data(), c.size() * 4));
        cpml_table(z, 0.0, zhi, d.pml_z, d.pml_z, d.dz, zh, b, c);
        CUDA_TRY(put(z.L.bz_h, b.data(), b.size() * 4));
        CUDA_TRY(put(z.L.cz_h, c.data(), c.size() * 4));
    }
    // permittivity at node planes (E_r, E_phi: cells k-1, k) and cell planes
    // (E_z: cell k): eps = a + d * (transverse density average)
    {
        const double de = d.eps_hi - d.eps_lo;
        auto design = [&](int k) { return k >= d.design_k0 && k < d.design_k1; };
        auto base = [&](int k) { return design(k) ? d.eps_lo : layer_eps_at(d, k); };
        std::vector<float> an(nz), dn(nz), ac(nz), dc(nz);
        for (int k = 0; k < nz; ++k) {
            const int km = std::max(k - 1, 0);
            an[k] = (float)(0.5 * (base(km) + base(k)));
            dn[k] = (float)(0.5 * de * ((design(km) ? 1 : 0) + (design(k) ? 1 : 0)));
            ac[k] = (float)base(k);
            dc[k] = (float)(design(k) ? de : 0.0);
        }
        CUDA_TRY(put(z.L.a_n, an.data(), nz * 4));
        CUDA_TRY(put(z.L.d_n, dn.data(), nz * 4));
        CUDA_TRY(put(z.L.a_c, ac.data(), nz * 4));
        CUDA_TRY(put(z.L.d_c, dc.data(), nz * 4));
    }
    // phases
    {
        std::vector<float2> pn(np), ph(np);
        std::vector<double2> en(np), eh(np);
        const bool bor = d.n_fold == 0;       // u-form: no azimuthal phase
        for (int j = 0; j < np; ++j) {
            const double a = bor ? 0.0 : d.m * j * z.dphi, b = bor ? 0.0 : d.m * (j + 0.5) * z.dphi;
            pn[j] = make_float2((float)std::cos(a), (float)std::sin(a));
            ph[j] = make_float2((float)std::cos(b), (float)std::sin(b));
            const double pn_ = bor ? 0.0 : j * z.dphi, ph_ = bor ? 0.0 : (j + 0.5) * z.dphi;
            en[j] = make_double2(std::cos(pn_), -std::sin(pn_));
            eh[j] = make_double2(std::cos(ph_), -std::sin(ph_));
        }
        CUDA_TRY(put(z.L.ph_n, pn.data(), np * 8));
        CUDA_TRY(put(z.L.ph_h, ph.data(), np * 8));
        CUDA_TRY(put(z.L.emph_n, en.data(), np * 16));
        CUDA_TRY(put(z.L.emph_h, eh.data(), np * 16));
    }
    // pulse, twiddles, adjoint pulse matrix
    {
        std::vector<float> pl(T);
        for (int n = 0; n < T; ++n) {
            const double u = (n + 0.5) * z.dt - z.t0;
            pl[n] = (float)(std::cos(2 * M_PI * z.f0 * u) * std::exp(-u * u / (2 * z.sigma * z.sigma)));
        }
        CUDA_TRY(put(z.L.pulse, pl.data(), (size_t)T * 4));
        std::vector<float2> tw((size_t)T * Q);
        for (int n = 0; n < T; ++n)
            for (int q = 0; q < Q; ++q) {
                const cd v = std::exp(cd(0, omega_q(z, q) * (n + 1) * z.dt)) * z.dt;
                tw[(size_t)n * Q + q] = make_float2((float)v.real(), (float)v.imag());
            }
        CUDA_TRY(put(z.L.twiddle, tw.data(), tw.size() * 8));
        // Broadband adjoint profiles: zero-mean first differences of
        // e^{+i w_l (t - 6 sigma)} Gaussians (centred at -w_l), combined with
        // the inverse of their discrete DFT matrix at -w_j so the profile of
        // column q has DFT delta_qj at -w_j.
        const double t0a = 6.0 * z.sigma;
        std::vector<cd> g((size_t)T * Q);
        for (int l = 0; l < Q; ++l) {
            auto p = [&](int n) {
                const double u = n * z.dt - t0a;
                return std::exp(cd(0, omega_q(z, l) * u)) * std::exp(-u * u / (2 * z.sigma * z.sigma));
            };
            cd prev = p(0);
            for (int n = 0; n < T; ++n) {
                const cd nx = p(n + 1);
                g[(size_t)n * Q + l] = nx - prev;
                prev = nx;
            }
        }
        std::vector<cd> Gm((size_t)Q * Q, 0.0);     // Gm[l][j] = sum_n g_l[n] e^{-i w_j t_{n+1/2}} dt
        for (int n = 0; n < T; ++n) {
            const double t = (n + 0.5) * z.dt;
            for (int jq = 0; jq < Q; ++jq) {
                const cd e = std::exp(cd(0, -omega_q(z, jq) * t)) * z.dt;
                for (int l = 0; l < Q; ++l) Gm[(size_t)l * Q + jq] += g[(size_t)n * Q + l] * e;
            }
        }
        double gscale = 0.0;
        for (const cd &v : Gm) gscale = std::max(gscale, std::abs(v));
        z.adjoint_ok = gscale > 0 && invert(Gm, Q, 1e-9 * gscale);
        std::vector<float2> at((size_t)T * Q, make_float2(0.f, 0.f));
        if (z.adjoint_ok) {
            for (int n = 0; n < T; ++n)
                for (int q = 0; q < Q; ++q) {
                    cd s = 0.0;
                    for (int l = 0; l < Q; ++l) s += Gm[(size_t)q * Q + l] * g[(size_t)n * Q + l];
                    at[(size_t)n * Q + q] = make_float2((float)s.real(), (float)s.imag());
                }
        }
        CUDA_TRY(put(z.L.adj_time, at.data(), at.size() * 8));
    }
    // Rayleigh-Sommerfeld (first kind) on-axis weights for the m = +1 run:
    // G(r) = (n/2) K(R) r dphi w_quad, K = (1/2pi)(z/R)(1/R - ik) e^{ikR}/R,
    // z = f - (z_monitor - z_design_top), k = 2 pi sqrt(eps_monitor) / lambda;
    // E_r sites: midpoint over the annulus cells, E_phi sites: trapezoid over
    // its nodes, times -i (S = c+ collects u_r - i u_phi); -w entries conjugate.
    {
        const double zf = d.focal - (d.monitor_k * d.dz - d.design_k1 * d.dz);
        const double ntop = std::sqrt(layer_eps_at(d, d.monitor_k));
        std::vector<double2> gr((size_t)Q * nr), gp((size_t)Q * nr);
        std::vector<float> wt(Q);
        for (int q = 0; q < Q; ++q) {
            const double kk = 2 * M_PI * ntop / z.lambda[q % z.lambda.size()];
            auto G = [&](double r) {
                const double R = std::sqrt(zf * zf + r * r);
                const cd K = (1.0 / (2 * M_PI)) * (zf / R) * (1.0 / R - cd(0, kk)) * std::exp(cd(0, kk * R)) / R;
                return 0.5 * (d.n_fold == 0 ? 1 : d.n_fold) * K * r * z.dphi;
            };
            const bool neg = q >= (int)z.lambda.size();
            for (int i = 0; i < nr; ++i) {
                cd a = 0.0, b = 0.0;
                if (i >= z.i_d0 && i < z.i_d1) a = G(d.r_lo + (i + 0.5) * d.dr) * d.dr;
                if (i >= z.i_d0 && i <= z.i_d1) {
                    const double wq = (i == z.i_d0 || i == z.i_d1) ? 0.5 * d.dr : d.dr;
                    b = G(d.r_lo + i * d.dr) * wq;
                }
                if (neg) { a = std::conj(a); b = std::conj(b); }
                b *= cd(0, -1);
                gr[(size_t)q * nr + i] = make_double2(a.real(), a.imag());
                gp[(size_t)q * nr + i] = make_double2(b.real(), b.imag());
            }
            wt[q] = (float)(2.0 * std::sin(omega_q(z, q) * z.dt / 2) / z.dt);
        }
        CUDA_TRY(put(z.L.Gr, gr.data(), gr.size() * 16));
        CUDA_TRY(put(z.L.Gp, gp.data(), gp.size() * 16));
        CUDA_TRY(put(z.L.wt, wt.data(), Q * 4));
        // radial quadrature (r dr) of the focal-plane evaluation: midpoint at
        // the E_r radii, trapezoid at the E_phi radii, over the design annulus
        std::vector<double> qr(nr), qw(nr), qp(nr), qwp(nr), kk(Q);
        for (int i = 0; i < nr; ++i) {
            qr[i] = d.r_lo + (i + 0.5) * d.dr;
            qw[i] = (i >= z.i_d0 && i < z.i_d1) ? qr[i] * d.dr : 0.0;
            qp[i] = d.r_lo + i * d.dr;
            qwp[i] = (i >= z.i_d0 && i <= z.i_d1) ? qp[i] * ((i == z.i_d0 || i == z.i_d1) ? 0.5 * d.dr : d.dr) : 0.0;
        }
        for (int q = 0; q < Q; ++q) kk[q] = 2 * M_PI * ntop / z.lambda[q % z.lambda.size()];
        CUDA_TRY(put(z.L.qr, qr.data(), nr * 8));
        CUDA_TRY(put(z.L.qw, qw.data(), nr * 8));
        CUDA_TRY(put(z.L.qp, qp.data(), nr * 8));
        CUDA_TRY(put(z.L.qwp, qwp.data(), nr * 8));
        CUDA_TRY(put(z.L.kk, kk.data(), Q * 8));
    }
    z.tables_dirty = false;
    return ZDA_OK;
}

static zda_status derive(zda_zone &z)
{
    const zda_zone_desc &d = z.d;
    const bool bor = d.n_fold == 0;
    if (d.n_r < 2 || d.n_phi < 1 || d.n_z < 2 || d.n_fold < 0 || d.dr <= 0 || d.dz <= 0)
        return fail(ZDA_ERR_ARG, "zone needs n_r>=2, n_phi>=1, n_z>=2, n_fold>=0, dr,dz>0");
    if (bor && (d.n_phi != 1 || d.r_lo < 0))
        return fail(ZDA_ERR_ARG, "continuous axisymmetry (n_fold = 0) needs n_phi = 1 and r_lo >= 0");
    if (!bor && d.r_lo <= 0) return fail(ZDA_ERR_ARG, "a wedge zone (n_fold > 0) needs r_lo > 0");
    if (d.r_lo == 0 && d.pml_r_in != 0) return fail(ZDA_ERR_ARG, "the axis zone has no inner r-PML");
    if (d.pml_r_in < 0 || d.pml_r_out < 0 || d.pml_z < 0 || d.pml_r_in + d.pml_r_out >= d.n_r ||
        2 * d.pml_z >= d.n_z)
        return fail(ZDA_ERR_ARG, "PML widths do not fit the grid");
    if (d.n_layers < 1 || d.n_layers > ZDA_MAX_LAYERS) return fail(ZDA_ERR_ARG, "n_layers out of range");
    if (d.design_k0 < 1 || d.design_k1 <= d.design_k0 || d.design_k1 >= d.n_z)
        return fail(ZDA_ERR_ARG, "design layer must satisfy 1 <= design_k0 < design_k1 < n_z");
    if (d.source_k < 1 || d.source_k >= d.n_z || d.monitor_k < 1 || d.monitor_k >= d.n_z)
        return fail(ZDA_ERR_ARG, "source_k / monitor_k outside the grid");
    if (d.n_steps < 1 || d.courant <= 0 || d.courant > 1) return fail(ZDA_ERR_ARG, "bad n_steps / courant");
    if (d.eps_lo <= 0 || d.eps_hi <= 0) return fail(ZDA_ERR_ARG, "permittivities must be positive");
    for (int l = 0; l < d.n_layers; ++l)
        if (d.layer_eps[l] <= 0) return fail(ZDA_ERR_ARG, "layer permittivities must be positive");
    z.tau = 2 * M_PI / (bor ? 1 : d.n_fold);
    z.dphi = z.tau / d.n_phi;
    if (bor) {
        // the i m / r terms act from r_lo (or dr/2 on the axis) outwards
        const double rmin = d.r_lo > 0 ? d.r_lo : 0.5 * d.dr;
        z.dt = d.courant / std::sqrt(1.0 / (d.dr * d.dr) + std::pow(d.m / rmin, 2) + 1.0 / (d.dz * d.dz));
    } else {
        z.dt = d.courant / std::sqrt(1.0 / (d.dr * d.dr) + 1.0 / std::pow(d.r_lo * z.dphi, 2) + 1.0 / (d.dz * d.dz));
    }
    z.nq = 2 * (int)z.lambda.size();
    z.i_d0 = d.pml_r_in;
    z.i_d1 = d.n_r - d.pml_r_out;
    z.nrd = z.i_d1 - z.i_d0;
    z.nk = d.design_k1 - d.design_k0 + 1;
    if (d.filter_radius > 0) {
        // taps past the design rows are dropped, so di_max never needs to exceed n_r_design - 1;
        // the tap count is capped (a radius of many cells would make the filter kernel run for ages)
        const double rc0 = d.r_lo + (z.i_d0 + 0.5) * d.dr;
        const double di = std::floor(d.filter_radius / d.dr), dj = std::floor(d.filter_radius / (rc0 * z.dphi));
        const double taps = (2 * std::min(di, (double)(z.nrd - 1)) + 1) * (2 * dj + 1);
        if (!(taps <= ZDA_MAX_FILTER_TAPS))
            return fail(ZDA_ERR_ARG, "filter_radius spans " + std::to_string(taps) + " taps per pixel (limit " +
                                         std::to_string(ZDA_MAX_FILTER_TAPS) + ")");
        z.di_max = (int)std::min(di, (double)(z.nrd - 1));
        z.dj_max = (int)dj;
    } else {
        z.di_max = z.dj_max = 0;
    }
    if (z.variant == 1 && (d.n_z > zda::fused_max_nz() || bor)) z.variant = 0;
    if ((z.variant == 3 || z.variant == 4 || z.variant == 5) && (bor || d.n_z % 2 || d.pml_z % 2)) z.variant = 0;
    compute_layout(z);
    z.tables_dirty = true;
    z.have_forward = false;
    return ZDA_OK;
}

static zda_status ready(zda_zone *z)
{
    if (!z) return fail(ZDA_ERR_ARG, "null zone");
    if (!z->ws) return fail(ZDA_ERR_STATE, "no workspace bound");
    if (z->ws_bytes < z->L.total) return fail(ZDA_ERR_OOM, "workspace smaller than zda_zone_workspace_bytes");
    CUDA_TRY(cudaSetDevice(z->ctx->device));
    if (z->tables_dirty) return upload(*z);
    return ZDA_OK;
}

static zda::StepParams step_params(zda_zone &z)
{
    using namespace zda;
    const zda_zone_desc &d = z.d;
    const size_t ncell = (size_t)d.n_r * d.n_phi * d.n_z;
    StepParams p{};
    p.nr = d.n_r; p.nphi = d.n_phi; p.nz = d.n_z;
    p.pr_in = d.pml_r_in; p.pr_out = d.pml_r_out; p.pz = d.pml_z;
    p.bor = d.n_fold == 0 ? 1 : 0;
    p.rpml_metric = z.rpml;
    p.m = (float)d.m;
    p.dt = (float)z.dt;
    p.inv_dr = (float)(1.0 / d.dr); p.inv_dz = (float)(1.0 / d.dz); p.inv_dphi = (float)(1.0 / z.dphi);
    const double ph = d.m * z.tau;
    p.bloch = make_float2((float)std::cos(ph), (float)std::sin(ph));
    p.bloch_inv = make_float2((float)std::cos(ph), (float)-std::sin(ph));
    float2 *F = P<float2>(z, z.L.fields);
    p.f = Fields{F, F + ncell, F + 2 * ncell, F + 3 * ncell, F + 4 * ncell, F + 5 * ncell};
    const size_t nzs = (size_t)d.n_r * d.n_phi * 2 * d.pml_z;
    float2 *Z = P<float2>(z, z.L.psi_z);
    const size_t nrs = (size_t)(d.pml_r_in + d.pml_r_out) * d.n_phi * d.n_z;
    float2 *R = P<float2>(z, z.L.psi_r);
    p.psi = Psi{Z, Z + nzs, R, R + nrs, Z + 2 * nzs, Z + 3 * nzs, R + 2 * nrs, R + 3 * nrs};
    float2 *M = P<float2>(z, z.L.psi_m);
    p.rm = Metric{P<float>(z, z.L.bm_n), P<float>(z, z.L.cm_n), P<float>(z, z.L.bm_h), P<float>(z, z.L.cm_h),
                  M, M + nrs, M + 2 * nrs, M + 3 * nrs};
    p.t = Tables{P<float>(z, z.L.inv_r_n), P<float>(z, z.L.inv_r_h), P<float>(z, z.L.br_n),
                 P<float>(z, z.L.cr_n), P<float>(z, z.L.br_h), P<float>(z, z.L.cr_h), P<float>(z, z.L.bz_n),
                 P<float>(z, z.L.cz_n), P<float>(z, z.L.bz_h), P<float>(z, z.L.cz_h), P<float>(z, z.L.a_n),
                 P<float>(z, z.L.d_n), P<float>(z, z.L.a_c), P<float>(z, z.L.d_c), P<float2>(z, z.L.ph_n),
                 P<float2>(z, z.L.ph_h), P<float>(z, z.L.pulse), P<float2>(z, z.L.twiddle),
                 P<float2>(z, z.L.adj_time)};
    const size_t plane = (size_t)d.n_r * d.n_phi;
    float *rb = P<float>(z, z.L.rb);
    p.rb_r = rb; p.rb_p = rb + plane; p.rb_z = rb + 2 * plane;
    p.beta_r = P<float2>(z, z.L.beta_r);
    p.beta_p = P<float2>(z, z.L.beta_p);
    p.src_rad = P<float2>(z, z.L.src_rad);
    p.dft_hist = P<float2>(z, z.L.dft_hist);
    p.nq = z.nq;
    p.src_scale = (float)(0.5 / d.dz);
    p.des_k0 = d.design_k0;
    p.des_nk = z.nk;
    // default block: 16 phi rows, or 4 for zones of at most 16 phi cells (longer z-runs per block;
    // measured 5-25 % faster on the 8-16-cell zones of the paper's lenses)
    p.pair_rows = (z.variant < 4 && zda::pair_rows_ok(z.tile_phi)) ? z.tile_phi : (d.n_phi <= 16 ? 4 : 16);
    p.e_blocks = (z.variant == 0 && z.i_ranges == 3) ? 3 : 2;
    return p;
}

static zda::FilterParams filter_params(const zda_zone &z)
{
    zda::FilterParams fp{};
    const zda_zone_desc &d = z.d;
    fp.nrd = z.nrd; fp.nphi = d.n_phi; fp.di_max = z.di_max; fp.dj_max = z.dj_max;
    fp.dr = (float)d.dr; fp.dphi = (float)z.dphi; fp.R = (float)d.filter_radius;
    fp.r_c0 = (float)(d.r_lo + (z.i_d0 + 0.5) * d.dr);
    fp.beta = (float)d.beta; fp.eta = (float)d.eta;
    fp.filter_on = d.filter_radius > 0 ? 1 : 0;
    return fp;
}

// rho (device, design grid) -> rho_bar, rho_t, rb_* in the workspace
static zda_status run_filter(zda_zone &z, const float *rho_dev, cudaStream_t s)
{
    const zda::FilterParams fp = filter_params(z);
    float *norm = P<float>(z, z.L.norm);
    if (fp.filter_on) { zda::launch_filter_norm(fp, norm, s); z.launches++; }
    zda::launch_filter_project(fp, rho_dev, norm, P<float>(z, z.L.rho_bar), P<float>(z, z.L.rho_t), s);
    const size_t plane = (size_t)z.d.n_r * z.d.n_phi;
    float *rb = P<float>(z, z.L.rb);
    zda::launch_rho_bar(P<float>(z, z.L.rho_t), z.d.n_r, z.d.n_phi, z.i_d0, z.i_d1, rb, rb + plane,
                        rb + 2 * plane, s);
    z.launches += 2;
    CUDA_TRY(cudaGetLastError());
    return ZDA_OK;
}

static zda_status clear_state(zda_zone &z, cudaStream_t s)
{
    CUDA_TRY(cudaMemsetAsync(P<int>(z, z.L.status) + 1, 0, sizeof(int), s));         // wait-timeout word
    CUDA_TRY(cudaMemsetAsync(z.ws + z.L.fields, 0, z.L.psi_r - z.L.fields, s));      // fields, psi_z
    CUDA_TRY(cudaMemsetAsync(z.ws + z.L.psi_r, 0, z.L.fields2 - z.L.psi_r, s));      // psi_r, psi_m
    if (z.variant == 1 || z.variant == 3) {                                           // fields2, psi_h2
        CUDA_TRY(cudaMemsetAsync(z.ws + z.L.fields2, 0, z.L.mon - z.L.fields2, s));
    }
    return ZDA_OK;
}

static int auto_i_ranges(const zda_zone &z)
{
    if (z.i_ranges > 0) return std::min(z.i_ranges, z.d.n_r);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = std::max(1, zda::fused_blocks_per_sm(z.tile_phi, z.d.n_z, z.d.pml_z));
    const int jt = (z.d.n_phi + z.tile_phi - 1) / z.tile_phi;
    // as many radius ranges as fit in one wave (all CTAs co-resident, so the
    // phi-halo rows of neighbouring tiles are read while still in L2), at
    // least 8 radii per range
    int ir = std::max(1, (sms * per_sm) / std::max(jt, 1));
    ir = std::min(ir, std::max(1, z.d.n_r / 8));
    return ir;
}

static zda::FusedParams fused_params(zda_zone &z, const zda::StepParams &p, int parity)
{
    using namespace zda;
    const zda_zone_desc &d = z.d;
    const size_t ncell = (size_t)d.n_r * d.n_phi * d.n_z;
    float2 *A = P<float2>(z, z.L.fields), *B = P<float2>(z, z.L.fields2);
    float2 *src = parity ? B : A, *dst = parity ? A : B;
    const size_t nzs = (size_t)d.n_r * d.n_phi * 2 * d.pml_z;
    const size_t nrs = (size_t)(d.pml_r_in + d.pml_r_out) * d.n_phi * d.n_z;
    float2 *H1 = P<float2>(z, z.L.psi_h2);
    // H-side CPML sets: set 0 = (psi_z[0..1], psi_r[0..1]) of the split layout, set 1 = psi_h2
    float2 *s0[4] = {p.psi.hr_z, p.psi.hp_z, p.psi.hp_r, p.psi.hz_r};
    float2 *s1[4] = {H1, H1 + nzs, H1 + 2 * nzs, H1 + 2 * nzs + nrs};
    float2 **rd = parity ? s1 : s0, **wr = parity ? s0 : s1;
    FusedParams f{};
    f.nr = d.n_r; f.nphi = d.n_phi; f.nz = d.n_z; f.nzs = d.n_z;
    f.pr_in = d.pml_r_in; f.pr_out = d.pml_r_out; f.pz = d.pml_z;
    f.tj = z.tile_phi;
    const int nir = auto_i_ranges(z);
    f.i_range = (d.n_r + nir - 1) / nir;
    f.dt = p.dt; f.inv_dr = p.inv_dr; f.inv_dz = p.inv_dz; f.inv_dphi = p.inv_dphi;
    f.bloch = p.bloch; f.bloch_inv = p.bloch_inv;
    f.Er = src; f.Ep = src + ncell; f.Ez = src + 2 * ncell;
    f.Hr = src + 3 * ncell; f.Hp = src + 4 * ncell; f.Hz = src + 5 * ncell;
    f.oEr = dst; f.oEp = dst + ncell; f.oEz = dst + 2 * ncell;
    f.oHr = dst + 3 * ncell; f.oHp = dst + 4 * ncell; f.oHz = dst + 5 * ncell;
    f.psH_hr_z = rd[0]; f.psH_hp_z = rd[1]; f.psH_hp_r = rd[2]; f.psH_hz_r = rd[3];
    f.opsH_hr_z = wr[0]; f.opsH_hp_z = wr[1]; f.opsH_hp_r = wr[2]; f.opsH_hz_r = wr[3];
    f.psE_er_z = p.psi.er_z; f.psE_ep_z = p.psi.ep_z; f.psE_ep_r = p.psi.ep_r; f.psE_ez_r = p.psi.ez_r;
    f.t = p.t;
    f.rb_r = p.rb_r; f.rb_p = p.rb_p; f.rb_z = p.rb_z;
    f.src_mode = p.src_mode; f.src_k = p.src_k; f.src_scale = p.src_scale;
    f.beta_r = p.beta_r; f.beta_p = p.beta_p;
    f.nq = p.nq;
    f.mon_k = p.mon_k; f.mon = p.mon;
    f.des_k0 = p.des_k0; f.des_nk = p.des_nk; f.des = p.des;
    f.src_rad = P<float2>(z, z.L.src_rad);
    f.err = P<int>(z, z.L.status) + 1;
    f.wait_limit = z.wait_limit;
    f.inject_timeout = z.inject_timeout;
    return f;
}

// decay probe (forward runs): after step n with (n + 1) % every == 0, the field
// energy of the state and of its one-step difference into sample n / every
static bool probe_due(const zda_zone &z, const zda::StepParams &p, int n)
{
    return z.probe_every > 0 && p.src_mode == zda::SRC_PLANE_WAVE && (n + 1) % z.probe_every == 0;
}

static zda::Fields fields_at(zda_zone &z, size_t off)
{
    const size_t ncell = (size_t)z.d.n_r * z.d.n_phi * z.d.n_z;
    float2 *F = P<float2>(z, off);
    return zda::Fields{F, F + ncell, F + 2 * ncell, F + 3 * ncell, F + 4 * ncell, F + 5 * ncell};
}

static void probe_sample(zda_zone &z, const zda::StepParams &p, int n, size_t cur_off, size_t prev_off,
                         cudaStream_t s)
{
    double *e = P<double>(z, z.L.energy);
    const int slot = n / z.probe_every;
    zda::launch_field_energy(p, fields_at(z, cur_off), fields_at(z, prev_off), z.d.r_lo, z.d.dr, z.dphi * z.d.dz,
                             P<double>(z, z.L.energy_part), e + 2 * slot, e + 2 * slot + 1, s);
    z.launches += 2;
}

static zda::TileParams tile_params(zda_zone &z, const zda::StepParams &p, int parity)
{
    using namespace zda;
    const zda_zone_desc &d = z.d;
    const size_t ncell = (size_t)d.n_r * d.n_phi * d.n_z;
    float2 *dst = parity ? P<float2>(z, z.L.fields) : P<float2>(z, z.L.fields2);
    const size_t nzs = (size_t)d.n_r * d.n_phi * 2 * d.pml_z;
    const size_t nrs = (size_t)(d.pml_r_in + d.pml_r_out) * d.n_phi * d.n_z;
    float2 *H1 = P<float2>(z, z.L.psi_h2);
    float2 *s0[4] = {p.psi.hr_z, p.psi.hp_z, p.psi.hp_r, p.psi.hz_r};
    float2 *s1[4] = {H1, H1 + nzs, H1 + 2 * nzs, H1 + 2 * nzs + nrs};
    float2 **rd = parity ? s1 : s0, **wr = parity ? s0 : s1;
    TileParams t{};
    t.p = p;
    for (int c = 0; c < 3; ++c) {
        t.oE[c] = dst + c * ncell;
        t.oH[c] = dst + (3 + c) * ncell;
    }
    for (int c = 0; c < 4; ++c) {
        t.psH_in[c] = rd[c];
        t.psH_out[c] = wr[c];
    }
    t.err = P<int>(z, z.L.status) + 1;
    t.wait_limit = z.wait_limit;
    t.inject_timeout = z.inject_timeout;
    return t;
}

// tensor maps of both field buffers for the tile step (encoded on the host;
// re-encoded when the workspace or the tile shape changes)
static zda_status tile_maps(zda_zone &z)
{
    if (z.tmaps_ws == z.ws && z.tmaps_tj == z.tile_phi) return ZDA_OK;
    const zda_zone_desc &d = z.d;
    const size_t ncell = (size_t)d.n_r * d.n_phi * d.n_z;
    for (int b = 0; b < 2; ++b) {
        float2 *F = b ? P<float2>(z, z.L.fields2) : P<float2>(z, z.L.fields);
        float2 *E[3] = {F, F + ncell, F + 2 * ncell}, *H[3] = {F + 3 * ncell, F + 4 * ncell, F + 5 * ncell};
        const char *why = "";
        if (!zda::encode_tile_maps(&z.tmaps[b], E, H, d.n_r, d.n_phi, d.n_z, z.tile_phi, &why))
            return fail(ZDA_ERR_CUDA, std::string("tile step: ") + why);
    }
    z.tmaps_ws = z.ws;
    z.tmaps_tj = z.tile_phi;
    return ZDA_OK;
}

static int tile_rchunks(const zda_zone &z)
{
    if (z.i_ranges > 0) return std::min(z.i_ranges, z.d.n_r);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return zda::tile_auto_rchunks(z.tile_phi, z.d.n_r, z.d.n_phi, z.d.n_z, sms);
}

// tensor maps of the field buffer for the E tile kernel (variant 4)
static zda_status tile_e_maps(zda_zone &z)
{
    if (z.emaps_ws == z.ws && z.emaps_tj == z.tile_phi) return ZDA_OK;
    const zda_zone_desc &d = z.d;
    const size_t ncell = (size_t)d.n_r * d.n_phi * d.n_z;
    float2 *F = P<float2>(z, z.L.fields);
    float2 *E[3] = {F, F + ncell, F + 2 * ncell}, *H[3] = {F + 3 * ncell, F + 4 * ncell, F + 5 * ncell};
    const char *why = "";
    if (!zda::encode_tile_e_maps(&z.emaps, E, H, d.n_r, d.n_phi, d.n_z, z.tile_phi, &why))
        return fail(ZDA_ERR_CUDA, std::string("E tile kernel: ") + why);
    z.emaps_ws = z.ws;
    z.emaps_tj = z.tile_phi;
    return ZDA_OK;
}

static int tile_e_rchunks(const zda_zone &z)
{
    if (z.i_ranges > 0) return std::min(z.i_ranges, z.d.n_r);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return zda::tile_e_auto_rchunks(z.tile_phi, z.d.n_r, z.d.n_phi, z.d.n_z, sms);
}

// tensor maps of the field buffer for the H tile kernel (variant 5)
static zda_status tile_h_maps(zda_zone &z)
{
    if (z.hmaps_ws == z.ws && z.hmaps_tj == z.tile_phi) return ZDA_OK;
    const zda_zone_desc &d = z.d;
    const size_t ncell = (size_t)d.n_r * d.n_phi * d.n_z;
    float2 *F = P<float2>(z, z.L.fields);
    float2 *E[3] = {F, F + ncell, F + 2 * ncell}, *H[3] = {F + 3 * ncell, F + 4 * ncell, F + 5 * ncell};
    const char *why = "";
    if (!zda::encode_tile_h_maps(&z.hmaps, E, H, d.n_r, d.n_phi, d.n_z, z.tile_phi, &why))
        return fail(ZDA_ERR_CUDA, std::string("H tile kernel: ") + why);
    z.hmaps_ws = z.ws;
    z.hmaps_tj = z.tile_phi;
    return ZDA_OK;
}

// kernels with bounded device-side waits report a timeout through the error word
static bool uses_waits(const zda_zone &z) { return z.variant == 1 || z.variant >= 3; }

static zda_status time_loop(zda_zone &z, zda::StepParams &p, cudaStream_t s)
{
    const int R = (int)z.ev_pending.size();
    if (z.variant == 3) {
        zda_status st = tile_maps(z);
        if (st) return st;
        const bool dft = p.des || p.mon;
        p.dft_ne = zda::dft_entries(p);
        const zda::TileParams tp[2] = {tile_params(z, p, 0), tile_params(z, p, 1)};
        const int nrc = tile_rchunks(z);
        const bool adj = p.src_mode == zda::SRC_ADJOINT;
        // timed samples: [tile step] between events 0 and 1, [DFT flush] between 2 and 3
        for (int n = 0; n < z.d.n_steps; ++n) {
            const bool timed = z.time_every > 0 && R > 0 && (n % z.time_every) == z.time_every - 1;
            int slot = 0;
            if (adj) zda::launch_adjoint_source_rad(p, n, s);
            if (timed) {
                slot = z.ev_next;
                z.ev_next = (z.ev_next + 1) % R;
                timing_drain_slot(z, slot);
                CUDA_TRY(cudaEventRecord(z.ev[4 * slot], s));
            }
            cudaError_t e = zda::launch_tile_step(z.tmaps[n & 1], tp[n & 1], n, z.tile_phi, nrc, s);
            if (e != cudaSuccess) return fail(ZDA_ERR_CUDA, std::string("tile step: ") + cudaGetErrorString(e));
            if (probe_due(z, p, n))
                probe_sample(z, p, n, (n & 1) ? z.L.fields : z.L.fields2, (n & 1) ? z.L.fields2 : z.L.fields, s);
            if (timed) {
                CUDA_TRY(cudaEventRecord(z.ev[4 * slot + 1], s));
                CUDA_TRY(cudaEventRecord(z.ev[4 * slot + 2], s));
            }
            if (dft && zda::dft_flush_due(p, n, z.d.n_steps)) {
                zda::launch_dft_flush(p, n, s);
                ++z.launches;
            }
            if (timed) {
                CUDA_TRY(cudaEventRecord(z.ev[4 * slot + 3], s));
                z.ev_pending[slot] = 1;
            }
        }
        z.last_parity = z.d.n_steps & 1;
        z.launches += (long long)z.d.n_steps * (adj ? 2 : 1);
        CUDA_TRY(cudaGetLastError());
        return ZDA_OK;
    }
    if (z.variant == 1) {
        zda::FusedParams f[2] = {fused_params(z, p, 0), fused_params(z, p, 1)};
        // timed samples: [stream kernel] between events 0 and 1, [DFT kernel] between 1 and 2
        for (int n = 0; n < z.d.n_steps; ++n) {
            const bool timed = z.time_every > 0 && R > 0 && (n % z.time_every) == z.time_every - 1;
            int slot = 0;
            const zda::FusedParams &fp = f[n & 1];
            cudaError_t e = zda::launch_fused_pre(fp, n, s);
            if (e != cudaSuccess) return fail(ZDA_ERR_CUDA, std::string("adjoint source step: ") + cudaGetErrorString(e));
            if (timed) {
                slot = z.ev_next;
                z.ev_next = (z.ev_next + 1) % R;
                timing_drain_slot(z, slot);
                CUDA_TRY(cudaEventRecord(z.ev[4 * slot], s));
            }
            e = zda::launch_fused_stream(fp, n, s);
            if (e != cudaSuccess) return fail(ZDA_ERR_CUDA, std::string("fused step: ") + cudaGetErrorString(e));
            if (probe_due(z, p, n))
                probe_sample(z, p, n, (n & 1) ? z.L.fields : z.L.fields2, (n & 1) ? z.L.fields2 : z.L.fields, s);
            if (timed) {
                CUDA_TRY(cudaEventRecord(z.ev[4 * slot + 1], s));
                CUDA_TRY(cudaEventRecord(z.ev[4 * slot + 2], s));
            }
            e = zda::launch_fused_post(fp, n, s);
            if (e != cudaSuccess) return fail(ZDA_ERR_CUDA, std::string("DFT step: ") + cudaGetErrorString(e));
            if (timed) {
                CUDA_TRY(cudaEventRecord(z.ev[4 * slot + 3], s));
                z.ev_pending[slot] = 1;
            }
        }
        z.last_parity = z.d.n_steps & 1;
        z.launches += (long long)z.d.n_steps * zda::fused_launches_per_step(f[0]);
        return ZDA_OK;
    }
    z.last_parity = 0;
    const bool pair = z.pair_kernels && zda::pair_kernels_apply(p);
    const bool dft = pair && (p.des || p.mon);
    p.dft_ne = zda::dft_entries(p);
    if (!pair) p.dft_hist = nullptr;
    const bool etile = pair && (z.variant == 4 || z.variant == 5), htile = pair && z.variant == 5;
    zda::TileParams etp{};
    int enrc = 1;
    if (etile) {
        zda_status st = tile_e_maps(z);
        if (st) return st;
        const size_t ncell = (size_t)z.d.n_r * z.d.n_phi * z.d.n_z;
        float2 *F = P<float2>(z, z.L.fields);
        if (htile) {
            st = tile_h_maps(z);
            if (st) return st;
        }
        etp.p = p;
        for (int c = 0; c < 3; ++c) {
            etp.oE[c] = F + c * ncell;
            etp.oH[c] = F + (3 + c) * ncell;
        }
        etp.err = P<int>(z, z.L.status) + 1;
        etp.wait_limit = z.wait_limit;
        etp.inject_timeout = z.inject_timeout;
        enrc = tile_e_rchunks(z);
    }
    for (int n = 0; n < z.d.n_steps; ++n) {
        const bool timed = z.time_every > 0 && R > 0 && (n % z.time_every) == z.time_every - 1;
        int slot = 0;
        if (pair && p.src_mode == zda::SRC_ADJOINT) zda::launch_adjoint_source_rad(p, n, s);
        if (timed) {
            slot = z.ev_next;
            z.ev_next = (z.ev_next + 1) % R;
            timing_drain_slot(z, slot);
            CUDA_TRY(cudaEventRecord(z.ev[4 * slot], s));
        }
        if (probe_due(z, p, n))                       // the state before this step, for the difference
            CUDA_TRY(cudaMemcpyAsync(z.ws + z.L.fields2, z.ws + z.L.fields,
                                     6 * (size_t)z.d.n_r * z.d.n_phi * z.d.n_z * sizeof(float2),
                                     cudaMemcpyDeviceToDevice, s));
        if (htile) {
            cudaError_t e = zda::launch_tile_h(z.hmaps, etp, z.tile_phi, enrc, s);
            if (e != cudaSuccess) return fail(ZDA_ERR_CUDA, std::string("H tile kernel: ") + cudaGetErrorString(e));
        } else if (pair) {
            zda::launch_update_h_pair(p, s);
        } else {
            zda::launch_update_h(p, s);
        }
        if (timed) CUDA_TRY(cudaEventRecord(z.ev[4 * slot + 1], s));
        if (etile) {
            cudaError_t e = zda::launch_tile_e(z.emaps, etp, n, z.tile_phi, enrc, s);
            if (e != cudaSuccess) return fail(ZDA_ERR_CUDA, std::string("E tile kernel: ") + cudaGetErrorString(e));
        } else if (pair) {
            zda::launch_update_e_pair(p, n, s);
        } else {
            zda::launch_update_e(p, n, s);
        }
        if (probe_due(z, p, n)) probe_sample(z, p, n, z.L.fields, z.L.fields2, s);
        if (timed) CUDA_TRY(cudaEventRecord(z.ev[4 * slot + 2], s));
        if (dft && zda::dft_flush_due(p, n, z.d.n_steps)) {
            zda::launch_dft_flush(p, n, s);
            ++z.launches;
        }
        if (timed) {
            CUDA_TRY(cudaEventRecord(z.ev[4 * slot + 3], s));
            z.ev_pending[slot] = 1;
        }
    }
    if (pair) z.launches += (long long)z.d.n_steps * (p.src_mode == zda::SRC_ADJOINT ? 1 : 0);
    z.launches += 2LL * z.d.n_steps;
    CUDA_TRY(cudaGetLastError());
    return ZDA_OK;
}

static zda_status check_wait_status(zda_zone &z, cudaStream_t s)
{
    int e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, P<int>(z, z.L.status) + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (e) return fail(ZDA_ERR_TIMEOUT, "a bounded device-side wait of the fused step gave up");
    return ZDA_OK;
}

// focal kernels: S (workspace) and the non-finite flag (status[0])
static zda_status focal_enqueue(zda_zone &z, const float2 *mon, cudaStream_t s)
{
    int *status = P<int>(z, z.L.status);
    CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    zda::launch_focal_partial(mon, P<double2>(z, z.L.Gr), P<double2>(z, z.L.Gp), P<double2>(z, z.L.emph_n),
                              P<double2>(z, z.L.emph_h), z.nq, z.d.n_r, z.d.n_phi, P<double2>(z, z.L.partial), s);
    zda::launch_focal_sum(P<double2>(z, z.L.partial), z.nq, z.d.n_r, P<double2>(z, z.L.S), status, s);
    z.launches += 2;
    CUDA_TRY(cudaGetLastError());
    return ZDA_OK;
}

static zda_status focal_finish(zda_zone &z, double *out_host, cudaStream_t s)
{
    int st = 0;
    if (out_host)
        CUDA_TRY(cudaMemcpyAsync(out_host, z.ws + z.L.S, z.nq * sizeof(double2), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&st, P<int>(z, z.L.status), sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (st) return fail(ZDA_ERR_NONFINITE, "non-finite focal phasor (the time loop diverged)");
    return ZDA_OK;
}

static zda_status focal(zda_zone &z, const float2 *mon, double *out_host, cudaStream_t s)
{
    zda_status st = focal_enqueue(z, mon, s);
    if (st) return st;
    return focal_finish(z, out_host, s);
}

// Everything of a forward run that is enqueued on the stream (no host sync):
// filter + projection, cleared state, the time loop with DFTs, focal kernels.
static zda_status forward_enqueue(zda_zone &z, const float *rho, cudaStream_t s)
{
    z.have_forward = false;
    zda_status st = run_filter(z, rho, s);
    if (st) return st;
    st = clear_state(z, s);
    if (st) return st;
    const size_t plane = (size_t)z.d.n_r * z.d.n_phi;
    CUDA_TRY(cudaMemsetAsync(z.ws + z.L.mon, 0, z.nq * 2 * plane * sizeof(float2), s));
    CUDA_TRY(cudaMemsetAsync(z.ws + z.L.des_f, 0, z.nq * 3 * plane * z.nk * sizeof(float2), s));
    zda::StepParams p = step_params(z);
    p.src_mode = zda::SRC_PLANE_WAVE;
    p.src_k = z.d.source_k;
    p.mon_k = z.d.monitor_k;
    p.mon = P<float2>(z, z.L.mon);
    p.des = P<float2>(z, z.L.des_f);
    st = time_loop(z, p, s);
    if (st) return st;
    z.probe_n = z.probe_every > 0 ? z.d.n_steps / z.probe_every : 0;
    return focal_enqueue(z, P<float2>(z, z.L.mon), s);
}

// Everything of an adjoint run that is enqueued (dI/dS already in g_in):
// adjoint profiles, the adjoint time loop, overlap, transposed chain.
static zda_status adjoint_enqueue(zda_zone &z, float *grad_rho, cudaStream_t s)
{
    const zda_zone_desc &d = z.d;
    const size_t plane = (size_t)d.n_r * d.n_phi;
    const double vol = d.dr * z.dphi * d.dz;
    zda::launch_adjoint_profiles(P<double2>(z, z.L.g_in), P<double2>(z, z.L.Gr), P<double2>(z, z.L.Gp),
                                 P<float>(z, z.L.wt), z.nq, d.n_r, d.r_lo, d.dr, vol, P<float2>(z, z.L.beta_r),
                                 P<float2>(z, z.L.beta_p), s);
    z.launches++;
    zda_status st = clear_state(z, s);
    if (st) return st;
    CUDA_TRY(cudaMemsetAsync(z.ws + z.L.des_a, 0, z.nq * 3 * plane * z.nk * sizeof(float2), s));
    zda::StepParams p = step_params(z);
    p.src_mode = zda::SRC_ADJOINT;
    p.src_k = d.monitor_k;
    p.mon_k = -1;
    p.mon = nullptr;
    p.des = P<float2>(z, z.L.des_a);
    st = time_loop(z, p, s);
    if (st) return st;
    zda::launch_site_gradient(P<float2>(z, z.L.des_f), P<float2>(z, z.L.des_a), P<float>(z, z.L.wt), z.nq,
                              d.n_r, d.n_phi, z.nk, d.r_lo, d.dr, vol, P<float>(z, z.L.site_grad), s);
    zda::launch_cell_gradient(P<float>(z, z.L.site_grad), d.n_r, d.n_phi, z.nk, z.i_d0, z.nrd,
                              (float)(d.eps_hi - d.eps_lo), P<float>(z, z.L.g_t), s);
    const zda::FilterParams fp = filter_params(z);
    zda::launch_filter_project_backward(fp, P<float>(z, z.L.rho_bar), P<float>(z, z.L.norm),
                                        P<float>(z, z.L.g_t), grad_rho, s);
    z.launches += 3;
    CUDA_TRY(cudaGetLastError());
    return ZDA_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

const char *zda_last_error(void) { return g_err.c_str(); }

zda_status zda_ctx_create(zda_ctx **out, int device)
{
    if (!out) return fail(ZDA_ERR_ARG, "null out");
    int n = 0;
    CUDA_TRY(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(ZDA_ERR_ARG, "device index out of range");
    CUDA_TRY(cudaSetDevice(device));
    *out = new zda_ctx{device};
    return ZDA_OK;
}

void zda_ctx_destroy(zda_ctx *ctx) { delete ctx; }

zda_status zda_zone_create(zda_ctx *ctx, const zda_zone_desc *desc, zda_zone **out)
{
    if (!ctx || !desc || !out) return fail(ZDA_ERR_ARG, "null argument");
    zda_zone *z = new zda_zone();
    z->ctx = ctx;
    z->d = *desc;
    // default step: split H update + E update on TMA tiles of 16 phi rows where the zone allows
    // (annular, even n_z and z-PML) and is large enough for them: at least four waves of thread
    // blocks (2 per SM) in radius ranges of about 21 radii.  Measured on GB300: 8 % faster per step
    // than the thread-per-pair E update on the 300 x 320 x 160 wide zone; slower on zones of 16 or
    // fewer phi cells and on the 200-phi-cell zones of the 40-zone lens, where the ranges get short.
    if (desc->n_fold > 0 && desc->n_z % 2 == 0 && desc->pml_z % 2 == 0) {
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            sms = 152;
        }
        const long long tiles = (long long)((desc->n_z + 31) / 32) * ((desc->n_phi + 15) / 16);
        if (tiles * (desc->n_r / 21) >= 8LL * sms) {
            z->variant = 4;
            z->tile_phi = 16;
        }
    }
    zda_status st = derive(*z);
    if (st != ZDA_OK) { delete z; return st; }
    *out = z;
    return ZDA_OK;
}

void zda_zone_destroy(zda_zone *zone) { delete zone; }

zda_status zda_set_wavelengths(zda_zone *z, const double *lambda, int n)
{
    if (!z || !lambda || n < 1 || 2 * n > ZDA_MAX_FREQ) return fail(ZDA_ERR_ARG, "bad wavelengths");
    for (int l = 0; l < n; ++l)
        if (!(lambda[l] > 0)) return fail(ZDA_ERR_ARG, "wavelengths must be positive");
    z->lambda.assign(lambda, lambda + n);
    return derive(*z);
}

zda_status zda_set_pulse(zda_zone *z, double f0, double sigma_t, double t0)
{
    if (!z || !(f0 > 0) || !(sigma_t > 0)) return fail(ZDA_ERR_ARG, "bad pulse");
    z->f0 = f0; z->sigma = sigma_t; z->t0 = t0;
    z->tables_dirty = true;
    z->have_forward = false;
    return ZDA_OK;
}

zda_status zda_zone_set_projection(zda_zone *z, double beta, double eta)
{
    if (!z || !(eta > 0 && eta < 1)) return fail(ZDA_ERR_ARG, "bad projection");
    z->d.beta = beta;
    z->d.eta = eta;
    z->have_forward = false;
    return ZDA_OK;
}

zda_status zda_zone_query(const zda_zone *z, zda_zone_info *info)
{
    if (!z || !info) return fail(ZDA_ERR_ARG, "null argument");
    info->dt = z->dt; info->dphi = z->dphi; info->tau = z->tau;
    info->n_freq = z->nq; info->n_r_design = z->nrd; info->design_nk = z->nk;
    info->workspace_bytes = z->L.total;
    info->cells = (long long)z->d.n_r * z->d.n_phi * z->d.n_z;
    return ZDA_OK;
}

zda_status zda_zone_workspace_bytes(const zda_zone *z, size_t *bytes)
{
    if (!z || !bytes) return fail(ZDA_ERR_ARG, "null argument");
    *bytes = z->L.total;
    return ZDA_OK;
}

zda_status zda_zone_bind_workspace(zda_zone *z, void *ws, size_t bytes)
{
    if (!z || !ws) return fail(ZDA_ERR_ARG, "null argument");
    if (((uintptr_t)ws) & 255) return fail(ZDA_ERR_ARG, "workspace must be 256-byte aligned");
    if (bytes < z->L.total) return fail(ZDA_ERR_OOM, "workspace smaller than zda_zone_workspace_bytes");
    z->ws = (char *)ws;
    z->ws_bytes = bytes;
    z->tables_dirty = true;
    z->have_forward = false;
    return ZDA_OK;
}

zda_status zda_filter_project(zda_zone *z, const float *rho, float *rho_t, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!rho || !rho_t) return fail(ZDA_ERR_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    z->have_forward = false;          // the permittivity tables now follow this rho
    st = run_filter(*z, rho, s);
    if (st) return st;
    CUDA_TRY(cudaMemcpyAsync(rho_t, z->ws + z->L.rho_t, (size_t)z->nrd * z->d.n_phi * 4, cudaMemcpyDeviceToDevice, s));
    return ZDA_OK;
}

zda_status zda_filter_project_backward(zda_zone *z, const float *rho, const float *g_t, float *g_rho, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!rho || !g_t || !g_rho) return fail(ZDA_ERR_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    z->have_forward = false;          // the permittivity tables now follow this rho
    st = run_filter(*z, rho, s);
    if (st) return st;
    const zda::FilterParams fp = filter_params(*z);
    zda::launch_filter_project_backward(fp, P<float>(*z, z->L.rho_bar), P<float>(*z, z->L.norm), g_t, g_rho, s);
    z->launches++;
    CUDA_TRY(cudaGetLastError());
    return ZDA_OK;
}

zda_status zda_forward(zda_zone *z, const float *rho, double *focal_out, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!rho || !focal_out) return fail(ZDA_ERR_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    st = forward_enqueue(*z, rho, s);
    if (st) return st;
    st = check_wait_status(*z, s);
    if (st) return st;
    st = focal_finish(*z, focal_out, s);
    if (st) return st;
    z->have_forward = true;
    return ZDA_OK;
}

zda_status zda_adjoint(zda_zone *z, const double *dI, float *grad_rho, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!dI || !grad_rho) return fail(ZDA_ERR_ARG, "null pointer");
    if (!z->have_forward) return fail(ZDA_ERR_STATE, "zda_adjoint needs a preceding zda_forward");
    if (!z->adjoint_ok)
        return fail(ZDA_ERR_ARG, "n_steps too short: the broadband adjoint pulses do not fit the run");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(z->ws + z->L.g_in, dI, z->nq * sizeof(double2), cudaMemcpyHostToDevice, s));
    st = adjoint_enqueue(*z, grad_rho, s);
    if (st) return st;
    if (uses_waits(*z)) return check_wait_status(*z, s);
    return ZDA_OK;
}

zda_status zda_iteration(zda_zone *z, const float *rho, double *I_out, float *grad_rho, int host_buffers,
                         void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!rho || !I_out || !grad_rho) return fail(ZDA_ERR_ARG, "null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nb = (size_t)z->nrd * z->d.n_phi * sizeof(float);
    const float *rho_dev = rho;
    float *g_dev = grad_rho;
    if (host_buffers) {
        CUDA_TRY(cudaMemcpyAsync(z->ws + z->L.rho_in, rho, nb, cudaMemcpyHostToDevice, s));
        rho_dev = P<float>(*z, z->L.rho_in);
        g_dev = P<float>(*z, z->L.g_rho);
    }
    std::vector<double> S(2 * z->nq), g(2 * z->nq);
    st = zda_forward(z, rho_dev, S.data(), stream);
    if (st) return st;
    double I = 0;
    for (int q = 0; q < z->nq; ++q) {
        I += 2.0 * (S[2 * q] * S[2 * q] + S[2 * q + 1] * S[2 * q + 1]);
        g[2 * q] = 4.0 * S[2 * q];
        g[2 * q + 1] = 4.0 * S[2 * q + 1];
    }
    st = zda_adjoint(z, g.data(), g_dev, stream);
    if (st) return st;
    if (host_buffers) CUDA_TRY(cudaMemcpyAsync(grad_rho, g_dev, nb, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *I_out = I;
    return ZDA_OK;
}

zda_status zda_focal_transform(zda_zone *z, const float *mon, double *out, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!mon || !out) return fail(ZDA_ERR_ARG, "null pointer");
    return focal(*z, (const float2 *)mon, out, (cudaStream_t)stream);
}

zda_status zda_focal_transform_nn(zda_zone *z, const float *y, int n, float scale, double *S, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!y || !S) return fail(ZDA_ERR_ARG, "null pointer");
    if (n < 1 || !(scale > 0.f)) return fail(ZDA_ERR_ARG, "n >= 1 and scale > 0 required");
    zda::launch_focal_nn(y, n, z->nq, z->i_d0, z->nrd, z->d.n_phi, z->d.n_r, scale, P<double2>(*z, z->L.Gr),
                         P<double2>(*z, z->L.Gp), P<double2>(*z, z->L.emph_n), P<double2>(*z, z->L.emph_h),
                         reinterpret_cast<double2 *>(S), (cudaStream_t)stream);
    z->launches++;
    CUDA_TRY(cudaGetLastError());
    return ZDA_OK;
}

zda_status zda_focal_transform_nn_transpose(zda_zone *z, const double *dS, int n, float scale, float *dy, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!dS || !dy) return fail(ZDA_ERR_ARG, "null pointer");
    if (n < 1 || !(scale > 0.f)) return fail(ZDA_ERR_ARG, "n >= 1 and scale > 0 required");
    zda::launch_focal_nn_T(reinterpret_cast<const double2 *>(dS), n, z->nq, z->i_d0, z->nrd, z->d.n_phi, z->d.n_r,
                           scale, P<double2>(*z, z->L.Gr), P<double2>(*z, z->L.Gp), P<double2>(*z, z->L.emph_n),
                           P<double2>(*z, z->L.emph_h), dy, (cudaStream_t)stream);
    z->launches++;
    CUDA_TRY(cudaGetLastError());
    return ZDA_OK;
}

zda_status zda_copy_fields(zda_zone *z, float *out, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!out) return fail(ZDA_ERR_ARG, "null pointer");
    const size_t n = 6 * (size_t)z->d.n_r * z->d.n_phi * z->d.n_z * sizeof(float2);
    const size_t off = ((z->variant == 1 || z->variant == 3) && z->last_parity) ? z->L.fields2 : z->L.fields;
    CUDA_TRY(cudaMemcpyAsync(out, z->ws + off, n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return ZDA_OK;
}

zda_status zda_copy_monitor_dft(zda_zone *z, float *out, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!out) return fail(ZDA_ERR_ARG, "null pointer");
    const size_t n = (size_t)z->nq * 2 * z->d.n_r * z->d.n_phi * sizeof(float2);
    CUDA_TRY(cudaMemcpyAsync(out, z->ws + z->L.mon, n, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return ZDA_OK;
}

zda_status zda_copy_design_dft(zda_zone *z, int which, float *out, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (!out || (which != 0 && which != 1)) return fail(ZDA_ERR_ARG, "bad argument");
    const size_t n = (size_t)z->nq * 3 * z->d.n_r * z->d.n_phi * z->nk * sizeof(float2);
    CUDA_TRY(cudaMemcpyAsync(out, z->ws + (which ? z->L.des_a : z->L.des_f), n, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
    return ZDA_OK;
}

long long zda_zone_launch_count(const zda_zone *z) { return z ? z->launches : -1; }

zda_status zda_zone_set_kernel(zda_zone *z, int variant, int tile_phi, int i_ranges)
{
    if (!z || variant < 0 || variant > 5 || i_ranges < 0) return fail(ZDA_ERR_ARG, "bad kernel choice");
    z->kernel_default = false;
    if (variant == 4 || variant == 5) {      // split step, E half (4) or both halves (5) on TMA-staged tiles
        if (z->d.n_fold == 0) return fail(ZDA_ERR_ARG, "the axis zone (continuous axisymmetry) uses the split step");
        if (z->rpml) return fail(ZDA_ERR_ARG, "the E tile kernel implements the real-radius r-PML only");
        if (z->d.n_z % 2 || z->d.pml_z % 2) return fail(ZDA_ERR_ARG, "the E tile kernel needs even n_z and pml_z");
        if (!zda::tile_e_shape_ok(tile_phi)) return fail(ZDA_ERR_ARG, "E tile kernel: tile_phi must be 8, 16 or 32");
        z->pair_kernels = true;
        z->variant = variant;
        z->tile_phi = tile_phi;
        z->i_ranges = i_ranges;
        z->have_forward = false;
        return ZDA_OK;
    }
    if (variant == 3) {                      // fused step on TMA-staged tiles streaming along r
        if (z->d.n_fold == 0) return fail(ZDA_ERR_ARG, "the axis zone (continuous axisymmetry) uses the split step");
        if (z->rpml) return fail(ZDA_ERR_ARG, "the tile step implements the real-radius r-PML only");
        if (z->d.n_z % 2 || z->d.pml_z % 2) return fail(ZDA_ERR_ARG, "the tile step needs even n_z and pml_z");
        if (!zda::tile_shape_ok(tile_phi)) return fail(ZDA_ERR_ARG, "tile step: tile_phi must be 4, 8 or 16");
        z->pair_kernels = true;
        z->variant = 3;
        z->tile_phi = tile_phi;
        z->i_ranges = i_ranges;
        z->have_forward = false;
        return ZDA_OK;
    }
    if (variant == 2) {                      // split step, one z-cell per thread
        z->variant = 0;
        z->pair_kernels = false;
        z->tile_phi = tile_phi;
        z->i_ranges = i_ranges;
        z->have_forward = false;
        return ZDA_OK;
    }
    z->pair_kernels = true;
    if (variant == 1) {
        if (z->d.n_fold == 0) return fail(ZDA_ERR_ARG, "the axis zone (continuous axisymmetry) uses the split step");
        if (z->rpml) return fail(ZDA_ERR_ARG, "the fused step implements the real-radius r-PML only");
        if (tile_phi != 2 && tile_phi != 4) return fail(ZDA_ERR_ARG, "fused step: tile_phi must be 2 or 4");
        if (z->d.n_z > zda::fused_max_nz()) return fail(ZDA_ERR_ARG, "fused step supports n_z <= 256");
        if (z->d.n_z % 2) return fail(ZDA_ERR_ARG, "fused step needs an even n_z (16-byte bulk copies)");
    }
    z->variant = variant;
    z->tile_phi = tile_phi;
    z->i_ranges = i_ranges;
    z->have_forward = false;
    return ZDA_OK;
}

zda_status zda_zone_set_radial_pml(zda_zone *z, int form)
{
    if (!z || (form != 0 && form != 1)) return fail(ZDA_ERR_ARG, "r-PML form must be 0 or 1");
    if (form == 1 && (z->variant == 1 || z->variant >= 3)) {
        if (!z->kernel_default)
            return fail(ZDA_ERR_ARG, "the fused and tiled steps implement the real-radius r-PML only");
        z->variant = 0;                      // the default tiled step gives way to the split step
        z->tile_phi = 2;
        z->i_ranges = 0;
    }
    if (z->rpml != form) {
        z->rpml = form;
        z->tables_dirty = true;
        z->have_forward = false;
    }
    return ZDA_OK;
}

zda_status zda_zone_get_radial_pml(const zda_zone *z, int *form)
{
    if (!z || !form) return fail(ZDA_ERR_ARG, "null argument");
    *form = z->rpml;
    return ZDA_OK;
}

zda_status zda_zone_time_steps(zda_zone *z, int steps, double *ms_out, void *stream)
{
    zda_status st = ready(z);
    if (st) return st;
    if (steps < 1 || !ms_out) return fail(ZDA_ERR_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    z->have_forward = false;                 // the fields are overwritten
    zda::StepParams p = step_params(*z);
    p.src_mode = zda::SRC_NONE;
    p.mon = nullptr;
    p.des = nullptr;
    p.mon_k = -1;
    cudaEvent_t a, b;
    CUDA_TRY(cudaEventCreate(&a));
    CUDA_TRY(cudaEventCreate(&b));
    const int saved_steps = z->d.n_steps;
    const int saved_every = z->time_every;
    z->d.n_steps = steps;
    z->time_every = 0;
    cudaError_t e = cudaEventRecord(a, s);
    if (e == cudaSuccess) st = time_loop(*z, p, s);
    if (e == cudaSuccess && st == ZDA_OK) e = cudaEventRecord(b, s);
    if (e == cudaSuccess && st == ZDA_OK) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess && st == ZDA_OK) e = cudaEventElapsedTime(&ms, a, b);
    z->d.n_steps = saved_steps;
    z->time_every = saved_every;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st) return st;
    if (e != cudaSuccess) return fail(ZDA_ERR_CUDA, std::string("timing: ") + cudaGetErrorString(e));
    *ms_out = ms;
    return check_wait_status(*z, s);
}

zda_status zda_zone_set_wait_limit(zda_zone *z, int polls, int inject_timeout)
{
    if (!z || polls < 1) return fail(ZDA_ERR_ARG, "bad wait limit");
    z->wait_limit = polls;
    z->inject_timeout = inject_timeout ? 1 : 0;
    return ZDA_OK;
}

zda_status zda_zone_get_kernel(const zda_zone *z, int *variant, int *tile_phi, int *i_ranges)
{
    if (!z || !variant || !tile_phi || !i_ranges) return fail(ZDA_ERR_ARG, "null argument");
    *variant = (z->variant == 0 && !z->pair_kernels) ? 2 : z->variant;
    *tile_phi = z->tile_phi;
    *i_ranges = z->variant == 1   ? auto_i_ranges(*z)
                : z->variant == 3 ? tile_rchunks(*z)
                : z->variant >= 4 ? tile_e_rchunks(*z)
                                  : z->i_ranges;
    return ZDA_OK;
}

zda_status zda_zone_set_timing(zda_zone *z, int every)
{
    if (!z || every < 0) return fail(ZDA_ERR_ARG, "bad argument");
    CUDA_TRY(cudaSetDevice(z->ctx->device));
    timing_release(*z);
    z->t_h_ms = z->t_e_ms = z->t_x_ms = 0;
    z->t_count = 0;
    if (every == 0) return ZDA_OK;
    const int R = 64;
    z->ev.resize(4 * R);
    for (auto &e : z->ev) CUDA_TRY(cudaEventCreate(&e));
    z->ev_pending.assign(R, 0);
    z->ev_next = 0;
    z->time_every = every;
    return ZDA_OK;
}

zda_status zda_zone_set_energy_probe(zda_zone *z, int every)
{
    if (!z || every < 0) return fail(ZDA_ERR_ARG, "bad argument");
    z->probe_every = every;
    z->probe_n = 0;
    return ZDA_OK;
}

zda_status zda_zone_energy_trace(zda_zone *z, double *w_host, double *wdot_host, int max_samples, int *n_samples)
{
    if (!z || !w_host || !wdot_host || !n_samples || max_samples < 0) return fail(ZDA_ERR_ARG, "null argument");
    if (!z->ws) return fail(ZDA_ERR_STATE, "no workspace bound");
    CUDA_TRY(cudaSetDevice(z->ctx->device));
    const int n = std::min(z->probe_n, max_samples);
    std::vector<double> buf(2 * (size_t)std::max(n, 1));
    if (n > 0) CUDA_TRY(cudaMemcpy(buf.data(), z->ws + z->L.energy, 2 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) {
        w_host[i] = buf[2 * i];
        wdot_host[i] = buf[2 * i + 1];
    }
    *n_samples = n;
    return ZDA_OK;
}

zda_status zda_zone_timing(zda_zone *z, double *ms3, long long *count)
{
    if (!z || !ms3 || !count) return fail(ZDA_ERR_ARG, "null argument");
    CUDA_TRY(cudaSetDevice(z->ctx->device));
    for (size_t s = 0; s < z->ev_pending.size(); ++s) timing_drain_slot(*z, (int)s);
    ms3[0] = z->t_h_ms;
    ms3[1] = z->t_e_ms;
    ms3[2] = z->t_x_ms;
    *count = z->t_count;
    z->t_h_ms = z->t_e_ms = z->t_x_ms = 0;
    z->t_count = 0;
    return ZDA_OK;
}


}  // extern "C"

// ------------------------------------------------------------------ lens
// A lens: concentric zones solved independently (section "Zoned discrete
// axisymmetry") whose focal phasors add up.  Each zone's whole forward (or
// adjoint) run is captured as one branch of a CUDA graph (the branches fork
// from one capture stream, so the zones run concurrently, each with its own
// dt and number of steps), joined by a device-side sum of the phasors.  One
// graph launch per run; the graph is captured on first use and again when a
// zone's configuration changes.
struct zda_lens {
    zda_ctx *ctx = nullptr;
    std::vector<zda_zone *> zones;
    int nq = 0;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool use_graph = true;
    cudaGraphExec_t g_fwd = nullptr, g_adj = nullptr;
    std::vector<std::vector<long long>> stamp_fwd, stamp_adj;
    std::vector<cudaStream_t> streams;     // [0] capture / join stream, [1 + z] zone branches
    std::vector<cudaEvent_t> events;       // [0] fork, [1 + z] joins
    bool have_forward = false;
    long long launches = 0;
    std::vector<const void *> bound_S;     // zones' phasor addresses when the workspace was bound
    ~zda_lens();
};

zda_lens::~zda_lens()
{
    if (g_fwd) cudaGraphExecDestroy(g_fwd);
    if (g_adj) cudaGraphExecDestroy(g_adj);
    for (cudaStream_t s : streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
}

static size_t lens_ws_ptrs(const zda_lens &L) { return 0; }
static size_t lens_ws_S(const zda_lens &L) { return align_up(L.zones.size() * sizeof(void *)); }
static size_t lens_ws_status(const zda_lens &L) { return lens_ws_S(L) + align_up(L.nq * sizeof(double2)); }
static size_t lens_ws_total(const zda_lens &L) { return lens_ws_status(L) + 256; }

static std::vector<long long> zone_stamp(const zda_zone &z)
{
    return {(long long)(uintptr_t)z.ws, z.variant, z.pair_kernels, z.tile_phi, z.i_ranges, z.probe_every, z.d.n_steps, z.nq,
            z.wait_limit, z.inject_timeout, (long long)z.lambda.size(), z.rpml};
}

static bool stamps_match(const zda_lens &L, const std::vector<std::vector<long long>> &st)
{
    if (st.size() != L.zones.size()) return false;
    for (size_t i = 0; i < L.zones.size(); ++i)
        if (st[i] != zone_stamp(*L.zones[i])) return false;
    return true;
}

// enqueue every zone's run on its branch stream and join on streams[0]
template <class F>
static zda_status lens_branches(zda_lens &L, F &&per_zone)
{
    cudaStream_t s0 = L.streams[0];
    CUDA_TRY(cudaEventRecord(L.events[0], s0));
    for (size_t z = 0; z < L.zones.size(); ++z) {
        cudaStream_t sz = L.streams[1 + z];
        CUDA_TRY(cudaStreamWaitEvent(sz, L.events[0], 0));
        zda_status st = per_zone(*L.zones[z], z, sz);
        if (st) return st;
        CUDA_TRY(cudaEventRecord(L.events[1 + z], sz));
        CUDA_TRY(cudaStreamWaitEvent(s0, L.events[1 + z], 0));
    }
    return ZDA_OK;
}

template <class F>
static zda_status lens_run(zda_lens &L, cudaGraphExec_t &exec, std::vector<std::vector<long long>> &stamp,
                           cudaStream_t user, F &&body)
{
    cudaStream_t s0 = L.streams[0];
    if (!L.use_graph) {
        CUDA_TRY(cudaEventRecord(L.events[0], user));
        CUDA_TRY(cudaStreamWaitEvent(s0, L.events[0], 0));
        zda_status st = body();
        if (st) return st;
        CUDA_TRY(cudaEventRecord(L.events[0], s0));
        CUDA_TRY(cudaStreamWaitEvent(user, L.events[0], 0));
        L.launches++;
        return ZDA_OK;
    }
    if (!exec || !stamps_match(L, stamp)) {
        if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
        std::vector<int> saved(L.zones.size());
        for (size_t z = 0; z < L.zones.size(); ++z) {       // no host waits inside a capture
            saved[z] = L.zones[z]->time_every;
            L.zones[z]->time_every = 0;
        }
        CUDA_TRY(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
        zda_status st = body();
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s0, &g);
        for (size_t z = 0; z < L.zones.size(); ++z) L.zones[z]->time_every = saved[z];
        if (st) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return fail(ZDA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { exec = nullptr; return fail(ZDA_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)); }
        stamp.clear();
        for (zda_zone *z : L.zones) stamp.push_back(zone_stamp(*z));
    }
    CUDA_TRY(cudaGraphLaunch(exec, user));
    L.launches++;
    return ZDA_OK;
}

extern "C" {

zda_status zda_lens_create(zda_ctx *ctx, zda_zone *const *zones, int n_zones, zda_lens **out)
{
    if (!ctx || !zones || n_zones < 1 || !out) return fail(ZDA_ERR_ARG, "bad argument");
    for (int z = 0; z < n_zones; ++z) {
        if (!zones[z] || zones[z]->ctx != ctx) return fail(ZDA_ERR_ARG, "zone missing or from another context");
        if (zones[z]->nq != zones[0]->nq) return fail(ZDA_ERR_ARG, "all zones of a lens need the same wavelengths");
        for (int y = 0; y < z; ++y)
            if (zones[y] == zones[z]) return fail(ZDA_ERR_ARG, "a zone appears twice");
    }
    CUDA_TRY(cudaSetDevice(ctx->device));
    zda_lens *L = new zda_lens();
    L->ctx = ctx;
    L->zones.assign(zones, zones + n_zones);
    L->nq = zones[0]->nq;
    L->streams.resize(n_zones + 1);
    L->events.resize(n_zones + 1);
    for (auto &s : L->streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) { delete L; return fail(ZDA_ERR_CUDA, "stream"); }
    for (auto &e : L->events)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { delete L; return fail(ZDA_ERR_CUDA, "event"); }
    *out = L;
    return ZDA_OK;
}

void zda_lens_destroy(zda_lens *lens) { delete lens; }

zda_status zda_lens_workspace_bytes(const zda_lens *L, size_t *bytes)
{
    if (!L || !bytes) return fail(ZDA_ERR_ARG, "null argument");
    *bytes = lens_ws_total(*L);
    return ZDA_OK;
}

zda_status zda_lens_bind_workspace(zda_lens *L, void *ws, size_t bytes)
{
    if (!L || !ws) return fail(ZDA_ERR_ARG, "null argument");
    if (((uintptr_t)ws) & 255) return fail(ZDA_ERR_ARG, "workspace must be 256-byte aligned");
    if (bytes < lens_ws_total(*L)) return fail(ZDA_ERR_OOM, "workspace smaller than zda_lens_workspace_bytes");
    CUDA_TRY(cudaSetDevice(L->ctx->device));
    L->ws = (char *)ws;
    L->ws_bytes = bytes;
    std::vector<const double2 *> ptrs;
    for (zda_zone *z : L->zones) {
        if (!z->ws) return fail(ZDA_ERR_STATE, "bind every zone's workspace before the lens workspace");
        ptrs.push_back((const double2 *)(z->ws + z->L.S));
    }
    L->bound_S.assign(ptrs.begin(), ptrs.end());
    CUDA_TRY(cudaMemcpy(L->ws + lens_ws_ptrs(*L), ptrs.data(), ptrs.size() * sizeof(void *), cudaMemcpyHostToDevice));
    if (L->g_fwd) { cudaGraphExecDestroy(L->g_fwd); L->g_fwd = nullptr; }
    if (L->g_adj) { cudaGraphExecDestroy(L->g_adj); L->g_adj = nullptr; }
    L->have_forward = false;
    return ZDA_OK;
}

zda_status zda_lens_set_graph(zda_lens *L, int use_graph)
{
    if (!L) return fail(ZDA_ERR_ARG, "null lens");
    L->use_graph = use_graph != 0;
    return ZDA_OK;
}

zda_status zda_lens_forward(zda_lens *L, const float *const *rho, double *focal_out, void *stream)
{
    if (!L || !rho || !focal_out) return fail(ZDA_ERR_ARG, "null argument");
    if (!L->ws) return fail(ZDA_ERR_STATE, "no lens workspace bound");
    cudaStream_t s = (cudaStream_t)stream;
    for (size_t z = 0; z < L->zones.size(); ++z) {
        zda_zone *Z = L->zones[z];
        if (!rho[z]) return fail(ZDA_ERR_ARG, "null density pointer");
        const void *now = Z->ws ? (const void *)(Z->ws + Z->L.S) : nullptr;
        if (now != L->bound_S[z]) return fail(ZDA_ERR_STATE, "a zone's workspace changed: re-bind the lens workspace");
        zda_status st = ready(Z);            // tables (host copies) before any capture
        if (st) return st;
        CUDA_TRY(cudaMemcpyAsync(Z->ws + Z->L.rho_in, rho[z], (size_t)Z->nrd * Z->d.n_phi * sizeof(float),
                                 cudaMemcpyDeviceToDevice, s));
    }
    L->have_forward = false;
    for (zda_zone *Z : L->zones) Z->have_forward = false;
    int *status = (int *)(L->ws + lens_ws_status(*L));
    auto body = [&]() -> zda_status {
        zda_status st = lens_branches(*L, [&](zda_zone &Z, size_t, cudaStream_t sz) {
            return forward_enqueue(Z, P<float>(Z, Z.L.rho_in), sz);
        });
        if (st) return st;
        CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), L->streams[0]));
        zda::launch_lens_sum((const double2 *const *)(L->ws + lens_ws_ptrs(*L)), (int)L->zones.size(), L->nq,
                             (double2 *)(L->ws + lens_ws_S(*L)), status, L->streams[0]);
        CUDA_TRY(cudaGetLastError());
        return ZDA_OK;
    };
    zda_status st = lens_run(*L, L->g_fwd, L->stamp_fwd, s, body);
    if (st) return st;
    int flag = 0;
    CUDA_TRY(cudaMemcpyAsync(focal_out, L->ws + lens_ws_S(*L), L->nq * sizeof(double2), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&flag, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (zda_zone *Z : L->zones) {
        if (uses_waits(*Z)) {
            st = check_wait_status(*Z, s);
            if (st) return st;
        }
    }
    if (flag) return fail(ZDA_ERR_NONFINITE, "non-finite lens focal phasor");
    for (zda_zone *Z : L->zones) Z->have_forward = true;
    L->have_forward = true;
    return ZDA_OK;
}

zda_status zda_lens_zone_focal(const zda_lens *L, int zone, double *focal_out)
{
    if (!L || zone < 0 || zone >= (int)L->zones.size() || !focal_out) return fail(ZDA_ERR_ARG, "bad argument");
    if (!L->have_forward) return fail(ZDA_ERR_STATE, "no lens forward yet");
    const zda_zone *Z = L->zones[zone];
    CUDA_TRY(cudaMemcpy(focal_out, Z->ws + Z->L.S, L->nq * sizeof(double2), cudaMemcpyDeviceToHost));
    return ZDA_OK;
}

zda_status zda_lens_adjoint(zda_lens *L, const double *dI, float *const *grad_rho, void *stream)
{
    if (!L || !dI || !grad_rho) return fail(ZDA_ERR_ARG, "null argument");
    if (!L->have_forward) return fail(ZDA_ERR_STATE, "zda_lens_adjoint needs a preceding zda_lens_forward");
    cudaStream_t s = (cudaStream_t)stream;
    for (zda_zone *Z : L->zones) {
        if (!Z->adjoint_ok)
            return fail(ZDA_ERR_ARG, "n_steps too short: the broadband adjoint pulses do not fit a zone's run");
        // every zone's phasors enter the lens sum with weight 1: same dI/dS
        CUDA_TRY(cudaMemcpyAsync(Z->ws + Z->L.g_in, dI, L->nq * sizeof(double2), cudaMemcpyHostToDevice, s));
    }
    auto body = [&]() -> zda_status {
        return lens_branches(*L, [&](zda_zone &Z, size_t, cudaStream_t sz) {
            return adjoint_enqueue(Z, P<float>(Z, Z.L.g_rho), sz);
        });
    };
    zda_status st = lens_run(*L, L->g_adj, L->stamp_adj, s, body);
    if (st) return st;
    for (size_t z = 0; z < L->zones.size(); ++z) {
        zda_zone *Z = L->zones[z];
        if (!grad_rho[z]) return fail(ZDA_ERR_ARG, "null gradient pointer");
        CUDA_TRY(cudaMemcpyAsync(grad_rho[z], Z->ws + Z->L.g_rho, (size_t)Z->nrd * Z->d.n_phi * sizeof(float),
                                 cudaMemcpyDeviceToDevice, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    for (zda_zone *Z : L->zones)
        if (uses_waits(*Z)) {
            st = check_wait_status(*Z, s);
            if (st) return st;
        }
    return ZDA_OK;
}

long long zda_lens_launch_count(const zda_lens *L) { return L ? L->launches : -1; }

static zda_status lens_field(zda_lens *L, const double *pts_dev, int pstride, int n_pts, int n_phi_samples,
                             double *field_dev, double *p_trans_host, void *stream)
{
    if (!L || !pts_dev || n_pts < 1 || n_phi_samples < 8 || !field_dev) return fail(ZDA_ERR_ARG, "bad argument");
    if (!L->have_forward) return fail(ZDA_ERR_STATE, "the lens field needs a preceding zda_lens_forward");
    cudaStream_t s = (cudaStream_t)stream;
    const int nl = L->nq / 2;
    double2 *ex = (double2 *)field_dev, *ey = ex + (size_t)nl * n_pts;
    CUDA_TRY(cudaMemsetAsync(field_dev, 0, (size_t)2 * nl * n_pts * sizeof(double2), s));
    std::vector<double> ptrans(nl, 0.0);
    for (zda_zone *Z : L->zones) {
        const zda_zone_desc &d = Z->d;
        zda::launch_phi_means(P<float2>(*Z, Z->L.mon), P<double2>(*Z, Z->L.emph_n), P<double2>(*Z, Z->L.emph_h),
                              Z->nq, d.n_r, d.n_phi, (d.n_fold == 1 || d.n_fold == 2) ? 1 : 0,
                              P<double2>(*Z, Z->L.umean), P<double>(*Z, Z->L.pt_row), s);
        const double zf = d.focal - (d.monitor_k * d.dz - d.design_k1 * d.dz);
        zda::launch_focal_plane(P<double2>(*Z, Z->L.umean), P<double>(*Z, Z->L.qr), P<double>(*Z, Z->L.qw),
                                P<double>(*Z, Z->L.qp), P<double>(*Z, Z->L.qwp), d.n_r, nl, pts_dev, pstride, n_pts, zf,
                                P<double>(*Z, Z->L.kk), n_phi_samples, ex, ey, s);
        CUDA_TRY(cudaGetLastError());
        Z->launches += 2;
        // transmitted power: (n_top/2) |E_t|^2 over the annulus, whole circle
        std::vector<double> row((size_t)nl * d.n_r);
        CUDA_TRY(cudaMemcpyAsync(row.data(), Z->ws + Z->L.pt_row, row.size() * 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        const double ntop = std::sqrt(layer_eps_at(d, d.monitor_k));
        const double copies = d.n_fold == 0 ? 1.0 : (double)d.n_fold;
        for (int l = 0; l < nl; ++l)
            for (int i = Z->i_d0; i < Z->i_d1; ++i)
                ptrans[l] += 0.5 * ntop * row[(size_t)l * d.n_r + i] * (d.r_lo + (i + 0.5) * d.dr) * d.dr * Z->dphi *
                             copies;
    }
    if (p_trans_host)
        for (int l = 0; l < nl; ++l) p_trans_host[l] = ptrans[l];
    CUDA_TRY(cudaStreamSynchronize(s));
    return ZDA_OK;
}

zda_status zda_zone_order_bound(const zda_zone_desc *d, const double *lambda_host, int n_lambda,
                                const double *pts_host, int n_pts, int stride, double *bound_host)
{
    if (!d || !lambda_host || n_lambda < 1 || !pts_host || n_pts < 1 || (stride != 2 && stride != 3) || !bound_host)
        return fail(ZDA_ERR_ARG, "bad argument");
    double lmin = lambda_host[0];
    for (int l = 1; l < n_lambda; ++l) lmin = std::min(lmin, lambda_host[l]);
    if (!(lmin > 0)) return fail(ZDA_ERR_ARG, "wavelengths must be positive");
    if (d->n_fold == 0) {                       // continuous axisymmetry: no other orders
        *bound_host = 0.0;
        return ZDA_OK;
    }
    const double k = 2.0 * M_PI * std::sqrt(layer_eps_at(*d, d->monitor_k)) / lmin;
    const double r_hi = d->r_lo + d->n_r * d->dr;
    const double zf0 = d->focal - (d->monitor_k * d->dz - d->design_k1 * d->dz);
    const double nu = std::max(d->n_fold - 2, 0);
    double worst = 0.0;
    for (int t = 0; t < n_pts; ++t) {
        const double *q = pts_host + (size_t)t * stride;
        const double zf = zf0 + (stride == 3 ? q[2] : 0.0);
        if (!(zf > 0)) {
            worst = HUGE_VAL;
            break;
        }
        const double x = k * r_hi * std::hypot(q[0], q[1]) / zf;
        double b;
        if (nu == 0) b = 1.0;
        else if (x <= 0) b = 0.0;
        else b = std::exp(std::min(nu * std::log(0.5 * x) - std::lgamma(nu + 1.0), 700.0));
        worst = std::max(worst, b);
    }
    *bound_host = worst;
    return ZDA_OK;
}

zda_status zda_lens_focal_plane(zda_lens *L, const double *pts_dev, int n_pts, int n_phi_samples, double *field_dev,
                                double *p_trans_host, void *stream)
{
    return lens_field(L, pts_dev, 2, n_pts, n_phi_samples, field_dev, p_trans_host, stream);
}

zda_status zda_lens_field_points(zda_lens *L, const double *pts_dev, int n_pts, int n_phi_samples, double *field_dev,
                                 void *stream)
{
    return lens_field(L, pts_dev, 3, n_pts, n_phi_samples, field_dev, nullptr, stream);
}

// device scratch of zda_lens_evaluate: line points, line field, disc points, disc field, FWHM, I(0),
// results (256-byte aligned pieces)
struct EvalScratch {
    size_t lp, lf, dp, df, fw, i0, out, total;
};

static EvalScratch eval_scratch(int nl, int n_line, int n_rad, int n_ang)
{
    EvalScratch e{};
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off += (b + 255) & ~(size_t)255;
        return o;
    };
    const size_t nd = (size_t)nl * n_rad * n_ang;
    e.lp = take((size_t)2 * n_line * 8);
    e.lf = take((size_t)2 * nl * n_line * 16);
    e.dp = take(2 * nd * 8);
    e.df = take((size_t)2 * nl * nd * 16);
    e.fw = take((size_t)nl * 8);
    e.i0 = take((size_t)nl * 8);
    e.out = take((size_t)8 * nl * 8);
    e.total = off;
    return e;
}

zda_status zda_lens_evaluate_scratch_bytes(const zda_lens *L, int n_line, int n_rad, int n_ang, size_t *bytes)
{
    if (!L || !bytes || n_line < 2 || n_rad < 1 || n_ang < 1) return fail(ZDA_ERR_ARG, "bad argument");
    *bytes = eval_scratch(L->nq / 2, n_line, n_rad, n_ang).total;
    return ZDA_OK;
}

zda_status zda_lens_evaluate(zda_lens *L, double lens_radius, double focal, const double *incident_host, double n_top,
                             int n_line, double x_max, int n_rad, int n_ang, int n_phi_samples, void *scratch_dev,
                             size_t scratch_bytes, double *out_host, double *line_dev, void *stream)
{
    if (!L || !incident_host || !out_host || !scratch_dev || !(lens_radius > 0) || !(focal > 0) || !(n_top > 0) ||
        n_line < 2 || !(x_max > 0) || n_rad < 1 || n_ang < 1 || n_phi_samples < 8)
        return fail(ZDA_ERR_ARG, "bad argument");
    if (!L->have_forward) return fail(ZDA_ERR_STATE, "the lens evaluation needs a preceding zda_lens_forward");
    const int nl = L->nq / 2;
    if (nl > ZDA_EVAL_MAX_LAMBDA) return fail(ZDA_ERR_ARG, "the lens evaluation takes at most 8 wavelengths");
    const EvalScratch e = eval_scratch(nl, n_line, n_rad, n_ang);
    if (scratch_bytes < e.total) return fail(ZDA_ERR_ARG, "scratch smaller than zda_lens_evaluate_scratch_bytes");
    if ((uintptr_t)scratch_dev % 256) return fail(ZDA_ERR_ARG, "scratch must be 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    char *scr = static_cast<char *>(scratch_dev);
    const size_t nd = (size_t)nl * n_rad * n_ang;
    double *lp = (double *)(scr + e.lp), *dp = (double *)(scr + e.dp);
    double *fw = (double *)(scr + e.fw), *i0 = (double *)(scr + e.i0), *out = (double *)(scr + e.out);
    zda::launch_eval_line_points(lp, n_line, x_max, s);
    std::vector<double> pt(nl, 0.0);
    zda_status st = lens_field(L, lp, 2, n_line, n_phi_samples, (double *)(scr + e.lf), pt.data(), stream);
    if (st) return st;
    zda::launch_eval_fwhm((const double2 *)(scr + e.lf), nl, n_line, x_max, n_top, line_dev, fw, i0, s);
    zda::launch_eval_disc_points(fw, nl, n_rad, n_ang, dp, s);
    CUDA_TRY(cudaGetLastError());
    st = lens_field(L, dp, 2, (int)nd, n_phi_samples, (double *)(scr + e.df), nullptr, stream);
    if (st) return st;
    zda::EvalScalars sc{};
    const std::vector<double> &lam = L->zones[0]->lambda;
    for (int l = 0; l < nl; ++l) {
        sc.incident[l] = incident_host[l];
        sc.p_trans[l] = pt[l];
        sc.lambda[l] = lam[l];
    }
    sc.area = M_PI * lens_radius * lens_radius;
    sc.focal = focal;
    sc.n_top = n_top;
    zda::launch_eval_finish((const double2 *)(scr + e.df), nl, n_rad, n_ang, fw, i0, sc, out, s);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(out_host, out, (size_t)8 * nl * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return ZDA_OK;
}

zda_status zda_zone_incident_intensity(zda_zone *z, double *out_dev, void *stream)
{
    if (!z || !out_dev) return fail(ZDA_ERR_ARG, "null argument");
    if (!z->have_forward) return fail(ZDA_ERR_STATE, "the incident intensity needs a preceding zda_forward");
    const zda_zone_desc &d = z->d;
    const int nl = z->nq / 2;
    const int i0 = d.pml_r_in, i1 = d.n_r - d.pml_r_out;
    if (i1 <= i0) return fail(ZDA_ERR_ARG, "no radius between the r-PMLs");
    const double dphi = d.n_fold == 0 ? 0.0 : 2.0 * M_PI / d.n_fold / d.n_phi;
    zda::launch_incident_intensity(P<float2>(*z, z->L.mon), nl, d.n_r, d.n_phi, i0, i1, dphi,
                                   std::sqrt(layer_eps_at(d, 0)), out_dev, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    return ZDA_OK;
}

zda_status zda_field_intensity(const double *field_dev, int n_lambda, int n_pts, double n_top, double *out_dev,
                               void *stream)
{
    if (!field_dev || !out_dev || n_lambda < 1 || n_pts < 1) return fail(ZDA_ERR_ARG, "bad argument");
    zda::launch_field_intensity((const double2 *)field_dev, n_lambda, n_pts, n_top, out_dev, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    return ZDA_OK;
}

zda_status zda_encircled_power(const double *radii_dev, const double *I_dev, int n_prof, int n, double *out_dev,
                               void *stream)
{
    if (!radii_dev || !I_dev || !out_dev || n_prof < 1 || n < 1) return fail(ZDA_ERR_ARG, "bad argument");
    zda::launch_encircled_power(radii_dev, I_dev, n_prof, n, out_dev, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    return ZDA_OK;
}

}  // extern "C"
