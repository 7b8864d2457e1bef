// Fused leap-frog step on TMA-staged (r, phi, z) tiles (sm_103a).
//
// One launch advances (E^n, H^{n-1/2}) to (E^{n+1}, H^{n+1/2}) (Eqs. 3-4)
// with the CPML auxiliaries, the sheet source and the history writes of the
// time-blocked running DFT, reading one field buffer and writing the other
// (ping-pong).  DRAM traffic per cell and step: one read and one write of
// the six components (96 B) against 144 B for the split H / E launches,
// which read the six components twice.
//
// Each CTA owns a column of TJ phi rows x 32 z-cells and streams along r
// over a range of radii [ib, ie).  Load group g(r) = {E^n at radius r+1,
// H^{n-1/2} at radius r} is one set of TMA tensor copies
// (cp.async.bulk.tensor, one box per component) of
//   E^n       rows j0-1 .. j0+TJ,   z k0-2 .. k0+33
//   H^{n-1/2} rows j0-1 .. j0+TJ-1, z k0-2 .. k0+31
// into a ring of NSLOT slots in shared memory ([row][z], z fastest; outside
// the grid the copy fills zeros, the PEC values there), completing on the
// slot's mbarrier.  Tiles at the wedge's phi edges also fetch the wrapped
// rows (phi row n_phi-1 below j0, row 0 above n_phi-1) into staging rows
// and apply the Bloch phase e^{-+i m tau} when they read them.  Iteration r
// runs two groups of warps side by side:
//   H items: H^{n+1/2}(r) on the H box (the tile plus the row j0-1 and the
//            z-cells k0-2, k0-1 below it, which the E update needs and the
//            neighbouring tiles own), in place in shared memory; tile sites
//            are also stored to the output buffer with their H-side CPML
//            auxiliaries (ping-ponged too: halo sites read the old set,
//            which their owner does not write);
//   E items: E^{n+1}(r-1) from H^{n+1/2}(r-1), H^{n+1/2}(r-2) and E^n(r-1),
//            E-side CPML in place (each site only by its owner), source,
//            DFT history, stored to the output buffer.
// Every cell takes the interior coefficient form; the CPML recursions and
// the source add their terms where they apply, so warps that straddle a
// CPML slab edge or the source plane do not run two versions of the update.
// After iteration r thread 0 waits for g(r+1) and the block barrier
// publishes it (and H(r)) to every thread; then g(r+NSLOT-2) is issued into
// the slot of g(r-2), whose last reader was E(r-1).  Each wait is bounded
// (polls and a 1 s deadline): on expiry the error word is set, every
// thread leaves the loop at the barrier, and thread 0 waits (bounded) for
// the copies still in flight before the CTA exits.  Same scheme as the
// split step (zda_pair.cu); results agree to FP32 rounding.
#include <cudaTypedefs.h>
#include <algorithm>
#include "zda_tile.h"

namespace zda {
namespace {

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void t_mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void t_mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// one poll; the thread may sleep in it up to 20 us (woken early when the phase completes)
__device__ __forceinline__ bool t_mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(20000)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t t_now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// bounded wait: at most `limit` polls and at most one second; false (and the
// error word set) if the phase never completed
__device__ __forceinline__ bool t_mbar_wait(uint32_t bar, uint32_t parity, int limit, int *err)
{
    const uint64_t t0 = t_now_ns();
    for (int it = 0; it < limit; ++it) {
        if (t_mbar_try(bar, parity)) return true;
        if ((it & 15) == 15 && t_now_ns() - t0 > 1000000000ull) break;
    }
    atomicOr(err, 1);
    return false;
}

// 3-D tensor copy global -> this CTA's shared memory, completing on `bar`
__device__ __forceinline__ void tma3(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

struct C2 { float2 a, b; };                       // the z-pair (k, k+1)

__device__ __forceinline__ C2 lds4(const float2 *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return C2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ C2 ldg4(const float2 *p)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return C2{make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void st4(float2 *p, C2 c)
{
    *reinterpret_cast<float4 *>(p) = make_float4(c.a.x, c.a.y, c.b.x, c.b.y);
}
__device__ __forceinline__ C2 cmul2(float2 s, C2 c) { return C2{c_mul(s, c.a), c_mul(s, c.b)}; }
__device__ __forceinline__ float2 f_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f_axpy(float s, float2 x, float2 y)      // y + s x
{
    return make_float2(fmaf(s, x.x, y.x), fmaf(s, x.y, y.y));
}
__device__ __forceinline__ float t_rcp(float x)          // hardware reciprocal, as in the split E update
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int TJ, int NS>
struct SG {                                                   // geometry of the radius-streamed tile step
    static constexpr int KP = TILE_KZ / 2;                    // z-pairs of a tile
    static constexpr int EZ = TILE_KZ + 4, HZ = TILE_KZ + 2;  // z extents of the slabs (from k0-2)
    static constexpr int EJ = TJ + 2, HJ = TJ + 1;            // rows of the E slab (j0-1 .. j0+TJ), H slab
    static constexpr int al(int x) { return (x + 15) & ~15; } // 128-byte aligned regions (float2 units)
    static constexpr int ES = al(EJ * EZ), HS = al(HJ * HZ), RW = al(EZ > HZ ? EZ : HZ);
    // one load group: E slab of radius r+1, H slab of radius r (3 components each), and the
    // wrapped rows of edge tiles: E low, E high, H low (3 components each)
    static constexpr int E_OFF = 0, H_OFF = 3 * ES, WEL = H_OFF + 3 * HS, WEH = WEL + 3 * RW, WHL = WEH + 3 * RW;
    static constexpr int GROUP = WHL + 3 * RW;
    static constexpr int NSLOT = NS;                       // ring of load groups (NS - 2 issued ahead)
    // threads: E items (row, pair 1..KP) | H items (row, pair 1..KP) | H z-halo items (row, pair 0)
    static constexpr int NE = TJ * KP, NH = HJ * KP, NHALO = HJ;
    static constexpr int NT = (NE + NH + NHALO + 31) / 32 * 32;
};

// H^{n+1/2} around an E pair (ke, ke+1) at radius i: the pair's own values,
// H_phi / H_r one cell below in z ([0]), the row below in phi (J) and the
// radius below (I).
struct HAround {
    float2 HPk[3], HRk[3];                  // index u + 1 = cell u, [0] = cell ke - 1
    float2 HZk[2], HZJ[2], HRJ[2], HZI[2], HPI[2];
};

// One E item: the z-pair (ke, ke+1) of phi row je, streamed along r.  Holds
// the pair's per-z coefficients; update() applies Eq. 4 (E^{n+1} from the H
// values around the pair) with the E-side CPML, the sheet source and the
// history writes of the time-blocked DFT, and stores the results.  Every
// cell takes the interior coefficient form; the CPML recursions and the
// source add their terms where they apply, so warps that straddle a CPML
// slab edge or the source plane do not run two versions of the update.
struct EItem {
    int je, ke, kze, src_u, dk0;
    bool valid, hist;
    float bzn[2], czn[2], an[2], dn[2], ac[2], dc[2];
    float2 src_pn, src_ph;
    float src_amp;
    float2 *hs;
    size_t plane, ndes;

    __device__ __forceinline__ void init(const StepParams &p, int n, int je_, int ke_)
    {
        je = je_;
        ke = ke_;
        valid = je < p.nphi && ke < p.nz;
        kze = (ke < p.pz) ? ke : ((ke >= p.nz - p.pz) ? ke - (p.nz - 2 * p.pz) : -1);
        src_u = -1;
        src_pn = src_ph = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 2; ++u) { bzn[u] = czn[u] = dn[u] = dc[u] = 0.f; an[u] = ac[u] = 1.f; }
        if (valid) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (kze >= 0) { bzn[u] = __ldg(p.t.bz_n + ke + u); czn[u] = __ldg(p.t.cz_n + ke + u) * p.inv_dz; }
                an[u] = __ldg(p.t.a_n + ke + u); dn[u] = __ldg(p.t.d_n + ke + u);
                ac[u] = __ldg(p.t.a_c + ke + u); dc[u] = __ldg(p.t.d_c + ke + u);
            }
            if (p.src_mode != SRC_NONE && (ke == p.src_k || ke + 1 == p.src_k)) {
                src_u = p.src_k - ke;
                src_pn = p.t.ph_n[je];
                src_ph = p.t.ph_h[je];
            }
        }
        src_amp = p.src_mode == SRC_PLANE_WAVE ? __ldg(p.t.pulse + n) * p.src_scale : 0.f;
        plane = (size_t)p.nr * p.nphi;
        ndes = p.des ? plane * p.des_nk : 0;
        hs = (p.dft_hist && (p.des || p.mon)) ? p.dft_hist + (size_t)(n % DFT_BLOCK) * p.dft_ne : nullptr;
        dk0 = ke - p.des_k0;
        hist = hs && valid && ((p.des && dk0 + 1 >= 0 && dk0 < p.des_nk) || (p.mon && (ke == p.mon_k || ke + 1 == p.mon_k)));
    }

    // per-radius values of an E radius: tab = (1/r_i, 1/r_{i+1/2}, CPML b, c at r_i), rb = rho-bar factors
    __device__ __forceinline__ static float4 tab_at(const StepParams &p, int i)
    {
        return make_float4(__ldg(p.t.inv_r_n + i), __ldg(p.t.inv_r_h + i), __ldg(p.t.br_n + i), __ldg(p.t.cr_n + i));
    }
    __device__ __forceinline__ void rb_at(const StepParams &p, int i, float &a, float &b, float &c) const
    {
        const int ij = i * p.nphi + je;
        a = __ldg(p.rb_r + ij); b = __ldg(p.rb_p + ij); c = __ldg(p.rb_z + ij);
    }

    // E^{n+1}(i) of the pair from E^n (er, ep, ez) and the H values h; stores E into oE
    __device__ __forceinline__ void update(const StepParams &p, int i, const float4 &tab, float rbr, float rbp, float rbz,
                                           const HAround &h, C2 er, C2 ep, C2 ez, float2 *const *oE) const
    {
        const float2 zero = make_float2(0.f, 0.f);
        const int nr = p.nr, nphi = p.nphi, nz = p.nz;
        const float dt = p.dt, cdz = p.inv_dz, cdr = p.inv_dr;
        const float irn = tab.x, irh = tab.y, brn = tab.z, crn = tab.w, crn_dr = tab.w * cdr;
        const int ir = (i < p.pr_in) ? i : ((i >= nr - p.pr_out) ? i - (nr - p.pr_in - p.pr_out) : -1);
        const int ij = i * nphi + je;
        const int zx = ij * (2 * p.pz) + (kze >= 0 ? kze : 0);
        const int rx = ((ir >= 0 ? ir : 0) * nphi + je) * nz + ke;
        float2 *ER[2] = {&er.a, &er.b}, *EP[2] = {&ep.a, &ep.b}, *EZ[2] = {&ez.a, &ez.b};
        C2 ps_r = C2{zero, zero}, ps_p = C2{zero, zero}, ps_pr = C2{zero, zero}, ps_zr = C2{zero, zero};
        if (kze >= 0) { ps_r = ldg4(p.psi.er_z + zx); ps_p = ldg4(p.psi.ep_z + zx); }
        if (ir >= 0) { ps_pr = ldg4(p.psi.ep_r + rx); ps_zr = ldg4(p.psi.ez_r + rx); }
        float2 *PR[2] = {&ps_r.a, &ps_r.b}, *PP[2] = {&ps_p.a, &ps_p.b};
        float2 *PPR[2] = {&ps_pr.a, &ps_pr.b}, *PZR[2] = {&ps_zr.a, &ps_zr.b};
        float2 jr = zero, jp = zero;                          // source current of this radius (cell src_u)
        if (src_u >= 0) {
            if (p.src_mode == SRC_PLANE_WAVE) {
                jr = c_scale(src_pn, src_amp);
                jp = make_float2(-src_ph.y * src_amp, src_ph.x * src_amp);
            } else {
                jr = c_mul(src_pn, p.src_rad[i]);
                jp = c_mul(src_ph, p.src_rad[nr + i]);
            }
        }
        const float cph_h = irh * p.inv_dphi, cph_n = irn * p.inv_dphi, cm = 0.5f * irn;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float cr = dt * t_rcp(an[u] + dn[u] * rbr), cp = dt * t_rcp(an[u] + dn[u] * rbp);
            const float cz = dt * t_rcp(ac[u] + dc[u] * rbz);
            const int kk = ke + u;
            // E_r: (1/r) dH_z/dphi - dH_phi/dz
            const float2 d_hp = f_sub(h.HPk[u + 1], h.HPk[u]);
            float2 t = f_sub(h.HZk[u], h.HZJ[u]);
            float2 a = make_float2(cph_h * t.x, cph_h * t.y);
            a = f_axpy(-cdz, d_hp, a);
            if (kze >= 0 && kk > 0) {
                *PR[u] = f_axpy(czn[u], d_hp, c_scale(*PR[u], bzn[u]));
                a = f_sub(a, *PR[u]);
            }
            // E_phi: dH_r/dz - dH_z/dr
            const float2 d_hr = f_sub(h.HRk[u + 1], h.HRk[u]), d_hzi = f_sub(h.HZk[u], h.HZI[u]);
            float2 b = make_float2(cdz * d_hr.x, cdz * d_hr.y);
            b = f_axpy(-cdr, d_hzi, b);
            const bool upd_p = kk > 0 && i > 0;
            if (kze >= 0 && upd_p) {
                *PP[u] = f_axpy(czn[u], d_hr, c_scale(*PP[u], bzn[u]));
                b = f_add(b, *PP[u]);
            }
            if (ir >= 0 && upd_p) {
                *PPR[u] = f_axpy(crn_dr, d_hzi, c_scale(*PPR[u], brn));
                b = f_sub(b, *PPR[u]);
            }
            if (u == src_u) { a = f_sub(a, jr); b = f_sub(b, jp); }
            if (kk > 0) *ER[u] = f_axpy(cr, a, *ER[u]);
            if (upd_p) *EP[u] = f_axpy(cp, b, *EP[u]);
            // E_z: (1/r) d(r H_phi)/dr - (1/r) dH_r/dphi
            t = f_sub(h.HPk[u + 1], h.HPI[u]);
            float2 c = make_float2(cdr * t.x, cdr * t.y);
            c = f_axpy(cm, f_add(h.HPk[u + 1], h.HPI[u]), c);
            if (ir >= 0 && i > 0) {
                *PZR[u] = f_axpy(crn, c, c_scale(*PZR[u], brn));
                c = f_add(c, *PZR[u]);
            }
            c = f_axpy(-cph_n, f_sub(h.HRk[u + 1], h.HRJ[u]), c);
            if (i > 0) *EZ[u] = f_axpy(cz, c, *EZ[u]);
        }
        const int o = i * (nphi * nz) + je * nz + ke;        // a zone's field < 2^31 cells
        st4(oE[0] + o, er);
        st4(oE[1] + o, ep);
        st4(oE[2] + o, ez);
        if (kze >= 0) { st4(p.psi.er_z + zx, ps_r); st4(p.psi.ep_z + zx, ps_p); }
        if (ir >= 0) { st4(p.psi.ep_r + rx, ps_pr); st4(p.psi.ez_r + rx, ps_zr); }
        if (hist) {                                           // history slot of the time-blocked DFT
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int dk = dk0 + u;
                if (p.des && dk >= 0 && dk < p.des_nk) {
                    const size_t e = (size_t)ij * p.des_nk + dk;
                    hs[e] = *ER[u];
                    hs[ndes + e] = *EP[u];
                    hs[2 * ndes + e] = *EZ[u];
                }
                if (p.mon && ke + u == p.mon_k) {
                    hs[3 * ndes + ij] = *ER[u];
                    hs[3 * ndes + plane + ij] = *EP[u];
                }
            }
        }
    }
};

template <int TJ, int NS, int MINB>
__global__ void __launch_bounds__(SG<TJ, NS>::NT, MINB)
    k_tile_step(const __grid_constant__ TileMaps m, const TileParams tp, const int n, const int i_range)
{
    using G = SG<TJ, NS>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_mem[G::NSLOT + 1];   // + one that nothing completes (tests)
    __shared__ int abort_s;                                   // the error word was already set at entry
    const uint32_t raw_s = s_addr(smem_raw);
    const uint32_t base_s = (raw_s + 127u) & ~127u;
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + (base_s - raw_s));

    const StepParams &p = tp.p;
    const int nr = p.nr, nphi = p.nphi, nz = p.nz;
    const int nzc = (nz + TILE_KZ - 1) / TILE_KZ;
    const int k0 = (blockIdx.x % nzc) * TILE_KZ;
    const int j0 = (blockIdx.x / nzc) * TJ;
    const int ib = blockIdx.y * i_range, ie = min(nr, ib + i_range);
    const int r0 = ib > 0 ? ib - 1 : 0;                       // radius ib-1: H recomputed, nothing stored
    const int tid = threadIdx.x;
    const bool wlo = j0 == 0;                                 // row j0-1 is the wrapped row n_phi-1
    const int s_hi = nphi - j0 + 1;                           // slab row of phi row n_phi (the wrapped row 0)
    const bool whi = s_hi <= TJ + 1;
    const int x = 2 * (k0 - 2);

    // load group g(r) = {E^n(r+1), H^{n-1/2}(r)}, r = r0-1 .. ie-1, in slot (r - r0 + 1) mod NSLOT
    auto slot_of = [&](int r) { return (unsigned)(r - r0 + 1) % (unsigned)G::NSLOT; };
    auto parity_of = [&](int r) { return ((unsigned)(r - r0 + 1) / (unsigned)G::NSLOT) & 1u; };
    auto group = [&](int r) { return sm + slot_of(r) * G::GROUP; };
    auto issue = [&](int r) {
        const unsigned sl = slot_of(r);
        const uint32_t g = base_s + (uint32_t)(sl * G::GROUP) * 8u;
        const uint32_t bar = s_addr(&bar_mem[sl]);
        uint32_t bytes = 3u * (G::EZ * G::EJ + G::HZ * G::HJ) * 8u;
        if (wlo) bytes += 3u * (G::EZ + G::HZ) * 8u;
        if (whi) bytes += 3u * G::EZ * 8u;
        t_mbar_expect_tx(bar, bytes);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            tma3(g + (G::E_OFF + c * G::ES) * 8u, &m.e[c], x, j0 - 1, r + 1, bar);
            tma3(g + (G::H_OFF + c * G::HS) * 8u, &m.h[c], x, j0 - 1, r, bar);
            if (wlo) {
                tma3(g + (G::WEL + c * G::RW) * 8u, &m.ew[c], x, nphi - 1, r + 1, bar);
                tma3(g + (G::WHL + c * G::RW) * 8u, &m.hw[c], x, nphi - 1, r, bar);
            }
            if (whi) tma3(g + (G::WEH + c * G::RW) * 8u, &m.ew[c], x, 0, r + 1, bar);
        }
    };
    // thread 0 alone waits for a group; the block barrier that follows publishes it to the others
    auto wait_group = [&](int r) { return t_mbar_wait(s_addr(&bar_mem[slot_of(r)]), parity_of(r), tp.wait_limit, tp.err); };

    if (tid == 0) {
        for (int s = 0; s <= G::NSLOT; ++s) t_mbar_init(s_addr(&bar_mem[s]), 1);
        // an earlier launch of this run gave up waiting: do nothing (the host reports the error)
        abort_s = *(volatile int *)tp.err;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (abort_s) return;
    // groups g(r0-1) .. g(r0+NSLOT-3) now; g(r+NSLOT-2) after iteration r, into the slot of g(r-2)
    constexpr int AHEAD = G::NSLOT - 2;
    int last_issued = min(ie - 1, r0 + AHEAD - 1);
    bool failed = false;
    if (tid == 0) {
        for (int r = r0 - 1; r <= last_issued; ++r) issue(r);
        if (tp.inject_timeout) failed = !t_mbar_wait(s_addr(&bar_mem[G::NSLOT]), 0, tp.wait_limit, tp.err);
        if (!failed) failed = !wait_group(r0 - 1);            // E^n(r0): read by H(r0)
        if (!failed && r0 < ie) failed = !wait_group(r0);     // E^n(r0+1), H(r0)
    }
    failed = __syncthreads_or(failed);

    const float2 zero = make_float2(0.f, 0.f);
    const float dt = p.dt;
    const int sj = nz, si = nphi * nz;                        // element strides (a zone's field < 2^31 cells)

    if (tid < G::NE) {
        // ================= E items: E^{n+1}(r-1) at iteration r, row se, pair pe (fixed)
        const int se = tid / G::KP + 1, pe = tid % G::KP + 1;
        EItem it;
        it.init(p, n, j0 - 1 + se, k0 - 2 + 2 * pe);
        const int he_own = G::H_OFF + se * G::HZ + 2 * pe, he_jm = G::H_OFF + (se - 1) * G::HZ + 2 * pe;
        const int ee_own = G::E_OFF + se * G::EZ + 2 * pe;
        // per-radius values of the next E radius, loaded one iteration ahead
        float rbr = 0.f, rbp = 0.f, rbz = 0.f, nrbr = 0.f, nrbp = 0.f, nrbz = 0.f;
        float4 tab = make_float4(0.f, 0.f, 0.f, 0.f), ntab = tab;
        if (ib < nr) {
            ntab = EItem::tab_at(p, ib);
            if (it.valid) it.rb_at(p, ib, nrbr, nrbp, nrbz);
        }
        for (int r = r0; r <= ie && !failed; ++r) {
            const int i = r - 1;                              // radius of this iteration's E update
            rbr = nrbr; rbp = nrbp; rbz = nrbz;
            tab = ntab;
            if (i + 1 >= 0 && i + 1 < nr) {
                ntab = EItem::tab_at(p, i + 1);
                if (it.valid) it.rb_at(p, i + 1, nrbr, nrbp, nrbz);
            }
            if (i >= ib && it.valid) {
                const float2 *gq = group(i);                  // H^{n+1/2}(i)
                const float2 *gp = group(i - 1);              // E^n(i), H^{n+1/2}(i-1)
                HAround h;
                const C2 hr = lds4(gq + he_own), hp = lds4(gq + he_own + G::HS), hz = lds4(gq + he_own + 2 * G::HS);
                const C2 hz_jm = lds4(gq + he_jm + 2 * G::HS), hr_jm = lds4(gq + he_jm);
                const C2 hz_im = lds4(gp + he_own + 2 * G::HS), hp_im = lds4(gp + he_own + G::HS);
                h.HPk[0] = gq[he_own + G::HS - 1]; h.HPk[1] = hp.a; h.HPk[2] = hp.b;
                h.HRk[0] = gq[he_own - 1]; h.HRk[1] = hr.a; h.HRk[2] = hr.b;
                h.HZk[0] = hz.a; h.HZk[1] = hz.b;
                h.HZJ[0] = hz_jm.a; h.HZJ[1] = hz_jm.b;
                h.HRJ[0] = hr_jm.a; h.HRJ[1] = hr_jm.b;
                h.HZI[0] = hz_im.a; h.HZI[1] = hz_im.b;
                h.HPI[0] = hp_im.a; h.HPI[1] = hp_im.b;
                it.update(p, i, tab, rbr, rbp, rbz, h, lds4(gp + ee_own), lds4(gp + ee_own + G::ES),
                          lds4(gp + ee_own + 2 * G::ES), tp.oE);
            }
            // g(r+1) landed (thread 0 waits); H(r) published; g(r-2) free.  A wait that
            // gave up ends the loop for every thread.
            if (tid == 0 && r + 1 < ie) failed = !wait_group(r + 1);
            if (__syncthreads_or(failed)) { failed = true; break; }
            if (tid == 0 && r + AHEAD < ie) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(r + AHEAD);
                last_issued = r + AHEAD;
            }
        }
    } else {
        // ================= H items: H^{n+1/2}(r) at iteration r, row sh, pair ph (fixed)
        const int th = tid - G::NE;
        const bool h_on = th < G::NH + G::NHALO;
        const int sh = th < G::NH ? th / G::KP : th - G::NH;
        const int ph = th < G::NH ? th % G::KP + 1 : 0;       // pair 0: the z-halo below the tile
        const int jh = j0 - 1 + sh, kh = k0 - 2 + 2 * ph;
        const bool h_valid = h_on && jh < nphi && kh >= 0 && kh < nz;
        const bool h_own = sh > 0 && ph > 0;
        const bool h_wlo = wlo && sh == 0, h_whi = whi && sh + 1 == s_hi;
        const int jhw = jh < 0 ? jh + nphi : jh;
        const int kzh = (kh < p.pz) ? kh : ((kh >= nz - p.pz) ? kh - (nz - 2 * p.pz) : -1);
        float bzh[2] = {0.f, 0.f}, czh[2] = {0.f, 0.f};
        if (h_valid && kzh >= 0) {
            bzh[0] = __ldg(p.t.bz_h + kh); bzh[1] = __ldg(p.t.bz_h + kh + 1);
            czh[0] = __ldg(p.t.cz_h + kh) * p.inv_dz; czh[1] = __ldg(p.t.cz_h + kh + 1) * p.inv_dz;
        }
        // shared offsets within a group: own row (slab or wrapped-row staging), row + 1
        const int e_own = h_wlo ? G::WEL + 2 * ph : G::E_OFF + sh * G::EZ + 2 * ph;
        const int e_cs = h_wlo ? G::RW : G::ES;               // component stride of that region
        const int e_up = h_whi ? G::WEH + 2 * ph : G::E_OFF + (sh + 1) * G::EZ + 2 * ph;
        const int e_ucs = h_whi ? G::RW : G::ES;
        const int h_rd = h_wlo ? G::WHL + 2 * ph : G::H_OFF + sh * G::HZ + 2 * ph;
        const int h_rcs = h_wlo ? G::RW : G::HS;
        const int h_wr = G::H_OFF + sh * G::HZ + 2 * ph;      // H^{n+1/2} always into the slab
        const float k_z = dt * p.inv_dz, k_r = dt * p.inv_dr;
        float4 tab = make_float4(0.f, 0.f, 0.f, 0.f), ntab = tab;   // 1/r_r, 1/r_{r+1/2}, CPML b, c at r_{r+1/2}
        auto tab_load = [&](int r, float4 &t) {
            if (r >= 0 && r < nr)
                t = make_float4(__ldg(p.t.inv_r_n + r), __ldg(p.t.inv_r_h + r), __ldg(p.t.br_h + r), __ldg(p.t.cr_h + r));
        };
        tab_load(r0, ntab);
        for (int r = r0; r <= ie && !failed; ++r) {
            tab = ntab;
            tab_load(r + 1, ntab);
            if (r < ie && h_valid) {
                const float2 *gp = group(r - 1);              // E^n(r)
                float2 *gc = group(r);                        // E^n(r+1), H(r)
                const float irn = tab.x, irh = tab.y;
                const int ir = (r < p.pr_in) ? r : ((r >= nr - p.pr_out) ? r - (nr - p.pr_in - p.pr_out) : -1);
                const C2 er = lds4(gp + e_own), ep = lds4(gp + e_own + e_cs), ez = lds4(gp + e_own + 2 * e_cs);
                const float2 ep_k2 = gp[e_own + e_cs + 2], er_k2 = gp[e_own + 2];
                const C2 ez_jp = lds4(gp + e_up + 2 * e_ucs), er_jp = lds4(gp + e_up);
                const C2 ez_ip = lds4(gc + e_own + 2 * e_cs), ep_ip = lds4(gc + e_own + e_cs);
                C2 hr = lds4(gc + h_rd), hp = lds4(gc + h_rd + h_rcs), hz = lds4(gc + h_rd + 2 * h_rcs);
                float2 EP[3] = {ep.a, ep.b, ep_k2}, ER[3] = {er.a, er.b, er_k2};
                float2 EZ[2] = {ez.a, ez.b}, EZJ[2] = {ez_jp.a, ez_jp.b}, ERJ[2] = {er_jp.a, er_jp.b};
                float2 EZI[2] = {ez_ip.a, ez_ip.b}, EPI[2] = {ep_ip.a, ep_ip.b};
                if (h_wlo) {                                  // row n_phi-1 seen from the wedge's low side
#pragma unroll
                    for (int u = 0; u < 3; ++u) { EP[u] = c_mul(p.bloch_inv, EP[u]); ER[u] = c_mul(p.bloch_inv, ER[u]); }
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        EZ[u] = c_mul(p.bloch_inv, EZ[u]); EZI[u] = c_mul(p.bloch_inv, EZI[u]);
                        EPI[u] = c_mul(p.bloch_inv, EPI[u]);
                    }
                    hr = cmul2(p.bloch_inv, hr); hp = cmul2(p.bloch_inv, hp); hz = cmul2(p.bloch_inv, hz);
                }
                if (h_whi) {                                  // row 0 seen from the wedge's high side
#pragma unroll
                    for (int u = 0; u < 2; ++u) { EZJ[u] = c_mul(p.bloch, EZJ[u]); ERJ[u] = c_mul(p.bloch, ERJ[u]); }
                }
                const int zx = (r * nphi + jhw) * (2 * p.pz) + (kzh >= 0 ? kzh : 0);
                const int rx = ((ir >= 0 ? ir : 0) * nphi + jhw) * nz + kh;
                C2 ps_r = C2{zero, zero}, ps_p = C2{zero, zero}, ps_pr = C2{zero, zero}, ps_zr = C2{zero, zero};
                if (kzh >= 0) {
                    ps_r = ldg4(tp.psH_in[0] + zx);
                    ps_p = ldg4(tp.psH_in[1] + zx);
                    if (h_wlo) { ps_r = cmul2(p.bloch_inv, ps_r); ps_p = cmul2(p.bloch_inv, ps_p); }
                }
                const float brh = tab.z, crh = tab.w * p.inv_dr;
                if (ir >= 0) {
                    ps_pr = ldg4(tp.psH_in[2] + rx);
                    ps_zr = ldg4(tp.psH_in[3] + rx);
                    if (h_wlo) { ps_pr = cmul2(p.bloch_inv, ps_pr); ps_zr = cmul2(p.bloch_inv, ps_zr); }
                }
                float2 *HR[2] = {&hr.a, &hr.b}, *HP[2] = {&hp.a, &hp.b}, *HZ[2] = {&hz.a, &hz.b};
                float2 *PR[2] = {&ps_r.a, &ps_r.b}, *PP[2] = {&ps_p.a, &ps_p.b};
                float2 *PPR[2] = {&ps_pr.a, &ps_pr.b}, *PZR[2] = {&ps_zr.a, &ps_zr.b};
                // one coefficient form for every cell; the CPML recursions add their terms where they apply
                const float k_phn = dt * irn * p.inv_dphi, k_m = 0.5f * dt * irh, k_phh = dt * irh * p.inv_dphi;
                const float c_m = 0.5f * irh * tab.w;
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float2 d_ep = f_sub(EP[u + 1], EP[u]), d_er = f_sub(ER[u + 1], ER[u]);
                    const float2 d_ezi = f_sub(EZI[u], EZ[u]), d_epi = f_sub(EPI[u], EP[u]);
                    const float2 s_epi = f_add(EPI[u], EP[u]);
                    // H_r
                    *HR[u] = f_axpy(-k_phn, f_sub(EZJ[u], EZ[u]), *HR[u]);
                    *HR[u] = f_axpy(k_z, d_ep, *HR[u]);
                    // H_phi
                    *HP[u] = f_axpy(-k_z, d_er, *HP[u]);
                    *HP[u] = f_axpy(k_r, d_ezi, *HP[u]);
                    if (kzh >= 0) {
                        *PR[u] = f_axpy(czh[u], d_ep, c_scale(*PR[u], bzh[u]));
                        *PP[u] = f_axpy(czh[u], d_er, c_scale(*PP[u], bzh[u]));
                        *HR[u] = f_axpy(dt, *PR[u], *HR[u]);
                        *HP[u] = f_axpy(-dt, *PP[u], *HP[u]);
                    }
                    // H_z
                    *HZ[u] = f_axpy(-k_r, d_epi, *HZ[u]);
                    *HZ[u] = f_axpy(-k_m, s_epi, *HZ[u]);
                    *HZ[u] = f_axpy(k_phh, f_sub(ERJ[u], ER[u]), *HZ[u]);
                    if (ir >= 0) {
                        *PPR[u] = f_axpy(crh, d_ezi, c_scale(*PPR[u], brh));
                        *PZR[u] = f_axpy(c_m, s_epi, f_axpy(crh, d_epi, c_scale(*PZR[u], brh)));
                        *HP[u] = f_axpy(dt, *PPR[u], *HP[u]);
                        *HZ[u] = f_axpy(-dt, *PZR[u], *HZ[u]);
                    }
                }
                st4(gc + h_wr, hr);
                st4(gc + h_wr + G::HS, hp);
                st4(gc + h_wr + 2 * G::HS, hz);
                if (h_own && r >= ib) {
                    const int o = r * si + jh * sj + kh;
                    st4(tp.oH[0] + o, hr);
                    st4(tp.oH[1] + o, hp);
                    st4(tp.oH[2] + o, hz);
                    if (kzh >= 0) { st4(tp.psH_out[0] + zx, ps_r); st4(tp.psH_out[1] + zx, ps_p); }
                    if (ir >= 0) { st4(tp.psH_out[2] + rx, ps_pr); st4(tp.psH_out[3] + rx, ps_zr); }
                }
            }
            if (__syncthreads_or(failed)) { failed = true; break; }   // matches the E warps' barrier
        }
    }
    if (failed && tid == 0)                                   // copies still in flight
        for (int r = max(r0 - 1, last_issued - G::NSLOT + 1); r <= last_issued; ++r) wait_group(r);
}

// ---------------------------------------------------------------- E update on TMA-staged tiles
// The E half of the split step as a radius-streamed tile kernel: the split
// H update (zda_pair.cu) has written H^{n+1/2}; this kernel reads it
// together with E^n through a ring of TMA load groups, so its loads are in
// flight several radii ahead of the arithmetic instead of one round trip per
// thread, and updates E in place.  Load group g(r) = {H^{n+1/2}(r) rows
// j0-1 .. j0+TJ-1 and z k0-2 .. k0+31, E^n(r) rows j0 .. j0+TJ-1 and z
// k0 .. k0+31, and for the tile at phi row 0 the wrapped H row n_phi-1};
// iteration r updates E(r) from g(r) and g(r-1).  After iteration r thread
// 0 waits for g(r+1) and the block barrier publishes it; then g(r+NSLOT-1)
// is issued into the slot of g(r-1).  The E box covers the tile's own cells
// only (no other CTA writes them), so reading E^n and writing E^{n+1} in
// the same buffer is safe; the group at r = ib-1 (the radius below the
// range, read for its H) carries no E box.
template <int TJ, int NS>
struct SE {                                                   // geometry of the E tile kernel
    static constexpr int KP = TILE_KZ / 2;                    // z-pairs of a tile
    static constexpr int HZ = TILE_KZ + 2, HJ = TJ + 1;       // H slab: z from k0-2, rows from j0-1
    static constexpr int al(int x) { return (x + 15) & ~15; } // 128-byte aligned regions (float2 units)
    static constexpr int HS = al(HJ * HZ), ES = al(TJ * TILE_KZ), RW = al(HZ);
    static constexpr int H_OFF = 0, E_OFF = 3 * HS, WHL = E_OFF + 3 * ES;
    static constexpr int GROUP = WHL + 3 * RW;
    static constexpr int NSLOT = NS;
    static constexpr int NT = TJ * KP;                        // one E item (z-pair) per thread
};

template <int TJ, int NS, int MINB>
__global__ void __launch_bounds__(SE<TJ, NS>::NT, MINB)
    k_tile_e(const __grid_constant__ TileEMaps m, const TileParams tp, const int n, const int i_range)
{
    using G = SE<TJ, NS>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_mem[G::NSLOT + 1];   // + one that nothing completes (tests)
    __shared__ int abort_s;
    const uint32_t raw_s = s_addr(smem_raw);
    const uint32_t base_s = (raw_s + 127u) & ~127u;
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + (base_s - raw_s));

    const StepParams &p = tp.p;
    const int nr = p.nr, nphi = p.nphi, nz = p.nz;
    const int nzc = (nz + TILE_KZ - 1) / TILE_KZ;
    const int k0 = (blockIdx.x % nzc) * TILE_KZ;
    const int j0 = (blockIdx.x / nzc) * TJ;
    const int ib = blockIdx.y * i_range, ie = min(nr, ib + i_range);
    const int tid = threadIdx.x;
    const bool wlo = j0 == 0;                                 // row j0-1 is the wrapped row n_phi-1
    const int xh = 2 * (k0 - 2), xe = 2 * k0;

    auto slot_of = [&](int r) { return (unsigned)(r - ib + 1) % (unsigned)G::NSLOT; };
    auto parity_of = [&](int r) { return ((unsigned)(r - ib + 1) / (unsigned)G::NSLOT) & 1u; };
    auto group = [&](int r) { return sm + slot_of(r) * G::GROUP; };
    auto issue = [&](int r) {
        const unsigned sl = slot_of(r);
        const uint32_t g = base_s + (uint32_t)(sl * G::GROUP) * 8u;
        const uint32_t bar = s_addr(&bar_mem[sl]);
        const bool with_e = r >= ib;
        uint32_t bytes = 3u * G::HZ * G::HJ * 8u;
        if (with_e) bytes += 3u * TILE_KZ * TJ * 8u;
        if (wlo) bytes += 3u * G::HZ * 8u;
        t_mbar_expect_tx(bar, bytes);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            tma3(g + (G::H_OFF + c * G::HS) * 8u, &m.h[c], xh, j0 - 1, r, bar);
            if (with_e) tma3(g + (G::E_OFF + c * G::ES) * 8u, &m.eo[c], xe, j0, r, bar);
            if (wlo) tma3(g + (G::WHL + c * G::RW) * 8u, &m.hw[c], xh, nphi - 1, r, bar);
        }
    };
    auto wait_group = [&](int r) { return t_mbar_wait(s_addr(&bar_mem[slot_of(r)]), parity_of(r), tp.wait_limit, tp.err); };

    if (tid == 0) {
        for (int s = 0; s <= G::NSLOT; ++s) t_mbar_init(s_addr(&bar_mem[s]), 1);
        abort_s = *(volatile int *)tp.err;                    // an earlier launch gave up waiting: do nothing
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (abort_s) return;
    // groups g(ib-1) .. g(ib+NSLOT-2) now (every slot); g(r+NSLOT-1) after iteration r
    constexpr int AHEAD = G::NSLOT - 1;
    int last_issued = min(ie - 1, ib - 1 + AHEAD);
    bool failed = false;
    if (tid == 0) {
        for (int r = ib - 1; r <= last_issued; ++r) issue(r);
        if (tp.inject_timeout) failed = !t_mbar_wait(s_addr(&bar_mem[G::NSLOT]), 0, tp.wait_limit, tp.err);
        if (!failed) failed = !wait_group(ib - 1);
        if (!failed && ib < ie) failed = !wait_group(ib);
    }
    failed = __syncthreads_or(failed);

    const int se = tid / G::KP, pe = tid % G::KP;
    EItem it;
    it.init(p, n, j0 + se, k0 + 2 * pe);
    const bool jm_wrap = wlo && se == 0;                      // row below is the wrapped row (Bloch phase)
    const int h_own = G::H_OFF + (se + 1) * G::HZ + 2 + 2 * pe;
    const int h_jm = jm_wrap ? G::WHL + 2 + 2 * pe : G::H_OFF + se * G::HZ + 2 + 2 * pe;
    const int jm_cs = jm_wrap ? G::RW : G::HS;                // component stride of that row's region
    const int e_own = G::E_OFF + se * TILE_KZ + 2 * pe;
    float rbr = 0.f, rbp = 0.f, rbz = 0.f, nrbr = 0.f, nrbp = 0.f, nrbz = 0.f;
    float4 tab = make_float4(0.f, 0.f, 0.f, 0.f), ntab = tab;
    if (ib < ie) {
        ntab = EItem::tab_at(p, ib);
        if (it.valid) it.rb_at(p, ib, nrbr, nrbp, nrbz);
    }
    for (int r = ib; r < ie && !failed; ++r) {
        rbr = nrbr; rbp = nrbp; rbz = nrbz;
        tab = ntab;
        if (r + 1 < ie) {                                     // next radius, one iteration ahead
            ntab = EItem::tab_at(p, r + 1);
            if (it.valid) it.rb_at(p, r + 1, nrbr, nrbp, nrbz);
        }
        if (it.valid) {
            const float2 *gq = group(r);                      // H^{n+1/2}(r), E^n(r)
            const float2 *gp = group(r - 1);                  // H^{n+1/2}(r-1)
            HAround h;
            const C2 hr = lds4(gq + h_own), hp = lds4(gq + h_own + G::HS), hz = lds4(gq + h_own + 2 * G::HS);
            C2 hz_jm = lds4(gq + h_jm + 2 * jm_cs), hr_jm = lds4(gq + h_jm);
            if (jm_wrap) { hz_jm = cmul2(p.bloch_inv, hz_jm); hr_jm = cmul2(p.bloch_inv, hr_jm); }
            const C2 hz_im = lds4(gp + h_own + 2 * G::HS), hp_im = lds4(gp + h_own + G::HS);
            h.HPk[0] = gq[h_own + G::HS - 1]; h.HPk[1] = hp.a; h.HPk[2] = hp.b;
            h.HRk[0] = gq[h_own - 1]; h.HRk[1] = hr.a; h.HRk[2] = hr.b;
            h.HZk[0] = hz.a; h.HZk[1] = hz.b;
            h.HZJ[0] = hz_jm.a; h.HZJ[1] = hz_jm.b;
            h.HRJ[0] = hr_jm.a; h.HRJ[1] = hr_jm.b;
            h.HZI[0] = hz_im.a; h.HZI[1] = hz_im.b;
            h.HPI[0] = hp_im.a; h.HPI[1] = hp_im.b;
            it.update(p, r, tab, rbr, rbp, rbz, h, lds4(gq + e_own), lds4(gq + e_own + G::ES),
                      lds4(gq + e_own + 2 * G::ES), tp.oE);
        }
        if (tid == 0 && r + 1 < ie) failed = !wait_group(r + 1);
        if (__syncthreads_or(failed)) { failed = true; break; }
        if (tid == 0 && r + AHEAD < ie) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(r + AHEAD);
            last_issued = r + AHEAD;
        }
    }
    if (failed && tid == 0)                                   // copies still in flight
        for (int r = max(ib - 1, last_issued - G::NSLOT + 1); r <= last_issued; ++r) wait_group(r);
}

// ---------------------------------------------------------------- H update on TMA-staged tiles
// E^n around an H pair (kh, kh+1) at radius r: the pair's own values and
// E_phi / E_r one cell above in z ([2]), the row above in phi (J) and the
// radius above (I).
struct EAround {
    float2 EP[3], ER[3];                    // index u = cell u, [2] = cell kh + 2
    float2 EZ[2], EZJ[2], ERJ[2], EZI[2], EPI[2];
};

// One H item: the z-pair (kh, kh+1) of phi row jh, streamed along r.
// update() applies Eq. 3 (H^{n+1/2} from the E values around the pair) with
// the H-side CPML in the same single coefficient form as the E items, and
// stores H and the auxiliaries in place.
struct HItem {
    int jh, kh, kzh;
    bool valid;
    float bzh[2], czh[2];

    __device__ __forceinline__ void init(const StepParams &p, int jh_, int kh_)
    {
        jh = jh_;
        kh = kh_;
        valid = jh < p.nphi && kh < p.nz;
        kzh = (kh < p.pz) ? kh : ((kh >= p.nz - p.pz) ? kh - (p.nz - 2 * p.pz) : -1);
        bzh[0] = bzh[1] = czh[0] = czh[1] = 0.f;
        if (valid && kzh >= 0) {
#pragma unroll
            for (int u = 0; u < 2; ++u) { bzh[u] = __ldg(p.t.bz_h + kh + u); czh[u] = __ldg(p.t.cz_h + kh + u) * p.inv_dz; }
        }
    }

    // per-radius values of an H radius: (1/r_r, 1/r_{r+1/2}, CPML b, c at r_{r+1/2})
    __device__ __forceinline__ static float4 tab_at(const StepParams &p, int r)
    {
        return make_float4(__ldg(p.t.inv_r_n + r), __ldg(p.t.inv_r_h + r), __ldg(p.t.br_h + r), __ldg(p.t.cr_h + r));
    }

    __device__ __forceinline__ void update(const StepParams &p, int r, const float4 &tab, const EAround &e, C2 hr, C2 hp,
                                           C2 hz, float2 *const *oH) const
    {
        const float2 zero = make_float2(0.f, 0.f);
        const int nr = p.nr, nphi = p.nphi, nz = p.nz;
        const float dt = p.dt, k_z = dt * p.inv_dz, k_r = dt * p.inv_dr;
        const float irn = tab.x, irh = tab.y, brh = tab.z, crh = tab.w * p.inv_dr;
        const int ir = (r < p.pr_in) ? r : ((r >= nr - p.pr_out) ? r - (nr - p.pr_in - p.pr_out) : -1);
        const int zx = (r * nphi + jh) * (2 * p.pz) + (kzh >= 0 ? kzh : 0);
        const int rx = ((ir >= 0 ? ir : 0) * nphi + jh) * nz + kh;
        C2 ps_r = C2{zero, zero}, ps_p = C2{zero, zero}, ps_pr = C2{zero, zero}, ps_zr = C2{zero, zero};
        if (kzh >= 0) { ps_r = ldg4(p.psi.hr_z + zx); ps_p = ldg4(p.psi.hp_z + zx); }
        if (ir >= 0) { ps_pr = ldg4(p.psi.hp_r + rx); ps_zr = ldg4(p.psi.hz_r + rx); }
        float2 *HR[2] = {&hr.a, &hr.b}, *HP[2] = {&hp.a, &hp.b}, *HZ[2] = {&hz.a, &hz.b};
        float2 *PR[2] = {&ps_r.a, &ps_r.b}, *PP[2] = {&ps_p.a, &ps_p.b};
        float2 *PPR[2] = {&ps_pr.a, &ps_pr.b}, *PZR[2] = {&ps_zr.a, &ps_zr.b};
        const float k_phn = dt * irn * p.inv_dphi, k_m = 0.5f * dt * irh, k_phh = dt * irh * p.inv_dphi;
        const float c_m = 0.5f * irh * tab.w;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float2 d_ep = f_sub(e.EP[u + 1], e.EP[u]), d_er = f_sub(e.ER[u + 1], e.ER[u]);
            const float2 d_ezi = f_sub(e.EZI[u], e.EZ[u]), d_epi = f_sub(e.EPI[u], e.EP[u]);
            const float2 s_epi = f_add(e.EPI[u], e.EP[u]);
            // H_r: -(1/r) dE_z/dphi + dE_phi/dz
            *HR[u] = f_axpy(-k_phn, f_sub(e.EZJ[u], e.EZ[u]), *HR[u]);
            *HR[u] = f_axpy(k_z, d_ep, *HR[u]);
            // H_phi: -dE_r/dz + dE_z/dr
            *HP[u] = f_axpy(-k_z, d_er, *HP[u]);
            *HP[u] = f_axpy(k_r, d_ezi, *HP[u]);
            if (kzh >= 0) {
                *PR[u] = f_axpy(czh[u], d_ep, c_scale(*PR[u], bzh[u]));
                *PP[u] = f_axpy(czh[u], d_er, c_scale(*PP[u], bzh[u]));
                *HR[u] = f_axpy(dt, *PR[u], *HR[u]);
                *HP[u] = f_axpy(-dt, *PP[u], *HP[u]);
            }
            // H_z: -(1/r) d(r E_phi)/dr + (1/r) dE_r/dphi
            *HZ[u] = f_axpy(-k_r, d_epi, *HZ[u]);
            *HZ[u] = f_axpy(-k_m, s_epi, *HZ[u]);
            *HZ[u] = f_axpy(k_phh, f_sub(e.ERJ[u], e.ER[u]), *HZ[u]);
            if (ir >= 0) {
                *PPR[u] = f_axpy(crh, d_ezi, c_scale(*PPR[u], brh));
                *PZR[u] = f_axpy(c_m, s_epi, f_axpy(crh, d_epi, c_scale(*PZR[u], brh)));
                *HP[u] = f_axpy(dt, *PPR[u], *HP[u]);
                *HZ[u] = f_axpy(-dt, *PZR[u], *HZ[u]);
            }
        }
        const int o = r * (nphi * nz) + jh * nz + kh;
        st4(oH[0] + o, hr);
        st4(oH[1] + o, hp);
        st4(oH[2] + o, hz);
        if (kzh >= 0) { st4(p.psi.hr_z + zx, ps_r); st4(p.psi.hp_z + zx, ps_p); }
        if (ir >= 0) { st4(p.psi.hp_r + rx, ps_pr); st4(p.psi.hz_r + rx, ps_zr); }
    }
};

// The H half of the split step as a radius-streamed tile kernel (the
// counterpart of k_tile_e): load group g(r) = {E^n(r) rows j0 .. j0+TJ and
// z k0 .. k0+33, H^{n-1/2}(r) over the tile's own cells, and for the tile
// holding phi row n_phi-1 the wrapped E row 0}; iteration r updates H(r)
// from g(r) and g(r+1) (E at the radius above), in place.  Groups run over
// r = ib .. ie (the last one, read for its E only, carries no H box).
template <int TJ, int NS>
struct SH {
    static constexpr int KP = TILE_KZ / 2;
    static constexpr int EZ = TILE_KZ + 2, EJ = TJ + 1;       // E slab: z from k0, rows from j0
    static constexpr int al(int x) { return (x + 15) & ~15; }
    static constexpr int ES = al(EJ * EZ), HS = al(TJ * TILE_KZ), RW = al(EZ);
    static constexpr int E_OFF = 0, H_OFF = 3 * ES, WEH = H_OFF + 3 * HS;
    static constexpr int GROUP = WEH + 3 * RW;
    static constexpr int NSLOT = NS;
    static constexpr int NT = TJ * KP;
};

template <int TJ, int NS, int MINB>
__global__ void __launch_bounds__(SH<TJ, NS>::NT, MINB)
    k_tile_h(const __grid_constant__ TileHMaps m, const TileParams tp, const int i_range)
{
    using G = SH<TJ, NS>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_mem[G::NSLOT + 1];   // + one that nothing completes (tests)
    __shared__ int abort_s;
    const uint32_t raw_s = s_addr(smem_raw);
    const uint32_t base_s = (raw_s + 127u) & ~127u;
    float2 *sm = reinterpret_cast<float2 *>(smem_raw + (base_s - raw_s));

    const StepParams &p = tp.p;
    const int nr = p.nr, nphi = p.nphi, nz = p.nz;
    const int nzc = (nz + TILE_KZ - 1) / TILE_KZ;
    const int k0 = (blockIdx.x % nzc) * TILE_KZ;
    const int j0 = (blockIdx.x / nzc) * TJ;
    const int ib = blockIdx.y * i_range, ie = min(nr, ib + i_range);
    const int tid = threadIdx.x;
    const int s_hi = nphi - j0;                               // slab row of phi row n_phi (the wrapped row 0)
    const bool whi = s_hi <= TJ;
    const int x = 2 * k0;

    auto slot_of = [&](int r) { return (unsigned)(r - ib) % (unsigned)G::NSLOT; };
    auto parity_of = [&](int r) { return ((unsigned)(r - ib) / (unsigned)G::NSLOT) & 1u; };
    auto group = [&](int r) { return sm + slot_of(r) * G::GROUP; };
    auto issue = [&](int r) {
        const unsigned sl = slot_of(r);
        const uint32_t g = base_s + (uint32_t)(sl * G::GROUP) * 8u;
        const uint32_t bar = s_addr(&bar_mem[sl]);
        const bool with_h = r < ie;
        uint32_t bytes = 3u * G::EZ * G::EJ * 8u;
        if (with_h) bytes += 3u * TILE_KZ * TJ * 8u;
        if (whi) bytes += 3u * G::EZ * 8u;
        t_mbar_expect_tx(bar, bytes);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            tma3(g + (G::E_OFF + c * G::ES) * 8u, &m.e[c], x, j0, r, bar);
            if (with_h) tma3(g + (G::H_OFF + c * G::HS) * 8u, &m.ho[c], x, j0, r, bar);
            if (whi) tma3(g + (G::WEH + c * G::RW) * 8u, &m.ew[c], x, 0, r, bar);
        }
    };
    auto wait_group = [&](int r) { return t_mbar_wait(s_addr(&bar_mem[slot_of(r)]), parity_of(r), tp.wait_limit, tp.err); };

    if (tid == 0) {
        for (int s = 0; s <= G::NSLOT; ++s) t_mbar_init(s_addr(&bar_mem[s]), 1);
        abort_s = *(volatile int *)tp.err;                    // an earlier launch gave up waiting: do nothing
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (abort_s) return;
    // groups g(ib) .. g(ib+NSLOT-1) now (every slot); g(r+NSLOT) after iteration r
    int last_issued = min(ie, ib + G::NSLOT - 1);
    bool failed = false;
    if (tid == 0) {
        for (int r = ib; r <= last_issued; ++r) issue(r);
        if (tp.inject_timeout) failed = !t_mbar_wait(s_addr(&bar_mem[G::NSLOT]), 0, tp.wait_limit, tp.err);
        if (!failed) failed = !wait_group(ib);
        if (!failed) failed = !wait_group(ib + 1);            // ib + 1 <= ie always
    }
    failed = __syncthreads_or(failed);

    const int se = tid / G::KP, pe = tid % G::KP;
    HItem it;
    it.init(p, j0 + se, k0 + 2 * pe);
    const bool jp_wrap = whi && se + 1 == s_hi;               // row above is the wrapped row (Bloch phase)
    const int e_own = G::E_OFF + se * G::EZ + 2 * pe;
    const int e_up = jp_wrap ? G::WEH + 2 * pe : G::E_OFF + (se + 1) * G::EZ + 2 * pe;
    const int up_cs = jp_wrap ? G::RW : G::ES;
    const int h_own = G::H_OFF + se * TILE_KZ + 2 * pe;
    float4 tab = make_float4(0.f, 0.f, 0.f, 0.f), ntab = HItem::tab_at(p, ib);
    for (int r = ib; r < ie && !failed; ++r) {
        tab = ntab;
        if (r + 1 < ie) ntab = HItem::tab_at(p, r + 1);       // next radius, one iteration ahead
        if (it.valid) {
            const float2 *gq = group(r);                      // E^n(r), H^{n-1/2}(r)
            const float2 *gn = group(r + 1);                  // E^n(r+1)
            EAround e;
            const C2 er = lds4(gq + e_own), ep = lds4(gq + e_own + G::ES), ez = lds4(gq + e_own + 2 * G::ES);
            C2 ez_jp = lds4(gq + e_up + 2 * up_cs), er_jp = lds4(gq + e_up);
            if (jp_wrap) { ez_jp = cmul2(p.bloch, ez_jp); er_jp = cmul2(p.bloch, er_jp); }
            const C2 ez_ip = lds4(gn + e_own + 2 * G::ES), ep_ip = lds4(gn + e_own + G::ES);
            e.EP[0] = ep.a; e.EP[1] = ep.b; e.EP[2] = gq[e_own + G::ES + 2];
            e.ER[0] = er.a; e.ER[1] = er.b; e.ER[2] = gq[e_own + 2];
            e.EZ[0] = ez.a; e.EZ[1] = ez.b;
            e.EZJ[0] = ez_jp.a; e.EZJ[1] = ez_jp.b;
            e.ERJ[0] = er_jp.a; e.ERJ[1] = er_jp.b;
            e.EZI[0] = ez_ip.a; e.EZI[1] = ez_ip.b;
            e.EPI[0] = ep_ip.a; e.EPI[1] = ep_ip.b;
            it.update(p, r, tab, e, lds4(gq + h_own), lds4(gq + h_own + G::HS), lds4(gq + h_own + 2 * G::HS), tp.oH);
        }
        if (tid == 0 && r + 2 <= ie) failed = !wait_group(r + 2);
        if (__syncthreads_or(failed)) { failed = true; break; }
        if (tid == 0 && r + G::NSLOT <= ie) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(r + G::NSLOT);
            last_issued = r + G::NSLOT;
        }
    }
    if (failed && tid == 0)                                   // copies still in flight
        for (int r = max(ib, last_issued - G::NSLOT + 1); r <= last_issued; ++r) wait_group(r);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

template <int TJ, int NS, int MINB>
cudaError_t launch_shape(const TileMaps &m, const TileParams &tp, int n, int n_rchunks, cudaStream_t s)
{
    using G = SG<TJ, NS>;
    const size_t bytes = (size_t)G::NSLOT * G::GROUP * sizeof(float2) + 128;
    int dev = 0;
    cudaGetDevice(&dev);
    static unsigned attr_done = 0;                            // per device (bit), set once
    if (dev < 32 && !(attr_done & (1u << dev))) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_step<TJ, NS, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (e != cudaSuccess) return e;
        attr_done |= 1u << dev;
    }
    const int nzc = (tp.p.nz + TILE_KZ - 1) / TILE_KZ, njt = (tp.p.nphi + TJ - 1) / TJ;
    const int nrc = std::max(1, std::min(n_rchunks, tp.p.nr));
    const int i_range = (tp.p.nr + nrc - 1) / nrc;
    dim3 g((unsigned)(nzc * njt), (unsigned)((tp.p.nr + i_range - 1) / i_range));
    k_tile_step<TJ, NS, MINB><<<g, G::NT, bytes, s>>>(m, tp, n, i_range);
    return cudaGetLastError();
}


template <int TJ, int NS, int MINB>
cudaError_t launch_e_shape(const TileEMaps &m, const TileParams &tp, int n, int n_rchunks, cudaStream_t s)
{
    using G = SE<TJ, NS>;
    const size_t bytes = (size_t)G::NSLOT * G::GROUP * sizeof(float2) + 128;
    int dev = 0;
    cudaGetDevice(&dev);
    static unsigned attr_done = 0;                            // per device (bit), set once
    if (dev < 32 && !(attr_done & (1u << dev))) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_e<TJ, NS, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (e != cudaSuccess) return e;
        attr_done |= 1u << dev;
    }
    const int nzc = (tp.p.nz + TILE_KZ - 1) / TILE_KZ, njt = (tp.p.nphi + TJ - 1) / TJ;
    const int nrc = std::max(1, std::min(n_rchunks, tp.p.nr));
    const int i_range = (tp.p.nr + nrc - 1) / nrc;
    dim3 g((unsigned)(nzc * njt), (unsigned)((tp.p.nr + i_range - 1) / i_range));
    k_tile_e<TJ, NS, MINB><<<g, G::NT, bytes, s>>>(m, tp, n, i_range);
    return cudaGetLastError();
}

template <int TJ, int NS, int MINB>
cudaError_t launch_h_shape(const TileHMaps &m, const TileParams &tp, int n_rchunks, cudaStream_t s)
{
    using G = SH<TJ, NS>;
    const size_t bytes = (size_t)G::NSLOT * G::GROUP * sizeof(float2) + 128;
    int dev = 0;
    cudaGetDevice(&dev);
    static unsigned attr_done = 0;                            // per device (bit), set once
    if (dev < 32 && !(attr_done & (1u << dev))) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_h<TJ, NS, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (e != cudaSuccess) return e;
        attr_done |= 1u << dev;
    }
    const int nzc = (tp.p.nz + TILE_KZ - 1) / TILE_KZ, njt = (tp.p.nphi + TJ - 1) / TJ;
    const int nrc = std::max(1, std::min(n_rchunks, tp.p.nr));
    const int i_range = (tp.p.nr + nrc - 1) / nrc;
    dim3 g((unsigned)(nzc * njt), (unsigned)((tp.p.nr + i_range - 1) / i_range));
    k_tile_h<TJ, NS, MINB><<<g, G::NT, bytes, s>>>(m, tp, i_range);
    return cudaGetLastError();
}

template <int TJ, int NS>
size_t e_shape_bytes() { return (size_t)SE<TJ, NS>::NSLOT * SE<TJ, NS>::GROUP * sizeof(float2) + 128; }

template <int TJ, int NS>
size_t shape_bytes() { return (size_t)SG<TJ, NS>::NSLOT * SG<TJ, NS>::GROUP * sizeof(float2) + 128; }

}  // namespace

// compiled shapes (phi rows: ring slots, thread blocks per SM the registers are sized for):
// 4: 5, 3;  8: 4, 2;  16: 4, 1 -- the measured best ring depth of each
bool tile_shape_ok(int tj) { return tj == 4 || tj == 8 || tj == 16; }

size_t tile_smem_bytes(int tj)
{
    if (tj == 4) return shape_bytes<4, 5>();
    if (tj == 8) return shape_bytes<8, 4>();
    if (tj == 16) return shape_bytes<16, 4>();
    return 0;
}

int tile_blocks_per_sm(int tj)
{
    const size_t b = tile_smem_bytes(tj);
    return b ? (int)std::min<size_t>(8, (227 * 1024) / (b + 1024)) : 0;
}

int tile_auto_rchunks(int tj, int nr, int nphi, int nz, int sms)
{
    const int per_wave = sms * std::max(1, tile_blocks_per_sm(tj));
    const int tiles = ((nz + TILE_KZ - 1) / TILE_KZ) * ((nphi + tj - 1) / tj);
    // radius chunks of about 21 radii (the measured optimum on a 300-radius zone: shorter chunks
    // recompute more halo radii, longer ones leave too few blocks to balance the SMs), at least four
    // waves of thread blocks and at least 8 radii per chunk
    const int waves4 = (4 * per_wave + tiles - 1) / std::max(tiles, 1);
    const int c = std::max(waves4, (nr + 10) / 21);
    return std::max(1, std::min(c, nr / 8));
}

bool encode_tile_maps(TileMaps *m, float2 *const E[3], float2 *const H[3], int nr, int nphi, int nz, int tj,
                      const char **why)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) {
        *why = "the driver's cuTensorMapEncodeTiled is not available";
        return false;
    }
    // FP32 view: x = 2 k (+1 for the imaginary part), y = phi row, z = radius
    const cuuint64_t dims[3] = {2ull * (cuuint64_t)nz, (cuuint64_t)nphi, (cuuint64_t)nr};
    const cuuint64_t strides[2] = {(cuuint64_t)nz * 8ull, (cuuint64_t)nphi * (cuuint64_t)nz * 8ull};
    const cuuint32_t es[3] = {1, 1, 1};
    const cuuint32_t be[3] = {2u * (TILE_KZ + 4), (cuuint32_t)(tj + 2), 1u};
    const cuuint32_t bew[3] = {2u * (TILE_KZ + 4), 1u, 1u};
    const cuuint32_t bh[3] = {2u * (TILE_KZ + 2), (cuuint32_t)(tj + 1), 1u};
    const cuuint32_t bhw[3] = {2u * (TILE_KZ + 2), 1u, 1u};
    auto one = [&](CUtensorMap *t, void *base, const cuuint32_t *box) {
        return enc(t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int c = 0; c < 3; ++c) {
        if (!one(&m->e[c], E[c], be) || !one(&m->ew[c], E[c], bew) || !one(&m->h[c], H[c], bh) ||
            !one(&m->hw[c], H[c], bhw)) {
            *why = "cuTensorMapEncodeTiled refused the field layout";
            return false;
        }
    }
    return true;
}

bool tile_e_shape_ok(int tj) { return tj == 8 || tj == 16 || tj == 32; }

size_t tile_e_smem_bytes(int tj)
{
    if (tj == 8) return e_shape_bytes<8, 6>();
    if (tj == 16) return e_shape_bytes<16, 4>();
    if (tj == 32) return e_shape_bytes<32, 4>();
    return 0;
}

int tile_e_auto_rchunks(int tj, int nr, int nphi, int nz, int sms)
{
    const size_t b = tile_e_smem_bytes(tj);
    const int per_wave = sms * std::max(1, b ? (int)std::min<size_t>(8, (227 * 1024) / (b + 1024)) : 1);
    const int tiles = ((nz + TILE_KZ - 1) / TILE_KZ) * ((nphi + tj - 1) / tj);
    // radius chunks of about 21 radii, at least four waves of thread blocks, at least 8 radii each
    const int waves4 = (4 * per_wave + tiles - 1) / std::max(tiles, 1);
    const int c = std::max(waves4, (nr + 10) / 21);
    return std::max(1, std::min(c, nr / 8));
}

bool encode_tile_e_maps(TileEMaps *m, float2 *const E[3], float2 *const H[3], int nr, int nphi, int nz, int tj,
                        const char **why)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) {
        *why = "the driver's cuTensorMapEncodeTiled is not available";
        return false;
    }
    const cuuint64_t dims[3] = {2ull * (cuuint64_t)nz, (cuuint64_t)nphi, (cuuint64_t)nr};
    const cuuint64_t strides[2] = {(cuuint64_t)nz * 8ull, (cuuint64_t)nphi * (cuuint64_t)nz * 8ull};
    const cuuint32_t es[3] = {1, 1, 1};
    const cuuint32_t beo[3] = {2u * TILE_KZ, (cuuint32_t)tj, 1u};
    const cuuint32_t bh[3] = {2u * (TILE_KZ + 2), (cuuint32_t)(tj + 1), 1u};
    const cuuint32_t bhw[3] = {2u * (TILE_KZ + 2), 1u, 1u};
    auto one = [&](CUtensorMap *t, void *base, const cuuint32_t *box) {
        return enc(t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int c = 0; c < 3; ++c) {
        if (!one(&m->eo[c], E[c], beo) || !one(&m->h[c], H[c], bh) || !one(&m->hw[c], H[c], bhw)) {
            *why = "cuTensorMapEncodeTiled refused the field layout";
            return false;
        }
    }
    return true;
}

bool encode_tile_h_maps(TileHMaps *m, float2 *const E[3], float2 *const H[3], int nr, int nphi, int nz, int tj,
                        const char **why)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) {
        *why = "the driver's cuTensorMapEncodeTiled is not available";
        return false;
    }
    const cuuint64_t dims[3] = {2ull * (cuuint64_t)nz, (cuuint64_t)nphi, (cuuint64_t)nr};
    const cuuint64_t strides[2] = {(cuuint64_t)nz * 8ull, (cuuint64_t)nphi * (cuuint64_t)nz * 8ull};
    const cuuint32_t es[3] = {1, 1, 1};
    const cuuint32_t be[3] = {2u * (TILE_KZ + 2), (cuuint32_t)(tj + 1), 1u};
    const cuuint32_t bew[3] = {2u * (TILE_KZ + 2), 1u, 1u};
    const cuuint32_t bho[3] = {2u * TILE_KZ, (cuuint32_t)tj, 1u};
    auto one = [&](CUtensorMap *t, void *base, const cuuint32_t *box) {
        return enc(t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    for (int c = 0; c < 3; ++c) {
        if (!one(&m->e[c], E[c], be) || !one(&m->ew[c], E[c], bew) || !one(&m->ho[c], H[c], bho)) {
            *why = "cuTensorMapEncodeTiled refused the field layout";
            return false;
        }
    }
    return true;
}

cudaError_t launch_tile_h(const TileHMaps &m, const TileParams &tp, int tj, int n_rchunks, cudaStream_t s)
{
    if (tj == 8) return launch_h_shape<8, 6, 2>(m, tp, n_rchunks, s);
    if (tj == 16) return launch_h_shape<16, 4, 2>(m, tp, n_rchunks, s);
    if (tj == 32) return launch_h_shape<32, 4, 1>(m, tp, n_rchunks, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_tile_e(const TileEMaps &m, const TileParams &tp, int n, int tj, int n_rchunks, cudaStream_t s)
{
    if (tj == 8) return launch_e_shape<8, 6, 2>(m, tp, n, n_rchunks, s);
    if (tj == 16) return launch_e_shape<16, 4, 2>(m, tp, n, n_rchunks, s);
    if (tj == 32) return launch_e_shape<32, 4, 1>(m, tp, n, n_rchunks, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_tile_step(const TileMaps &m, const TileParams &tp, int n, int tj, int n_rchunks, cudaStream_t s)
{
    if (tj == 4) return launch_shape<4, 5, 3>(m, tp, n, n_rchunks, s);
    if (tj == 8) return launch_shape<8, 4, 2>(m, tp, n, n_rchunks, s);
    if (tj == 16) return launch_shape<16, 4, 1>(m, tp, n, n_rchunks, s);
    return cudaErrorInvalidValue;
}

}  // namespace zda
