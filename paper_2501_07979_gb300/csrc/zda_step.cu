// Fused leap-frog step (sm_103a): one launch advances (E^n, H^{n-1/2}) to
// (E^{n+1}, H^{n+1/2}) (Eqs. 3-4), with the CPML auxiliaries, the sheet
// source and the running DFTs fused in.
//
// Data movement: each CTA owns a phi-tile of TJ rows x all z for a range of
// radii and streams along r.  Lanes run along z (coalesced 256-byte rows per
// component and warp), the TJ rows are register-blocked in each thread.  At
// radius i the thread loads E^n(i+1) and H^{n-1/2}(i), computes H^{n+1/2}(i)
// for its rows plus the low phi-halo row (recomputed, so no other CTA's
// result is needed), then E^{n+1}(i) from H^{n+1/2}(i), H^{n+1/2}(i-1) (kept
// in registers from the previous radius) and the z-neighbour (warp shuffle,
// shared memory across warp boundaries).  E^n(i) is carried in registers
// from the previous radius.  Reads and writes go to separate buffers
// (ping-pong), so halo reads never see a neighbour's updated values; the
// H-side CPML auxiliaries are ping-ponged for the same reason, the E-side
// ones are updated in place (only their owner touches them).  DRAM traffic
// is one read and one write of the six field components per cell and step
// (96 B) plus the CPML slabs and DFT accumulators; the halo rows come from L2.
#include "zda_internal.h"
#include "zda_step.h"

namespace zda {

template <int TJ>
struct Slots {
    int jj[TJ + 2];       // global phi index of slot s (row j0 - 1 + s), wrapped
    float2 ph[TJ + 2];    // Bloch phase applied to values loaded for slot s
    bool own[TJ + 2];     // slot s is an owned row of this tile
};

__device__ __forceinline__ float2 ld2(const float2 *p) { return __ldg(p); }

template <int TJ, int NKW>
__global__ void __launch_bounds__(32 * NKW, (NKW <= 2) ? 4 : 2) k_fused_step(const FusedParams p, const int n)
{
    const int lane = threadIdx.x, w = threadIdx.y;
    const int k = 32 * w + lane;
    const int nz = p.nz, nphi = p.nphi, nr = p.nr;
    const bool kin = k < nz;
    const int j0 = blockIdx.x * TJ;
    const int ib = blockIdx.y * p.i_range;
    const int ie = min(nr, ib + p.i_range);
    const size_t sj = (size_t)p.nzs, si = (size_t)nphi * p.nzs;
    const float2 zero = make_float2(0.f, 0.f);
    const float dt = p.dt;

    __shared__ float2 xch[2][NKW][TJ][2];    // lane-31 H_phi, H_r of each warp, double-buffered

    Slots<TJ> sl;
#pragma unroll
    for (int s = 0; s < TJ + 2; ++s) {
        int j = j0 - 1 + s;
        float2 ph = make_float2(1.f, 0.f);
        while (j < 0) { j += nphi; ph = c_mul(ph, p.bloch_inv); }
        while (j >= nphi) { j -= nphi; ph = c_mul(ph, p.bloch); }
        sl.jj[s] = j;
        sl.ph[s] = ph;
        sl.own[s] = (s >= 1 && s <= TJ && j0 - 1 + s < nphi);
    }
    const bool edge = (j0 == 0) || (j0 + TJ >= nphi);   // some slot carries a Bloch phase

    auto LD = [&](const float2 *base, int i, int s) -> float2 {
        if (!kin || i >= nr) return zero;
        float2 v = ld2(base + (size_t)i * si + (size_t)sl.jj[s] * sj + k);
        return edge ? c_mul(sl.ph[s], v) : v;
    };
    auto LDk1 = [&](const float2 *base, int i, int s) -> float2 {   // value at k + 1 (lane 31 only)
        if (k + 1 >= nz) return zero;
        float2 v = ld2(base + (size_t)i * si + (size_t)sl.jj[s] * sj + k + 1);
        return edge ? c_mul(sl.ph[s], v) : v;
    };

    const int kz = (k < p.pz) ? k : ((k >= nz - p.pz) ? k - (nz - 2 * p.pz) : -1);
    const bool zpml = kin && kz >= 0;
    const float bzh = zpml ? __ldg(p.t.bz_h + k) : 0.f, czh = zpml ? __ldg(p.t.cz_h + k) : 0.f;
    const float bzn = zpml ? __ldg(p.t.bz_n + k) : 0.f, czn = zpml ? __ldg(p.t.cz_n + k) : 0.f;
    const float a_n = kin ? __ldg(p.t.a_n + k) : 1.f, d_n = kin ? __ldg(p.t.d_n + k) : 0.f;
    const float a_c = kin ? __ldg(p.t.a_c + k) : 1.f, d_c = kin ? __ldg(p.t.d_c + k) : 0.f;
    const int dkk = k - p.des_k0;
    const bool in_des = kin && p.des != nullptr && dkk >= 0 && dkk < p.des_nk;
    const bool in_mon = kin && p.mon != nullptr && k == p.mon_k;
    const bool in_src = kin && k == p.src_k && p.src_mode != SRC_NONE;
    float src_amp = 0.f;
    if (in_src && p.src_mode == SRC_PLANE_WAVE) src_amp = __ldg(p.t.pulse + n) * p.src_scale;

    // E^n(i) per slot (slot TJ+1 only needs E_r and E_z)
    float2 Er[TJ + 2], Ep[TJ + 2], Ez[TJ + 2];
    float2 Hpp[TJ + 1], Hpz[TJ + 1];           // H^{n+1/2}(i-1): H_phi, H_z for slots 1..TJ
    const int i_first = (ib > 0) ? ib - 1 : ib;
#pragma unroll
    for (int s = 0; s < TJ + 2; ++s) {
        Er[s] = LD(p.Er, i_first, s);
        Ez[s] = LD(p.Ez, i_first, s);
        Ep[s] = (s <= TJ) ? LD(p.Ep, i_first, s) : zero;
    }
#pragma unroll
    for (int s = 0; s <= TJ; ++s) { Hpp[s] = zero; Hpz[s] = zero; }

    int par = 0;
    for (int i = i_first; i < ie; ++i) {
        const bool emit = i >= ib;
        const float irn = __ldg(p.t.inv_r_n + i), irh = __ldg(p.t.inv_r_h + i);
        const int ir = (i < p.pr_in) ? i : ((i >= nr - p.pr_out) ? i - (nr - p.pr_in - p.pr_out) : -1);
        const bool rpml = kin && ir >= 0;
        const float brh = rpml ? __ldg(p.t.br_h + i) : 0.f, crh = rpml ? __ldg(p.t.cr_h + i) : 0.f;
        const float brn = rpml ? __ldg(p.t.br_n + i) : 0.f, crn = rpml ? __ldg(p.t.cr_n + i) : 0.f;

        // ---- loads: E^n(i+1), H^{n-1/2}(i)
        float2 nEr[TJ + 2], nEp[TJ + 2], nEz[TJ + 2];
#pragma unroll
        for (int s = 0; s < TJ + 2; ++s) {
            nEr[s] = LD(p.Er, i + 1, s);
            nEz[s] = LD(p.Ez, i + 1, s);
            nEp[s] = (s <= TJ) ? LD(p.Ep, i + 1, s) : zero;
        }
        float2 Hr[TJ + 1], Hp[TJ + 1], Hz[TJ + 1];
#pragma unroll
        for (int s = 0; s <= TJ; ++s) {
            Hr[s] = LD(p.Hr, i, s);
            Hp[s] = LD(p.Hp, i, s);
            Hz[s] = LD(p.Hz, i, s);
        }

        // ---- H^{n+1/2}(i) for slots 0..TJ
#pragma unroll
        for (int s = 0; s <= TJ; ++s) {
            // z-neighbours E_phi(k+1), E_r(k+1): shuffle, lane 31 from memory
            float2 ep1, er1;
            ep1.x = __shfl_down_sync(0xffffffffu, Ep[s].x, 1);
            ep1.y = __shfl_down_sync(0xffffffffu, Ep[s].y, 1);
            er1.x = __shfl_down_sync(0xffffffffu, Er[s].x, 1);
            er1.y = __shfl_down_sync(0xffffffffu, Er[s].y, 1);
            if (lane == 31) {
                ep1 = LDk1(p.Ep, i, s);
                er1 = LDk1(p.Er, i, s);
            } else if (k + 1 >= nz) {
                ep1 = zero;
                er1 = zero;
            }
            const size_t zx = ((size_t)i * nphi + sl.jj[s]) * (2 * p.pz) + (zpml ? kz : 0);
            const size_t rx = ((size_t)(rpml ? ir : 0) * nphi + sl.jj[s]) * nz + k;
            const float2 phs = edge ? sl.ph[s] : make_float2(1.f, 0.f);
            const bool store_psi = sl.own[s] && emit;
            // H_r: (1/r) dE_z/dphi - dE_phi/dz
            {
                const float2 dph = c_scale(c_sub(Ez[s + 1], Ez[s]), irn * p.inv_dphi);
                float2 dz = c_scale(c_sub(ep1, Ep[s]), p.inv_dz);
                if (zpml) {
                    float2 ps = c_mul(phs, ld2(p.psH_hr_z + zx));
                    ps = c_add(c_scale(ps, bzh), c_scale(dz, czh));
                    if (store_psi) p.opsH_hr_z[zx] = ps;
                    dz = c_add(dz, ps);
                }
                Hr[s] = c_sub(Hr[s], c_scale(c_sub(dph, dz), dt));
            }
            // H_phi: dE_r/dz - dE_z/dr
            {
                float2 dz = c_scale(c_sub(er1, Er[s]), p.inv_dz);
                float2 drr = c_scale(c_sub(nEz[s], Ez[s]), p.inv_dr);
                if (zpml) {
                    float2 ps = c_mul(phs, ld2(p.psH_hp_z + zx));
                    ps = c_add(c_scale(ps, bzh), c_scale(dz, czh));
                    if (store_psi) p.opsH_hp_z[zx] = ps;
                    dz = c_add(dz, ps);
                }
                if (rpml) {
                    float2 ps = c_mul(phs, ld2(p.psH_hp_r + rx));
                    ps = c_add(c_scale(ps, brh), c_scale(drr, crh));
                    if (store_psi) p.opsH_hp_r[rx] = ps;
                    drr = c_add(drr, ps);
                }
                Hp[s] = c_sub(Hp[s], c_scale(c_sub(dz, drr), dt));
            }
            // H_z: (1/r) d(r E_phi)/dr - (1/r) dE_r/dphi
            {
                float2 drr = c_add(c_scale(c_sub(nEp[s], Ep[s]), p.inv_dr),
                                   c_scale(c_add(nEp[s], Ep[s]), 0.5f * irh));
                const float2 dph = c_scale(c_sub(Er[s + 1], Er[s]), irh * p.inv_dphi);
                if (rpml) {
                    float2 ps = c_mul(phs, ld2(p.psH_hz_r + rx));
                    ps = c_add(c_scale(ps, brh), c_scale(drr, crh));
                    if (store_psi) p.opsH_hz_r[rx] = ps;
                    drr = c_add(drr, ps);
                }
                Hz[s] = c_sub(Hz[s], c_scale(c_sub(drr, dph), dt));
            }
        }

        // ---- z-neighbour exchange across warp boundaries: H_phi, H_r at k-1
        if (lane == 31) {
#pragma unroll
            for (int s = 1; s <= TJ; ++s) {
                xch[par][w][s - 1][0] = Hp[s];
                xch[par][w][s - 1][1] = Hr[s];
            }
        }
        __syncthreads();

        if (emit) {
            const size_t plane = (size_t)nr * nphi;
#pragma unroll
            for (int s = 1; s <= TJ; ++s) {
                float2 hpk, hrk;             // H_phi(k-1), H_r(k-1)
                hpk.x = __shfl_up_sync(0xffffffffu, Hp[s].x, 1);
                hpk.y = __shfl_up_sync(0xffffffffu, Hp[s].y, 1);
                hrk.x = __shfl_up_sync(0xffffffffu, Hr[s].x, 1);
                hrk.y = __shfl_up_sync(0xffffffffu, Hr[s].y, 1);
                if (lane == 0) {
                    if (w > 0) {
                        hpk = xch[par][w - 1][s - 1][0];
                        hrk = xch[par][w - 1][s - 1][1];
                    } else {
                        hpk = zero;
                        hrk = zero;
                    }
                }
                if (!sl.own[s] || !kin) continue;
                const int j = sl.jj[s];
                const size_t ij = (size_t)i * nphi + j;
                const size_t c = (size_t)i * si + (size_t)j * sj + k;
                const size_t zx = ij * (2 * p.pz) + (zpml ? kz : 0);
                const size_t rx = ((size_t)(rpml ? ir : 0) * nphi + j) * nz + k;

                float2 jr = zero, jp = zero;
                if (in_src) {
                    if (p.src_mode == SRC_PLANE_WAVE) {
                        const float2 pn = p.t.ph_n[j], pq = p.t.ph_h[j];
                        jr = c_scale(pn, src_amp);
                        jp = make_float2(-pq.y * src_amp, pq.x * src_amp);
                    } else {
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
                float2 er = Er[s], ep = Ep[s], ez = Ez[s];
                // E_r (k > 0)
                if (k > 0) {
                    const float2 dph = c_scale(c_sub(Hz[s], Hz[s - 1]), irh * p.inv_dphi);
                    float2 dz = c_scale(c_sub(Hp[s], hpk), p.inv_dz);
                    if (zpml) {
                        float2 ps = p.psE_er_z[zx];
                        ps = c_add(c_scale(ps, bzn), c_scale(dz, czn));
                        p.psE_er_z[zx] = ps;
                        dz = c_add(dz, ps);
                    }
                    const float ie_ = 1.0f / (a_n + d_n * __ldg(p.rb_r + ij));
                    er = c_add(er, c_scale(c_sub(c_sub(dph, dz), jr), dt * ie_));
                }
                // E_phi (i > 0, k > 0)
                if (i > 0 && k > 0) {
                    float2 dz = c_scale(c_sub(Hr[s], hrk), p.inv_dz);
                    float2 drr = c_scale(c_sub(Hz[s], Hpz[s]), p.inv_dr);
                    if (zpml) {
                        float2 ps = p.psE_ep_z[zx];
                        ps = c_add(c_scale(ps, bzn), c_scale(dz, czn));
                        p.psE_ep_z[zx] = ps;
                        dz = c_add(dz, ps);
                    }
                    if (rpml) {
                        float2 ps = p.psE_ep_r[rx];
                        ps = c_add(c_scale(ps, brn), c_scale(drr, crn));
                        p.psE_ep_r[rx] = ps;
                        drr = c_add(drr, ps);
                    }
                    const float ie_ = 1.0f / (a_n + d_n * __ldg(p.rb_p + ij));
                    ep = c_add(ep, c_scale(c_sub(c_sub(dz, drr), jp), dt * ie_));
                }
                // E_z (i > 0)
                if (i > 0) {
                    float2 drr = c_add(c_scale(c_sub(Hp[s], Hpp[s]), p.inv_dr),
                                       c_scale(c_add(Hp[s], Hpp[s]), 0.5f * irn));
                    const float2 dph = c_scale(c_sub(Hr[s], Hr[s - 1]), irn * p.inv_dphi);
                    if (rpml) {
                        float2 ps = p.psE_ez_r[rx];
                        ps = c_add(c_scale(ps, brn), c_scale(drr, crn));
                        p.psE_ez_r[rx] = ps;
                        drr = c_add(drr, ps);
                    }
                    const float ie_ = 1.0f / (a_c + d_c * __ldg(p.rb_z + ij));
                    ez = c_add(ez, c_scale(c_sub(drr, dph), dt * ie_));
                }
                p.oHr[c] = Hr[s];
                p.oHp[c] = Hp[s];
                p.oHz[c] = Hz[s];
                p.oEr[c] = er;
                p.oEp[c] = ep;
                p.oEz[c] = ez;

                if (in_mon) {
                    const float2 e2[2] = {er, ep};
                    dft_update<2, 2>(p.mon + ij, 2 * plane, plane, p.t.twiddle + (size_t)n * p.nq, p.nq, e2);
                }
                if (in_des) {
                    const size_t comp = plane * p.des_nk;
                    const float2 e3[3] = {er, ep, ez};
                    dft_update<3, 2>(p.des + ij * p.des_nk + dkk, 3 * comp, comp, p.t.twiddle + (size_t)n * p.nq,
                                  p.nq, e3);
                }
            }
        }
        // carry: H^{n+1/2}(i) -> H(i-1) of the next radius; E^n(i+1) -> E^n(i)
#pragma unroll
        for (int s = 1; s <= TJ; ++s) { Hpp[s] = Hp[s]; Hpz[s] = Hz[s]; }
#pragma unroll
        for (int s = 0; s < TJ + 2; ++s) { Er[s] = nEr[s]; Ep[s] = nEp[s]; Ez[s] = nEz[s]; }
        par ^= 1;
    }
}

template <int TJ, int NKW>
static cudaError_t launch_tj(const FusedParams &p, int n, cudaStream_t s)
{
    dim3 b(32, NKW), g((p.nphi + TJ - 1) / TJ, (p.nr + p.i_range - 1) / p.i_range);
    k_fused_step<TJ, NKW><<<g, b, 0, s>>>(p, n);
    return cudaGetLastError();
}

template <int TJ>
static cudaError_t launch_nkw(const FusedParams &p, int n, cudaStream_t s)
{
    const int nkw = (p.nz + 31) / 32;
    switch (nkw) {
    case 1: return launch_tj<TJ, 1>(p, n, s);
    case 2: return launch_tj<TJ, 2>(p, n, s);
    case 3: return launch_tj<TJ, 3>(p, n, s);
    case 4: return launch_tj<TJ, 4>(p, n, s);
    case 5: return launch_tj<TJ, 5>(p, n, s);
    case 6: return launch_tj<TJ, 6>(p, n, s);
    case 7: return launch_tj<TJ, 7>(p, n, s);
    case 8: return launch_tj<TJ, 8>(p, n, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused_step(const FusedParams &p, int n, cudaStream_t s)
{
    switch (p.tj) {
    case 2: return launch_nkw<2>(p, n, s);
    case 4: return launch_nkw<4>(p, n, s);
    default: return cudaErrorInvalidValue;
    }
}

int fused_max_nz() { return 8 * 32; }

template <int TJ, int NKW>
static int occ_tj()
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fused_step<TJ, NKW>, 32 * NKW, 0);
    return nb;
}

template <int TJ>
static int occ_nkw(int nkw)
{
    switch (nkw) {
    case 1: return occ_tj<TJ, 1>();
    case 2: return occ_tj<TJ, 2>();
    case 3: return occ_tj<TJ, 3>();
    case 4: return occ_tj<TJ, 4>();
    case 5: return occ_tj<TJ, 5>();
    case 6: return occ_tj<TJ, 6>();
    case 7: return occ_tj<TJ, 7>();
    case 8: return occ_tj<TJ, 8>();
    default: return 0;
    }
}

int fused_blocks_per_sm(int tj, int nz)
{
    const int nkw = (nz + 31) / 32;
    return tj == 2 ? occ_nkw<2>(nkw) : (tj == 4 ? occ_nkw<4>(nkw) : 0);
}

}  // namespace zda
