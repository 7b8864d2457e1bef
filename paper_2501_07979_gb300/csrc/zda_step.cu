// Fused leap-frog step (sm_103a): one launch advances (E^n, H^{n-1/2}) to
// (E^{n+1}, H^{n+1/2}) (Eqs. 3-4) with the CPML auxiliaries and the sheet
// source; the running DFTs follow in k_dft_step (one fully parallel launch,
// so their read-modify-writes never sit on the streaming chain below).
//
// Each CTA owns a phi-tile of TJ rows x all z for a range of radii and
// streams along r.  Lanes run along z; the TJ rows are register-blocked per
// thread.  Stage r of a ring of S shared-memory stages holds, for radius r,
// E^n of the rows j0-1 .. j0+TJ (3 components), H^{n-1/2} of j0-1 .. j0+TJ-1
// and the z-slab CPML auxiliaries; one thread fills it with 1-D bulk async
// copies (each (radius, row, component) column is a contiguous run of n_z
// complex values) that complete on the stage's mbarrier.  Iteration i reads
// stages i and i+1, computes H^{n+1/2}(i) for its rows plus the low phi-halo
// row (recomputed, so no other CTA's result is needed) and E^{n+1}(i) from
// H^{n+1/2}(i), H^{n+1/2}(i-1) (registers) and the z-neighbour (warp shuffle,
// shared memory across warps), stores both, and after the iteration's
// barrier the stage of radius i is refilled with radius i+S.  Reads and
// writes use separate field buffers (ping-pong), so halo reads never see a
// neighbour's new values; the H-side CPML auxiliaries are ping-ponged too,
// the E-side ones updated in place by their owner.  DRAM traffic per cell and
// step: one read and one write of the six components (96 B) plus the CPML
// slabs; the halo rows of neighbouring tiles come from L2.
//
// Every mbarrier wait is bounded: on expiry the kernel sets the error word
// (ZDA_ERR_TIMEOUT on the host), carries on without the data, and before
// exiting waits (bounded) for its copies still in flight.
#include "zda_internal.h"
#include "zda_step.h"

namespace zda {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false (and the error word set) if the phase never completed
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int limit, int *err)
{
    for (int it = 0; it < limit; ++it)
        if (mbar_try(bar, parity)) return true;
    atomicOr(err, 1);
    return false;
}

template <int TJ>
struct StageLayout {
    int nz, pz2;                      // n_z, 2 pml_z
    __device__ int e_off(int s, int c) const { return (s * 3 + c) * nz; }
    __device__ int h_off(int s, int c) const { return ((TJ + 2) * 3 + s * 3 + c) * nz; }
    __device__ int ph_off(int s, int t) const { return (2 * TJ + 3) * 3 * nz + (s * 2 + t) * pz2; }
    __device__ int pe_off(int s, int t) const { return (2 * TJ + 3) * 3 * nz + (TJ + 1) * 2 * pz2 + (s * 2 + t) * pz2; }
    __device__ int elems() const { return (2 * TJ + 3) * 3 * nz + (2 * TJ + 1) * 2 * pz2; }
};

template <int TJ, int NKW, int S>
__global__ void __launch_bounds__(32 * NKW, 1) k_stream_step(const FusedParams p, const int n)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);                 // S stage barriers + 1 spare
    float2 (*xch)[NKW][TJ][2] = reinterpret_cast<float2 (*)[NKW][TJ][2]>(smem_raw + 128);
    float2 *stages = reinterpret_cast<float2 *>(smem_raw + 128 + 2 * NKW * TJ * 2 * sizeof(float2));

    const int lane = threadIdx.x, w = threadIdx.y;
    const int tid = w * 32 + lane;
    const int k = 32 * w + lane;
    const int nz = p.nz, nphi = p.nphi, nr = p.nr;
    const bool kin = k < nz;
    const int j0 = blockIdx.x * TJ;
    const int ib = blockIdx.y * p.i_range;
    const int ie = min(nr, ib + p.i_range);
    const int i_first = (ib > 0) ? ib - 1 : ib;
    const int last_r = min(ie, nr - 1);                   // last radius whose E is staged
    const size_t sj = (size_t)nz, si = (size_t)nphi * nz;
    const float2 zero = make_float2(0.f, 0.f);
    const float dt = p.dt;
    StageLayout<TJ> L{nz, 2 * p.pz};
    const int st_elems = L.elems();

    // slots: row j0-1+s, wrapped into the wedge with its Bloch phase
    int jj[TJ + 2];
    float2 ph[TJ + 2];
    bool own[TJ + 2];
#pragma unroll
    for (int s = 0; s < TJ + 2; ++s) {
        int j = j0 - 1 + s;
        float2 q = make_float2(1.f, 0.f);
        while (j < 0) { j += nphi; q = c_mul(q, p.bloch_inv); }
        while (j >= nphi) { j -= nphi; q = c_mul(q, p.bloch); }
        jj[s] = j;
        ph[s] = q;
        own[s] = (s >= 1 && s <= TJ && j0 - 1 + s < nphi);
    }
    const bool edge = (j0 == 0) || (j0 + TJ >= nphi);

    const int kz = (k < p.pz) ? k : ((k >= nz - p.pz) ? k - (nz - 2 * p.pz) : -1);
    const bool zpml = kin && kz >= 0;

    if (tid == 0) {
        for (int s = 0; s <= S; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ---- producer: stage radius r (thread 0 only)
    auto fill = [&](int r) {
        const int slot = (r - i_first) % S;
        float2 *st = stages + (size_t)slot * st_elems;
        uint64_t *bar = &bars[slot];
        const bool need_h = r < ie;
        const uint32_t col = (uint32_t)nz * 8u, pcol = (uint32_t)(2 * p.pz) * 8u;
        uint32_t bytes = (TJ + 2) * 3 * col;
        if (need_h) bytes += (TJ + 1) * 3 * col;
        if (need_h && p.pz > 0) {
            bytes += (TJ + 1) * 2 * pcol;
            for (int s = 1; s <= TJ; ++s)
                if (own[s]) bytes += 2 * pcol;
        }
        mbar_expect_tx(bar, bytes);
        const float2 *Ec[3] = {p.Er, p.Ep, p.Ez};
        const float2 *Hc[3] = {p.Hr, p.Hp, p.Hz};
        for (int s = 0; s < TJ + 2; ++s)
            for (int c = 0; c < 3; ++c)
                bulk_g2s(st + L.e_off(s, c), Ec[c] + (size_t)r * si + (size_t)jj[s] * sj, col, bar);
        if (need_h) {
            for (int s = 0; s <= TJ; ++s)
                for (int c = 0; c < 3; ++c)
                    bulk_g2s(st + L.h_off(s, c), Hc[c] + (size_t)r * si + (size_t)jj[s] * sj, col, bar);
            if (p.pz > 0) {
                const float2 *Pz[2] = {p.psH_hr_z, p.psH_hp_z};
                const float2 *Ez2[2] = {p.psE_er_z, p.psE_ep_z};
                for (int s = 0; s <= TJ; ++s)
                    for (int t = 0; t < 2; ++t)
                        bulk_g2s(st + L.ph_off(s, t), Pz[t] + ((size_t)r * nphi + jj[s]) * (2 * p.pz), pcol, bar);
                for (int s = 1; s <= TJ; ++s)
                    if (own[s])
                        for (int t = 0; t < 2; ++t)
                            bulk_g2s(st + L.pe_off(s - 1, t), Ez2[t] + ((size_t)r * nphi + jj[s]) * (2 * p.pz), pcol,
                                     bar);
            }
        }
    };
    auto parity_of = [&](int r) -> uint32_t { return (uint32_t)(((r - i_first) / S) & 1); };

    if (tid == 0)
        for (int r = i_first; r <= last_r && r < i_first + S; ++r) fill(r);

    // per-lane constants
    const float bzh = zpml ? __ldg(p.t.bz_h + k) : 0.f, czh = zpml ? __ldg(p.t.cz_h + k) : 0.f;
    const float bzn = zpml ? __ldg(p.t.bz_n + k) : 0.f, czn = zpml ? __ldg(p.t.cz_n + k) : 0.f;
    const float a_n = kin ? __ldg(p.t.a_n + k) : 1.f, d_n = kin ? __ldg(p.t.d_n + k) : 0.f;
    const float a_c = kin ? __ldg(p.t.a_c + k) : 1.f, d_c = kin ? __ldg(p.t.d_c + k) : 0.f;
    const bool in_src = kin && k == p.src_k && p.src_mode != SRC_NONE;
    float2 srcw[TJ + 1][2];                                 // source phase patterns of the owned rows
    float src_amp = 0.f;
#pragma unroll
    for (int s = 1; s <= TJ; ++s) {
        srcw[s][0] = p.t.ph_n[jj[s]];
        srcw[s][1] = p.t.ph_h[jj[s]];
    }
    if (in_src && p.src_mode == SRC_PLANE_WAVE) src_amp = __ldg(p.t.pulse + n) * p.src_scale;
    const bool adj_src = in_src && p.src_mode == SRC_ADJOINT;

    // per-radius tables, prefetched one radius ahead
    auto rtab = [&](int i, float (&t)[6]) {
        t[0] = __ldg(p.t.inv_r_n + i);
        t[1] = __ldg(p.t.inv_r_h + i);
        t[2] = __ldg(p.t.br_h + i);
        t[3] = __ldg(p.t.cr_h + i);
        t[4] = __ldg(p.t.br_n + i);
        t[5] = __ldg(p.t.cr_n + i);
    };
    float tab[6], tab_next[6];
    rtab(i_first, tab);
#pragma unroll
    for (int t = 0; t < 6; ++t) tab_next[t] = tab[t];
    float rbr[TJ + 1], rbp[TJ + 1], rbz[TJ + 1], rbr_n[TJ + 1], rbp_n[TJ + 1], rbz_n[TJ + 1];
#pragma unroll
    for (int s = 1; s <= TJ; ++s) {
        const size_t ij = (size_t)ib * nphi + jj[s];
        rbr[s] = __ldg(p.rb_r + ij);
        rbp[s] = __ldg(p.rb_p + ij);
        rbz[s] = __ldg(p.rb_z + ij);
        rbr_n[s] = rbr[s];
        rbp_n[s] = rbp[s];
        rbz_n[s] = rbz[s];
    }

    float2 asr = zero, asp = zero, asr_n = zero, asp_n = zero;   // adjoint radial source at i, i+1
    if (adj_src) {
        asr = p.src_rad[ib];
        asp = p.src_rad[nr + ib];
    }

    float2 Hpp[TJ + 1], Hpz[TJ + 1];                      // H^{n+1/2}(i-1): H_phi, H_z of the owned rows
#pragma unroll
    for (int s = 0; s <= TJ; ++s) { Hpp[s] = zero; Hpz[s] = zero; }

    auto SLD = [&](const float2 *st, int off, int s) -> float2 {   // stage value with Bloch phase
        float2 v = st[off + k];
        return edge ? c_mul(ph[s], v) : v;
    };

    int par = 0;
    for (int i = i_first; i < ie; ++i) {
        const bool emit = i >= ib;
        if (i + 1 < ie) rtab(i + 1, tab_next);
        if (emit && i + 1 < ie) {
#pragma unroll
            for (int s = 1; s <= TJ; ++s) {
                const size_t ij = (size_t)(i + 1) * nphi + jj[s];
                rbr_n[s] = __ldg(p.rb_r + ij);
                rbp_n[s] = __ldg(p.rb_p + ij);
                rbz_n[s] = __ldg(p.rb_z + ij);
            }
            if (adj_src) {
                asr_n = p.src_rad[i + 1];
                asp_n = p.src_rad[nr + i + 1];
            }
        }
        const float irn = tab[0], irh = tab[1];
        const int ir = (i < p.pr_in) ? i : ((i >= nr - p.pr_out) ? i - (nr - p.pr_in - p.pr_out) : -1);
        const bool rpml = kin && ir >= 0;
        const float brh = tab[2], crh = tab[3], brn = tab[4], crn = tab[5];

        const bool has_next = i + 1 <= last_r;
        mbar_wait(&bars[(i - i_first) % S], parity_of(i), p.wait_limit, p.err);
        if (has_next) mbar_wait(&bars[(i + 1 - i_first) % S], parity_of(i + 1), p.wait_limit, p.err);
        if (p.inject_timeout) mbar_wait(&bars[S], 0, p.wait_limit, p.err);     // never completes
        const float2 *st0 = stages + (size_t)((i - i_first) % S) * st_elems;
        const float2 *st1 = stages + (size_t)((i + 1 - i_first) % S) * st_elems;

        // ---- H^{n+1/2}(i) for slots 0..TJ
        float2 Hr[TJ + 1], Hp[TJ + 1], Hz[TJ + 1];
#pragma unroll
        for (int s = 0; s <= TJ; ++s) {
            float2 er = zero, ep = zero, ez = zero, er1 = zero, ep1 = zero, ez_j1 = zero, er_j1 = zero;
            float2 nez = zero, nep = zero, hr = zero, hp = zero, hz = zero;
            if (kin) {
                er = SLD(st0, L.e_off(s, 0), s);
                ep = SLD(st0, L.e_off(s, 1), s);
                ez = SLD(st0, L.e_off(s, 2), s);
                if (k + 1 < nz) {
                    er1 = SLD(st0, L.e_off(s, 0) + 1, s);
                    ep1 = SLD(st0, L.e_off(s, 1) + 1, s);
                }
                er_j1 = SLD(st0, L.e_off(s + 1, 0), s + 1);
                ez_j1 = SLD(st0, L.e_off(s + 1, 2), s + 1);
                if (has_next) {
                    nep = SLD(st1, L.e_off(s, 1), s);
                    nez = SLD(st1, L.e_off(s, 2), s);
                }
                hr = SLD(st0, L.h_off(s, 0), s);
                hp = SLD(st0, L.h_off(s, 1), s);
                hz = SLD(st0, L.h_off(s, 2), s);
            }
            const bool store_psi = own[s] && emit;
            const size_t rx = ((size_t)(rpml ? ir : 0) * nphi + jj[s]) * nz + k;
            const size_t zx = ((size_t)i * nphi + jj[s]) * (2 * p.pz) + (zpml ? kz : 0);
            // H_r: (1/r) dE_z/dphi - dE_phi/dz
            {
                const float2 dph = c_scale(c_sub(ez_j1, ez), irn * p.inv_dphi);
                float2 dz = c_scale(c_sub(ep1, ep), p.inv_dz);
                if (zpml) {
                    float2 ps = SLD(st0, L.ph_off(s, 0) - k + kz, s);
                    ps = c_add(c_scale(ps, bzh), c_scale(dz, czh));
                    if (store_psi) p.opsH_hr_z[zx] = ps;
                    dz = c_add(dz, ps);
                }
                Hr[s] = c_sub(hr, c_scale(c_sub(dph, dz), dt));
            }
            // H_phi: dE_r/dz - dE_z/dr
            {
                float2 dz = c_scale(c_sub(er1, er), p.inv_dz);
                float2 drr = c_scale(c_sub(nez, ez), p.inv_dr);
                if (zpml) {
                    float2 ps = SLD(st0, L.ph_off(s, 1) - k + kz, s);
                    ps = c_add(c_scale(ps, bzh), c_scale(dz, czh));
                    if (store_psi) p.opsH_hp_z[zx] = ps;
                    dz = c_add(dz, ps);
                }
                if (rpml) {
                    float2 ps = p.psH_hp_r[rx];
                    if (edge) ps = c_mul(ph[s], ps);
                    ps = c_add(c_scale(ps, brh), c_scale(drr, crh));
                    if (store_psi) p.opsH_hp_r[rx] = ps;
                    drr = c_add(drr, ps);
                }
                Hp[s] = c_sub(hp, c_scale(c_sub(dz, drr), dt));
            }
            // H_z: (1/r) d(r E_phi)/dr - (1/r) dE_r/dphi
            {
                float2 drr = c_add(c_scale(c_sub(nep, ep), p.inv_dr), c_scale(c_add(nep, ep), 0.5f * irh));
                const float2 dph = c_scale(c_sub(er_j1, er), irh * p.inv_dphi);
                if (rpml) {
                    float2 ps = p.psH_hz_r[rx];
                    if (edge) ps = c_mul(ph[s], ps);
                    ps = c_add(c_scale(ps, brh), c_scale(drr, crh));
                    if (store_psi) p.opsH_hz_r[rx] = ps;
                    drr = c_add(drr, ps);
                }
                Hz[s] = c_sub(hz, c_scale(c_sub(drr, dph), dt));
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
#pragma unroll
            for (int s = 1; s <= TJ; ++s) {
                float2 hpk, hrk;                               // H_phi(k-1), H_r(k-1)
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
                if (!own[s] || !kin) continue;
                const int j = jj[s];
                const size_t c = (size_t)i * si + (size_t)j * sj + k;
                const size_t zx = ((size_t)i * nphi + j) * (2 * p.pz) + (zpml ? kz : 0);
                const size_t rx = ((size_t)(rpml ? ir : 0) * nphi + j) * nz + k;

                float2 jr = zero, jp = zero;
                if (in_src) {
                    if (p.src_mode == SRC_PLANE_WAVE) {
                        jr = c_scale(srcw[s][0], src_amp);
                        jp = make_float2(-srcw[s][1].y * src_amp, srcw[s][1].x * src_amp);
                    } else if (adj_src) {
                        jr = c_mul(srcw[s][0], asr);
                        jp = c_mul(srcw[s][1], asp);
                    }
                }
                float2 er = st0[L.e_off(s, 0) + k], ep = st0[L.e_off(s, 1) + k], ez = st0[L.e_off(s, 2) + k];
                // E_r (k > 0)
                if (k > 0) {
                    const float2 dph = c_scale(c_sub(Hz[s], Hz[s - 1]), irh * p.inv_dphi);
                    float2 dz = c_scale(c_sub(Hp[s], hpk), p.inv_dz);
                    if (zpml) {
                        float2 ps = st0[L.pe_off(s - 1, 0) + kz];
                        ps = c_add(c_scale(ps, bzn), c_scale(dz, czn));
                        p.psE_er_z[zx] = ps;
                        dz = c_add(dz, ps);
                    }
                    const float ie_ = 1.0f / (a_n + d_n * rbr[s]);
                    er = c_add(er, c_scale(c_sub(c_sub(dph, dz), jr), dt * ie_));
                }
                // E_phi (i > 0, k > 0)
                if (i > 0 && k > 0) {
                    float2 dz = c_scale(c_sub(Hr[s], hrk), p.inv_dz);
                    float2 drr = c_scale(c_sub(Hz[s], Hpz[s]), p.inv_dr);
                    if (zpml) {
                        float2 ps = st0[L.pe_off(s - 1, 1) + kz];
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
                    const float ie_ = 1.0f / (a_n + d_n * rbp[s]);
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
                    const float ie_ = 1.0f / (a_c + d_c * rbz[s]);
                    ez = c_add(ez, c_scale(c_sub(drr, dph), dt * ie_));
                }
                p.oHr[c] = Hr[s];
                p.oHp[c] = Hp[s];
                p.oHz[c] = Hz[s];
                p.oEr[c] = er;
                p.oEp[c] = ep;
                p.oEz[c] = ez;
            }
        }
#pragma unroll
        for (int s = 1; s <= TJ; ++s) {
            Hpp[s] = Hp[s];
            Hpz[s] = Hz[s];
            if (emit) { rbr[s] = rbr_n[s]; rbp[s] = rbp_n[s]; rbz[s] = rbz_n[s]; }
        }
        if (emit) { asr = asr_n; asp = asp_n; }
#pragma unroll
        for (int t = 0; t < 6; ++t) tab[t] = tab_next[t];
        par ^= 1;
        __syncthreads();                                 // stage of radius i is free
        if (tid == 0 && i + S <= last_r) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fill(i + S);
        }
    }
    // copies still in flight (only after a timed-out wait): wait for them
    if (tid == 0)
        for (int r = max(i_first, last_r - S + 1); r <= last_r; ++r)
            mbar_wait(&bars[(r - i_first) % S], parity_of(r), p.wait_limit, p.err);
}

// Adjoint source of step n on the monitor plane, per radius:
// sum_q beta_q(r) k_q(t_{n+1/2}) for the E_r and E_phi sites (the e^{i phi}
// factor is applied per row by the step kernel).
__global__ void k_adjoint_source_step(const FusedParams p, const int n)
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

// Running DFTs of E^{n+1} (monitor plane: E_r, E_phi; design volume: all
// three components), one thread per site, accumulators read-modify-written
// in chunks (see dft_update).
__global__ void k_dft_step(const FusedParams p, const int n)
{
    const int nz = p.nz, nphi = p.nphi, nr = p.nr;
    const size_t plane = (size_t)nr * nphi;
    const size_t sj = (size_t)nz, si = (size_t)nphi * nz;
    const float2 *tw = p.t.twiddle + (size_t)n * p.nq;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t ndes = p.des ? plane * p.des_nk : 0;
    if (t < ndes) {
        const int kk = (int)(t % p.des_nk);
        const size_t ij = t / p.des_nk;
        const size_t c = (ij / nphi) * si + (ij % nphi) * sj + p.des_k0 + kk;
        const float2 e3[3] = {p.oEr[c], p.oEp[c], p.oEz[c]};
        const size_t comp = plane * p.des_nk;
        dft_update<3>(p.des + t, 3 * comp, comp, tw, p.nq, e3);
        return;
    }
    const size_t u = t - ndes;
    if (p.mon && u < plane) {
        const size_t c = (u / nphi) * si + (u % nphi) * sj + p.mon_k;
        const float2 e2[2] = {p.oEr[c], p.oEp[c]};
        dft_update<2>(p.mon + u, 2 * plane, plane, tw, p.nq, e2);
    }
}

template <int TJ, int NKW, int S>
static size_t smem_bytes(int nz, int pz)
{
    const size_t st = ((size_t)(2 * TJ + 3) * 3 * nz + (size_t)(2 * TJ + 1) * 2 * (2 * pz)) * sizeof(float2);
    return 128 + 2 * NKW * TJ * 2 * sizeof(float2) + S * st;
}

template <int TJ, int NKW, int S>
static cudaError_t launch_tj(const FusedParams &p, int n, cudaStream_t s)
{
    const size_t sm = smem_bytes<TJ, NKW, S>(p.nz, p.pz);
    cudaError_t e = cudaFuncSetAttribute(k_stream_step<TJ, NKW, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 b(32, NKW), g((p.nphi + TJ - 1) / TJ, (p.nr + p.i_range - 1) / p.i_range);
    k_stream_step<TJ, NKW, S><<<g, b, sm, s>>>(p, n);
    return cudaGetLastError();
}

cudaError_t launch_fused_pre(const FusedParams &p, int n, cudaStream_t s)
{
    if (p.src_mode != SRC_ADJOINT) return cudaSuccess;
    k_adjoint_source_step<<<(p.nr + 127) / 128, 128, 0, s>>>(p, n);
    return cudaGetLastError();
}

cudaError_t launch_fused_post(const FusedParams &p, int n, cudaStream_t s)
{
    if (!p.des && !p.mon) return cudaSuccess;
    const size_t nsite = (p.des ? (size_t)p.nr * p.nphi * p.des_nk : 0) + (p.mon ? (size_t)p.nr * p.nphi : 0);
    k_dft_step<<<(unsigned)((nsite + 255) / 256), 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

#define ZDA_STAGES 3

template <int TJ>
static cudaError_t launch_nkw(const FusedParams &p, int n, cudaStream_t s)
{
    switch ((p.nz + 31) / 32) {
    case 1: return launch_tj<TJ, 1, ZDA_STAGES>(p, n, s);
    case 2: return launch_tj<TJ, 2, ZDA_STAGES>(p, n, s);
    case 3: return launch_tj<TJ, 3, ZDA_STAGES>(p, n, s);
    case 4: return launch_tj<TJ, 4, ZDA_STAGES>(p, n, s);
    case 5: return launch_tj<TJ, 5, ZDA_STAGES>(p, n, s);
    case 6: return launch_tj<TJ, 6, ZDA_STAGES>(p, n, s);
    case 7: return launch_tj<TJ, 7, ZDA_STAGES>(p, n, s);
    case 8: return launch_tj<TJ, 8, ZDA_STAGES>(p, n, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused_stream(const FusedParams &p, int n, cudaStream_t s)
{
    switch (p.tj) {
    case 2: return launch_nkw<2>(p, n, s);
    case 4: return launch_nkw<4>(p, n, s);
    default: return cudaErrorInvalidValue;
    }
}

int fused_launches_per_step(const FusedParams &p)
{
    return 1 + ((p.des || p.mon) ? 1 : 0) + (p.src_mode == SRC_ADJOINT ? 1 : 0);
}

int fused_max_nz() { return 8 * 32; }

template <int TJ, int NKW>
static int occ_tj(int nz, int pz)
{
    const size_t sm = smem_bytes<TJ, NKW, ZDA_STAGES>(nz, pz);
    if (cudaFuncSetAttribute(k_stream_step<TJ, NKW, ZDA_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm) != cudaSuccess)
        return 0;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream_step<TJ, NKW, ZDA_STAGES>, 32 * NKW, sm);
    return nb;
}

template <int TJ>
static int occ_nkw(int nkw, int nz, int pz)
{
    switch (nkw) {
    case 1: return occ_tj<TJ, 1>(nz, pz);
    case 2: return occ_tj<TJ, 2>(nz, pz);
    case 3: return occ_tj<TJ, 3>(nz, pz);
    case 4: return occ_tj<TJ, 4>(nz, pz);
    case 5: return occ_tj<TJ, 5>(nz, pz);
    case 6: return occ_tj<TJ, 6>(nz, pz);
    case 7: return occ_tj<TJ, 7>(nz, pz);
    case 8: return occ_tj<TJ, 8>(nz, pz);
    default: return 0;
    }
}

int fused_blocks_per_sm(int tj, int nz, int pz)
{
    const int nkw = (nz + 31) / 32;
    return tj == 2 ? occ_nkw<2>(nkw, nz, pz) : (tj == 4 ? occ_nkw<4>(nkw, nz, pz) : 0);
}

}  // namespace zda
