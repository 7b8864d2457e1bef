// Tensor-core kernels of the surrogate network (sm_103a): BF16 operands
// staged in shared memory by bulk copies (cp.async.bulk on mbarriers),
// tcgen05.mma accumulating in FP32 in tensor memory, epilogues reading TMEM
// with tcgen05.ld.  Activations are planar (see zda_nn_internal.h): each
// 8-channel plane of a window is one contiguous run of rows, which is also
// the canonical no-swizzle operand layout (core matrix = 8 rows x 16 B).
//
// k_conv_tc  -- forward convolution and its input-gradient (transposed)
//               convolution.  A tile is mt x 128 consecutive padded
//               positions with all N output channels.  One window of the
//               input (the tile's positions plus a halo of Wp + 1 rows on
//               each side) serves all taps: tap t is the same window seen
//               from start row halo + off(t), i.e. a different descriptor
//               start address, so no im2col copy is ever made.
// k_wgrad_tc -- weight gradient: both operands MN-major (channels contiguous),
//               reduction over positions; M = 128 rows hold 128 / c_in taps'
//               shifted copies of the input, each copied pre-shifted.
//
// Roles of k_conv_tc (352 threads): warp 0 lane 0 = producer, warps 1 and 10
// lane 0 = MMA issuers (M tile 0 / 1 of each tile, warp 1 also allocates
// TMEM), warps 2..9 = epilogue (warp w reads TMEM lanes 32 (w mod 4) ..).  Every mbarrier wait is bounded; a timeout sets
// the error word and the CTA skips its stores, frees TMEM and exits.
#include <cuda_bf16.h>

#include <algorithm>

#include "zda_nn_internal.h"
#include "zda_nn_tc.cuh"

namespace zda {
namespace nn {

static __device__ __forceinline__ bool bf16_pos(uint16_t b) { return !(b & 0x8000u) && b != 0; }

static __device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Bounded wait that also gives up when another role has aborted.
static __device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, int limit, volatile int *abort,
                                                     int *err, int code)
{
    for (int it = 0; it < limit; ++it) {
        if (mb_try(bar, parity)) return true;
        if ((it & 63) == 63 && *abort) return false;
    }
    *abort = 1;
    if (err) atomicCAS(err, 0, code);
    return false;
}

// Epilogue of one 16-channel chunk (channels cc .. cc + 15) of one position.
__device__ __forceinline__ void epilogue_chunk(const ConvParams &p, float *v, int cc, int pos, bool valid, bool inner,
                                               const float *bias)
{
    if (p.epi == EPI_F32 || p.epi == EPI_GRAD_F32) {
        // straight into the caller's [n][H][W][out_ld] tensor (interior positions only)
        if (!inner || cc >= p.out_ld) return;
        const int HW = p.Hp * p.Wp, rem = pos % HW, y = rem / p.Wp, x = rem % p.Wp;
        const size_t pix = ((size_t)(pos / HW) * (p.Hp - 2) + (y - 1)) * (p.Wp - 2) + (x - 1);
        float *o = static_cast<float *>(p.out0) + pix * p.out_ld + cc;
        const int nc = p.out_ld - cc < 16 ? p.out_ld - cc : 16;
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] += bias[i];
        if ((p.out_ld & 3) == 0) {
            float4 *o4 = reinterpret_cast<float4 *>(o);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (4 * i < nc) o4[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (i < nc) o[i] = v[i];
        }
        return;
    }
    const int half = cc >= p.out_ld ? 1 : 0;
    const int c = cc - half * p.out_ld;           // channel within the output tensor
    if (p.epi == EPI_RELU_BF16) {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = inner ? fmaxf(v[i] + bias[i], 0.f) : 0.f;
    } else {   // EPI_GRAD_BF16
        const uint16_t *mk = half ? p.mask1 : p.mask0;
        if (mk && inner) {
            const uint4 m0 = __ldg(reinterpret_cast<const uint4 *>(mk + ((size_t)(c / 8) * p.rows + LEAD + pos) * 8));
            const uint4 m1 = __ldg(reinterpret_cast<const uint4 *>(mk + ((size_t)(c / 8 + 1) * p.rows + LEAD + pos) * 8));
            const uint16_t *h0 = reinterpret_cast<const uint16_t *>(&m0);
            const uint16_t *h1 = reinterpret_cast<const uint16_t *>(&m1);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (!bf16_pos(h0[i])) v[i] = 0.f;
                if (!bf16_pos(h1[i])) v[8 + i] = 0.f;
            }
        }
        if (!inner) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
    }
    uint16_t *ob = static_cast<uint16_t *>(half ? p.out1 : p.out0);
    *reinterpret_cast<uint4 *>(ob + ((size_t)(c / 8) * p.rows + LEAD + pos) * 8) =
        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    *reinterpret_cast<uint4 *>(ob + ((size_t)(c / 8 + 1) * p.rows + LEAD + pos) * 8) =
        make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]), pack_bf16(v[14], v[15]));
}

// The MMAs of one tap for M tile m0 of the tile: NKS K-steps of 16 channels each.
template <int NKS>
__device__ __forceinline__ void issue_tap(uint32_t d0, uint32_t dn, int m0, uint64_t a0, uint32_t a_ks, uint64_t b0,
                                          uint32_t b_ks, uint32_t idesc, uint32_t acc0)
{
    const uint64_t am = a0 + (uint64_t)(m0 * 128);            // 128 rows x 16 B
    const uint32_t dm = d0 + m0 * dn;
    tc_mma(dm, am, b0, idesc, acc0);
#pragma unroll
    for (int ks = 1; ks < NKS; ++ks) tc_mma(dm, am + (uint64_t)(ks * a_ks), b0 + (uint64_t)(ks * b_ks), idesc, 1u);
}

// All MMAs of one unit (up to 32 input channels) of one tile with resident
// weights, fully unrolled over taps, M tiles and K steps.  abase: descriptor
// of the window at row `halo` (a tap adds its row offset: one 16-byte unit
// per row); bbase: descriptor of the unit's half of the first weight block
// of its group.
template <int TAPS, int NKS>
__device__ __forceinline__ void issue_unit(uint32_t d0, uint32_t dn, int m0, uint64_t abase, int Wp, uint64_t bbase,
                                           uint32_t wunits, uint32_t a_ks, uint32_t b_ks, uint32_t idesc, int uu)
{
#pragma unroll
    for (int tap = 0; tap < TAPS; ++tap) {
        const int off = TAPS == 9 ? (tap / 3 - 1) * Wp + (tap % 3 - 1) : 0;
        const uint64_t a0 = abase + (uint64_t)(int64_t)off;
        const uint64_t b0 = bbase + (uint64_t)(tap * wunits);
        issue_tap<NKS>(d0, dn, m0, a0, a_ks, b0, b_ks, idesc, (uu | tap) != 0);
    }
}

__device__ __forceinline__ void mb_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent, warp-specialised convolution.  Warp 0 (one lane) streams, per
// tile and input unit, the bulk-copied window into one of two stages; the
// weight blocks are either loaded once per CTA (resident: every layer whose
// weights fit beside the two windows) or streamed per tap through a ring
// (the concatenating layers); warp 1 (one lane) issues the MMAs
// into one of two TMEM accumulators (2 x mt x N columns); warps 2..9 drain
// the other accumulator (warp w reads lane quarter w mod 4, column half
// (w - 2) / 4) while the next tile's MMAs run.
__global__ void __launch_bounds__(CONV_THREADS, 1)
    k_conv_tc(const ConvParams p)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw = su32(smem), base = (raw + 1023u) & ~1023u;   // copy destinations: 1024-aligned
    // a unit = up to 4 planes (32 channels) of one input group; window stages hold one unit
    const int upl = p.cg / 8 < 4 ? p.cg / 8 : 4, uh = (p.cg / 8) / upl, nunits = p.ngroups * uh;
    const uint32_t win_bytes = (uint32_t)upl * p.plane;
    const uint32_t wslot = (uint32_t)p.N * p.cg * 2;              // one (group, tap) weight block
    const uint32_t uslot = (uint32_t)p.N * upl * 16;              // its share for one unit (streamed ring)
    const uint32_t sWin = base, sW = base + 2 * win_bytes;
    const uint32_t sBar = sW + (p.resident ? p.ngroups * p.taps * wslot : p.slots * uslot);
    const uint32_t winFull = sBar, winEmpty = sBar + 16, accFull = sBar + 32, accEmpty = sBar + 48;
    const uint32_t wFull = sBar + 64, wEmpty = wFull + 8 * p.slots;
    const uint32_t sMisc = wEmpty + 8 * p.slots;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + (sMisc - raw));
    volatile int *abort = reinterpret_cast<volatile int *>(smem + (sMisc + 4 - raw));

    const int tile_pos = p.mt * 128;
    const int ntiles = (p.P + tile_pos - 1) / tile_pos;
    const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t acc_cols = (uint32_t)(p.mt * p.N);

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mb_init(winFull + 8 * s, 1);
            mb_init(winEmpty + 8 * s, 2);          // one commit per MMA warp
            mb_init(accFull + 8 * s, 2);
            mb_init(accEmpty + 8 * s, 8);          // one arrival per epilogue warp
        }
        for (int s = 0; s < p.slots; ++s) {
            mb_init(wFull + 8 * s, 1);
            mb_init(wEmpty + 8 * s, 2);
        }
        *abort = 0;
        mb_fence_init();
    }
    if (warp == 1) tm_alloc(sMisc, p.ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer
            int u = 0, it = 0;
            bool ok = true;
            if (p.resident && my_tiles > 0) {
                mb_expect_tx(wFull, (uint32_t)(p.ngroups * p.taps) * wslot);
                for (int blk = 0; blk < p.ngroups * p.taps; ++blk)
                    bulk_load(sW + blk * wslot, p.wimg + (size_t)blk * p.N * p.cg, wslot, wFull);
            }
            for (int t = 0; t < my_tiles && ok; ++t) {
                const int p0 = ((int)blockIdx.x + t * (int)gridDim.x) * tile_pos;
                for (int uu = 0; uu < nunits && ok; ++uu, ++u) {
                    const int g = uu / uh, hf = uu % uh;
                    const int s = u & 1, k = u >> 1;
                    if (k > 0 && !wait_or_abort(winEmpty + 8 * s, (k - 1) & 1, p.wait_limit, abort, p.err, 11)) {
                        ok = false;
                        break;
                    }
                    const uint16_t *src = g == 0 ? p.in0 : p.in1;
                    const uint32_t dst = sWin + s * win_bytes;
                    mb_expect_tx(winFull + 8 * s, (uint32_t)upl * p.R * 16);
                    for (int j = 0; j < upl; ++j)
                        bulk_load(dst + j * p.plane, src + ((size_t)(hf * upl + j) * p.rows + LEAD + p0 - p.halo) * 8,
                                  (uint32_t)p.R * 16, winFull + 8 * s);
                    for (int tap = 0; tap < p.taps && !p.resident; ++tap, ++it) {
                        const int sl = it % p.slots, kk = it / p.slots;
                        if (kk > 0 && !wait_or_abort(wEmpty + 8 * sl, (kk - 1) & 1, p.wait_limit, abort, p.err, 12)) {
                            ok = false;
                            break;
                        }
                        mb_expect_tx(wFull + 8 * sl, uslot);
                        bulk_load(sW + sl * uslot,
                                  p.wimg + (size_t)(g * p.taps + tap) * p.N * p.cg + (size_t)hf * p.N * upl * 8, uslot,
                                  wFull + 8 * sl);
                    }
                }
            }
        }
    } else if (warp == 1 || warp == 10) {
        if (lane == 0) {
            // ---------------- MMA issuers: warp 1 issues M tile 0, warp 10 M tile 1 (separate accumulators)
            const int m0 = warp == 1 ? 0 : 1;
            const uint32_t idesc = idesc_bf16(128, p.N, 0, 0);
            const uint32_t a_ks = (2 * (uint32_t)p.plane) >> 4, b_ks = ((uint32_t)p.N * 32) >> 4;
            const int taps = p.taps, Wp = p.Wp, halo = p.halo, nks = upl / 2, N = p.N;
            const uint32_t plane = (uint32_t)p.plane;
            const bool resident = p.resident != 0;
            int u = 0, it = 0;
            bool ok = true;
            if (resident && my_tiles > 0) ok = wait_or_abort(wFull, 0, p.wait_limit, abort, p.err, 17);
            for (int t = 0; t < my_tiles && ok; ++t) {
                const int b = t & 1, kb = t >> 1;
                if (kb > 0 && !wait_or_abort(accEmpty + 8 * b, (kb - 1) & 1, p.wait_limit, abort, p.err, 13)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d0 = tmem + b * acc_cols;
                for (int uu = 0; uu < nunits && ok; ++uu, ++u) {
                    const int g = uu / uh, hf = uu % uh;
                    const int s = u & 1, k = u >> 1;
                    if (!wait_or_abort(winFull + 8 * s, k & 1, p.wait_limit, abort, p.err, 14)) {
                        ok = false;
                        break;
                    }
                    const uint32_t win = sWin + s * win_bytes;
                    if (resident) {
                        tc_fence_after();
                        // descriptors advance by plain adds: the start-address field is the low
                        // 14 bits in 16-byte units and every address stays below 256 KB
                        const uint64_t abase = sdesc(win + (uint32_t)halo * 16, plane, 128);
                        const uint64_t bbase = sdesc(sW + (uint32_t)(g * taps) * wslot, 128, 256) +
                                               (uint64_t)(hf * nks * b_ks);
                        const uint32_t wunits = wslot >> 4;
                        const int kind = taps * 8 + nks;
                        if (kind == 9 * 8 + 2) issue_unit<9, 2>(d0, N, m0, abase, Wp, bbase, wunits, a_ks, b_ks, idesc, uu);
                        else if (kind == 9 * 8 + 1) issue_unit<9, 1>(d0, N, m0, abase, Wp, bbase, wunits, a_ks, b_ks, idesc, uu);
                        else if (kind == 1 * 8 + 2) issue_unit<1, 2>(d0, N, m0, abase, Wp, bbase, wunits, a_ks, b_ks, idesc, uu);
                        else issue_unit<1, 1>(d0, N, m0, abase, Wp, bbase, wunits, a_ks, b_ks, idesc, uu);
                    } else {
                        for (int tap = 0; tap < taps; ++tap, ++it) {
                            const int sl = it % p.slots, kk = it / p.slots;
                            if (!wait_or_abort(wFull + 8 * sl, kk & 1, p.wait_limit, abort, p.err, 15)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const int off = taps == 9 ? (tap / 3 - 1) * Wp + (tap % 3 - 1) : 0;
                            const uint64_t a0 = sdesc(win + (uint32_t)(halo + off) * 16, plane, 128);
                            const uint64_t b0 = sdesc(sW + sl * uslot, 128, 256);
                            const uint32_t acc0 = (uu | tap) != 0;
                            if (nks == 2) issue_tap<2>(d0, N, m0, a0, a_ks, b0, b_ks, idesc, acc0);
                            else issue_tap<1>(d0, N, m0, a0, a_ks, b0, b_ks, idesc, acc0);
                            tc_commit(wEmpty + 8 * sl);
                        }
                    }
                    if (ok) tc_commit(winEmpty + 8 * s);
                }
                if (ok) tc_commit(accFull + 8 * b);
            }
        }
    } else {
        // ---------------- epilogue (warps 2..9)
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int HW = p.Hp * p.Wp, nchunk = p.N / 16;
        // this warp's chunks: c16 = h, h + 2, h + 4, h + 6 (those < nchunk); biases in registers
        float bias_r[2][16];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = (h + 2 * j) * 16 + i;
                bias_r[j][i] = (p.bias && c < p.nbias) ? __ldg(p.bias + c) : 0.f;
            }
        for (int t = 0; t < my_tiles; ++t) {
            const int b = t & 1, kb = t >> 1;
            bool ok = true;
            if (lane == 0) ok = wait_or_abort(accFull + 8 * b, kb & 1, p.wait_limit, abort, p.err, 16);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            tc_fence_after();
            const int p0 = ((int)blockIdx.x + t * (int)gridDim.x) * tile_pos;
            for (int m = 0; m < p.mt; ++m) {
                const int pos = p0 + m * 128 + q * 32 + lane;
                const bool valid = pos < p.P;             // rows up to the tile end exist (zeroed past P)
                const int rem = pos % HW, y = rem / p.Wp, x = rem % p.Wp;
                const bool inner = valid && y > 0 && y < p.Hp - 1 && x > 0 && x < p.Wp - 1;
                const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + b * acc_cols + m * p.N;
                for (int c16 = h; c16 < nchunk; c16 += 4) {
                    float va[16], vb[16];
                    const bool two = c16 + 2 < nchunk;
                    if (two) tm_ld16x2(trow + c16 * 16, trow + (c16 + 2) * 16, va, vb);
                    else tm_ld16(trow + c16 * 16, va);
                    epilogue_chunk(p, va, c16 * 16, pos, valid, inner, bias_r[0]);   // biases only when N <= 64
                    if (two) epilogue_chunk(p, vb, (c16 + 2) * 16, pos, valid, inner, bias_r[1]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mb_arrive(accEmpty + 8 * b);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tm_dealloc(tmem, p.ncols);
}

__global__ void __launch_bounds__(WG_THREADS, 1)
    k_wgrad_tc(const WgradParams p)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw = su32(smem), base = (raw + 1023u) & ~1023u;
    const uint32_t planeb = (uint32_t)p.kt * 16;
    const uint32_t a_bytes = 16 * planeb, b_bytes = (uint32_t)(p.N / 8) * planeb;
    const uint32_t stage = a_bytes + b_bytes;
    const uint32_t sBar = base + WG_STAGES * stage;
    const uint32_t barF = sBar, barE = sBar + 8 * WG_STAGES, bar_done = barE + 8 * WG_STAGES;
    const uint32_t sTmem = bar_done + 8;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + (sTmem - raw));
    const int g = blockIdx.x, split = blockIdx.y;
    const int tile0 = split * p.tiles_per_cta;
    const int tile1 = min(p.ntiles, tile0 + p.tiles_per_cta);
    const int ntile = max(0, tile1 - tile0);
    const uint32_t ncols = p.N < 32 ? 32 : p.N;

    if (threadIdx.x == 0) {
        for (int s = 0; s < WG_STAGES; ++s) {
            mb_init(barF + 8 * s, 1);
            mb_init(barE + 8 * s, 1);
        }
        mb_init(bar_done, 1);
        mb_fence_init();
    }
    if (warp == 2) tm_alloc(sTmem, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        for (int i = 0; i < ntile; ++i) {
            const int s = i % WG_STAGES, u = i / WG_STAGES;
            if (u > 0 && !mb_wait(barE + 8 * s, (u - 1) & 1, p.wait_limit, p.err, 21)) break;
            const uint32_t sa = base + s * stage, sb = sa + a_bytes;
            const int y = (tile0 + i) * p.kt;
            mb_expect_tx(barF + 8 * s, stage);
            for (int j = 0; j < p.ntap_grp; ++j) {
                int t = g * p.ntap_grp + j;
                if (t >= p.taps) t = p.taps - 1;                 // padding copy: its rows are discarded
                const int off = p.taps == 9 ? (t / 3 - 1) * p.Wp + (t % 3 - 1) : 0;
                for (int c = 0; c < p.cin_planes; ++c) {
                    const bool second = p.two_inputs && c >= 8;
                    const uint16_t *x = second ? p.x1 : p.x0;
                    const int cc = second ? c - 8 : c;
                    bulk_load(sa + (j * p.cin_planes + c) * planeb, x + ((size_t)cc * p.rows + LEAD + y + off) * 8, planeb,
                              barF + 8 * s);
                }
            }
            for (int c = 0; c < p.N / 8; ++c)
                bulk_load(sb + c * planeb, p.dy + ((size_t)c * p.rows + LEAD + y) * 8, planeb, barF + 8 * s);
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16(128, p.N, 1, 1);
        bool ok = true;
        for (int i = 0; i < ntile; ++i) {
            const int s = i % WG_STAGES, u = i / WG_STAGES;
            if (!mb_wait(barF + 8 * s, u & 1, p.wait_limit, p.err, 22)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sa = base + s * stage, sb = sa + a_bytes;
            const uint64_t ad = sdesc(sa, 128, planeb), bd = sdesc(sb, 128, planeb);
            tc_mma(tmem, ad, bd, idesc, i != 0);
#pragma unroll 8
            for (int ks = 1; ks < p.kt / 16; ++ks)            // 16 rows x 16 B = 16 units per step
                tc_mma(tmem, ad + (uint64_t)(ks * 16), bd + (uint64_t)(ks * 16), idesc, 1u);
            tc_commit(barE + 8 * s);
        }
        if (ok && ntile > 0) tc_commit(bar_done);
    }
    __syncwarp();

    const bool done = ntile == 0 || mb_wait(bar_done, 0, p.wait_limit, p.err, 23);
    tc_fence_after();
    const int row = warp * 32 + lane;
    float *out = p.partial + (((size_t)split * p.ngroups + g) * 128 + row) * p.N;
    for (int c16 = 0; c16 < p.N / 16; ++c16) {
        float v[16];
        tm_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c16 * 16, v);
        if (!done) continue;
        float4 *o = reinterpret_cast<float4 *>(out + c16 * 16);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            o[i] = ntile > 0 ? make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3])
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) tm_dealloc(tmem, ncols);
}

size_t conv_smem_bytes(const ConvParams &p)
{
    const size_t upl = p.cg / 8 < 4 ? p.cg / 8 : 4;
    const size_t wbytes = p.resident ? (size_t)p.ngroups * p.taps * p.N * p.cg * 2 : (size_t)p.slots * p.N * upl * 16;
    return 2 * upl * p.plane + wbytes + 64 + 16 * p.slots + 8 + 1024;
}

size_t wgrad_smem_bytes(const WgradParams &p)
{
    return (size_t)WG_STAGES * (16 + p.N / 8) * p.kt * 16 + 16 * WG_STAGES + 16 + 1024;
}

// Resident CTAs x TMEM columns must stay within the SM's 512 columns, or a
// CTA's allocation would wait for another CTA to exit.
static size_t smem_for_tmem(size_t smem, uint32_t ncols)
{
    const size_t per_sm = 228 * 1024;
    const size_t max_ctas = 512 / ncols;
    const size_t need = per_sm / (max_ctas + 1) + 1;   // (max_ctas + 1) CTAs no longer fit
    return smem < need ? need : smem;
}

cudaError_t launch_conv(const ConvParams &p, cudaStream_t s)
{
    const size_t smem = smem_for_tmem(conv_smem_bytes(p), p.ncols);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_tc, CONV_THREADS, smem)) != cudaSuccess)
        return e;
    per_sm = std::max(1, std::min(per_sm, (int)(512 / p.ncols)));
    if (p.mt != 2) return cudaErrorInvalidValue;     // the MMA issue loop is unrolled for two M tiles
    const int ntiles = (p.P + p.mt * 128 - 1) / (p.mt * 128);
    const int grid = std::max(1, std::min(ntiles, sms * per_sm));
    k_conv_tc<<<grid, CONV_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_wgrad(const WgradParams &p, int splits, cudaStream_t s)
{
    size_t smem = smem_for_tmem(wgrad_smem_bytes(p), p.N < 32 ? 32 : p.N);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_wgrad_tc<<<dim3(p.ngroups, splits), WG_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace zda
