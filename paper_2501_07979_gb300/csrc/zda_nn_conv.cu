// Tensor-core kernels of the surrogate network (sm_103a): BF16 operands
// staged in shared memory by TMA / bulk copies, tcgen05.mma accumulating in
// FP32 in tensor memory, epilogues reading TMEM with tcgen05.ld.
//
// k_conv_tc  -- forward convolution and its input-gradient (transposed)
//               convolution.  A CTA owns mt x 128 consecutive padded
//               positions and all N output channels.  One TMA window of the
//               input (the CTA's positions plus a halo of Wp + 1 rows on each
//               side) serves all taps: tap t is the same window seen from
//               start row halo + off(t), i.e. a different descriptor start
//               address, so no im2col copy is ever made.  Weights stream
//               through a ring of per-tap slots (bulk copies).
// k_wgrad_tc -- weight gradient: both operands MN-major (channels contiguous),
//               reduction over positions; M = 128 rows hold 128 / c_in taps'
//               shifted copies of the input, each loaded pre-shifted by TMA.
//
// Roles (128 threads): warp 0 lane 0 = producer (TMA), warp 1 lane 0 = MMA
// issuer, warp 2 = TMEM allocator, all four warps = epilogue (warp w reads
// TMEM lanes 32w .. 32w + 31).  Every mbarrier wait is bounded; a timeout sets
// the error word and the CTA skips its stores, frees TMEM and exits.
#include <cuda_bf16.h>

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

__global__ void __launch_bounds__(CONV_THREADS, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1, const ConvParams p)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t raw = su32(smem), base = (raw + 1023u) & ~1023u;   // TMA destinations: 1024-aligned window
    const uint32_t a_bytes = (uint32_t)(p.cg / 8) * p.plane;
    const uint32_t wslot = (uint32_t)p.N * p.cg * 2;
    const uint32_t sA = base, sW = base + a_bytes;
    const uint32_t sBar = sW + p.slots * wslot;             // 8-byte barriers
    const uint32_t barA_full = sBar, barA_free = sBar + 8, bar_done = sBar + 16;
    const uint32_t barW_full = sBar + 24, barW_empty = barW_full + 8 * p.slots;
    const uint32_t sTmem = barW_empty + 8 * p.slots;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + (sTmem - raw));

    const int p0 = blockIdx.x * p.mt * 128;

    if (threadIdx.x == 0) {
        mb_init(barA_full, 1);
        mb_init(barA_free, 1);
        mb_init(bar_done, 1);
        for (int s = 0; s < p.slots; ++s) {
            mb_init(barW_full + 8 * s, 1);
            mb_init(barW_empty + 8 * s, 1);
        }
        mb_fence_init();
    }
    if (warp == 2) tm_alloc(sTmem, p.ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // ---------------- producer
        int it = 0;
        for (int g = 0; g < p.ngroups; ++g) {
            if (g > 0 && !mb_wait(barA_free, (g - 1) & 1, p.wait_limit, p.err, 11)) break;
            const CUtensorMap *tm = g == 0 ? &tm0 : &tm1;
            mb_expect_tx(barA_full, a_bytes);
            for (int c8 = 0; c8 < p.cg / 8; ++c8)
                for (int k = 0; k < p.npiece; ++k)
                    tma_load_2d(sA + c8 * p.plane + k * p.br * 16, tm, c8 * 8, p0 - p.halo + k * p.br, barA_full);
            bool ok = true;
            for (int t = 0; t < p.taps; ++t, ++it) {
                const int s = it % p.slots, u = it / p.slots;
                if (u > 0 && !mb_wait(barW_empty + 8 * s, (u - 1) & 1, p.wait_limit, p.err, 12)) {
                    ok = false;
                    break;
                }
                mb_expect_tx(barW_full + 8 * s, wslot);
                bulk_load(sW + s * wslot, p.wimg + (size_t)(g * p.taps + t) * p.N * p.cg, wslot, barW_full + 8 * s);
            }
            if (!ok) break;
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = idesc_bf16(128, p.N, 0, 0);
        int it = 0;
        bool ok = true;
        for (int g = 0; g < p.ngroups && ok; ++g) {
            if (!mb_wait(barA_full, g & 1, p.wait_limit, p.err, 13)) {
                ok = false;
                break;
            }
            for (int t = 0; t < p.taps; ++t, ++it) {
                const int s = it % p.slots, u = it / p.slots;
                if (!mb_wait(barW_full + 8 * s, u & 1, p.wait_limit, p.err, 14)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int off = p.taps == 9 ? (t / 3 - 1) * p.Wp + (t % 3 - 1) : 0;
                for (int m = 0; m < p.mt; ++m) {
                    const uint32_t row0 = (uint32_t)(p.halo + off + m * 128);
                    for (int ks = 0; ks < p.cg / 16; ++ks) {
                        const uint64_t ad = sdesc(sA + 2 * ks * p.plane + row0 * 16, p.plane, 128);
                        const uint64_t bd = sdesc(sW + s * wslot + ks * p.N * 32, 128, 256);
                        tc_mma(tmem + m * p.N, ad, bd, idesc, (g | t | ks) != 0);
                    }
                }
                tc_commit(barW_empty + 8 * s);
            }
            if (ok) tc_commit(barA_free);
        }
        if (ok) tc_commit(bar_done);
    }
    __syncwarp();

    // ---------------- epilogue
    const bool done = mb_wait(bar_done, 0, p.wait_limit, p.err, 15);
    tc_fence_after();
    const int HW = p.Hp * p.Wp;
    for (int m = 0; m < p.mt; ++m) {
        const int pos = p0 + m * 128 + warp * 32 + lane;
        const bool valid = done && pos < p.P;
        const int rem = pos % HW, y = rem / p.Wp, x = rem % p.Wp;
        const bool inner = y > 0 && y < p.Hp - 1 && x > 0 && x < p.Wp - 1;
        for (int c16 = 0; c16 < p.N / 16; ++c16) {
            float v[16];
            tm_ld16(tmem + ((uint32_t)(warp * 32) << 16) + m * p.N + c16 * 16, v);
            if (!valid) continue;
            const int cc = c16 * 16;
            if (p.epi == EPI_RELU_BF16 || p.epi == EPI_F32) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float t = v[i] + ((p.bias && cc + i < p.nbias) ? __ldg(p.bias + cc + i) : 0.f);
                    if (p.epi == EPI_RELU_BF16) t = fmaxf(t, 0.f);
                    v[i] = inner ? t : 0.f;
                }
                if (p.epi == EPI_RELU_BF16) {
                    uint4 *o = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(p.out0) + (size_t)pos * p.out_ld + cc);
                    o[0] = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                      pack_bf16(v[6], v[7]));
                    o[1] = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                                      pack_bf16(v[14], v[15]));
                } else {
                    float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(p.out0) + (size_t)pos * p.out_ld + cc);
#pragma unroll
                    for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
            } else if (p.epi == EPI_GRAD_BF16) {
                const int half = cc >= p.out_ld ? 1 : 0;
                const int c = cc - half * p.out_ld;
                const uint16_t *mk = half ? p.mask1 : p.mask0;
                if (mk) {
                    const uint4 *mp = reinterpret_cast<const uint4 *>(mk + (size_t)pos * p.out_ld + c);
                    uint4 q[2] = {__ldg(mp), __ldg(mp + 1)};
                    const uint16_t *h = reinterpret_cast<const uint16_t *>(q);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (!bf16_pos(h[i])) v[i] = 0.f;
                }
                if (!inner) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = 0.f;
                }
                uint4 *o = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(half ? p.out1 : p.out0) +
                                                     (size_t)pos * p.out_ld + c);
                o[0] = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                  pack_bf16(v[6], v[7]));
                o[1] = make_uint4(pack_bf16(v[8], v[9]), pack_bf16(v[10], v[11]), pack_bf16(v[12], v[13]),
                                  pack_bf16(v[14], v[15]));
            } else {   // EPI_GRAD_F32
                if (cc >= p.out_ld) continue;
                float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(p.out0) + (size_t)pos * p.out_ld + cc);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    o[i] = inner ? make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3])
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) tm_dealloc(tmem, p.ncols);
}

__global__ void __launch_bounds__(CONV_THREADS, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap tx0, const __grid_constant__ CUtensorMap tx1,
               const __grid_constant__ CUtensorMap tdy, const WgradParams p)
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
                    tma_load_2d(sa + (j * p.cin_planes + c) * planeb, second ? &tx1 : &tx0, (second ? c - 8 : c) * 8,
                                y + off, barF + 8 * s);
                }
            }
            for (int c = 0; c < p.N / 8; ++c) tma_load_2d(sb + c * planeb, &tdy, c * 8, y, barF + 8 * s);
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
            for (int ks = 0; ks < p.kt / 16; ++ks) {
                const uint64_t ad = sdesc(sa + ks * 256, 128, planeb);
                const uint64_t bd = sdesc(sb + ks * 256, 128, planeb);
                tc_mma(tmem, ad, bd, idesc, (i | ks) != 0);
            }
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
    return (size_t)(p.cg / 8) * p.plane + (size_t)p.slots * p.N * p.cg * 2 + 24 + 16 * p.slots + 16 + 1024;
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

cudaError_t launch_conv(const CUtensorMap &tm0, const CUtensorMap &tm1, const ConvParams &p, cudaStream_t s)
{
    size_t smem = smem_for_tmem(conv_smem_bytes(p), p.ncols);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (p.P + p.mt * 128 - 1) / (p.mt * 128);
    k_conv_tc<<<grid, CONV_THREADS, smem, s>>>(tm0, tm1, p);
    return cudaGetLastError();
}

cudaError_t launch_wgrad(const CUtensorMap &tx0, const CUtensorMap &tx1, const CUtensorMap &tdy, const WgradParams &p,
                         int splits, cudaStream_t s)
{
    size_t smem = smem_for_tmem(wgrad_smem_bytes(p), p.N < 32 ? 32 : p.N);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_wgrad_tc<<<dim3(p.ngroups, splits), CONV_THREADS, smem, s>>>(tx0, tx1, tdy, p);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace zda
