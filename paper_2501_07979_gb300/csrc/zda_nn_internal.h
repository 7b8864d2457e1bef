// Internal declarations of the surrogate network (libzda, sm_103a).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace zda {
namespace nn {

enum Epilogue {
    EPI_RELU_BF16 = 0,   // bias + ReLU -> bf16 (forward convolutions)
    EPI_F32 = 1,         // bias -> f32, no activation (head)
    EPI_GRAD_BF16 = 2,   // optional sign mask -> bf16, optionally split in two outputs (input gradients)
    EPI_GRAD_F32 = 3     // -> f32 (gradient of the network input)
};

// Implicit-GEMM 3x3 (or 1x1) convolution on zero-bordered ("padded") NHWC
// activations: output position p, tap t reads input position p + off(t),
// off = (dy - 1) Wp + (dx - 1), so every tap's A operand is the same shared
// memory window seen from another start row.
struct ConvParams {
    int P;                 // positions (rows) of the activation arrays: n Hp Wp
    int Hp, Wp;            // padded image size
    int taps;              // 9 or 1
    int halo;              // window rows before the CTA's first position
    int br, npiece;        // TMA box rows, boxes per channel-chunk plane
    int plane;             // bytes per 8-channel plane of the window (npiece br 16)
    int cg;                // input channels per group (16, 32 or 64)
    int ngroups;           // 1, or 2 when the input is the concatenation of two tensors
    int N;                 // GEMM N = output channels (16 .. 128)
    int mt;                // 128-row M tiles per CTA (one window)
    int slots;             // weight ring slots
    uint32_t ncols;        // TMEM columns allocated
    const uint16_t *wimg;  // weight images [ngroups][taps][N cg] (bf16, operand layout)
    const float *bias;     // [nbias] or null (channels >= nbias get no bias)
    int nbias;
    int epi;
    void *out0, *out1;     // outputs [P][out_ld]; out1 receives channels >= out_ld when N = 2 out_ld
    int out_ld;
    const uint16_t *mask0, *mask1;   // gradient masks (post-activation tensors, [P][out_ld]) or null
    int *err;
    int wait_limit;
};

// Weight gradient: D[(tap copy, c_in)][c_out] = sum_p X[p + off(tap)][c_in] dY[p][c_out],
// M = 128 rows = several taps' copies of the input, reduction over positions.
struct WgradParams {
    int P, Hp, Wp;
    int taps;              // 9 or 1
    int cin_planes;        // input channels / 8 per tap copy (2, 4, 8 or 16)
    int ntap_grp;          // taps per 128-row group (16 / cin_planes)
    int ngroups;           // ceil(taps / ntap_grp)
    int two_inputs;        // planes 8..15 come from the second tensor (concatenated input)
    int N;                 // output channels (GEMM N)
    int kt;                // positions per stage (128)
    int ntiles;            // ceil(P / kt)
    int tiles_per_cta;
    float *partial;        // [splits][ngroups][128][N]
    int *err;
    int wait_limit;
};

constexpr int CONV_THREADS = 128;
constexpr int WG_KT = 128;
constexpr int WG_STAGES = 2;

size_t conv_smem_bytes(const ConvParams &p);
size_t wgrad_smem_bytes(const WgradParams &p);
cudaError_t launch_conv(const CUtensorMap &tm0, const CUtensorMap &tm1, const ConvParams &p, cudaStream_t s);
cudaError_t launch_wgrad(const CUtensorMap &tx0, const CUtensorMap &tx1, const CUtensorMap &tdy, const WgradParams &p,
                         int splits, cudaStream_t s);

}  // namespace nn
}  // namespace zda
