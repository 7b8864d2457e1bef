// Internal declarations of the surrogate network (libzda, sm_103a).
#pragma once
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

// Activation layout ("planar"): a tensor of C channels (a multiple of 8)
// over the zero-bordered positions of one level (n samples x (H + 2) x
// (W + 2)) is stored as C / 8 planes of `rows` rows of 8 channels (16 B);
// position p lives at row LEAD + p.  The rows before LEAD and after the
// last 256-position tile are zero, so every convolution window is one
// contiguous run of rows per plane (a single bulk copy).
constexpr int LEAD = 256;

// Implicit-GEMM 3x3 (or 1x1) convolution: output position p, tap t reads
// input position p + off(t), off = (dy - 1) Wp + (dx - 1), so every tap's A
// operand is the same shared-memory window seen from another start row.
struct ConvParams {
    int P;                 // positions of the level: n Hp Wp
    int Hp, Wp;            // padded image size
    int taps;              // 9 or 1
    int halo;              // window rows before the tile's first position (Wp + 1, or 0)
    int R;                 // window rows: mt 128 + 2 halo
    int plane;             // bytes per 8-channel plane of the window in shared memory (>= R 16)
    long rows;             // rows per plane of the input / output tensors
    int cg;                // input channels per group (16, 32 or 64)
    int ngroups;           // 1, or 2 when the input is the concatenation of two tensors
    int N;                 // GEMM N = output channels (16 .. 128)
    int mt;                // 128-row M tiles per tile (one window)
    int slots;             // weight ring slots (streamed weights)
    int resident;          // 1: all weight blocks loaded once per CTA (no ring)
    uint32_t ncols;        // TMEM columns allocated
    const uint16_t *in0, *in1;   // planar inputs of group 0 / 1 (cg channels each)
    const uint16_t *wimg;  // weight images [ngroups][taps][N cg] (bf16, operand layout)
    const float *bias;     // [nbias] or null (channels >= nbias get no bias)
    int nbias;
    int epi;
    void *out0, *out1;     // bf16 planar outputs of out_ld channels (out1: channels >= out_ld when
                           // N = 2 out_ld), or the caller's f32 tensor [n][H][W][out_ld]
                           // (EPI_F32, EPI_GRAD_F32: interior positions only)
    int out_ld;
    const uint16_t *mask0, *mask1;   // gradient masks: planar post-activation tensors (out_ld channels) or null
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
    long rows;             // rows per plane of x0, x1 and dy
    const uint16_t *x0, *x1, *dy;   // planar input(s) and output gradient
    float *partial;        // [splits][ngroups][128][N]
    int *err;
    int wait_limit;
};

constexpr int CONV_THREADS = 352;   // persistent convolution: producer, 2 MMA and 8 epilogue warps
constexpr int WG_THREADS = 128;
constexpr int WG_KT = 128;
constexpr int WG_STAGES = 2;

size_t conv_smem_bytes(const ConvParams &p);
size_t wgrad_smem_bytes(const WgradParams &p);
cudaError_t launch_conv(const ConvParams &p, cudaStream_t s);
cudaError_t launch_wgrad(const WgradParams &p, int splits, cudaStream_t s);

}  // namespace nn
}  // namespace zda
