// Zone surrogate network: host orchestration, C ABI (include/zda_nn.h) and
// the bandwidth-bound helper kernels (packing, pooling, upsampling, gradient
// combination, reductions, loss, Adam).  The convolutions and their
// gradients run in the tensor-core kernels of zda_nn_conv.cu.
//
// Activations live in zero-bordered NHWC arrays: level l (H_l = H >> l,
// W_l = W >> l) of n samples is a [n][H_l + 2][W_l + 2][C] array whose
// border positions hold zeros, so a 3x3 convolution with zero padding is a
// sum over nine constant position offsets (see k_conv_tc).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "zda.h"
#include "zda_internal.h"
#include "zda_nn.h"
#include "zda_nn_internal.h"

using namespace zda::nn;

namespace {

zda_status nn_fail(zda_status s, const std::string &m)
{
    zda_internal_set_error(m.c_str());
    return s;
}

#define NN_CUDA(expr)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return nn_fail(ZDA_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int C = 64;      // network width
constexpr int NL = 15;     // parameterised layers
constexpr int LEV = 4;     // resolution levels

__device__ __forceinline__ float bf2f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }
__device__ __forceinline__ uint16_t f2bf(float f)
{
    __nv_bfloat16 h = __float2bfloat16_rn(f);
    return *reinterpret_cast<uint16_t *>(&h);
}
__device__ __forceinline__ bool interior(int y, int x, int Hp, int Wp) { return y > 0 && y < Hp - 1 && x > 0 && x < Wp - 1; }

// ---------------------------------------------------------------- helper kernels
// Planar element offset of (channel plane c8, position pos) in a tensor of `rows` rows per plane.
__device__ __forceinline__ size_t pofs(long rows, int c8, long pos) { return ((size_t)c8 * rows + LEAD + pos) * 8; }

// x [n][H][W][ic] f32 -> planar bf16, 16 channels (2 planes), positions < Pt (zero border, zero tail)
__global__ void k_pack_input(const float *x, int n, int H, int W, int ic, long Pt, long rows, uint16_t *out)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * Pt) return;
    const int c8 = (int)(i / Pt);
    const long pos = i % Pt;
    const int Hp = H + 2, Wp = W + 2;
    const long P = (long)n * Hp * Wp;
    const int rem = (int)(pos % (Hp * Wp)), y = rem / Wp, xx = rem % Wp;
    uint16_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (pos < P && interior(y, xx, Hp, Wp)) {
        const float *src = x + (((pos / (Hp * Wp)) * H + (y - 1)) * W + (xx - 1)) * ic;
        for (int e = 0; e < 8; ++e) {
            const int c = c8 * 8 + e;
            if (c < ic) r[e] = f2bf(src[c]);
        }
    }
    *reinterpret_cast<uint4 *>(out + pofs(rows, c8, pos)) = *reinterpret_cast<uint4 *>(r);
}

// [n][H][W][nc] f32 -> planar bf16, 32 channels (4 planes), positions < Pt (zeros elsewhere)
__global__ void k_pack_grad(const float *dy, int n, int H, int W, int nc, long Pt, long rows, uint16_t *out)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * Pt) return;
    const int c8 = (int)(i / Pt);
    const long pos = i % Pt;
    const int Hp = H + 2, Wp = W + 2;
    const long P = (long)n * Hp * Wp;
    const int rem = (int)(pos % (Hp * Wp)), y = rem / Wp, x = rem % Wp;
    uint16_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (pos < P && interior(y, x, Hp, Wp)) {
        const float *src = dy + (((pos / (Hp * Wp)) * H + (y - 1)) * W + (x - 1)) * nc;
        for (int e = 0; e < 8; ++e) {
            const int c = c8 * 8 + e;
            if (c < nc) r[e] = f2bf(src[c]);
        }
    }
    *reinterpret_cast<uint4 *>(out + pofs(rows, c8, pos)) = *reinterpret_cast<uint4 *>(r);
}

// The position-parallel kernels below run one thread per (plane, position)
// over Pt positions (the 256-rounded tail is written as zeros), 64 channels.
struct Lev {
    int n, H, W;        // samples, interior size of this level
    long rows, Pt;      // rows per plane, positions covered (multiple of 256)
};

__device__ __forceinline__ bool decode(const Lev &L, long pos, long &s, int &y, int &x)
{
    const int Hp = L.H + 2, Wp = L.W + 2;
    s = pos / (Hp * Wp);
    const int rem = (int)(pos % (Hp * Wp));
    y = rem / Wp;
    x = rem % Wp;
    return s < L.n && interior(y, x, Hp, Wp);
}

// avgpool: coarse interior (i, j) = mean of fine interior (2i .. 2i+1, 2j .. 2j+1)
__global__ void k_pool(const uint16_t *in, Lev F, uint16_t *out, Lev Cc)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * Cc.Pt) return;
    const int c8 = (int)(i / Cc.Pt);
    const long pos = i % Cc.Pt;
    long s;
    int y, x;
    uint4 o = make_uint4(0, 0, 0, 0);
    if (decode(Cc, pos, s, y, x)) {
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const long fp = (s * (F.H + 2) + 2 * y - 1 + a) * (F.W + 2) + 2 * x - 1 + b;
                const uint4 q = *reinterpret_cast<const uint4 *>(in + pofs(F.rows, c8, fp));
                const uint16_t *h = reinterpret_cast<const uint16_t *>(&q);
                for (int e = 0; e < 8; ++e) acc[e] += bf2f(h[e]);
            }
        uint16_t r[8];
        for (int e = 0; e < 8; ++e) r[e] = f2bf(0.25f * acc[e]);
        o = *reinterpret_cast<uint4 *>(r);
    }
    *reinterpret_cast<uint4 *>(out + pofs(Cc.rows, c8, pos)) = o;
}

// nearest upsampling: fine interior (i, j) = coarse interior (i / 2, j / 2)
__global__ void k_up(const uint16_t *in, Lev Cc, uint16_t *out, Lev F)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * F.Pt) return;
    const int c8 = (int)(i / F.Pt);
    const long pos = i % F.Pt;
    long s;
    int y, x;
    uint4 o = make_uint4(0, 0, 0, 0);
    if (decode(F, pos, s, y, x)) {
        const long cp = (s * (Cc.H + 2) + (y - 1) / 2 + 1) * (Cc.W + 2) + (x - 1) / 2 + 1;
        o = *reinterpret_cast<const uint4 *>(in + pofs(Cc.rows, c8, cp));
    }
    *reinterpret_cast<uint4 *>(out + pofs(F.rows, c8, pos)) = o;
}

// transpose of nearest upsampling (sum over each 2x2 block) times the sign
// mask of the coarse activation: coarse output
__global__ void k_up_bwd_mask(const uint16_t *g, Lev F, const uint16_t *act, uint16_t *out, Lev Cc)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * Cc.Pt) return;
    const int c8 = (int)(i / Cc.Pt);
    const long pos = i % Cc.Pt;
    long s;
    int y, x;
    uint4 o = make_uint4(0, 0, 0, 0);
    if (decode(Cc, pos, s, y, x)) {
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const long fp = (s * (F.H + 2) + 2 * y - 1 + a) * (F.W + 2) + 2 * x - 1 + b;
                const uint4 q = *reinterpret_cast<const uint4 *>(g + pofs(F.rows, c8, fp));
                const uint16_t *h = reinterpret_cast<const uint16_t *>(&q);
                for (int e = 0; e < 8; ++e) acc[e] += bf2f(h[e]);
            }
        const uint4 mq = *reinterpret_cast<const uint4 *>(act + pofs(Cc.rows, c8, pos));
        const uint16_t *m = reinterpret_cast<const uint16_t *>(&mq);
        uint16_t r[8];
        for (int e = 0; e < 8; ++e) r[e] = f2bf(bf2f(m[e]) > 0.f ? acc[e] : 0.f);
        o = *reinterpret_cast<uint4 *>(r);
    }
    *reinterpret_cast<uint4 *>(out + pofs(Cc.rows, c8, pos)) = o;
}

// skip gradient of level l: mask(act > 0) * (g_skip + transpose of avgpool applied to g_coarse)
__global__ void k_skip_combine(const uint16_t *gs, const uint16_t *gc, Lev Cc, const uint16_t *act, uint16_t *out,
                               Lev F)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 8 * F.Pt) return;
    const int c8 = (int)(i / F.Pt);
    const long pos = i % F.Pt;
    long s;
    int y, x;
    uint4 o = make_uint4(0, 0, 0, 0);
    if (decode(F, pos, s, y, x)) {
        const uint4 a = *reinterpret_cast<const uint4 *>(gs + pofs(F.rows, c8, pos));
        const long cp = (s * (Cc.H + 2) + (y - 1) / 2 + 1) * (Cc.W + 2) + (x - 1) / 2 + 1;
        const uint4 b = *reinterpret_cast<const uint4 *>(gc + pofs(Cc.rows, c8, cp));
        const uint4 mq = *reinterpret_cast<const uint4 *>(act + pofs(F.rows, c8, pos));
        const uint16_t *ha = reinterpret_cast<const uint16_t *>(&a), *hb = reinterpret_cast<const uint16_t *>(&b),
                       *m = reinterpret_cast<const uint16_t *>(&mq);
        uint16_t r[8];
        for (int e = 0; e < 8; ++e) r[e] = f2bf(bf2f(m[e]) > 0.f ? bf2f(ha[e]) + 0.25f * bf2f(hb[e]) : 0.f);
        o = *reinterpret_cast<uint4 *>(r);
    }
    *reinterpret_cast<uint4 *>(out + pofs(F.rows, c8, pos)) = o;
}

// column sums of a planar bf16 tensor of `planes` planes over positions < P
// (channels < nc): partial[block][c]; thread t covers channel t % 8 of rows
// t / 8, t / 8 + 32, ... of each plane.
__global__ void k_colsum(const uint16_t *g, long rows, long P, int planes, int nc, float *partial)
{
    __shared__ float red[256];
    const int e = threadIdx.x % 8, r0 = threadIdx.x / 8;
    for (int c8 = 0; c8 < planes; ++c8) {
        float acc = 0.f;
        for (long p = (long)blockIdx.x * 32 + r0; p < P; p += (long)gridDim.x * 32) acc += bf2f(g[pofs(rows, c8, p) + e]);
        red[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x < 8) {
            float s = 0.f;
            for (int r = 0; r < 32; ++r) s += red[r * 8 + threadIdx.x];
            const int c = c8 * 8 + threadIdx.x;
            if (c < nc) partial[(size_t)blockIdx.x * nc + c] = s;
        }
        __syncthreads();
    }
}

// Layer gradient from the wgrad partials [splits][ngroups][128][N] and the
// bias partials [nblk][cout]: grads[w[co][t][ci]], grads[b[co]].
__global__ void k_layer_grad(const float *wpart, int splits, int ngroups, int ntap_grp, int cin_pad, int N,
                             const float *bpart, int nblk, int cout, int cin, int taps, float *grad)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nw = (long)cout * taps * cin;
    if (i < nw) {
        const int ci = (int)(i % cin), t = (int)((i / cin) % taps), co = (int)(i / ((long)cin * taps));
        const int g = t / ntap_grp, row = (t % ntap_grp) * cin_pad + ci;
        float s = 0.f;
        for (int k = 0; k < splits; ++k) s += wpart[(((size_t)k * ngroups + g) * 128 + row) * N + co];
        grad[i] = s;
    } else if (i < nw + cout) {
        const int co = (int)(i - nw);
        float s = 0.f;
        for (int k = 0; k < nblk; ++k) s += bpart[(size_t)k * cout + co];
        grad[i] = s;
    }
}

struct PackLayer {
    long off;          // parameter offset of w
    int k, cin, cout;  // kernel size, true channels
    int cin_pad;       // input channels in the activation (16 for the input layer, else cin)
    int nf;            // forward GEMM N (cout padded to 32 for the head, else 64)
    long img_f, img_d; // element offsets of the forward / input-gradient images
};

// Operand image of one (group, tap) block, K-major, no swizzle: element
// (n, k) of an N x cg block at ks = k / 16: ks N 16 + (n / 8) 128 + ((k / 8) % 2) 64 + (n % 8) 8 + k % 8.
__device__ __forceinline__ long img_index(int n, int k, int N)
{
    return (long)(k / 16) * N * 16 + (n / 8) * 128 + ((k / 8) % 2) * 64 + (n % 8) * 8 + (k % 8);
}

__global__ void k_pack_weights(const float *params, PackLayer L, uint16_t *img)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int taps = L.k * L.k;
    const int cg = L.cin_pad > 64 ? 64 : L.cin_pad;
    const long nf_tot = (long)taps * L.nf * L.cin_pad;           // forward image elements
    const long nd_tot = (long)taps * L.cin_pad * L.nf;           // input-gradient image elements
    if (i < nf_tot) {
        // forward: group g (64 channels), tap t, row n = c_out, column k = c_in within the group
        const int k = (int)(i % cg), n = (int)((i / cg) % L.nf), t = (int)((i / ((long)cg * L.nf)) % taps);
        const int g = (int)(i / ((long)cg * L.nf * taps));
        const int ci = g * cg + k;
        float v = 0.f;
        if (n < L.cout && ci < L.cin) v = params[L.off + (((long)n * taps + t) * L.cin) + ci];
        img[L.img_f + (long)(g * taps + t) * L.nf * cg + img_index(n, k, L.nf)] = f2bf(v);
    } else if (i < nf_tot + nd_tot) {
        // input gradient: tap t' (flipped), row n = c_in, column k = c_out
        const long j = i - nf_tot;
        const int k = (int)(j % L.nf), n = (int)((j / L.nf) % L.cin_pad), tp = (int)(j / ((long)L.nf * L.cin_pad));
        const int ty = tp / L.k, tx = tp % L.k;
        const int t = (L.k - 1 - ty) * L.k + (L.k - 1 - tx);
        float v = 0.f;
        if (k < L.cout && n < L.cin) v = params[L.off + (((long)k * taps + t) * L.cin) + n];
        img[L.img_d + (long)tp * L.cin_pad * L.nf + img_index(n, k, L.cin_pad)] = f2bf(v);
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, long n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_mse(const float *y, const float *t, long n, float *dy, float *partial)
{
    __shared__ float red[256];
    float acc = 0.f;
    const float sc = 2.f / (float)n;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = sc * d;
        acc += d * d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_mse_final(const float *partial, int nblk, long n, float *loss)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[b];
    *loss = (float)(s / (double)n);
}

unsigned nblocks(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- layers
struct Layer {
    const char *name;
    int k, cin, cout, level;
    int cin_pad, nf;
    long off;          // parameter offset
    long img_f, img_d; // image offsets (elements)
};

}  // namespace

struct zda_nn {
    int device = 0;
    zda_nn_desc d{};
    int H[LEV], W[LEV];
    long rows[LEV];        // rows per plane of the level's planar tensors (batch capacity)
    Layer L[NL];
    long nparam = 0, img_elems = 0;
    double flops = 0;
    // workspace
    uint8_t *ws = nullptr;
    size_t ws_bytes = 0, need = 0;
    struct Off {
        size_t params, grads, m, v, img, x16, gy, wpart, bpart, mpart, err;
        size_t act[LEV][8];   // per level: enc_a, enc_b, in (pooled input), up, dec_a, dec_b, (level 3: bot_a, bot_b)
        size_t g[LEV][4];     // per level: gA, gB, gU, gS
    } o{};
    size_t wpart_floats = 0;
    int bpart_blocks = 240;
    int adam_step = 0;
    long long launches = 0;
    int n_fwd = 0;
    bool bound = false;
    // optional CUDA-event timing of the convolution launches
    bool timing = false;
    std::vector<cudaEvent_t> ev;       // pairs (before, after)
    std::vector<double> ev_flops;      // useful FLOPs of each timed launch
    size_t ev_used = 0;
    ~zda_nn()
    {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

namespace {

enum { A_ENCA = 0, A_ENCB, A_IN, A_UP, A_DECA, A_DECB };
enum { G_A = 0, G_B, G_U, G_S };

template <class T> T *at(zda_nn *net, size_t off) { return reinterpret_cast<T *>(net->ws + off); }

long pos_count(const zda_nn *net, int lev, int n) { return (long)n * (net->H[lev] + 2) * (net->W[lev] + 2); }
long pos_tiles(const zda_nn *net, int lev, int n) { return (pos_count(net, lev, n) + 255) / 256 * 256; }
Lev lev(const zda_nn *net, int l, int n) { return Lev{n, net->H[l], net->W[l], net->rows[l], pos_tiles(net, l, n)}; }

void build_layers(zda_nn *net)
{
    const int ic = net->d.in_ch, oc = net->d.out_ch;
    const char *names[NL] = {"enc0a", "enc0b", "enc1a", "enc1b", "enc2a", "enc2b", "bota", "botb",
                             "dec2a", "dec2b", "dec1a", "dec1b", "dec0a", "dec0b", "head"};
    const int lev[NL] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0, 0};
    long off = 0, img = 0;
    double fl = 0;
    for (int i = 0; i < NL; ++i) {
        Layer &l = net->L[i];
        l.name = names[i];
        l.level = lev[i];
        l.k = i == NL - 1 ? 1 : 3;
        l.cin = i == 0 ? ic : ((i == 8 || i == 10 || i == 12) ? 2 * C : C);
        l.cout = i == NL - 1 ? oc : C;
        l.cin_pad = i == 0 ? 16 : l.cin;
        l.nf = i == NL - 1 ? 32 : C;
        l.off = off;
        off += (long)l.cout * l.k * l.k * l.cin + l.cout;
        l.img_f = img;
        img += (long)l.k * l.k * l.nf * l.cin_pad;
        l.img_d = img;
        img += (long)l.k * l.k * l.nf * l.cin_pad;
        fl += 2.0 * net->H[l.level] * net->W[l.level] * l.k * l.k * l.cin * l.cout;
    }
    net->nparam = off;
    net->img_elems = img;
    net->flops = fl;
}

int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Convolution (forward or input gradient) of one layer.
//   in0 / in1 : input tensors (in1 = second half of a concatenated input or null)
//   cg        : channels per input tensor;  N : GEMM output channels
zda_status conv(zda_nn *net, int lv, int n, int taps, const uint16_t *in0, const uint16_t *in1, int cg, int N,
                const uint16_t *wimg, const float *bias, int nbias, int epi, void *out0, void *out1, int out_ld,
                const uint16_t *mask0, const uint16_t *mask1, cudaStream_t s, double flops = 0.0)
{
    ConvParams p{};
    p.Hp = net->H[lv] + 2;
    p.Wp = net->W[lv] + 2;
    p.P = (int)pos_count(net, lv, n);
    p.taps = taps;
    p.halo = taps == 9 ? p.Wp + 1 : 0;
    p.mt = 2;
    p.R = p.mt * 128 + 2 * p.halo;
    p.plane = round_up(p.R, 8) * 16;
    p.rows = net->rows[lv];
    p.cg = cg;
    p.ngroups = in1 ? 2 : 1;
    p.N = N;
    // weights resident if they fit beside the two window stages, else a ring
    // of as many per-tap slots as fit (at most 8)
    const size_t budget = 220 * 1024;
    const size_t upl = std::min(cg / 8, 4);                    // window planes per unit (32 channels)
    const size_t win2 = 2 * upl * p.plane, wslot = (size_t)N * cg * 2, uslot = (size_t)N * upl * 16;
    p.resident = win2 + (size_t)p.ngroups * taps * wslot <= budget ? 1 : 0;
    p.slots = p.resident ? 1 : (int)std::max<size_t>(2, std::min<size_t>(8, (budget - win2) / uslot));
    uint32_t nc = 32;
    while (nc < (uint32_t)(2 * p.mt * N)) nc <<= 1;   // two accumulators (double buffering)
    p.ncols = nc;
    p.in0 = in0;
    p.in1 = in1;
    p.wimg = wimg;
    p.bias = bias;
    p.nbias = nbias;
    p.epi = epi;
    p.out0 = out0;
    p.out1 = out1;
    p.out_ld = out_ld;
    p.mask0 = mask0;
    p.mask1 = mask1;
    p.err = at<int>(net, net->o.err);
    p.wait_limit = 1 << 22;
    const bool timed = net->timing && flops > 0.0;
    if (timed) {
        if (net->ev_used + 2 > net->ev.size()) {
            for (int k = 0; k < 64; ++k) {
                cudaEvent_t ev;
                NN_CUDA(cudaEventCreate(&ev));
                net->ev.push_back(ev);
            }
        }
        NN_CUDA(cudaEventRecord(net->ev[net->ev_used], s));
    }
    cudaError_t e = launch_conv(p, s);
    if (e != cudaSuccess) return nn_fail(ZDA_ERR_CUDA, std::string("conv launch: ") + cudaGetErrorString(e));
    if (timed) {
        NN_CUDA(cudaEventRecord(net->ev[net->ev_used + 1], s));
        net->ev_used += 2;
        net->ev_flops.push_back(flops);
    }
    net->launches++;
    return ZDA_OK;
}

// Weight + bias gradient of layer li: x0 (/x1) its input, g the gradient of its
// pre-activation output ([P][ldg] bf16).
zda_status layer_grad(zda_nn *net, int li, int n, const uint16_t *x0, const uint16_t *x1, const uint16_t *g, int ldg,
                      cudaStream_t s)
{
    const Layer &l = net->L[li];
    WgradParams p{};
    p.Hp = net->H[l.level] + 2;
    p.Wp = net->W[l.level] + 2;
    p.P = (int)pos_count(net, l.level, n);
    p.taps = l.k * l.k;
    p.cin_planes = l.cin_pad / 8;
    p.ntap_grp = 16 / p.cin_planes;
    p.ngroups = (p.taps + p.ntap_grp - 1) / p.ntap_grp;
    p.two_inputs = x1 != nullptr;
    p.N = ldg;
    p.kt = WG_KT;
    p.ntiles = (p.P + p.kt - 1) / p.kt;
    int splits = std::max(1, std::min(p.ntiles, (304 + p.ngroups - 1) / p.ngroups));
    p.tiles_per_cta = (p.ntiles + splits - 1) / splits;
    splits = (p.ntiles + p.tiles_per_cta - 1) / p.tiles_per_cta;
    if ((size_t)splits * p.ngroups * 128 * p.N > net->wpart_floats)
        return nn_fail(ZDA_ERR_OOM, "weight-gradient partial buffer too small");
    p.rows = net->rows[l.level];
    p.x0 = x0;
    p.x1 = x1;
    p.dy = g;
    p.partial = at<float>(net, net->o.wpart);
    p.err = at<int>(net, net->o.err);
    p.wait_limit = 1 << 22;
    cudaError_t e = launch_wgrad(p, splits, s);
    if (e != cudaSuccess) return nn_fail(ZDA_ERR_CUDA, std::string("wgrad launch: ") + cudaGetErrorString(e));
    k_colsum<<<net->bpart_blocks, 256, 0, s>>>(g, p.rows, p.P, ldg / 8, l.cout, at<float>(net, net->o.bpart));
    const long nw = (long)l.cout * p.taps * l.cin + l.cout;
    k_layer_grad<<<nblocks(nw), 256, 0, s>>>(at<float>(net, net->o.wpart), splits, p.ngroups, p.ntap_grp, l.cin_pad,
                                             p.N, at<float>(net, net->o.bpart), net->bpart_blocks, l.cout, l.cin,
                                             p.taps, at<float>(net, net->o.grads) + l.off);
    net->launches += 3;
    e = cudaGetLastError();
    if (e != cudaSuccess) return nn_fail(ZDA_ERR_CUDA, std::string("gradient reduction: ") + cudaGetErrorString(e));
    return ZDA_OK;
}

zda_status pack_all(zda_nn *net, cudaStream_t s)
{
    for (int i = 0; i < NL; ++i) {
        const Layer &l = net->L[i];
        PackLayer pl{l.off, l.k, l.cin, l.cout, l.cin_pad, l.nf, l.img_f, l.img_d};
        const long tot = 2L * l.k * l.k * l.nf * l.cin_pad;
        k_pack_weights<<<nblocks(tot), 256, 0, s>>>(at<float>(net, net->o.params), pl, at<uint16_t>(net, net->o.img));
        net->launches++;
    }
    NN_CUDA(cudaGetLastError());
    return ZDA_OK;
}

// useful forward FLOPs of layer i over n samples (true channel counts, H_l x W_l outputs)
double lf(const zda_nn *net, int i, int n)
{
    const Layer &l = net->L[i];
    return 2.0 * n * net->H[l.level] * net->W[l.level] * l.k * l.k * l.cin * l.cout;
}

const uint16_t *A(zda_nn *net, int lev, int k) { return at<uint16_t>(net, net->o.act[lev][k]); }
uint16_t *Aw(zda_nn *net, int lev, int k) { return at<uint16_t>(net, net->o.act[lev][k]); }
uint16_t *Gb(zda_nn *net, int lev, int k) { return at<uint16_t>(net, net->o.g[lev][k]); }
const uint16_t *Wf(zda_nn *net, int i) { return at<uint16_t>(net, net->o.img) + net->L[i].img_f; }
const uint16_t *Wd(zda_nn *net, int i) { return at<uint16_t>(net, net->o.img) + net->L[i].img_d; }
const float *Bias(zda_nn *net, int i) { return at<float>(net, net->o.params) + net->L[i].off + (long)net->L[i].cout * net->L[i].k * net->L[i].k * net->L[i].cin; }

}  // namespace

// ======================================================================== ABI
extern "C" {

zda_status zda_nn_create(int device, const zda_nn_desc *d, zda_nn **out)
{
    if (!d || !out) return nn_fail(ZDA_ERR_ARG, "null argument");
    *out = nullptr;
    if (d->batch < 1 || d->height < 8 || d->width < 8 || d->height % 8 || d->width % 8 || d->height > 1024 ||
        d->width > 176 || d->in_ch < 1 || d->in_ch > 16 || d->out_ch < 1 || d->out_ch > 32)
        return nn_fail(ZDA_ERR_ARG, "invalid network descriptor (H multiple of 8 in 8..1024, W multiple of 8 in "
                                    "8..176; 1..16 inputs; 1..32 outputs; batch >= 1)");
    const long P0 = (long)d->batch * (d->height + 2) * (d->width + 2);
    if (P0 * 64 > (1L << 31) - 1) return nn_fail(ZDA_ERR_ARG, "batch x image too large for 32-bit positions");
    zda_nn *net = new zda_nn();
    net->device = device;
    net->d = *d;
    for (int l = 0; l < LEV; ++l) {
        net->H[l] = d->height >> l;
        net->W[l] = d->width >> l;
        net->rows[l] = LEAD + pos_tiles(net, l, d->batch) + 256;   // zero lead rows, tiles, zero trail rows
    }
    build_layers(net);
    // workspace layout
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t r = o;
        o += (bytes + 255) / 256 * 256;
        return r;
    };
    const int B = d->batch;
    net->o.params = take(net->nparam * 4);
    net->o.grads = take(net->nparam * 4);
    net->o.m = take(net->nparam * 4);
    net->o.v = take(net->nparam * 4);
    net->o.img = take(net->img_elems * 2);
    net->o.x16 = take((size_t)net->rows[0] * 16 * 2);
    net->o.gy = take((size_t)net->rows[0] * 32 * 2);
    for (int l = 0; l < LEV; ++l) {
        const size_t t = (size_t)net->rows[l] * C * 2;
        for (int k = 0; k < 6; ++k) net->o.act[l][k] = take(t);
        for (int k = 0; k < 4; ++k) net->o.g[l][k] = take(t);
    }
    size_t wp = 0;
    for (int i = 0; i < NL; ++i) {
        const Layer &l = net->L[i];
        const int taps = l.k * l.k, ntg = 16 / (l.cin_pad / 8), ng = (taps + ntg - 1) / ntg;
        const size_t splits = (size_t)std::min<long>((pos_count(net, l.level, B) + 127) / 128, (304 + ng - 1) / ng) + 1;
        wp = std::max(wp, splits * ng * 128 * (size_t)(i == NL - 1 ? 32 : 64));
    }
    net->wpart_floats = wp;
    net->o.wpart = take(wp * 4);
    net->o.bpart = take((size_t)net->bpart_blocks * 64 * 4);
    net->o.mpart = take(1024 * 4);
    net->o.err = take(16);
    net->need = o;
    *out = net;
    return ZDA_OK;
}

void zda_nn_destroy(zda_nn *net) { delete net; }

zda_status zda_nn_param_count(const zda_nn *net, size_t *count)
{
    if (!net || !count) return nn_fail(ZDA_ERR_ARG, "null argument");
    *count = (size_t)net->nparam;
    return ZDA_OK;
}

zda_status zda_nn_forward_flops(const zda_nn *net, double *flops)
{
    if (!net || !flops) return nn_fail(ZDA_ERR_ARG, "null argument");
    *flops = net->flops;
    return ZDA_OK;
}

zda_status zda_nn_workspace_bytes(const zda_nn *net, size_t *bytes)
{
    if (!net || !bytes) return nn_fail(ZDA_ERR_ARG, "null argument");
    *bytes = net->need;
    return ZDA_OK;
}

zda_status zda_nn_bind_workspace(zda_nn *net, void *ws, size_t bytes)
{
    if (!net || !ws) return nn_fail(ZDA_ERR_ARG, "null argument");
    if (bytes < net->need) return nn_fail(ZDA_ERR_OOM, "workspace smaller than zda_nn_workspace_bytes");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return nn_fail(ZDA_ERR_ARG, "workspace must be 256-byte aligned");
    NN_CUDA(cudaSetDevice(net->device));
    net->ws = static_cast<uint8_t *>(ws);
    net->ws_bytes = bytes;
    NN_CUDA(cudaMemset(ws, 0, net->need));
    net->bound = true;
    net->adam_step = 0;
    net->n_fwd = 0;
    return ZDA_OK;
}

static zda_status need_bound(zda_nn *net)
{
    if (!net) return nn_fail(ZDA_ERR_ARG, "null network");
    if (!net->bound) return nn_fail(ZDA_ERR_STATE, "no workspace bound");
    cudaError_t e = cudaSetDevice(net->device);
    if (e != cudaSuccess) return nn_fail(ZDA_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return ZDA_OK;
}

zda_status zda_nn_set_params(zda_nn *net, const float *params, int host, void *stream)
{
    zda_status st = need_bound(net);
    if (st != ZDA_OK) return st;
    if (!params) return nn_fail(ZDA_ERR_ARG, "null parameters");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t b = net->nparam * 4;
    NN_CUDA(cudaMemcpyAsync(at<float>(net, net->o.params), params, b,
                            host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    NN_CUDA(cudaMemsetAsync(at<float>(net, net->o.m), 0, b, s));
    NN_CUDA(cudaMemsetAsync(at<float>(net, net->o.v), 0, b, s));
    net->adam_step = 0;
    st = pack_all(net, s);
    if (st != ZDA_OK) return st;
    if (host) NN_CUDA(cudaStreamSynchronize(s));
    return ZDA_OK;
}

static zda_status copy_out(zda_nn *net, size_t off, float *dst, int host, void *stream)
{
    zda_status st = need_bound(net);
    if (st != ZDA_OK) return st;
    if (!dst) return nn_fail(ZDA_ERR_ARG, "null output");
    cudaStream_t s = (cudaStream_t)stream;
    NN_CUDA(cudaMemcpyAsync(dst, at<float>(net, off), net->nparam * 4,
                            host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (host) NN_CUDA(cudaStreamSynchronize(s));
    return ZDA_OK;
}

zda_status zda_nn_get_params(zda_nn *net, float *params, int host, void *stream)
{
    return copy_out(net, net ? net->o.params : 0, params, host, stream);
}

zda_status zda_nn_get_grads(zda_nn *net, float *grads, int host, void *stream)
{
    return copy_out(net, net ? net->o.grads : 0, grads, host, stream);
}

zda_status zda_nn_forward(zda_nn *net, const float *x, int n, float *y, void *stream)
{
    zda_status st = need_bound(net);
    if (st != ZDA_OK) return st;
    if (!x || !y) return nn_fail(ZDA_ERR_ARG, "null tensor");
    if (n < 1 || n > net->d.batch) return nn_fail(ZDA_ERR_ARG, "n outside 1..batch");
    cudaStream_t s = (cudaStream_t)stream;
    const int H = net->d.height, W = net->d.width;
    uint16_t *x16 = at<uint16_t>(net, net->o.x16);
    k_pack_input<<<nblocks(2 * pos_tiles(net, 0, n)), 256, 0, s>>>(x, n, H, W, net->d.in_ch, pos_tiles(net, 0, n),
                                                                  net->rows[0], x16);
    net->launches++;
#define TRY(e)                          \
    do {                                \
        zda_status st_ = (e);           \
        if (st_ != ZDA_OK) return st_;  \
    } while (0)
    const uint16_t *inp = x16;
    int cin = 16;
    for (int l = 0; l < 3; ++l) {
        TRY(conv(net, l, n, 9, inp, nullptr, cin, C, Wf(net, 2 * l), Bias(net, 2 * l), C, EPI_RELU_BF16, Aw(net, l, A_ENCA),
                 nullptr, C, nullptr, nullptr, s, lf(net, 2 * l, n)));
        TRY(conv(net, l, n, 9, A(net, l, A_ENCA), nullptr, C, C, Wf(net, 2 * l + 1), Bias(net, 2 * l + 1), C, EPI_RELU_BF16,
                 Aw(net, l, A_ENCB), nullptr, C, nullptr, nullptr, s, lf(net, 2 * l + 1, n)));
        k_pool<<<nblocks(8 * pos_tiles(net, l + 1, n)), 256, 0, s>>>(A(net, l, A_ENCB), lev(net, l, n),
                                                                    Aw(net, l + 1, A_IN), lev(net, l + 1, n));
        net->launches++;
        inp = A(net, l + 1, A_IN);
        cin = C;
    }
    TRY(conv(net, 3, n, 9, inp, nullptr, C, C, Wf(net, 6), Bias(net, 6), C, EPI_RELU_BF16, Aw(net, 3, A_ENCA), nullptr, C,
             nullptr, nullptr, s, lf(net, 6, n)));
    TRY(conv(net, 3, n, 9, A(net, 3, A_ENCA), nullptr, C, C, Wf(net, 7), Bias(net, 7), C, EPI_RELU_BF16,
             Aw(net, 3, A_ENCB), nullptr, C, nullptr, nullptr, s, lf(net, 7, n)));
    const uint16_t *below = A(net, 3, A_ENCB);
    for (int l = 2; l >= 0; --l) {
        const int li = 8 + 2 * (2 - l);
        k_up<<<nblocks(8 * pos_tiles(net, l, n)), 256, 0, s>>>(below, lev(net, l + 1, n), Aw(net, l, A_UP),
                                                              lev(net, l, n));
        net->launches++;
        TRY(conv(net, l, n, 9, A(net, l, A_UP), A(net, l, A_ENCB), C, C, Wf(net, li), Bias(net, li), C, EPI_RELU_BF16,
                 Aw(net, l, A_DECA), nullptr, C, nullptr, nullptr, s, lf(net, li, n)));
        TRY(conv(net, l, n, 9, A(net, l, A_DECA), nullptr, C, C, Wf(net, li + 1), Bias(net, li + 1), C, EPI_RELU_BF16,
                 Aw(net, l, A_DECB), nullptr, C, nullptr, nullptr, s, lf(net, li + 1, n)));
        below = A(net, l, A_DECB);
    }
    TRY(conv(net, 0, n, 1, below, nullptr, C, 32, Wf(net, 14), Bias(net, 14), net->d.out_ch, EPI_F32, y, nullptr,
             net->d.out_ch, nullptr, nullptr, s, lf(net, 14, n)));
    NN_CUDA(cudaGetLastError());
    net->n_fwd = n;
    return ZDA_OK;
}

zda_status zda_nn_backward(zda_nn *net, const float *dy, float *dx, void *stream)
{
    zda_status st = need_bound(net);
    if (st != ZDA_OK) return st;
    if (!dy) return nn_fail(ZDA_ERR_ARG, "null gradient");
    if (net->n_fwd < 1) return nn_fail(ZDA_ERR_STATE, "backward before forward");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = net->n_fwd, H = net->d.height, W = net->d.width;
    uint16_t *gy = at<uint16_t>(net, net->o.gy);
    k_pack_grad<<<nblocks(4 * pos_tiles(net, 0, n)), 256, 0, s>>>(dy, n, H, W, net->d.out_ch, pos_tiles(net, 0, n),
                                                                 net->rows[0], gy);
    net->launches++;
    // head
    TRY(layer_grad(net, 14, n, A(net, 0, A_DECB), nullptr, gy, 32, s));
    TRY(conv(net, 0, n, 1, gy, nullptr, 32, C, Wd(net, 14), nullptr, 0, EPI_GRAD_BF16, Gb(net, 0, G_B), nullptr, C,
             A(net, 0, A_DECB), nullptr, s));
    // decoder, top level first: G_B holds the gradient of dec_b's pre-activation
    for (int l = 0; l <= 2; ++l) {
        const int li = 8 + 2 * (2 - l);
        TRY(layer_grad(net, li + 1, n, A(net, l, A_DECA), nullptr, Gb(net, l, G_B), C, s));
        TRY(conv(net, l, n, 9, Gb(net, l, G_B), nullptr, C, C, Wd(net, li + 1), nullptr, 0, EPI_GRAD_BF16,
                 Gb(net, l, G_A), nullptr, C, A(net, l, A_DECA), nullptr, s));
        TRY(layer_grad(net, li, n, A(net, l, A_UP), A(net, l, A_ENCB), Gb(net, l, G_A), C, s));
        TRY(conv(net, l, n, 9, Gb(net, l, G_A), nullptr, C, 2 * C, Wd(net, li), nullptr, 0, EPI_GRAD_BF16,
                 Gb(net, l, G_U), Gb(net, l, G_S), C, nullptr, nullptr, s));
        const uint16_t *below = l == 2 ? A(net, 3, A_ENCB) : A(net, l + 1, A_DECB);
        k_up_bwd_mask<<<nblocks(8 * pos_tiles(net, l + 1, n)), 256, 0, s>>>(Gb(net, l, G_U), lev(net, l, n), below,
                                                                           Gb(net, l + 1, G_B), lev(net, l + 1, n));
        net->launches++;
    }
    // bottleneck (level 3: A_ENCA = bot_a, A_ENCB = bot_b)
    TRY(layer_grad(net, 7, n, A(net, 3, A_ENCA), nullptr, Gb(net, 3, G_B), C, s));
    TRY(conv(net, 3, n, 9, Gb(net, 3, G_B), nullptr, C, C, Wd(net, 7), nullptr, 0, EPI_GRAD_BF16, Gb(net, 3, G_A),
             nullptr, C, A(net, 3, A_ENCA), nullptr, s));
    TRY(layer_grad(net, 6, n, A(net, 3, A_IN), nullptr, Gb(net, 3, G_A), C, s));
    TRY(conv(net, 3, n, 9, Gb(net, 3, G_A), nullptr, C, C, Wd(net, 6), nullptr, 0, EPI_GRAD_BF16, Gb(net, 3, G_U),
             nullptr, C, nullptr, nullptr, s));
    // encoder, coarse to fine: G_U of level l + 1 holds the gradient of in_{l+1}
    for (int l = 2; l >= 0; --l) {
        k_skip_combine<<<nblocks(8 * pos_tiles(net, l, n)), 256, 0, s>>>(Gb(net, l, G_S), Gb(net, l + 1, G_U),
                                                                        lev(net, l + 1, n), A(net, l, A_ENCB),
                                                                        Gb(net, l, G_B), lev(net, l, n));
        net->launches++;
        TRY(layer_grad(net, 2 * l + 1, n, A(net, l, A_ENCA), nullptr, Gb(net, l, G_B), C, s));
        TRY(conv(net, l, n, 9, Gb(net, l, G_B), nullptr, C, C, Wd(net, 2 * l + 1), nullptr, 0, EPI_GRAD_BF16,
                 Gb(net, l, G_A), nullptr, C, A(net, l, A_ENCA), nullptr, s));
        const uint16_t *in = l == 0 ? at<uint16_t>(net, net->o.x16) : A(net, l, A_IN);
        TRY(layer_grad(net, 2 * l, n, in, nullptr, Gb(net, l, G_A), C, s));
        if (l > 0)
            TRY(conv(net, l, n, 9, Gb(net, l, G_A), nullptr, C, C, Wd(net, 2 * l), nullptr, 0, EPI_GRAD_BF16,
                     Gb(net, l, G_U), nullptr, C, nullptr, nullptr, s));
        else if (dx) {
            TRY(conv(net, 0, n, 9, Gb(net, 0, G_A), nullptr, C, 16, Wd(net, 0), nullptr, 0, EPI_GRAD_F32, dx, nullptr,
                     net->d.in_ch, nullptr, nullptr, s));
        }
    }
    NN_CUDA(cudaGetLastError());
    return ZDA_OK;
}

zda_status zda_nn_mse(zda_nn *net, const float *y, const float *t, int n, float *dy, float *loss, void *stream)
{
    zda_status st = need_bound(net);
    if (st != ZDA_OK) return st;
    if (!y || !t || !dy || !loss) return nn_fail(ZDA_ERR_ARG, "null tensor");
    if (n < 1 || n > net->d.batch) return nn_fail(ZDA_ERR_ARG, "n outside 1..batch");
    cudaStream_t s = (cudaStream_t)stream;
    const long cnt = (long)n * net->d.height * net->d.width * net->d.out_ch;
    const int nb = (int)std::min<long>(1024, nblocks(cnt));
    k_mse<<<nb, 256, 0, s>>>(y, t, cnt, dy, at<float>(net, net->o.mpart));
    k_mse_final<<<1, 32, 0, s>>>(at<float>(net, net->o.mpart), nb, cnt, loss);
    net->launches += 2;
    NN_CUDA(cudaGetLastError());
    return ZDA_OK;
}

zda_status zda_nn_adam(zda_nn *net, float lr, float b1, float b2, float eps, void *stream)
{
    zda_status st = need_bound(net);
    if (st != ZDA_OK) return st;
    if (!(lr >= 0.f) || !(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) || !(eps > 0.f))
        return nn_fail(ZDA_ERR_ARG, "invalid Adam hyper-parameters");
    cudaStream_t s = (cudaStream_t)stream;
    net->adam_step++;
    const float c1 = (float)(1.0 - std::pow((double)b1, net->adam_step));
    const float c2 = (float)(1.0 - std::pow((double)b2, net->adam_step));
    k_adam<<<nblocks(net->nparam), 256, 0, s>>>(at<float>(net, net->o.params), at<float>(net, net->o.grads),
                                                at<float>(net, net->o.m), at<float>(net, net->o.v), net->nparam, lr, b1,
                                                b2, eps, c1, c2);
    net->launches++;
    NN_CUDA(cudaGetLastError());
    return pack_all(net, s);
}

long long zda_nn_launch_count(const zda_nn *net) { return net ? net->launches : 0; }

zda_status zda_nn_set_timing(zda_nn *net, int on)
{
    if (!net) return nn_fail(ZDA_ERR_ARG, "null network");
    net->timing = on != 0;
    net->ev_used = 0;
    net->ev_flops.clear();
    return ZDA_OK;
}

zda_status zda_nn_timing(zda_nn *net, double *conv_ms, double *conv_flops, int *launches)
{
    if (!net || !conv_ms || !conv_flops || !launches) return nn_fail(ZDA_ERR_ARG, "null argument");
    double ms = 0.0, fl = 0.0;
    for (size_t k = 0; k + 1 < net->ev_used; k += 2) {
        NN_CUDA(cudaEventSynchronize(net->ev[k + 1]));
        float t = 0.f;
        NN_CUDA(cudaEventElapsedTime(&t, net->ev[k], net->ev[k + 1]));
        ms += t;
        fl += net->ev_flops[k / 2];
    }
    *conv_ms = ms;
    *conv_flops = fl;
    *launches = (int)(net->ev_used / 2);
    net->ev_used = 0;
    net->ev_flops.clear();
    return ZDA_OK;
}

zda_status zda_nn_check(zda_nn *net, void *stream)
{
    zda_status st = need_bound(net);
    if (st != ZDA_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int err = 0;
    NN_CUDA(cudaMemcpyAsync(&err, at<int>(net, net->o.err), 4, cudaMemcpyDeviceToHost, s));
    NN_CUDA(cudaStreamSynchronize(s));
    if (err) {
        NN_CUDA(cudaMemsetAsync(at<int>(net, net->o.err), 0, 4, s));
        return nn_fail(ZDA_ERR_TIMEOUT, "tensor-core kernel wait gave up (site " + std::to_string(err) + ")");
    }
    return ZDA_OK;
}

}  // extern "C"
