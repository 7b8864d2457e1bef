// zda_filter_project_noalloc: the density filter + projection step for
// callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: for example a host
// program that embeds the solver inside another framework whose memory pool
// owns the whole device (an extra cudaMalloc there can fail, or fragment the
// pool), or a latency-critical optimisation loop that is not allowed to
// allocate once it has started.  This entry point needs no zone, no context
// and no workspace: the caller passes the zone description, the input
// density and the output buffer, and the one piece of scratch memory the
// filter needs (its per-row weight sums) lives in a fixed device array
// compiled into the library.
//
// That array (ZDA_NOALLOC_MAX_ROWS floats, 64 KiB) exists on every GPU that
// loads the library, for the lifetime of the process.  Its device address is
// looked up once per device and kept: after a cudaDeviceReset the module may
// be loaded again at another address, so this entry point must not be used
// on a device after cudaDeviceReset in the same process.  All calls on a device
// share it: every call rewrites the rows it reads before reading them (nothing
// needs to start at zero), and two calls whose kernels overlap on the GPU
// (e.g. on different streams without ordering) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "zda.h"
#include "zda_internal.h"

#define ZDA_NOALLOC_MAX_ROWS 16384
#define ZDA_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) float g_noalloc_norm[ZDA_NOALLOC_MAX_ROWS];

namespace {

std::mutex g_mu;
float *g_norm_ptr[ZDA_NOALLOC_MAX_DEVICES];
bool g_ready[ZDA_NOALLOC_MAX_DEVICES];

struct NaParams {
    int nrd, nphi, di_max, dj_max, filter_on;
    float dr, dphi, R, r_c0, beta, eta;
};

__device__ __forceinline__ float na_weight(const NaParams &p, int i, int di, int dj)
{
    const float rc = p.r_c0 + i * p.dr;
    const float a = di * p.dr, b = rc * dj * p.dphi;
    return fmaxf(0.f, 1.f - sqrtf(a * a + b * b) / p.R);
}

__global__ void k_na_norm(const NaParams p, float *norm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.nrd) return;
    float s = 0.f;
    for (int di = -p.di_max; di <= p.di_max; ++di) {
        if (i + di < 0 || i + di >= p.nrd) continue;
        for (int dj = -p.dj_max; dj <= p.dj_max; ++dj) s += na_weight(p, i, di, dj);
    }
    norm[i] = s;
}

__global__ void k_na_filter_project(const NaParams p, const float *__restrict__ rho,
                                    const float *__restrict__ norm, float *rho_t)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= p.nphi || i >= p.nrd) return;
    float v;
    if (p.filter_on) {
        float s = 0.f;
        for (int di = -p.di_max; di <= p.di_max; ++di) {
            const int ii = i + di;
            if (ii < 0 || ii >= p.nrd) continue;
            for (int dj = -p.dj_max; dj <= p.dj_max; ++dj) {
                const float w = na_weight(p, i, di, dj);
                if (w == 0.f) continue;
                int jj = (j + dj) % p.nphi;
                if (jj < 0) jj += p.nphi;
                s = fmaf(w, __ldg(rho + (size_t)ii * p.nphi + jj), s);
            }
        }
        v = s / norm[i];
    } else {
        v = rho[(size_t)i * p.nphi + j];
    }
    if (p.beta > 0.f) {
        const float te = tanhf(p.beta * p.eta);
        v = (te + tanhf(p.beta * (v - p.eta))) / (te + tanhf(p.beta * (1.f - p.eta)));
    }
    rho_t[(size_t)i * p.nphi + j] = v;
}

zda_status na_fail(zda_status s, const std::string &m)
{
    zda_internal_set_error(m.c_str());       // reported by zda_last_error()
    return s;
}

}  // namespace

extern "C" zda_status zda_filter_project_noalloc(const zda_zone_desc *d, const float *rho_dev,
                                                 float *rho_tilde_dev, void *stream)
{
    if (!d || !rho_dev || !rho_tilde_dev) return na_fail(ZDA_ERR_ARG, "null argument");
    // the checks of zda_zone_create that concern the filter: wedge zones and
    // the axis zone (continuous axisymmetry: n_fold = 0, one phi cell)
    const bool bor = d->n_fold == 0;
    if (d->n_fold < 0 || d->n_phi < 1 || d->n_r < 2 || d->dr <= 0)
        return na_fail(ZDA_ERR_ARG, "zone needs n_r >= 2, n_phi >= 1, n_fold >= 0, dr > 0");
    if (bor && (d->n_phi != 1 || d->r_lo < 0))
        return na_fail(ZDA_ERR_ARG, "continuous axisymmetry (n_fold = 0) needs n_phi = 1 and r_lo >= 0");
    if (!bor && d->r_lo <= 0) return na_fail(ZDA_ERR_ARG, "a wedge zone (n_fold > 0) needs r_lo > 0");
    if (d->pml_r_in < 0 || d->pml_r_out < 0 || d->pml_r_in + d->pml_r_out >= d->n_r)
        return na_fail(ZDA_ERR_ARG, "PML widths do not fit the grid");
    const int nrd = d->n_r - d->pml_r_in - d->pml_r_out;
    if (nrd > ZDA_NOALLOC_MAX_ROWS)
        return na_fail(ZDA_ERR_ARG, "n_r_design = " + std::to_string(nrd) + " exceeds the no-allocation limit of " +
                                        std::to_string(ZDA_NOALLOC_MAX_ROWS) + " rows");
    const double dphi = 2.0 * M_PI / (bor ? 1 : d->n_fold) / d->n_phi;
    const double rc0 = d->r_lo + (d->pml_r_in + 0.5) * d->dr;
    double di = 0, dj = 0;
    if (d->filter_radius > 0) {                  // the same tap bound as zda_zone_create
        di = std::min(std::floor(d->filter_radius / d->dr), (double)(nrd - 1));
        dj = std::floor(d->filter_radius / (rc0 * dphi));
        const double taps = (2 * di + 1) * (2 * dj + 1);
        if (!(taps <= ZDA_MAX_FILTER_TAPS))
            return na_fail(ZDA_ERR_ARG, "filter_radius spans " + std::to_string(taps) + " taps per pixel (limit " +
                                            std::to_string(ZDA_MAX_FILTER_TAPS) + ")");
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(ZDA_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= ZDA_NOALLOC_MAX_DEVICES) return na_fail(ZDA_ERR_ARG, "device index too large");
    float *norm = nullptr;
    {
        // once per device, with that device current: the host-side symbol is
        // only a stand-in, the kernels need the array's device address
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ready[dev]) {
            e = cudaGetSymbolAddress((void **)&g_norm_ptr[dev], g_noalloc_norm);
            if (e != cudaSuccess)
                return na_fail(ZDA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_ready[dev] = true;
        }
        norm = g_norm_ptr[dev];
    }
    NaParams p{};
    p.nrd = nrd;
    p.nphi = d->n_phi;
    p.dr = (float)d->dr;
    p.dphi = (float)dphi;
    p.R = (float)d->filter_radius;
    p.r_c0 = (float)rc0;
    p.beta = (float)d->beta;
    p.eta = (float)d->eta;
    p.filter_on = d->filter_radius > 0 ? 1 : 0;
    p.di_max = (int)di;
    p.dj_max = (int)dj;
    cudaStream_t s = (cudaStream_t)stream;
    if (p.filter_on) k_na_norm<<<(nrd + 127) / 128, 128, 0, s>>>(p, norm);
    dim3 g((p.nphi + 127) / 128, nrd);
    k_na_filter_project<<<g, 128, 0, s>>>(p, rho_dev, norm, rho_tilde_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(ZDA_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return ZDA_OK;
}
