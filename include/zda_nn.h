/* zda_nn.h -- C ABI of the zone surrogate in libzda (sm_103a).
 *
 * A learned warm start for each zone's topology optimisation: a 4-level
 * convolutional U-Net (width 64, 3x3 convolutions, 2x2 average pooling,
 * nearest-neighbour upsampling with skip concatenation, 1x1 head) mapping a
 * zone's density patch rho (n_r_design x n_phi pixels, plus optional
 * conditioning channels) to the zone's monitor-plane DFT over the design
 * annulus (2 transverse components x signed frequencies x re/im channels),
 * i.e. the near field that the focal transform of "Results and Discussion"
 * integrates.  The paper has no learned component: the plain FDTD solve of
 * zda.h stays the reference and the measure of the surrogate's error.
 *
 * Precision: bfloat16 weights, activations and activation gradients; FP32
 * accumulation in tensor memory (tcgen05.mma kind::f16); FP32 biases, head
 * output, loss, weight gradients and Adam state.
 *
 * Memory: the library allocates no device memory.  zda_nn_workspace_bytes
 * gives the size of one caller-allocated device workspace (parameters,
 * gradients, Adam moments, bfloat16 weight images, every activation and
 * gradient buffer of a batch of `batch` samples); zda_nn_bind_workspace
 * hands it over (the caller keeps ownership and frees it after
 * zda_nn_destroy).
 *
 * Layouts: user tensors are FP32, [n][H][W][channels] with channels fastest
 * (H = rows = radial design pixels, W = columns = azimuthal pixels).
 * Parameters are one flat FP32 vector, layer by layer in network order
 * (enc0a, enc0b, enc1a, enc1b, enc2a, enc2b, bota, botb, dec2a, dec2b,
 * dec1a, dec1b, dec0a, dec0b, head); each layer stores its weights
 * w[c_out][ky][kx][c_in] (row-major) followed by its bias b[c_out].  The
 * decoder's first convolution of level l takes the concatenation
 * [upsampled coarser output, encoder output of level l] (128 channels).
 *
 * Calls are asynchronous on the given stream unless they say otherwise;
 * every call returns a zda_status (zda_last_error() has the message).
 */
#ifndef ZDA_NN_H
#define ZDA_NN_H

#include <stddef.h>

#include "zda.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct zda_nn zda_nn;

typedef struct {
    int batch;      /* largest number of samples per call (>= 1) */
    int height;     /* H, a multiple of 8, 8 .. 1024 */
    int width;      /* W, a multiple of 8, 8 .. 176 (the convolution's shared-memory window
                       holds 2 x (256 + 2 (W + 3)) positions x 64 channels) */
    int in_ch;      /* input channels, 1 .. 16 */
    int out_ch;     /* output channels, 1 .. 32 */
} zda_nn_desc;

/* Create a network for `device` (ZDA_ERR_ARG on an invalid descriptor). */
zda_status zda_nn_create(int device, const zda_nn_desc *desc, zda_nn **out);
void zda_nn_destroy(zda_nn *net);

/* Number of FP32 parameters (the length of the flat parameter vector). */
zda_status zda_nn_param_count(const zda_nn *net, size_t *count_host);
/* Forward FLOPs of one sample (2 per multiply-add, H x W output pixels per convolution). */
zda_status zda_nn_forward_flops(const zda_nn *net, double *flops_host);

zda_status zda_nn_workspace_bytes(const zda_nn *net, size_t *bytes_host);
/* Bind the workspace (device memory of at least zda_nn_workspace_bytes,
 * 256-byte aligned).  Parameters start at zero; set them before use. */
zda_status zda_nn_bind_workspace(zda_nn *net, void *workspace_dev, size_t bytes);

/* Parameters in / out (flat FP32 vector of zda_nn_param_count entries, on
 * the device, or on the host when host != 0; host copies synchronise the
 * stream).  Setting parameters resets the Adam state. */
zda_status zda_nn_set_params(zda_nn *net, const float *params, int host, void *stream);
zda_status zda_nn_get_params(zda_nn *net, float *params, int host, void *stream);
/* Gradient of the last zda_nn_backward (same layout as the parameters). */
zda_status zda_nn_get_grads(zda_nn *net, float *grads, int host, void *stream);

/* y = net(x): x_dev [n][H][W][in_ch], y_dev [n][H][W][out_ch] (device,
 * FP32), 1 <= n <= batch.  Keeps the activations for zda_nn_backward. */
zda_status zda_nn_forward(zda_nn *net, const float *x_dev, int n, float *y_dev, void *stream);

/* Backward pass of the last forward: dy_dev = dL/dy [n][H][W][out_ch];
 * writes dL/dparams into the gradient buffer and, when dx_dev is not null,
 * dL/dx [n][H][W][in_ch] into dx_dev. */
zda_status zda_nn_backward(zda_nn *net, const float *dy_dev, float *dx_dev, void *stream);

/* Mean squared error of y against target ([n][H][W][out_ch] each, device):
 * writes dL/dy = 2 (y - target) / (n H W out_ch) to dy_dev and the loss to
 * *loss_dev (one FP32 on the device). */
zda_status zda_nn_mse(zda_nn *net, const float *y_dev, const float *target_dev, int n, float *dy_dev,
                      float *loss_dev, void *stream);

/* One Adam update (Kingma and Ba, Algorithm 1) of the parameters with the
 * current gradient; the step counter starts at 1 after zda_nn_set_params. */
zda_status zda_nn_adam(zda_nn *net, float lr, float beta1, float beta2, float eps, void *stream);

/* CUDA-event timing of the forward convolution launches (k_conv_tc), on
 * the launching stream: with on != 0 every forward convolution is bracketed
 * by two events.  zda_nn_timing waits for them and returns the summed
 * durations (ms), the useful FLOPs of those launches (true channel counts,
 * H x W outputs per sample) and the number of launches, then resets. */
zda_status zda_nn_set_timing(zda_nn *net, int on);
zda_status zda_nn_timing(zda_nn *net, double *conv_ms_host, double *conv_flops_host, int *launches_host);

/* Kernel launches issued by this network so far. */
long long zda_nn_launch_count(const zda_nn *net);

/* Device-side error word of the tensor-core kernels (bounded waits):
 * synchronises the stream; ZDA_ERR_TIMEOUT if a wait gave up since the last
 * call (the word is then cleared). */
zda_status zda_nn_check(zda_nn *net, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ZDA_NN_H */
