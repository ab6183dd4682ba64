/*
 * fehom_unet.h -- C ABI of the learned warm start of the PCG solve in fehom.h.
 *
 * The paper's method has no learned part; this is an addition to it.  A periodic 3-D
 * convolutional U-Net maps the phase field of a cubic cell (through a per-phase input feature,
 * e.g. log10 of the conductivity) to a guess of the fluctuation fields of n_out unit macroscopic
 * loads.  The guess is passed to fehom_solve as its initial iterate x0; PCG (Sec. 4.1) still runs
 * to the same tolerance, measured against the right-hand side (stopping rule of Sec. 6), so a poor
 * guess costs iterations but never accuracy.
 *
 * Network (levels L, widths w_0 < ... < w_{L-1}, every w_l a multiple of 16):
 *   encoder level l: [2x2x2 mean pool of level l-1 output, l > 0]
 *                    -> conv3x3x3 + ReLU (w_{l-1} or 1 -> w_l) -> conv3x3x3 + ReLU (w_l -> w_l)
 *   decoder level l = L-2 .. 0: concat(skip = encoder output of level l, nearest 2x upsampling of
 *                    the level below) -> conv3x3x3 + ReLU (w_l + w_{l+1} -> w_l) -> conv + ReLU (w_l -> w_l)
 *   head: 1x1x1 linear map w_0 -> n_out; prediction x0 = out_scale * head output.
 * Every 3x3x3 convolution is periodic: y[o, v] = b[o] + sum_t sum_i W[t][o][i] x[i, v + off(t)],
 * off(t) = (dz, dy, dx) in {-1, 0, 1}^3, t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1), v = (z, y, x).
 *
 * Numerics: activations and gradients are stored in BF16 (channels-last, [sample][voxel][channel],
 * voxel index x + n (y + n z)); the convolutions (all but the first, whose input has one channel)
 * run on the tcgen05 tensor cores with BF16 operands and FP32 accumulation in tensor memory; master
 * weights, their gradients and the Adam state are FP32.  Adam: beta1 0.9, beta2 0.999, eps 1e-8,
 * bias-corrected.  Loss (fehom_unet_set_loss) of the residual r = head output - target / out_scale,
 * count = batch * n_out * n^3 target values: FEHOM_LOSS_MSE (default) sum r^2 / count;
 * FEHOM_LOSS_H1 (sum over the three axes of the squared periodic forward differences of r, plus
 * l2_weight * sum r^2) / count, a discrete H^1 seminorm, closer to the energy norm in which PCG
 * measures the error of its initial iterate.
 *
 * Parameters form one flat FP32 vector; per 3x3x3 layer in the order e0a, e0, e1a, e1, ...,
 * e{L-1}a, e{L-1}, d{L-2}a, d{L-2}, ..., d0a, d0 the weight W[27][Cout][Cin] then the bias
 * b[Cout]; last the head Wo[n_out][w_0] and bo[n_out].
 *
 * Buffers: ids (uint8, [batch][n^3]), features (float, [batch][n_phases]: the input value of each
 * phase of each sample), targets and predictions (double, [batch][n_out][n^3], the component-
 * blocked field layout of fehom.h with c = 1) are device pointers on the network's device, owned by
 * the caller.  Host pointers are marked.  Every call returns a status; fehom_unet_last_error()
 * describes the last failure.  Calls are asynchronous on the network's stream unless they return
 * a host value (loss, parameters), which synchronises the stream.
 */
#ifndef FEHOM_UNET_H
#define FEHOM_UNET_H

#include "fehom.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fehom_unet fehom_unet; /* opaque, owned by the library */

/* Allocates the network and its activation, gradient and optimiser buffers for up to max_batch
 * samples of an n^3 grid.  n must be a multiple of 2^(n_levels-1) (and <= 512); 1 <= n_levels <= 6;
 * widths[n_levels] multiples of 16 with w_0 <= 32, w_l <= 256, w_l + w_{l+1} <= 256;
 * 1 <= n_phases <= 256; 1 <= n_out <= 4.  stream: cudaStream_t or NULL (a blocking stream the
 * network creates).  Parameters start at zero: set them with fehom_unet_set_params. */
fehom_status fehom_unet_create(fehom_unet** out, int64_t n, int n_levels, const int* widths, int n_phases,
                               int n_out, int max_batch, void* stream);
void fehom_unet_destroy(fehom_unet* net);
const char* fehom_unet_last_error(const fehom_unet* net); /* NULL net: the last failed create */

typedef enum { FEHOM_LOSS_MSE = 0, FEHOM_LOSS_H1 = 1 } fehom_unet_loss;

/* Selects the training loss (see above); l2_weight >= 0 is used by FEHOM_LOSS_H1 only. */
fehom_status fehom_unet_set_loss(fehom_unet* net, int kind, double l2_weight);

/* Number of FP32 parameters (the length of the flat vector described above). */
fehom_status fehom_unet_param_count(const fehom_unet* net, int64_t* n_params);
/* Copies theta (host, n_params floats) in; resets the Adam moments and step count. */
fehom_status fehom_unet_set_params(fehom_unet* net, const float* theta);
/* Copies the current FP32 parameters out (host, n_params floats); synchronises. */
fehom_status fehom_unet_get_params(fehom_unet* net, float* theta);

/* Forward pass of batch <= max_batch samples; writes x0[b][l][v] = out_scale * output (double, device). */
fehom_status fehom_unet_predict(fehom_unet* net, int batch, const uint8_t* ids, const float* features,
                                double out_scale, double* x0);
/* Loss and its gradient for a batch without changing the parameters.  loss (host, may be NULL);
 * grad (host, n_params floats, may be NULL).  Synchronises. */
fehom_status fehom_unet_loss_grad(fehom_unet* net, int batch, const uint8_t* ids, const float* features,
                                  const double* target, double out_scale, double* loss, float* grad);
/* One Adam step with learning rate lr on the batch's loss.  loss (host) may be NULL; when given, the
 * call synchronises and returns the loss before the update. */
fehom_status fehom_unet_train_step(fehom_unet* net, int batch, const uint8_t* ids, const float* features,
                                   const double* target, double out_scale, double lr, double* loss);

/* Kernel-level entry points of the tensor-core convolution, for tests and measurement (no network).
 * fehom_conv3_bf16: y[b][v][o] = relu?(bias[o] + sum_t sum_i w[t][o][i] x[b][v + off(t)][i]) in FP32;
 *   x bf16 [B][D*H*W][Cin], w bf16 [27][Cout][Cin], bias float [Cout] or NULL, y float [B][D*H*W][Cout];
 *   Cin and Cout multiples of 16, Cout <= 256.
 * fehom_conv3_wgrad_bf16: dw[t][o][i] = sum_b sum_v dy[b][v][o] x[b][v + off(t)][i] in FP32;
 *   x bf16 [B][D*H*W][Cin], dy bf16 [B][D*H*W][Cout], dw float [27][Cout][Cin] (overwritten);
 *   Cin and Cout multiples of 16, Cout <= 128.  Allocates its scratch and synchronises.
 * All pointers are device pointers; stream: cudaStream_t or NULL (the legacy default stream). */
fehom_status fehom_conv3_bf16(int B, int D, int H, int W, int Cin, int Cout, const void* x, const void* w,
                              const float* bias, int relu, float* y, void* stream);
fehom_status fehom_conv3_wgrad_bf16(int B, int D, int H, int W, int Cin, int Cout, const void* x,
                                    const void* dy, float* dw, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FEHOM_UNET_H */
