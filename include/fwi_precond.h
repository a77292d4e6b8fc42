/*
 * fwi_precond.h -- C ABI of the kernels of the learned gradient preconditioner.
 *
 * The gradients dJ/dlambda, dJ/dmu of a multiparameter inversion suffer from
 * cross-talk between the two parameters (Sec. 3.3.3 of arXiv:1504.08340, where
 * the paper counters it by biasing the lambda search direction, Eq. (25)). The
 * learned preconditioner is a small 3D convolutional network that maps the raw
 * gradients and the current model, (g_lambda, g_mu, lambda, mu) on the interior
 * material grid, to a model update. These calls are its building blocks: 3x3x3
 * convolutions (stride 1, zero padding 1) forward and backward, ReLU, a mean
 * squared error and Adam, for inference and training on the GPU.
 *
 * Layouts and precisions:
 *   - activations: BF16 [C][D][H][W] (W fastest), one sample;
 *   - weights: BF16 [C_out][C_in][3][3][3] (kz, ky, kx; kx fastest) for the
 *     forward and backward-data convolutions, with an FP32 master copy that
 *     fwi_nn_adam updates; biases FP32 [C_out];
 *   - gradients of activations, weights and biases: FP32;
 *   - every product is accumulated in FP32, the loss in FP64; every sum runs in
 *     a fixed order, so results repeat bit for bit.
 * BF16 values are passed as their 16-bit patterns (uint16_t).
 *
 * Every pointer is a device pointer usable on `stream` (a cudaStream_t; null is
 * the legacy default stream). The calls only enqueue work on that stream and
 * return; the caller owns every array. Errors: FWI_E_INVAL (a null pointer or a
 * size out of range, checked before any device work), FWI_E_CUDA (a launch
 * failed).
 */
#ifndef FWI_PRECOND_H
#define FWI_PRECOND_H

#include <stdint.h>

#include "fwi.h"

#ifdef __cplusplus
extern "C" {
#endif

/* y[co] = act(b[co] + sum_ci sum_t w[co][ci][t] x[ci][p + t - 1]) for every voxel p,
 * out-of-grid taps reading zero; act is ReLU when relu != 0, else the identity.
 * x: BF16 [cin][D][H][W]; w: BF16 [cout][cin][27]; b: FP32 [cout] or null (zero);
 * y: BF16 [cout][D][H][W], rounded to nearest even from the FP32 sum.
 * Runs on the tensor cores (tcgen05 MMAs, BF16 operands, FP32 accumulation in tensor
 * memory) as an implicit GEMM over tiles of 8 x 16 voxels of one plane: a TMA box brings
 * the tile of x with its halo, and the 27 taps are shifted views of it. Two scratch copies
 * are allocated and freed in stream order (cudaMallocAsync): x with its channels padded to
 * a multiple of 32 (BF16, group-major) and the weights packed for the MMAs. A wait inside
 * the kernel that gives up (not expected in operation) writes NaN to the outputs of its
 * tile. FWI_E_INVAL for sizes the tiling cannot take (D > 65535); FWI_E_CUDA also when the
 * scratch cannot be allocated. */
fwi_status fwi_nn_conv3d_forward(const uint16_t *x, const uint16_t *w, const float *b, int cin, int cout, int D,
                                 int H, int W, int relu, uint16_t *y, void *stream);

/* The transposed convolution: dx[ci][p] = sum_co sum_t w[co][ci][t] dy[co][p - t + 1],
 * the gradient of sum(dy * y) with respect to x for the pre-activation y.
 * dy: FP32 [cout][D][H][W]; w: BF16 [cout][cin][27]; dx: FP32 [cin][D][H][W].
 * On the tensor cores in the tile form of the forward call (taps mirrored), with dy taken
 * as three BF16 parts per value (hi, lo, lo2; their sum is dy to 2^-24), so the exact BF16
 * products keep FP32 accuracy; the sums run in FP32 on the tensor cores. */
fwi_status fwi_nn_conv3d_backward_data(const float *dy, const uint16_t *w, int cin, int cout, int D, int H, int W,
                                       float *dx, void *stream);

/* Floats of scratch fwi_nn_conv3d_backward_weight needs for these sizes (0 on bad sizes). */
int64_t fwi_nn_conv3d_backward_weight_work(int cin, int cout, int D, int H, int W);

/* dw[co][ci][t] = sum_p dy[co][p] x[ci][p + t - 1] and db[co] = sum_p dy[co][p]: the
 * gradients of sum(dy * y) with respect to the weights and biases. On the tensor cores:
 * per slice of 2048 voxels one GEMM of the im2col matrix of x (with a row of ones for db)
 * against dy taken as three BF16 parts per value (so the products keep FP32 accuracy),
 * FP32 partial sums into `work`, then the slices added in order. Copies of x
 * (channels-last) and of the split dy are allocated and freed in stream order.
 * dy: FP32 [cout][D][H][W]; x: BF16 [cin][D][H][W]; dw: FP32 [cout][cin][27];
 * db: FP32 [cout] or null; work: FP32 scratch (fwi_nn_conv3d_backward_weight_work). */
fwi_status fwi_nn_conv3d_backward_weight(const float *dy, const uint16_t *x, int cin, int cout, int D, int H, int W,
                                         float *dw, float *db, float *work, void *stream);

/* ReLU backward through the stored (post-ReLU, BF16) output: out[i] = y[i] > 0 ? dy[i] : 0. */
fwi_status fwi_nn_relu_backward(const float *dy, const uint16_t *y, int64_t n, float *out, void *stream);

/* Mean squared error of y (BF16) against t (FP32) over n values:
 * *loss = sum (y - t)^2 / (2 n) in FP64 (device scalar), dy = (y - t) / n (FP32).
 * work: FP64 scratch of 1024 values. */
fwi_status fwi_nn_mse(const uint16_t *y, const float *t, int64_t n, float *dy, double *loss, double *work,
                      void *stream);

/* Adam step t >= 1 on n parameters: m = beta1 m + (1 - beta1) g, v = beta2 v + (1 - beta2) g^2,
 * master -= lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps); then w = BF16(master)
 * when w is not null. master, g, m, v: FP32 [n]; w: BF16 [n] or null. */
fwi_status fwi_nn_adam(float *master, uint16_t *w, const float *g, float *m, float *v, int64_t n, float lr,
                       float beta1, float beta2, float eps, int t, void *stream);

/* 2x average pooling and nearest-neighbour upsampling between a fine grid D x H x W
 * and the coarse grid ceil(D/2) x ceil(H/2) x ceil(W/2), for the U-Net's contracting and
 * expanding paths; coarse cell q covers the fine voxels 2q and 2q + 1 along each axis,
 * clipped to the fine grid (D, H, W are always the fine sizes).
 * pool2_forward:     y[c][q] = mean of x[c][p] over the cell (FP32 sum, BF16 result);
 * pool2_backward:    dx[c][p] = dy[c][q(p)] / (voxels of the cell q(p));
 * upsample2_forward: y[c][p] = x[c][q(p)];
 * upsample2_backward: dx[c][q] = sum of dy[c][p] over the cell, in a fixed order.
 * x, y: BF16 [C][grid]; dy, dx: FP32 [C][grid]. With accumulate != 0 the backward calls
 * add into dx (the gradient of an activation that also feeds a skip connection). */
fwi_status fwi_nn_pool2_forward(const uint16_t *x, int C, int D, int H, int W, uint16_t *y, void *stream);
fwi_status fwi_nn_pool2_backward(const float *dy, int C, int D, int H, int W, int accumulate, float *dx, void *stream);
fwi_status fwi_nn_upsample2_forward(const uint16_t *x, int C, int D, int H, int W, uint16_t *y, void *stream);
fwi_status fwi_nn_upsample2_backward(const float *dy, int C, int D, int H, int W, int accumulate, float *dx,
                                     void *stream);

/* FP32 -> BF16 (round to nearest even) and BF16 -> FP32, n values. */
fwi_status fwi_nn_to_bf16(const float *x, int64_t n, uint16_t *y, void *stream);
fwi_status fwi_nn_from_bf16(const uint16_t *x, int64_t n, float *y, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FWI_PRECOND_H */
