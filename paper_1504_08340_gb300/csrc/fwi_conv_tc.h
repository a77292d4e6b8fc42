// fwi_conv_tc.h -- the tensor-core (tcgen05) convolutions of the learned
// preconditioner (fwi_conv_tc.cu), called by fwi_nn_conv3d_forward,
// fwi_nn_conv3d_backward_data and fwi_nn_conv3d_backward_weight. Not public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fwi_tc {
// y[co][p] = act(b[co] + sum_ci sum_t w[co][ci][t] x[ci][p + off(t)]) with the layouts of
// fwi_nn_conv3d_forward, in the tile form (a TMA box of x per 8 x 16 voxel tile, the taps as
// shifted MMA views); enqueues the weight pack and a group-major copy of x into
// stream-ordered scratch, the convolution and the scratch's release on s. Returns the first
// CUDA error (cudaErrorInvalidValue for sizes the tiling cannot take).
cudaError_t conv3d_forward_tc(const uint16_t *x, const uint16_t *w, const float *b, int cin, int cout, int D, int H,
                              int W, int relu, uint16_t *y, cudaStream_t s);
// dx[ci][p] = sum_co sum_t w[co][ci][t] dy[co][p - off(t)] with the layouts of
// fwi_nn_conv3d_backward_data, in the tile form with the taps mirrored: the FP32 dy enters
// as three BF16 parts (hi, lo, lo2) per channel, so the tensor-core products stay exact.
cudaError_t conv3d_backward_data_tc(const float *dy, const uint16_t *w, int cin, int cout, int D, int H, int W,
                                    float *dx, cudaStream_t s);
// dw[co][ci][t] = sum_p dy[co][p] x[ci][p + off(t)], db[co] = sum_p dy[co][p] with the
// layouts of fwi_nn_conv3d_backward_weight: per 2048-voxel slice one GEMM (im2col of x
// against the three BF16 parts of dy, plus a row of ones for db) into `work`, then the
// slices added in order. conv3d_backward_weight_tc_work: the floats `work` must hold.
int64_t conv3d_backward_weight_tc_work(int cin, int cout, int D, int H, int W);
cudaError_t conv3d_backward_weight_tc(const float *dy, const uint16_t *x, int cin, int cout, int D, int H, int W,
                                      float *dw, float *db, float *work, cudaStream_t s);
}  // namespace fwi_tc
