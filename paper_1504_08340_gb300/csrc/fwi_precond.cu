// fwi_precond.cu -- kernels of the learned gradient preconditioner (sm_103a): 3x3x3
// convolutions forward and backward, ReLU backward, mean squared error and Adam, with
// BF16 storage of activations and weights and FP32 accumulation (fwi_precond.h).
//
// The three convolutions (forward, backward data, weight gradient) run on the tensor
// cores as implicit GEMMs (fwi_conv_tc.cu). Every sum runs in a fixed order (the MMAs in
// a fixed sequence; weight gradients over fixed voxel slices, then the slices in order),
// so results repeat bit for bit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "fwi_conv_tc.h"
#include "fwi_precond.h"

namespace {

constexpr int kT = 256;                 // threads per block
constexpr int64_t kMaxVox = int64_t(1) << 34;
constexpr int kRedBlocks = 1024;

__device__ __forceinline__ float bf2f(uint16_t u) { return __uint_as_float((unsigned)u << 16); }
__device__ __forceinline__ uint16_t f2bf(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }

__global__ void __launch_bounds__(kT) relu_bwd_kernel(const float *__restrict__ dy, const uint16_t *__restrict__ y,
                                                      int64_t n, float *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    out[i] = bf2f(y[i]) > 0.f ? dy[i] : 0.f;
}

__global__ void __launch_bounds__(kT) mse_partial_kernel(const uint16_t *__restrict__ y, const float *__restrict__ t,
                                                         int64_t n, float inv_n, float *__restrict__ dy,
                                                         double *__restrict__ part) {
  __shared__ double sh[kT];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const float e = bf2f(y[i]) - t[i];
    dy[i] = e * inv_n;
    s += (double)e * (double)e;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = kT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void mse_final_kernel(const double *__restrict__ part, int nblocks, int64_t n, double *loss) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < nblocks; i++) s += part[i];
  *loss = s / (2.0 * (double)n);
}

__global__ void __launch_bounds__(kT) adam_kernel(float *__restrict__ master, uint16_t *__restrict__ w,
                                                  const float *__restrict__ g, float *__restrict__ m,
                                                  float *__restrict__ v, int64_t n, float lr, float b1, float b2,
                                                  float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float p = master[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    master[i] = p;
    if (w) w[i] = f2bf(p);
  }
}

__global__ void __launch_bounds__(kT) to_bf16_kernel(const float *__restrict__ x, int64_t n, uint16_t *__restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) y[i] = f2bf(x[i]);
}

__global__ void __launch_bounds__(kT) from_bf16_kernel(const uint16_t *__restrict__ x, int64_t n, float *__restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) y[i] = bf2f(x[i]);
}

// ---- 2x pooling and upsampling between a fine grid D x H x W and the coarse grid
// ceil(D/2) x ceil(H/2) x ceil(W/2); coarse cell q covers fine voxels 2q .. 2q + 1 along each
// axis, clipped to the fine grid. Activations BF16, gradients FP32.
struct Cells {
  int D, H, W, Dc, Hc, Wc;
  __device__ __forceinline__ int count(int q0, int q1, int q2) const {  // fine voxels of a coarse cell
    return (2 * q0 + 1 < D ? 2 : 1) * (2 * q1 + 1 < H ? 2 : 1) * (2 * q2 + 1 < W ? 2 : 1);
  }
};

// y[c][q] = mean of x[c][p] over the fine voxels p of coarse cell q (FP32 sum, rounded to BF16)
__global__ void __launch_bounds__(kT) pool2_fwd_kernel(const uint16_t *__restrict__ x, int C, Cells g,
                                                       uint16_t *__restrict__ y) {
  const int64_t nc = (int64_t)g.Dc * g.Hc * g.Wc, n = nc * C;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const int64_t c = i / nc, q = i % nc;
    const int q2 = (int)(q % g.Wc), q1 = (int)((q / g.Wc) % g.Hc), q0 = (int)(q / ((int64_t)g.Wc * g.Hc));
    const uint16_t *xc = x + c * (int64_t)g.D * g.H * g.W;
    float s = 0.f;
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        for (int e = 0; e < 2; e++) {
          const int z = 2 * q0 + a, yy = 2 * q1 + b, xx = 2 * q2 + e;
          if (z < g.D && yy < g.H && xx < g.W) s += bf2f(xc[((int64_t)z * g.H + yy) * g.W + xx]);
        }
    y[i] = f2bf(s / (float)g.count(q0, q1, q2));
  }
}

// dx[c][p] (+)= dy[c][cell(p)] / count(cell(p))
__global__ void __launch_bounds__(kT) pool2_bwd_kernel(const float *__restrict__ dy, int C, Cells g, int acc,
                                                       float *__restrict__ dx) {
  const int64_t nf = (int64_t)g.D * g.H * g.W, n = nf * C;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const int64_t c = i / nf, p = i % nf;
    const int x2 = (int)(p % g.W), x1 = (int)((p / g.W) % g.H), x0 = (int)(p / ((int64_t)g.W * g.H));
    const int q0 = x0 >> 1, q1 = x1 >> 1, q2 = x2 >> 1;
    const float v = dy[c * (int64_t)g.Dc * g.Hc * g.Wc + ((int64_t)q0 * g.Hc + q1) * g.Wc + q2] / (float)g.count(q0, q1, q2);
    dx[i] = acc ? dx[i] + v : v;
  }
}

// y[c][p] = x[c][cell(p)] (nearest neighbour)
__global__ void __launch_bounds__(kT) up2_fwd_kernel(const uint16_t *__restrict__ x, int C, Cells g,
                                                     uint16_t *__restrict__ y) {
  const int64_t nf = (int64_t)g.D * g.H * g.W, n = nf * C;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const int64_t c = i / nf, p = i % nf;
    const int x2 = (int)(p % g.W), x1 = (int)((p / g.W) % g.H), x0 = (int)(p / ((int64_t)g.W * g.H));
    y[i] = x[c * (int64_t)g.Dc * g.Hc * g.Wc + ((int64_t)(x0 >> 1) * g.Hc + (x1 >> 1)) * g.Wc + (x2 >> 1)];
  }
}

// dx[c][q] (+)= sum of dy[c][p] over the fine voxels p of cell q, in a fixed order
__global__ void __launch_bounds__(kT) up2_bwd_kernel(const float *__restrict__ dy, int C, Cells g, int acc,
                                                     float *__restrict__ dx) {
  const int64_t nc = (int64_t)g.Dc * g.Hc * g.Wc, n = nc * C;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    const int64_t c = i / nc, q = i % nc;
    const int q2 = (int)(q % g.Wc), q1 = (int)((q / g.Wc) % g.Hc), q0 = (int)(q / ((int64_t)g.Wc * g.Hc));
    const float *dc = dy + c * (int64_t)g.D * g.H * g.W;
    float s = 0.f;
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        for (int e = 0; e < 2; e++) {
          const int z = 2 * q0 + a, yy = 2 * q1 + b, xx = 2 * q2 + e;
          if (z < g.D && yy < g.H && xx < g.W) s += dc[((int64_t)z * g.H + yy) * g.W + xx];
        }
    dx[i] = acc ? dx[i] + s : s;
  }
}

Cells cells(int D, int H, int W) { return Cells{D, H, W, (D + 1) / 2, (H + 1) / 2, (W + 1) / 2}; }

bool sizes_ok(int cin, int cout, int D, int H, int W) {
  if (cin < 1 || cout < 1 || D < 1 || H < 1 || W < 1) return false;
  if (cin > 65535 || cout > 65535) return false;  // grid y / z limits
  return (int64_t)D * H * W <= kMaxVox;
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + kT - 1) / kT;
  return (unsigned)(b < 1 ? 1 : (b > 65536 ? 65536 : b));  // grid-stride loops cover the rest
}

fwi_status launched() { return cudaGetLastError() == cudaSuccess ? FWI_OK : FWI_E_CUDA; }

// sizes the tensor-core tiling cannot take come back as cudaErrorInvalidValue, before any
// device work
fwi_status tc_status(cudaError_t e) {
  return e == cudaSuccess ? FWI_OK : (e == cudaErrorInvalidValue ? FWI_E_INVAL : FWI_E_CUDA);
}

}  // namespace

extern "C" {

fwi_status fwi_nn_conv3d_forward(const uint16_t *x, const uint16_t *w, const float *b, int cin, int cout, int D,
                                 int H, int W, int relu, uint16_t *y, void *stream) {
  if (!x || !w || !y || !sizes_ok(cin, cout, D, H, W)) return FWI_E_INVAL;
  return tc_status(fwi_tc::conv3d_forward_tc(x, w, b, cin, cout, D, H, W, relu, y, (cudaStream_t)stream));
}

fwi_status fwi_nn_conv3d_backward_data(const float *dy, const uint16_t *w, int cin, int cout, int D, int H, int W,
                                       float *dx, void *stream) {
  if (!dy || !w || !dx || !sizes_ok(cin, cout, D, H, W)) return FWI_E_INVAL;
  return tc_status(fwi_tc::conv3d_backward_data_tc(dy, w, cin, cout, D, H, W, dx, (cudaStream_t)stream));
}

int64_t fwi_nn_conv3d_backward_weight_work(int cin, int cout, int D, int H, int W) {
  if (!sizes_ok(cin, cout, D, H, W)) return 0;
  return fwi_tc::conv3d_backward_weight_tc_work(cin, cout, D, H, W);
}

fwi_status fwi_nn_conv3d_backward_weight(const float *dy, const uint16_t *x, int cin, int cout, int D, int H, int W,
                                         float *dw, float *db, float *work, void *stream) {
  if (!dy || !x || !dw || !work || !sizes_ok(cin, cout, D, H, W)) return FWI_E_INVAL;
  return tc_status(fwi_tc::conv3d_backward_weight_tc(dy, x, cin, cout, D, H, W, dw, db, work, (cudaStream_t)stream));
}

fwi_status fwi_nn_relu_backward(const float *dy, const uint16_t *y, int64_t n, float *out, void *stream) {
  if (!dy || !y || !out || n < 1) return FWI_E_INVAL;
  relu_bwd_kernel<<<grid_for(n), kT, 0, (cudaStream_t)stream>>>(dy, y, n, out);
  return launched();
}

fwi_status fwi_nn_mse(const uint16_t *y, const float *t, int64_t n, float *dy, double *loss, double *work,
                      void *stream) {
  if (!y || !t || !dy || !loss || !work || n < 1) return FWI_E_INVAL;
  int64_t nb = (n + kT - 1) / kT;
  if (nb > kRedBlocks) nb = kRedBlocks;
  const cudaStream_t s = (cudaStream_t)stream;
  mse_partial_kernel<<<(unsigned)nb, kT, 0, s>>>(y, t, n, (float)(1.0 / (double)n), dy, work);
  mse_final_kernel<<<1, 32, 0, s>>>(work, (int)nb, n, loss);
  return launched();
}

fwi_status fwi_nn_adam(float *master, uint16_t *w, const float *g, float *m, float *v, int64_t n, float lr,
                       float beta1, float beta2, float eps, int t, void *stream) {
  if (!master || !g || !m || !v || n < 1 || t < 1 || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) || !(lr > 0.f))
    return FWI_E_INVAL;
  // bias corrections 1 / (1 - beta^t), in FP64 on the host
  const double p1 = std::pow((double)beta1, t), p2 = std::pow((double)beta2, t);
  adam_kernel<<<grid_for(n), kT, 0, (cudaStream_t)stream>>>(master, w, g, m, v, n, lr, beta1, beta2, eps,
                                                            (float)(1.0 / (1.0 - p1)), (float)(1.0 / (1.0 - p2)));
  return launched();
}

fwi_status fwi_nn_pool2_forward(const uint16_t *x, int C, int D, int H, int W, uint16_t *y, void *stream) {
  if (!x || !y || !sizes_ok(C, 1, D, H, W)) return FWI_E_INVAL;
  const Cells g = cells(D, H, W);
  pool2_fwd_kernel<<<grid_for((int64_t)C * g.Dc * g.Hc * g.Wc), kT, 0, (cudaStream_t)stream>>>(x, C, g, y);
  return launched();
}

fwi_status fwi_nn_pool2_backward(const float *dy, int C, int D, int H, int W, int accumulate, float *dx, void *stream) {
  if (!dy || !dx || !sizes_ok(C, 1, D, H, W)) return FWI_E_INVAL;
  pool2_bwd_kernel<<<grid_for((int64_t)C * D * H * W), kT, 0, (cudaStream_t)stream>>>(dy, C, cells(D, H, W),
                                                                                      accumulate != 0, dx);
  return launched();
}

fwi_status fwi_nn_upsample2_forward(const uint16_t *x, int C, int D, int H, int W, uint16_t *y, void *stream) {
  if (!x || !y || !sizes_ok(C, 1, D, H, W)) return FWI_E_INVAL;
  up2_fwd_kernel<<<grid_for((int64_t)C * D * H * W), kT, 0, (cudaStream_t)stream>>>(x, C, cells(D, H, W), y);
  return launched();
}

fwi_status fwi_nn_upsample2_backward(const float *dy, int C, int D, int H, int W, int accumulate, float *dx,
                                     void *stream) {
  if (!dy || !dx || !sizes_ok(C, 1, D, H, W)) return FWI_E_INVAL;
  const Cells g = cells(D, H, W);
  up2_bwd_kernel<<<grid_for((int64_t)C * g.Dc * g.Hc * g.Wc), kT, 0, (cudaStream_t)stream>>>(dy, C, g,
                                                                                             accumulate != 0, dx);
  return launched();
}

fwi_status fwi_nn_to_bf16(const float *x, int64_t n, uint16_t *y, void *stream) {
  if (!x || !y || n < 1) return FWI_E_INVAL;
  to_bf16_kernel<<<grid_for(n), kT, 0, (cudaStream_t)stream>>>(x, n, y);
  return launched();
}

fwi_status fwi_nn_from_bf16(const uint16_t *x, int64_t n, float *y, void *stream) {
  if (!x || !y || n < 1) return FWI_E_INVAL;
  from_bf16_kernel<<<grid_for(n), kT, 0, (cudaStream_t)stream>>>(x, n, y);
  return launched();
}

}  // extern "C"
