// fwi_opt.cu -- device vector kernels of the reduced-space update (Sec. 3.2 of
// arXiv:1504.08340): the model vector m = (lambda, mu) on the interior nodes, its
// gradient in the Mtilde inner product (g = Mtilde^-1 g_mis, Eq. (18) with R = 0),
// the L-BFGS two-loop recursion's dot products and axpys (FP64), and the trial
// material of Algorithm 1's backtracking line search (Eq. (19)).
#include <cuda_runtime.h>

#include "fwi_internal.h"

namespace fwi {
namespace {

constexpr int kT = 256;

__global__ void __launch_bounds__(kT) wdot_kernel(const double *a, const double *b, const double *w, int64_t nmat,
                                                  double *part) {
  __shared__ double sh[kT];
  double acc = 0.0;
  const int64_t n = 2 * nmat;  // lambda half, then mu half; the weight repeats
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    acc += a[i] * w[i < nmat ? i : i - nmat] * b[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kT) sum_parts(const double *part, int nb, double *out) {
  __shared__ double sh[kT];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += kT) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void axpby_kernel(double *y, double a, const double *x, double b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// g = Mtilde^-1 g_mis, frozen parameters (mask bit 1: lambda, bit 2: mu) get 0
__global__ void riesz_kernel(const double *gl, const double *gm, const double *mt, double *g, int64_t nmat,
                             int mask) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nmat; i += (int64_t)gridDim.x * blockDim.x) {
    g[i] = (mask & 1) ? gl[i] / mt[i] : 0.0;
    g[nmat + i] = (mask & 2) ? gm[i] / mt[i] : 0.0;
  }
}

// trial material m + alpha d in FP32, and its admissibility: flags[0] = 1 when a
// value is not finite, mu <= 0 or lambda + 2 mu <= 0; flags[1] = max (lambda + 2 mu)
// as float bits (non-negative floats order like their bit patterns)
__global__ void trial_kernel(const double *m, const double *d, double alpha, float *lam, float *mu, int64_t nmat,
                             unsigned *flags) {
  unsigned bad = 0, pmax = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nmat; i += (int64_t)gridDim.x * blockDim.x) {
    const float l = (float)(m[i] + alpha * d[i]);
    const float u = (float)(m[nmat + i] + alpha * d[nmat + i]);
    lam[i] = l;
    mu[i] = u;
    const float p = l + 2.f * u;
    if (!isfinite(l) || !isfinite(u) || !(u > 0.f) || !(p > 0.f)) bad = 1;
    else pmax = max(pmax, __float_as_uint(p));
  }
  if (bad) atomicOr(flags, 1u);
  if (pmax) atomicMax(flags + 1, pmax);
}

__global__ void pack_kernel(const float *lam, const float *mu, double *m, int64_t nmat) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nmat; i += (int64_t)gridDim.x * blockDim.x) {
    m[i] = lam[i];
    m[nmat + i] = mu[i];
  }
}

__global__ void absmax_kernel(const double *x, int64_t n, unsigned long long *out) {
  unsigned long long best = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = fabs(x[i]);
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    best = b > best ? b : best;
  }
  if (best) atomicMax(out, best);
}

inline int grid_for(int64_t n) {
  int64_t b = (n + kT - 1) / kT;
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

}  // namespace

void opt_wdot(const double *a, const double *b, const double *w, int64_t nmat, double *part, double *out,
              cudaStream_t s) {
  const int nb = grid_for(2 * nmat);
  wdot_kernel<<<nb, kT, 0, s>>>(a, b, w, nmat, part);
  sum_parts<<<1, kT, 0, s>>>(part, nb, out);
}

void opt_axpby(double *y, double a, const double *x, double b, int64_t n, cudaStream_t s) {
  axpby_kernel<<<grid_for(n), kT, 0, s>>>(y, a, x, b, n);
}

void opt_riesz(const double *gl, const double *gm, const double *mt, double *g, int64_t nmat, int mask,
               cudaStream_t s) {
  riesz_kernel<<<grid_for(nmat), kT, 0, s>>>(gl, gm, mt, g, nmat, mask);
}

void opt_trial(const double *m, const double *d, double alpha, float *lam, float *mu, int64_t nmat, unsigned *flags,
               cudaStream_t s) {
  trial_kernel<<<grid_for(nmat), kT, 0, s>>>(m, d, alpha, lam, mu, nmat, flags);
}

void opt_pack(const float *lam, const float *mu, double *m, int64_t nmat, cudaStream_t s) {
  pack_kernel<<<grid_for(nmat), kT, 0, s>>>(lam, mu, m, nmat);
}

void opt_absmax(const double *x, int64_t n, unsigned long long *out, cudaStream_t s) {
  absmax_kernel<<<grid_for(n), kT, 0, s>>>(x, n, out);
}

}  // namespace fwi
