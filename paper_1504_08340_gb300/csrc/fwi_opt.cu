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

__global__ void __launch_bounds__(kT) dot_kernel(const double *a, const double *b, int64_t n, double *part) {
  __shared__ double sh[kT];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) acc += a[i] * b[i];
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

// ---- regularisation, Eqs. (8)/(9), gradients (C.1b)-(C.1e), on a nodal field f of the
// interior (material) grid (mx, my, mz nodes, spacing h/2). Quadrature points are the
// element nodes; grad chi_a(q) is nonzero only when q lies on one of the three lines
// through a inside the element, where d chi_a / dx_j (q) = (2/h) D[q_j][a_j], with D the
// derivative matrix of the quadratic Lagrange basis at the nodes -1, 0, 1 and weights
// w = (1/3, 4/3, 1/3).
__device__ __forceinline__ double lgl_d(int q, int a) {
  return q == 0 ? (a == 0 ? -1.5 : (a == 1 ? 2.0 : -0.5))
                : (q == 1 ? (a == 0 ? -0.5 : (a == 1 ? 0.0 : 0.5)) : (a == 0 ? 0.5 : (a == 1 ? -2.0 : 1.5)));
}
__device__ __forceinline__ double lgl_w(int q) { return q == 1 ? 4.0 / 3.0 : 1.0 / 3.0; }

struct RegGrid {
  const float *f;
  int m[3];     // nodes per axis
  double h;     // element size
  double eps;   // TV parameter
};

// d f_h / dx_d at local point q of the element with first node e0 (global node indices)
__device__ __forceinline__ double reg_deriv(const RegGrid &r, const int e0[3], const int q[3], int d) {
  double s = 0.0;
#pragma unroll
  for (int b = 0; b < 3; b++) {
    int n[3] = {e0[0] + q[0], e0[1] + q[1], e0[2] + q[2]};
    n[d] = e0[d] + b;
    s += lgl_d(q[d], b) * (double)__ldg(r.f + ((int64_t)n[2] * r.m[1] + n[1]) * r.m[0] + n[0]);
  }
  return (2.0 / r.h) * s;
}

// g_a = sum over the elements around node a and the points q on its three lines of
// W detJ grad chi_a(q) . grad f_h(q), divided by (|grad f_h(q)|^2 + eps)^(1/2) for TV
template <bool TV>
__global__ void __launch_bounds__(kT) reg_grad_kernel(RegGrid r, double *g) {
  const int64_t n = (int64_t)r.m[0] * r.m[1] * r.m[2];
  const double hh = 0.5 * r.h, wdet = hh * hh * hh;
  for (int64_t mi = (int64_t)blockIdx.x * kT + threadIdx.x; mi < n; mi += (int64_t)gridDim.x * kT) {
    const int c[3] = {(int)(mi % r.m[0]), (int)((mi / r.m[0]) % r.m[1]), (int)(mi / ((int64_t)r.m[0] * r.m[1]))};
    double acc = 0.0;
    // the (one or two) elements along each axis: first node 2e, local index c - 2e
    for (int sz = 0; sz < 2; sz++)
      for (int sy = 0; sy < 2; sy++)
        for (int sx = 0; sx < 2; sx++) {
          const int sd[3] = {sx, sy, sz};
          int e0[3], a[3];
          bool ok = true;
          for (int d = 0; d < 3; d++) {
            // side 0: the element below (node is its local 2, or local 1 for odd c);
            // side 1: the element above (local 0), only for even c
            int e;
            if (c[d] & 1) {
              if (sd[d]) { ok = false; break; }
              e = (c[d] - 1) / 2;
            } else {
              e = sd[d] ? c[d] / 2 : c[d] / 2 - 1;
              if (e < 0 || 2 * e + 2 > r.m[d] - 1) { ok = false; break; }
            }
            e0[d] = 2 * e;
            a[d] = c[d] - 2 * e;
          }
          if (!ok) continue;
          for (int J = 0; J < 3; J++)
            for (int qj = 0; qj < 3; qj++) {
              const double cj = (2.0 / r.h) * lgl_d(qj, a[J]);
              if (cj == 0.0) continue;
              int q[3] = {a[0], a[1], a[2]};
              q[J] = qj;
              const double W = lgl_w(q[0]) * lgl_w(q[1]) * lgl_w(q[2]) * wdet;
              const double gJ = reg_deriv(r, e0, q, J);
              double scale = 1.0;
              if (TV) {
                double s2 = gJ * gJ;
                for (int d = 0; d < 3; d++)
                  if (d != J) {
                    const double gd = reg_deriv(r, e0, q, d);
                    s2 += gd * gd;
                  }
                scale = 1.0 / sqrt(s2 + r.eps);
              }
              acc += W * cj * gJ * scale;
            }
        }
    g[mi] = acc;
  }
}

// per-block partial sums of the functional: W detJ |grad f_h|^2 / 2 (TN) or
// W detJ (|grad f_h|^2 + eps)^(1/2) (TV) over the elements and their 27 points
template <bool TV>
__global__ void __launch_bounds__(kT) reg_value_kernel(RegGrid r, double *part) {
  __shared__ double sh[kT];
  const int ne[3] = {(r.m[0] - 1) / 2, (r.m[1] - 1) / 2, (r.m[2] - 1) / 2};
  const int64_t nel = (int64_t)ne[0] * ne[1] * ne[2];
  const double hh = 0.5 * r.h, wdet = hh * hh * hh;
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * kT + threadIdx.x; e < nel; e += (int64_t)gridDim.x * kT) {
    const int e0[3] = {2 * (int)(e % ne[0]), 2 * (int)((e / ne[0]) % ne[1]), 2 * (int)(e / ((int64_t)ne[0] * ne[1]))};
    for (int cq = 0; cq < 27; cq++) {
      const int q[3] = {cq % 3, (cq / 3) % 3, cq / 9};
      const double gx = reg_deriv(r, e0, q, 0), gy = reg_deriv(r, e0, q, 1), gz = reg_deriv(r, e0, q, 2);
      const double s2 = gx * gx + gy * gy + gz * gz;
      const double W = lgl_w(q[0]) * lgl_w(q[1]) * lgl_w(q[2]) * wdet;
      acc += TV ? W * sqrt(s2 + r.eps) : 0.5 * W * s2;
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
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

void opt_dot(const double *a, const double *b, int64_t n, double *part, double *out, cudaStream_t s) {
  const int nb = grid_for(n);
  dot_kernel<<<nb, kT, 0, s>>>(a, b, n, part);
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

void opt_regularization(const float *f, const int m[3], double h, bool tv, double eps, double *g, double *part,
                        double *value, cudaStream_t s) {
  RegGrid r{f, {m[0], m[1], m[2]}, h, eps};
  const int64_t n = (int64_t)m[0] * m[1] * m[2];
  const int64_t nel = (int64_t)((m[0] - 1) / 2) * ((m[1] - 1) / 2) * ((m[2] - 1) / 2);
  const int nb = grid_for(nel);
  if (tv) {
    reg_grad_kernel<true><<<grid_for(n), kT, 0, s>>>(r, g);
    reg_value_kernel<true><<<nb, kT, 0, s>>>(r, part);
  } else {
    reg_grad_kernel<false><<<grid_for(n), kT, 0, s>>>(r, g);
    reg_value_kernel<false><<<nb, kT, 0, s>>>(r, part);
  }
  sum_parts<<<1, kT, 0, s>>>(part, nb, value);
}

void opt_absmax(const double *x, int64_t n, unsigned long long *out, cudaStream_t s) {
  absmax_kernel<<<grid_for(n), kT, 0, s>>>(x, n, out);
}

}  // namespace fwi
