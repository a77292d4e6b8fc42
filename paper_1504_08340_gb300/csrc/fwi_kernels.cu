// fwi_kernels.cu -- CUDA kernels of the gradient path other than the RK4 stage
// (sm_103a): point loads, receiver sampling, the FP64 gradient integrals
// (C.1f)/(C.1g) of arXiv:1504.08340 and the FP64 misfit reduction.
//
// Element-wise derivatives at a node use the one-sided / centred 3-point stencils
// of the 27-node LGL element along each axis (see fwi_stage.cu):
//   C (odd coordinate): (v[c+1] - v[c-1]) / h
//   L (element below):  (v[c-2] - 4 v[c-1] + 3 v[c]) / h
//   R (element above):  (-3 v[c] + 4 v[c+1] - v[c+2]) / h
#include <cuda_runtime.h>

#include "fwi_internal.h"

namespace fwi {
namespace {

enum { kC = 0, kL = 1, kR = 2 };

struct Axis {
  int ns;       // elements along this axis that contain the node (1 or 2)
  int type[2];  // side type of each
  bool rd[2];   // element index along this axis inside the interior range
};

__device__ __forceinline__ Axis axis_info(int c, int n, int lo, int hi) {
  Axis a;
  a.ns = 0;
  a.type[0] = a.type[1] = kC;
  a.rd[0] = a.rd[1] = false;
  if (c & 1) {
    int e = (c - 1) >> 1;
    a.type[0] = kC;
    a.rd[0] = e >= lo && e < hi;
    a.ns = 1;
  } else {
    if (c >= 2) {
      int e = (c >> 1) - 1;
      a.type[a.ns] = kL;
      a.rd[a.ns] = e >= lo && e < hi;
      a.ns++;
    }
    if (c <= n - 3) {
      int e = c >> 1;
      a.type[a.ns] = kR;
      a.rd[a.ns] = e >= lo && e < hi;
      a.ns++;
    }
  }
  return a;
}

// element-wise derivative stencil (times h) of field f at index i, axis stride s
__device__ __forceinline__ float dstc(const float *__restrict__ f, int64_t i, int64_t s, int type) {
  if (type == kC) return __ldg(f + i + s) - __ldg(f + i - s);
  if (type == kL) return __ldg(f + i - 2 * s) - 4.f * __ldg(f + i - s) + 3.f * __ldg(f + i);
  return -3.f * __ldg(f + i) + 4.f * __ldg(f + i + s) - __ldg(f + i + 2 * s);
}

__global__ void point_kernel(PointArgs p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.npts * p.nshot) return;
  const int b = t / p.npts, i = t - b * p.npts;  // shot of the batch, point
  const int k = p.mode == 0 ? b : i;             // sources: one point per shot
  const int64_t n = p.node[k];
  float *buf = p.buf + (int64_t)b * p.sstride;
  const float *table = p.mode == 0 ? p.table : p.table + (int64_t)b * p.tstride;
  for (int c = 0; c < 3; c++) {
    float amp;
    if (p.mode == 0) {
      amp = table[p.i0];
      if (p.i1 >= 0) amp = 0.5f * (amp + table[p.i1]);
    } else {
      amp = table[((int64_t)p.i0 * p.npts + i) * 3 + c];
      if (p.i1 >= 0) amp = 0.5f * (amp + table[((int64_t)p.i1 * p.npts + i) * 3 + c]);
    }
    buf[(int64_t)(18 + c) * p.stride + n] += p.cdt * amp * p.vec[k * 3 + c];
  }
}

__global__ void sample_kernel(const float *buf, int64_t stride, int nrec, const int64_t *node, float *tr,
                              int nshot, int64_t sstride, int64_t tstride) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrec * 3 * nshot) return;
  const int b = t / (nrec * 3), i = t - b * nrec * 3;
  const int r = i / 3, c = i % 3;
  tr[(int64_t)b * tstride + i] = buf[(int64_t)b * sstride + (int64_t)(9 + c) * stride + node[r]];
}

// (C.1f)/(C.1g) at one time level. One thread per interior node; the sum over the
// interior elements around the node of the element-wise gradients' products.
__global__ void __launch_bounds__(256) gradient_kernel(Geo g, const float *__restrict__ ws0,
                                                       const float *__restrict__ uh0, double wdt,
                                                       double *gl, double *gm, int nshot, int64_t sstride,
                                                       int64_t hstride) {
  const int64_t mi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (mi >= g.nmat) return;
  const int i = (int)(mi % g.m[0]);
  const int64_t t = mi / g.m[0];
  const int j = (int)(t % g.m[1]);
  const int k = (int)(t / g.m[1]);
  const int I = i + 2 * g.lo[0], J = j + 2 * g.lo[1], K = k + 2 * g.lo[2];
  const int c3[3] = {I, J, K};
  const int64_t node = ((int64_t)K * g.n[1] + J) * g.px + I;
  const int64_t sn[3] = {1, (int64_t)g.px, (int64_t)g.px * g.n[1]};
  const int64_t sm[3] = {1, (int64_t)g.m[0], (int64_t)g.m[0] * g.m[1]};
  Axis ax[3] = {axis_info(I, g.n[0], g.lo[0], g.hi[0]), axis_info(J, g.n[1], g.lo[1], g.hi[1]),
                axis_info(K, g.n[2], g.lo[2], g.hi[2])};
  float W = g.wdetj;
#pragma unroll
  for (int x = 0; x < 3; x++) W *= (c3[x] & 1) ? (4.f / 3.f) : (1.f / 3.f);
  double accl = gl[mi], accm = gm[mi];
  // the shots of a batch in order: shot b's adjoint state at ws0 + b sstride, its
  // displacement history level at uh0 + b hstride
#pragma unroll 1
  for (int b = 0; b < nshot; b++) {
  const float *__restrict__ ws = ws0 + b * sstride;
  const float *__restrict__ uh = uh0 + b * hstride;
  // all loops have fixed trip counts and are unrolled, so the arrays stay in registers
  float dw[3][2][3], du[3][2][3];  // [axis][side][component]
#pragma unroll
  for (int x = 0; x < 3; x++)
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const bool used = s < ax[x].ns && ax[x].rd[s];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        dw[x][s][c] = used ? dstc(ws + (int64_t)(9 + c) * g.stride, node, sn[x], ax[x].type[s]) * g.inv_h : 0.f;
        du[x][s][c] = used ? dstc(uh + (int64_t)c * g.nmat, mi, sm[x], ax[x].type[s]) * g.inv_h : 0.f;
      }
    }
  float sl = 0.f, smu = 0.f;
#pragma unroll
  for (int sx = 0; sx < 2; sx++)
#pragma unroll
    for (int sy = 0; sy < 2; sy++)
#pragma unroll
      for (int sz = 0; sz < 2; sz++) {
        if (sx >= ax[0].ns || sy >= ax[1].ns || sz >= ax[2].ns) continue;
        if (!(ax[0].rd[sx] && ax[1].rd[sy] && ax[2].rd[sz])) continue;
        const int s[3] = {sx, sy, sz};
        float Gw[3][3], Gu[3][3];  // G[i][j] = d v_i / d x_j
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
          for (int b = 0; b < 3; b++) {
            Gw[a][b] = dw[b][s[b]][a];
            Gu[a][b] = du[b][s[b]][a];
          }
        const float divw = Gw[0][0] + Gw[1][1] + Gw[2][2];
        const float divu = Gu[0][0] + Gu[1][1] + Gu[2][2];
        sl += divw * divu;
        smu += 2.f * (Gw[0][0] * Gu[0][0] + Gw[1][1] * Gu[1][1] + Gw[2][2] * Gu[2][2]) +
               (Gw[0][1] + Gw[1][0]) * (Gu[1][0] + Gu[0][1]) + (Gw[0][2] + Gw[2][0]) * (Gu[2][0] + Gu[0][2]) +
               (Gw[1][2] + Gw[2][1]) * (Gu[2][1] + Gu[1][2]);
      }
  accl -= wdt * (double)W * (double)sl;
  accm -= wdt * (double)W * (double)smu;
  }
  gl[mi] = accl;
  gm[mi] = accm;
}

constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads) residual_kernel(const float *tr, const float *ob, float *res,
                                                               int64_t n, int64_t per_step, int nsteps,
                                                               double dt, double *part, int *flag) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float tv = tr[i];
    if (!isfinite(tv)) bad = 1;
    const float e = tv - ob[i];
    res[i] = e;
    const int64_t step = i / per_step;
    const double wn = (step == 0 || step == nsteps) ? 0.5 : 1.0;
    acc += 0.5 * wn * dt * (double)e * (double)e;
  }
  if (bad) *flag = 1;
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kRedThreads) sum_kernel(const double *part, int nb, double *out) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void finite_kernel(const double *x, int64_t n, int *flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) *flag = 1;
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

void launch_point(const PointArgs &p, cudaStream_t s) {
  if (p.npts <= 0 || p.nshot <= 0) return;
  point_kernel<<<blocks_for((int64_t)p.npts * p.nshot, 128), 128, 0, s>>>(p);
}

void launch_sample(const float *buf, int64_t stride, int nrec, const int64_t *node, float *traces,
                   cudaStream_t s, int nshot, int64_t sstride, int64_t tstride) {
  if (nrec <= 0 || nshot <= 0) return;
  sample_kernel<<<blocks_for((int64_t)nrec * 3 * nshot, 256), 256, 0, s>>>(buf, stride, nrec, node, traces, nshot,
                                                                           sstride, tstride);
}

void launch_gradient(const Geo &g, const float *w_state, const float *u_hist, double wdt, double *gl,
                     double *gm, cudaStream_t s, int nshot, int64_t sstride, int64_t hstride) {
  gradient_kernel<<<blocks_for(g.nmat, 256), 256, 0, s>>>(g, w_state, u_hist, wdt, gl, gm, nshot, sstride,
                                                          hstride);
}

int misfit_blocks(int64_t n) {
  int64_t b = (n + kRedThreads - 1) / kRedThreads;
  if (b < 1) b = 1;
  return (int)(b > 1024 ? 1024 : b);
}

void launch_residual(const float *traces, const float *observed, float *resid, int64_t n, int64_t per_step,
                     int nsteps, double dt, double *part, int *flag, cudaStream_t s) {
  residual_kernel<<<misfit_blocks(n), kRedThreads, 0, s>>>(traces, observed, resid, n, per_step, nsteps, dt,
                                                          part, flag);
}

void launch_sum(const double *part, int nblocks, double *out, cudaStream_t s) {
  sum_kernel<<<1, kRedThreads, 0, s>>>(part, nblocks, out);
}

// lambda, mu at node (i, j, k) of the state layout: the material-grid value, with the
// coordinates clamped to the interior box for PML nodes (the material extended into
// the PML); the row padding gets zero
__global__ void extend_material_kernel(Geo g, float *lam_n, float *mu_n) {
  const int64_t n = (int64_t)g.px * g.n[1] * g.n[2];
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(idx % g.px);
    const int64_t r = idx / g.px;
    const int J = (int)(r % g.n[1]), K = (int)(r / g.n[1]);
    if (I >= g.n[0]) {
      lam_n[idx] = 0.f;
      mu_n[idx] = 0.f;
      continue;
    }
    int i = I - 2 * g.lo[0], j = J - 2 * g.lo[1], k = K - 2 * g.lo[2];
    i = i < 0 ? 0 : (i >= g.m[0] ? g.m[0] - 1 : i);
    j = j < 0 ? 0 : (j >= g.m[1] ? g.m[1] - 1 : j);
    k = k < 0 ? 0 : (k >= g.m[2] ? g.m[2] - 1 : k);
    const int64_t mi = ((int64_t)k * g.m[1] + j) * g.m[0] + i;
    lam_n[idx] = g.lam[mi];
    mu_n[idx] = g.mu[mi];
  }
}

void launch_extend_material(const Geo &g, float *lam_n, float *mu_n, cudaStream_t s) {
  const int64_t n = (int64_t)g.px * g.n[1] * g.n[2];
  int64_t b = (n + 255) / 256;
  extend_material_kernel<<<(int)(b > 4096 ? 4096 : b), 256, 0, s>>>(g, lam_n, mu_n);
}

void launch_check_finite(const double *x, int64_t n, int *flag, cudaStream_t s) {
  finite_kernel<<<misfit_blocks(n), kRedThreads, 0, s>>>(x, n, flag);
}

}  // namespace fwi
