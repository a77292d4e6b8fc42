// fwi_kernels.cu -- CUDA kernels of the gradient path other than the RK4 stage
// (sm_103a): point loads, receiver sampling, the FP64 gradient integrals
// (C.1f)/(C.1g) of arXiv:1504.08340 and the FP64 misfit reduction.
//
// Element-wise derivatives at a node use the one-sided / centred 3-point stencils
// of the 27-node LGL element along each axis:
//   C (odd coordinate): (v[c+1] - v[c-1]) / h
//   L (element below):  (v[c-2] - 4 v[c-1] + 3 v[c]) / h
//   R (element above):  (-3 v[c] + 4 v[c+1] - v[c+2]) / h
#include <cuda_runtime.h>

#include "fwi_internal.h"

namespace fwi {
namespace {

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__global__ void point_kernel(PointArgs p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.npts * p.nshot) return;
  const int b = t / p.npts, i = t - b * p.npts;  // shot of the batch, point
  const int k = p.mode == 0 ? b : i;             // sources: one point per shot
  const int64_t n = p.node[k];
  if (!guard(p.oob, kSitePoint, n, p.nnode_pad)) return;
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
                              int nshot, int64_t sstride, int64_t tstride, unsigned long long *oob) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrec * 3 * nshot) return;
  const int b = t / (nrec * 3), i = t - b * nrec * 3;
  const int r = i / 3, c = i % 3;
  const int64_t n = node[r];
  if (!guard(oob, kSiteSample, n, stride)) return;
  tr[(int64_t)b * tstride + i] = buf[(int64_t)b * sstride + (int64_t)(9 + c) * stride + n];
}

// (C.1f)/(C.1g) at one time level, in FP64: for every interior node, the sum over the
// interior elements around it of W detJ times the products of the element-wise
// gradients of w and u. A block owns a 32 x 8 tile of interior nodes in
// (x, y) and marches up a chunk of kGKC levels in z. Plane k of the six fields (w and
// u, three components each) is staged with its two-node x/y halo in a six-slot ring
// by 4-byte cp.async; the copies of plane k + 3 are in flight while level k is
// computed from planes k-2 .. k+2, so a level costs one barrier. Every derivative
// candidate of an axis (C, or L and R) is formed from the five staged values and the
// one the node's parity asks for is selected, so the x parity alternating across a
// warp costs no divergence in the stencils.
constexpr int kGX = 32, kGY = 8, kGKC = 16, kGH = 2;
constexpr int kGW = kGX + 2 * kGH, kGR = kGY + 2 * kGH, kGP = kGW * kGR;  // staged positions per plane
constexpr int kGSlots = 6, kGFields = 6;
constexpr size_t kGSmem = sizeof(float) * kGSlots * kGFields * kGP;

__device__ __forceinline__ void cp_async4(float *dst, const float *src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}

// copies of plane k (0 <= k < m[2]) of the tile at (x0, y0) into its ring slot; halo
// positions outside the interior grid are zero-filled (the stencils never select them)
__device__ __forceinline__ void grad_stage_plane(const Geo &g, const float *ws, const float *uh, float *ring, int k,
                                                 int x0, int y0, int tid) {
  float *slot = ring + ((k + kGSlots) % kGSlots) * (kGFields * kGP);
  for (int p = tid; p < kGP; p += kGX * kGY) {
    const int hy = p / kGW, hx = p - hy * kGW;
    const int i = x0 - kGH + hx, j = y0 - kGH + hy;
    const bool v = i >= 0 && i < g.m[0] && j >= 0 && j < g.m[1];
    const int64_t node =
        v ? ((int64_t)(k + 2 * g.lo[2]) * g.n[1] + (j + 2 * g.lo[1])) * g.px + (i + 2 * g.lo[0]) : 0;
    const int64_t mi = v ? ((int64_t)k * g.m[1] + j) * g.m[0] + i : 0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      cp_async4(slot + c * kGP + p, ws + (int64_t)(9 + c) * g.stride + node, v ? 4 : 0);
      cp_async4(slot + (3 + c) * kGP + p, uh + (int64_t)c * g.nmat + mi, v ? 4 : 0);
    }
  }
}

// the candidates of one axis from the five values f[-2..2] along it: side 0 is C (odd
// coordinate) or L (even), side 1 is R
__device__ __forceinline__ void grad_axis(float a, float b, float c, float d, float e, bool odd, float inv_h,
                                          float &s0, float &s1) {
  s0 = (odd ? d - b : a - 4.f * b + 3.f * c) * inv_h;
  s1 = (-3.f * c + 4.f * d - e) * inv_h;
}

__global__ void __launch_bounds__(kGX *kGY, 3) gradient_kernel(Geo g, const float *__restrict__ ws0,
                                                                     const float *__restrict__ uh0, double wdt,
                                                                     double *gl, double *gm, int nshot,
                                                                     int64_t sstride, int64_t hstride) {
  extern __shared__ float ring[];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kGX + tx;
  const int x0 = blockIdx.x * kGX, y0 = blockIdx.y * kGY, k0 = blockIdx.z * kGKC;
  const int m2 = g.m[2], k1 = min(k0 + kGKC, m2);
  const int i = x0 + tx, j = y0 + ty;
  const bool own = i < g.m[0] && j < g.m[1];
  // element sides present along each axis: odd coordinate -> the one element it is
  // the centre of; even -> below (L) if it is not the first node, above (R) if it is
  // not the last
  const bool ox = i & 1, oy = j & 1;
  const bool vx[2] = {ox || i >= 2, !ox && i <= g.m[0] - 3};
  const bool vy[2] = {oy || j >= 2, !oy && j <= g.m[1] - 3};
  const float Wxy = g.wdetj * (ox ? 4.f / 3.f : 1.f / 3.f) * (oy ? 4.f / 3.f : 1.f / 3.f);
  const int q = (ty + kGH) * kGW + tx + kGH;  // the node's staged position
#pragma unroll 1
  for (int b = 0; b < nshot; b++) {
    const float *ws = ws0 + b * sstride;
    const float *uh = uh0 + b * hstride;
    for (int k = max(k0 - 2, 0); k <= min(k0 + 2, m2 - 1); k++) grad_stage_plane(g, ws, uh, ring, k, x0, y0, tid);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
#pragma unroll 1
    for (int k = k0; k < k1; k++) {
      if (k + 3 <= min(k1 + 1, m2 - 1)) grad_stage_plane(g, ws, uh, ring, k + 3, x0, y0, tid);
      cp_async_commit();
      if (own) {
        const bool oz = k & 1;
        const bool vz[2] = {oz || k >= 2, !oz && k <= m2 - 3};
        const float *sl5[5];
#pragma unroll
        for (int d = 0; d < 5; d++) sl5[d] = ring + ((k - 2 + d + kGSlots) % kGSlots) * (kGFields * kGP) + q;
        float dv[3][2][kGFields];  // [axis][side][field]
#pragma unroll
        for (int f = 0; f < kGFields; f++) {
          const float *c = sl5[2] + f * kGP;
          grad_axis(c[-2], c[-1], c[0], c[1], c[2], ox, g.inv_h, dv[0][0][f], dv[0][1][f]);
          grad_axis(c[-2 * kGW], c[-kGW], c[0], c[kGW], c[2 * kGW], oy, g.inv_h, dv[1][0][f], dv[1][1][f]);
          grad_axis(sl5[0][f * kGP], sl5[1][f * kGP], c[0], sl5[3][f * kGP], sl5[4][f * kGP], oz, g.inv_h,
                    dv[2][0][f], dv[2][1][f]);
        }
        float sl = 0.f, smu = 0.f;
#pragma unroll
        for (int sx = 0; sx < 2; sx++)
#pragma unroll
          for (int sy = 0; sy < 2; sy++)
#pragma unroll
            for (int sz = 0; sz < 2; sz++) {
              if (!(vx[sx] && vy[sy] && vz[sz])) continue;
              const int sd[3] = {sx, sy, sz};
              float Gw[3][3], Gu[3][3];  // G[a][b] = d v_a / d x_b
#pragma unroll
              for (int a = 0; a < 3; a++)
#pragma unroll
                for (int x = 0; x < 3; x++) {
                  Gw[a][x] = dv[x][sd[x]][a];
                  Gu[a][x] = dv[x][sd[x]][3 + a];
                }
              const float divw = Gw[0][0] + Gw[1][1] + Gw[2][2];
              const float divu = Gu[0][0] + Gu[1][1] + Gu[2][2];
              sl += divw * divu;
              smu += 2.f * (Gw[0][0] * Gu[0][0] + Gw[1][1] * Gu[1][1] + Gw[2][2] * Gu[2][2]) +
                     (Gw[0][1] + Gw[1][0]) * (Gu[1][0] + Gu[0][1]) + (Gw[0][2] + Gw[2][0]) * (Gu[2][0] + Gu[0][2]) +
                     (Gw[1][2] + Gw[2][1]) * (Gu[2][1] + Gu[1][2]);
            }
        const float W = Wxy * (oz ? 4.f / 3.f : 1.f / 3.f);
        const int64_t mi = ((int64_t)k * g.m[1] + j) * g.m[0] + i;
        if (guard(g.oob, kSiteGradient, mi, g.nmat)) {
          gl[mi] -= wdt * (double)W * (double)sl;
          gm[mi] -= wdt * (double)W * (double)smu;
        }
      }
      cp_async_wait_all();
      __syncthreads();
    }
  }
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
                   cudaStream_t s, int nshot, int64_t sstride, int64_t tstride, unsigned long long *oob) {
  if (nrec <= 0 || nshot <= 0) return;
  sample_kernel<<<blocks_for((int64_t)nrec * 3 * nshot, 256), 256, 0, s>>>(buf, stride, nrec, node, traces, nshot,
                                                                           sstride, tstride, oob);
}

void launch_gradient(const Geo &g, const float *w_state, const float *u_hist, double wdt, double *gl,
                     double *gm, cudaStream_t s, int nshot, int64_t sstride, int64_t hstride) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(gradient_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem);
    attr = true;
  }
  const dim3 grid((g.m[0] + kGX - 1) / kGX, (g.m[1] + kGY - 1) / kGY, (g.m[2] + kGKC - 1) / kGKC);
  gradient_kernel<<<grid, dim3(kGX, kGY), kGSmem, s>>>(g, w_state, u_hist, wdt, gl, gm, nshot, sstride,
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

// ---- compact forward-state snapshots (checkpointed adjoint sweep)
// Slots 0..5 hold the fields 9, 10, 11, 18, 19, 20 (u and udot) of every entry; slots
// 6..26 hold the other 21 fields (ubar and the three stress levels) at the PML nodes of
// `list` only, npad values each: those fields are zero at every other entry of any state.
namespace {
__device__ __forceinline__ int snap_field(int slot) {
  if (slot < 3) return 9 + slot;
  if (slot < 6) return 15 + slot;              // 18, 19, 20
  const int k = slot - 6;                      // 0..20
  return k < 9 ? k : (k < 15 ? k + 3 : k + 6);  // 0..8, 12..17, 21..26
}

template <bool PACK>
__global__ void __launch_bounds__(256) snapshot_kernel(float *state, float *snap, const int *__restrict__ list,
                                                       int64_t npml, int64_t npad, int64_t stride, int64_t sstride,
                                                       int64_t snap_stride, unsigned long long *oob) {
  const int slot = blockIdx.y;
  float *st = state + (int64_t)blockIdx.z * sstride + (int64_t)snap_field(slot) * stride;
  float *sn = snap + (int64_t)blockIdx.z * snap_stride;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, dt = (int64_t)gridDim.x * blockDim.x;
  if (slot < 6) {  // dense: stride is a multiple of 64 floats and every base is 256-byte aligned
    float4 *a = reinterpret_cast<float4 *>(sn + (int64_t)slot * stride);
    float4 *b = reinterpret_cast<float4 *>(st);
    for (int64_t i = t0; i < stride / 4; i += dt) {
      if (PACK) __stcs(a + i, __ldcs(b + i));
      else __stcs(b + i, __ldcs(a + i));
    }
  } else {
    float *a = sn + 6 * stride + (int64_t)(slot - 6) * npad;
    for (int64_t p = t0; p < npml; p += dt) {
      const int64_t n = __ldg(list + p);
      if (!guard(oob, kSiteSnapshot, n, stride)) continue;
      if (PACK) __stcs(a + p, __ldcs(st + n));
      else __stcs(st + n, __ldcs(a + p));
    }
  }
}
}  // namespace

void launch_snapshot(float *state, float *snap, const int *list, int64_t npml, int64_t npad, int64_t stride,
                     int nshot, int64_t sstride, int64_t snap_stride, bool pack, cudaStream_t s,
                     unsigned long long *oob) {
  const dim3 grid(296, 27, nshot);
  if (pack)
    snapshot_kernel<true><<<grid, 256, 0, s>>>(state, snap, list, npml, npad, stride, sstride, snap_stride, oob);
  else
    snapshot_kernel<false><<<grid, 256, 0, s>>>(state, snap, list, npml, npad, stride, sstride, snap_stride, oob);
}

void launch_check_finite(const double *x, int64_t n, int *flag, cudaStream_t s) {
  finite_kernel<<<misfit_blocks(n), kRedThreads, 0, s>>>(x, n, flag);
}

}  // namespace fwi
