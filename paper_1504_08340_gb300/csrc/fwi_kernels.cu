// fwi_kernels.cu -- CUDA kernels of the per-shot gradient path (sm_103a).
//
// Discretisation (Sec. 2 of arXiv:1504.08340): 27-node hexahedral spectral
// elements with LGL quadrature on a structured box. Because the quadrature
// points coincide with the nodes and the box is structured, every element-level
// quantity evaluated at a node reduces to short one-dimensional stencils along
// the three axes, and the assembled (summed over elements) operator at a node is
// a sum over the at most 8 elements around it. The stage kernel therefore works
// node-by-node ("gather"), fuses the matrix-free operator of (6) with the RK4
// stage update, writes every output exactly once, and needs no atomics: results
// are bitwise reproducible.
//
// Stencils along an axis, for a node at coordinate c (node spacing h/2):
//  element-wise derivative at the node, inside the element on side
//    C (c odd, node is the element's middle node):   (v[c+1] - v[c-1]) / h
//    L (c even, element on the low side, local 2):   (v[c-2] - 4 v[c-1] + 3 v[c]) / h
//    R (c even, element on the high side, local 0):  (-3 v[c] + 4 v[c+1] - v[c+2]) / h
//  quadrature of d phi_a/dx_j along the element line through the node,
//  sum_q w_q (2/h) D[q][a] g(x_q), with GLL weights (1/3, 4/3, 1/3):
//    C: (4 g[c-1] - 4 g[c+1]) / (3h)
//    L: (-g[c-2] + 4 g[c-1] + 3 g[c]) / (3h)
//    R: (-3 g[c] - 4 g[c+1] + g[c+2]) / (3h)
#include <cuda_runtime.h>

#include "fwi_internal.h"

namespace fwi {
namespace {

enum { kC = 0, kL = 1, kR = 2 };

// line points (offsets along the axis) of the element on one side, their
// quadrature coefficient (units 1/(3h)) and the side type of the point itself
__constant__ int kLineOff[3][3] = {{-1, 0, 1}, {-2, -1, 0}, {0, 1, 2}};
__constant__ float kLineCoef[3][3] = {{4.f, 0.f, -4.f}, {-1.f, 4.f, 3.f}, {-3.f, -4.f, 1.f}};
// point p of a line has local index p inside the element: 0 -> R, 1 -> C, 2 -> L
__device__ __forceinline__ int point_type(int p) { return p == 0 ? kR : (p == 1 ? kC : kL); }

// symmetric component index of (i, j): xx yy zz yz xz xy
__device__ __forceinline__ int sym(int i, int j) {
  return i == j ? i : (i + j == 1 ? 5 : (i + j == 2 ? 4 : 3));
}

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

__device__ __forceinline__ int clampi(int v, int a, int b) { return v < a ? a : (v > b ? b : v); }

__device__ __forceinline__ int64_t mat_index(const Geo &g, int I, int J, int K) {
  int i = clampi(I - 2 * g.lo[0], 0, g.m[0] - 1);
  int j = clampi(J - 2 * g.lo[1], 0, g.m[1] - 1);
  int k = clampi(K - 2 * g.lo[2], 0, g.m[2] - 1);
  return ((int64_t)k * g.m[1] + j) * g.m[0] + i;
}

// Rate of the first-order system at one node (forward: Eq. (6); adjoint: the
// reversed-time transposed system, see fwi_rhs in fwi.h), then the RK4 stage
// update of that node.
template <bool ADJ>
__global__ void __launch_bounds__(256) stage_kernel(Geo g, StageArgs a) {
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nnode) return;
  const int I = (int)(node % g.n[0]);
  const int64_t t = node / g.n[0];
  const int J = (int)(t % g.n[1]);
  const int K = (int)(t / g.n[1]);
  const int c3[3] = {I, J, K};
  const int64_t st[3] = {1, (int64_t)g.n[0], (int64_t)g.n[0] * g.n[1]};
  const Axis ax[3] = {axis_info(I, g.n[0], g.lo[0], g.hi[0]), axis_info(J, g.n[1], g.lo[1], g.hi[1]),
                      axis_info(K, g.n[2], g.lo[2], g.hi[2])};
  const bool dir = I == 0 || I == g.n[0] - 1 || J == 0 || J == g.n[1] - 1 || K == g.n[2] - 1 ||
                   (g.top_dir && K == 0);
  int nel = ax[0].ns * ax[1].ns * ax[2].ns, nrd = 0;
  for (int sx = 0; sx < ax[0].ns; sx++)
    for (int sy = 0; sy < ax[1].ns; sy++)
      for (int sz = 0; sz < ax[2].ns; sz++) nrd += (ax[0].rd[sx] && ax[1].rd[sy] && ax[2].rd[sz]);
  const int npml = nel - nrd;
  const bool pml = npml > 0;

  const int64_t S = g.stride;
  const float *__restrict__ Y = a.Y;
  auto F = [&](int f) { return Y + (int64_t)f * S; };

  // stretch coefficients at the node (reading R1, products of eps_x eps_y eps_z)
  const float alx = __ldg(g.alpha[0] + I), aly = __ldg(g.alpha[1] + J), alz = __ldg(g.alpha[2] + K);
  const float bex = __ldg(g.beta[0] + I), bey = __ldg(g.beta[1] + J), bez = __ldg(g.beta[2] + K);
  const float ca = alx * aly * alz;
  const float cb = alx * aly * bez + alx * bey * alz + bex * aly * alz;
  const float cc = alx * bey * bez + bex * aly * bez + bex * bey * alz;
  const float cd = bex * bey * bez;
  const float Le[3] = {aly * alz, alx * alz, alx * aly};
  const float Lp[3] = {aly * bez + bey * alz, alx * bez + bex * alz, alx * bey + bex * aly};
  const float Lw[3] = {bey * bez, bex * bez, bex * bey};

  float rate[27];
#pragma unroll
  for (int f = 0; f < 27; f++) rate[f] = 0.f;

  // ---------------------------------------------------------- u rows
  if (!dir) {
    float frd[3] = {0.f, 0.f, 0.f}, fpml[3] = {0.f, 0.f, 0.f};
    for (int j = 0; j < 3; j++) {
      const int k = (j + 1) % 3, l = (j + 2) % 3;
      const float invw = (c3[j] & 1) ? 0.75f : 3.0f;
      for (int sj = 0; sj < ax[j].ns; sj++) {
        const int ty = ax[j].type[sj];
        int cpml = 0, crd = 0;
        for (int sk = 0; sk < ax[k].ns; sk++)
          for (int sl = 0; sl < ax[l].ns; sl++) {
            bool rd = ax[j].rd[sj] && ax[k].rd[sk] && ax[l].rd[sl];
            crd += rd;
            cpml += !rd;
          }
        // interior elements: sum of the element-wise stresses sigma_ij along the line
        if (crd) {
          float acc[3] = {0.f, 0.f, 0.f};
          for (int p = 0; p < 3; p++) {
            const float cf = kLineCoef[ty][p];
            if (cf == 0.f) continue;
            const int off = kLineOff[ty][p];
            const int64_t q = node + off * st[j];
            int cq[3] = {I, J, K};
            cq[j] += off;
            const int64_t mq = mat_index(g, cq[0], cq[1], cq[2]);
            const float lq = __ldg(g.lam + mq), mq_ = __ldg(g.mu + mq);
            const int pt = point_type(p);
            float dj[3];
#pragma unroll
            for (int c = 0; c < 3; c++) dj[c] = dstc(F(9 + c), q, st[j], pt);
            float dll[2] = {0.f, 0.f}, dlj[2] = {0.f, 0.f};
            for (int sl = 0; sl < ax[l].ns; sl++) {
              dll[sl] = dstc(F(9 + l), q, st[l], ax[l].type[sl]);
              dlj[sl] = dstc(F(9 + j), q, st[l], ax[l].type[sl]);
            }
            float sjj = 0.f, skj = 0.f, slj = 0.f;
            for (int sk = 0; sk < ax[k].ns; sk++) {
              const float dkk = dstc(F(9 + k), q, st[k], ax[k].type[sk]);
              const float dkj = dstc(F(9 + j), q, st[k], ax[k].type[sk]);
              for (int sl = 0; sl < ax[l].ns; sl++) {
                if (!(ax[j].rd[sj] && ax[k].rd[sk] && ax[l].rd[sl])) continue;
                const float tr = dj[j] + dkk + dll[sl];
                sjj += lq * tr + 2.f * mq_ * dj[j];
                skj += mq_ * (dj[k] + dkj);
                slj += mq_ * (dj[l] + dlj[sl]);
              }
            }
            acc[j] += cf * sjj;
            acc[k] += cf * skj;
            acc[l] += cf * slj;
          }
          frd[0] += invw * acc[0];
          frd[1] += invw * acc[1];
          frd[2] += invw * acc[2];
        }
        // PML elements: divergence of Sdot Le + S Lp + Sbar Lw (forward) or of the
        // same with tau(T) = mu (T + diag T) + lambda tr(T) I in place of S (adjoint)
        if (cpml) {
          float acc[3] = {0.f, 0.f, 0.f};
          const float Lv[3] = {Lw[j], Lp[j], Le[j]};  // levels 0 (history), 1, 2 (rate)
          for (int p = 0; p < 3; p++) {
            const float cf = kLineCoef[ty][p];
            if (cf == 0.f) continue;
            const int64_t q = node + kLineOff[ty][p] * st[j];
            float qj = 0.f, qk = 0.f, ql = 0.f;
            if (!ADJ) {
#pragma unroll
              for (int lv = 0; lv < 3; lv++) {
                const int b = 9 * lv + 3;
                qj += Lv[lv] * __ldg(F(b + sym(j, j)) + q);
                qk += Lv[lv] * __ldg(F(b + sym(k, j)) + q);
                ql += Lv[lv] * __ldg(F(b + sym(l, j)) + q);
              }
            } else {
              int cq[3] = {I, J, K};
              cq[j] += kLineOff[ty][p];
              const int64_t mq = mat_index(g, cq[0], cq[1], cq[2]);
              const float lq = __ldg(g.lam + mq), mq_ = __ldg(g.mu + mq);
#pragma unroll
              for (int lv = 0; lv < 3; lv++) {
                const int b = 9 * lv + 3;
                const float tjj = __ldg(F(b + j) + q), tkk = __ldg(F(b + k) + q), tll = __ldg(F(b + l) + q);
                const float tkj = __ldg(F(b + sym(k, j)) + q), tlj = __ldg(F(b + sym(l, j)) + q);
                qj += Lv[lv] * (2.f * mq_ * tjj + lq * (tjj + tkk + tll));
                qk += Lv[lv] * (mq_ * tkj);
                ql += Lv[lv] * (mq_ * tlj);
              }
            }
            acc[j] += cf * qj;
            acc[k] += cf * qk;
            acc[l] += cf * ql;
          }
          const float wgt = invw * (float)cpml;
          fpml[0] += wgt * acc[0];
          fpml[1] += wgt * acc[1];
          fpml[2] += wgt * acc[2];
        }
      }
    }
    const float s_rd = g.inv_h * g.inv_h * (1.f / 3.f), s_pml = g.inv_h * (1.f / 3.f);
    const float inv_m = 1.f / (g.rho * ca * (float)nel);
    const float inv_a = 1.f / ca;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const float u0 = __ldg(F(c) + node), u1 = __ldg(F(9 + c) + node), u2 = __ldg(F(18 + c) + node);
      rate[c] = pml ? u1 : 0.f;
      rate[9 + c] = u2;
      rate[18 + c] = -(s_rd * frd[c] + s_pml * fpml[c]) * inv_m - (cb * u2 + cc * u1 + cd * u0) * inv_a;
    }
  }

  // ---------------------------------------------------------- S rows (PML nodes)
  if (pml) {
    // element-summed derivatives of the three displacement levels, weighted by Lambda
    float H[3][3];  // H[i][j] = (1/npml) sum_lv Lambda^lv_jj sum_e d_j^e v^lv_i
    for (int j = 0; j < 3; j++) {
      const int k = (j + 1) % 3, l = (j + 2) % 3;
      float hs[3] = {0.f, 0.f, 0.f};
      for (int sj = 0; sj < ax[j].ns; sj++) {
        int cpml = 0;
        for (int sk = 0; sk < ax[k].ns; sk++)
          for (int sl = 0; sl < ax[l].ns; sl++) cpml += !(ax[j].rd[sj] && ax[k].rd[sk] && ax[l].rd[sl]);
        if (!cpml) continue;
        const int ty = ax[j].type[sj];
#pragma unroll
        for (int i = 0; i < 3; i++) {
          const float d = Le[j] * dstc(F(18 + i), node, st[j], ty) + Lp[j] * dstc(F(9 + i), node, st[j], ty) +
                          Lw[j] * dstc(F(i), node, st[j], ty);
          hs[i] += (float)cpml * d;
        }
      }
      const float sc = g.inv_h / (float)npml;
      H[0][j] = hs[0] * sc;
      H[1][j] = hs[1] * sc;
      H[2][j] = hs[2] * sc;
    }
    // P(H): diagonal H_ii, off-diagonal H_ij + H_ji, in the order xx yy zz yz xz xy
    float src[6] = {H[0][0], H[1][1], H[2][2], H[1][2] + H[2][1], H[0][2] + H[2][0], H[0][1] + H[1][0]};
    if (!ADJ) {
      const int64_t mi = mat_index(g, I, J, K);
      const float lq = __ldg(g.lam + mi), mq_ = __ldg(g.mu + mi);
      const float tr = src[0] + src[1] + src[2];
#pragma unroll
      for (int c = 0; c < 3; c++) src[c] = 2.f * mq_ * src[c] + lq * tr;
#pragma unroll
      for (int c = 3; c < 6; c++) src[c] = mq_ * src[c];
    }
    const float inv_a = 1.f / ca;
#pragma unroll
    for (int c = 0; c < 6; c++) {
      const float s0 = __ldg(F(3 + c) + node), s1 = __ldg(F(12 + c) + node), s2 = __ldg(F(21 + c) + node);
      rate[3 + c] = s1;
      rate[12 + c] = s2;
      rate[21 + c] = (src[c] - cb * s2 - cc * s1 - cd * s0) * inv_a;
    }
  }

  // ---------------------------------------------------------- stage update
  float *__restrict__ out = a.out;
  if (a.stage == 0) {
#pragma unroll
    for (int f = 0; f < 27; f++) out[(int64_t)f * S + node] = rate[f];
    return;
  }
#pragma unroll
  for (int f = 0; f < 27; f++) {
    const int c = f % 9, lv = f / 9;
    const bool active = c < 3 ? (!dir && (lv > 0 || pml)) : pml;
    if (!active) continue;
    const int64_t idx = (int64_t)f * S + node;
    float v;
    if (a.stage < 4) {
      v = __ldg(a.X + idx) + a.cdt * rate[f];
    } else {
      v = (-__ldg(a.X + idx) + __ldg(a.Y2 + idx) + 2.f * __ldg(a.Y3 + idx) + __ldg(Y + idx)) * (1.f / 3.f) +
          a.cdt * rate[f];
    }
    out[idx] = v;
    if (a.hist && lv == 1 && c < 3) {
      const int i = I - 2 * g.lo[0], j = J - 2 * g.lo[1], k = K - 2 * g.lo[2];
      if (i >= 0 && i < g.m[0] && j >= 0 && j < g.m[1] && k >= 0 && k < g.m[2])
        a.hist[(int64_t)c * g.nmat + ((int64_t)k * g.m[1] + j) * g.m[0] + i] = v;
    }
  }
}

__global__ void point_kernel(PointArgs p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.npts) return;
  const int64_t n = p.node[i];
  for (int c = 0; c < 3; c++) {
    float amp;
    if (p.mode == 0) {
      amp = p.table[p.i0];
      if (p.i1 >= 0) amp = 0.5f * (amp + p.table[p.i1]);
    } else {
      amp = p.table[((int64_t)p.i0 * p.npts + i) * 3 + c];
      if (p.i1 >= 0) amp = 0.5f * (amp + p.table[((int64_t)p.i1 * p.npts + i) * 3 + c]);
    }
    p.buf[(int64_t)(18 + c) * p.stride + n] += p.cdt * amp * p.vec[i * 3 + c];
  }
}

__global__ void sample_kernel(const float *buf, int64_t stride, int nrec, const int64_t *node, float *tr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrec * 3) return;
  const int r = i / 3, c = i % 3;
  tr[i] = buf[(int64_t)(9 + c) * stride + node[r]];
}

// (C.1f)/(C.1g) at one time level. One thread per interior node; the sum over the
// interior elements around the node of the element-wise gradients' products.
__global__ void __launch_bounds__(256) gradient_kernel(Geo g, const float *__restrict__ ws,
                                                       const float *__restrict__ uh, double wdt,
                                                       double *gl, double *gm) {
  const int64_t mi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (mi >= g.nmat) return;
  const int i = (int)(mi % g.m[0]);
  const int64_t t = mi / g.m[0];
  const int j = (int)(t % g.m[1]);
  const int k = (int)(t / g.m[1]);
  const int I = i + 2 * g.lo[0], J = j + 2 * g.lo[1], K = k + 2 * g.lo[2];
  const int c3[3] = {I, J, K};
  const int64_t node = ((int64_t)K * g.n[1] + J) * g.n[0] + I;
  const int64_t sn[3] = {1, (int64_t)g.n[0], (int64_t)g.n[0] * g.n[1]};
  const int64_t sm[3] = {1, (int64_t)g.m[0], (int64_t)g.m[0] * g.m[1]};
  Axis ax[3] = {axis_info(I, g.n[0], g.lo[0], g.hi[0]), axis_info(J, g.n[1], g.lo[1], g.hi[1]),
                axis_info(K, g.n[2], g.lo[2], g.hi[2])};
  float dw[3][2][3], du[3][2][3];  // [axis][side][component]
  for (int x = 0; x < 3; x++)
    for (int s = 0; s < ax[x].ns; s++) {
      if (!ax[x].rd[s]) continue;
      for (int c = 0; c < 3; c++) {
        dw[x][s][c] = dstc(ws + (int64_t)(9 + c) * g.stride, node, sn[x], ax[x].type[s]) * g.inv_h;
        du[x][s][c] = dstc(uh + (int64_t)c * g.nmat, mi, sm[x], ax[x].type[s]) * g.inv_h;
      }
    }
  float sl = 0.f, smu = 0.f;
  for (int sx = 0; sx < ax[0].ns; sx++)
    for (int sy = 0; sy < ax[1].ns; sy++)
      for (int sz = 0; sz < ax[2].ns; sz++) {
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
  float W = g.wdetj;
  for (int x = 0; x < 3; x++) W *= (c3[x] & 1) ? (4.f / 3.f) : (1.f / 3.f);
  gl[mi] -= wdt * (double)W * (double)sl;
  gm[mi] -= wdt * (double)W * (double)smu;
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

void launch_stage(const Geo &g, const StageArgs &a, bool adjoint, cudaStream_t s) {
  const unsigned nb = blocks_for(g.nnode, 256);
  if (adjoint)
    stage_kernel<true><<<nb, 256, 0, s>>>(g, a);
  else
    stage_kernel<false><<<nb, 256, 0, s>>>(g, a);
}

void launch_point(const PointArgs &p, cudaStream_t s) {
  if (p.npts <= 0) return;
  point_kernel<<<blocks_for(p.npts, 128), 128, 0, s>>>(p);
}

void launch_sample(const float *buf, int64_t stride, int nrec, const int64_t *node, float *traces,
                   cudaStream_t s) {
  if (nrec <= 0) return;
  sample_kernel<<<blocks_for((int64_t)nrec * 3, 256), 256, 0, s>>>(buf, stride, nrec, node, traces);
}

void launch_gradient(const Geo &g, const float *w_state, const float *u_hist, double wdt, double *gl,
                     double *gm, cudaStream_t s) {
  gradient_kernel<<<blocks_for(g.nmat, 256), 256, 0, s>>>(g, w_state, u_hist, wdt, gl, gm);
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

void launch_check_finite(const double *x, int64_t n, int *flag, cudaStream_t s) {
  finite_kernel<<<misfit_blocks(n), kRedThreads, 0, s>>>(x, n, flag);
}

}  // namespace fwi
