// fwi_stage.cu -- fused RK4 stage kernels (sm_103a): rate of the first-order
// system (6) (or of the reversed-time transposed adjoint system) at every node,
// followed by the node's RK4 stage update.
//
// Discretisation (Sec. 2 of arXiv:1504.08340): 27-node hexahedral spectral
// elements with LGL quadrature on a structured box. Quadrature points are the
// nodes, so every element-level quantity at a node is a 3-point stencil along
// each axis, taken inside one of the (at most two) elements along that axis that
// contain the node. A node's side along an axis has one of three types:
//   C (odd coordinate, middle node):     d/dx v = (v[c+1] - v[c-1]) / h
//   L (element below, node is local 2):  d/dx v = (v[c-2] - 4 v[c-1] + 3 v[c]) / h
//   R (element above, node is local 0):  d/dx v = (-3 v[c] + 4 v[c+1] - v[c+2]) / h
// and the quadrature of d phi_a/dx_j along the element line through the node,
// sum_q w_q (2/h) D[q][a] g(x_q) with GLL weights (1/3, 4/3, 1/3), is
//   C: (4 g[c-1] - 4 g[c+1]) / (3h), L: (-g[c-2] + 4 g[c-1] + 3 g[c]) / (3h),
//   R: (-3 g[c] - 4 g[c+1] + g[c+2]) / (3h).
// An element is interior (regular domain) exactly when its index along every axis
// lies in the interior range, so the set of interior elements around a node is a
// product of per-axis side sets and every sum over elements factorises per axis.
//
// Three kernels per stage write disjoint node sets:
//  interior_kernel (fwi_interior.cu): nodes all of whose elements are interior
//    (the bulk of the regular domain): displacement only, K_RD u, no PML terms;
//  pml_kernel (fwi_pml.cu): nodes all of whose elements are PML elements;
//  shell_kernel (here): the nodes in between, shared by interior and PML
//    elements (and the fixed outer faces when there is no PML), with the
//    general per-node formulas below.
// Every output is written once by one thread: no atomics, bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>

#include "fwi_internal.h"

namespace fwi {
namespace {

enum { kC = 0, kL = 1, kR = 2 };

struct Ax {
  int ns;       // elements along this axis containing the node: 1 or 2
  int t0, t1;   // their side types
  bool r0, r1;  // element index along this axis inside the interior range
};

__device__ __forceinline__ Ax make_ax(int c, int n, int lo, int hi) {
  Ax a;
  a.t1 = kR;
  a.r1 = false;
  if (c & 1) {
    const int e = (c - 1) >> 1;
    a.ns = 1;
    a.t0 = kC;
    a.r0 = e >= lo && e < hi;
  } else if (c == 0) {
    a.ns = 1;
    a.t0 = kR;
    a.r0 = 0 >= lo && 0 < hi;
  } else if (c == n - 1) {
    const int e = (c >> 1) - 1;
    a.ns = 1;
    a.t0 = kL;
    a.r0 = e >= lo && e < hi;
  } else {
    const int e = (c >> 1) - 1;
    a.ns = 2;
    a.t0 = kL;
    a.r0 = e >= lo && e < hi;
    a.t1 = kR;
    a.r1 = e + 1 >= lo && e + 1 < hi;
  }
  return a;
}

__device__ __forceinline__ int nrd(const Ax &a) { return (int)a.r0 + (a.ns == 2 ? (int)a.r1 : 0); }

// element-wise derivative (times h) of field f at index i along stride s, side type t
__device__ __forceinline__ float dst(const float *__restrict__ f, int64_t i, int64_t s, int t) {
  if (t == kC) return __ldg(f + i + s) - __ldg(f + i - s);
  if (t == kL) return __ldg(f + i - 2 * s) - 4.f * __ldg(f + i - s) + 3.f * __ldg(f + i);
  return -3.f * __ldg(f + i) + 4.f * __ldg(f + i + s) - __ldg(f + i + 2 * s);
}

// sum over the sides of `a` that are interior elements (all sides when all_sides)
__device__ __forceinline__ float dsum(const float *__restrict__ f, int64_t i, int64_t s, const Ax &a,
                                      bool all_sides) {
  if (a.ns == 2 && (all_sides || (a.r0 && a.r1)))  // L + R in one 4-point stencil
    return __ldg(f + i - 2 * s) - 4.f * __ldg(f + i - s) + 4.f * __ldg(f + i + s) - __ldg(f + i + 2 * s);
  float v = 0.f;
  if (all_sides || a.r0) v += dst(f, i, s, a.t0);
  if (a.ns == 2 && !all_sides && a.r1) v += dst(f, i, s, a.t1);
  return v;
}

// line point p (0..2) of the element on side type t: offset, quadrature coefficient
// (units 1/(3h)) and the side type of the point inside that element
__device__ __forceinline__ int line_off(int t, int p) { return t == kC ? p - 1 : (t == kL ? p - 2 : p); }
__device__ __forceinline__ float line_coef(int t, int p) {
  if (t == kC) return p == 0 ? 4.f : (p == 2 ? -4.f : 0.f);
  if (t == kL) return p == 0 ? -1.f : (p == 1 ? 4.f : 3.f);
  return p == 0 ? -3.f : (p == 1 ? -4.f : 1.f);
}
__device__ __forceinline__ int point_type(int p) { return p == 0 ? kR : (p == 1 ? kC : kL); }

// symmetric component index: xx yy zz yz xz xy
__host__ __device__ constexpr int sym(int i, int j) { return i == j ? i : (i + j == 1 ? 5 : (i + j == 2 ? 4 : 3)); }


// RK4 stage update of one field value with stage-input value yv (see StageArgs;
// in stage 1 X is the stage input)
__device__ __forceinline__ float stage_value(const StageArgs &a, int64_t idx, float yv, float rate) {
  if (a.stage == 0) return rate;
  if (a.stage == 1) return yv + a.cdt * rate;
  if (a.stage < 4) return __ldcs(a.X + idx) + a.cdt * rate;
  return (-__ldcs(a.X + idx) + __ldcs(a.Y2 + idx) + 2.f * __ldcs(a.Y3 + idx) + yv) * (1.f / 3.f) + a.cdt * rate;
}

__device__ __forceinline__ void write_hist(const Geo &g, const StageArgs &a, int I, int J, int K, int c, float v) {
  const int i = I - 2 * g.lo[0], j = J - 2 * g.lo[1], k = K - 2 * g.lo[2];
  if (i >= 0 && i < g.m[0] && j >= 0 && j < g.m[1] && k >= 0 && k < g.m[2])
    a.hist[(int64_t)c * g.nmat + ((int64_t)k * g.m[1] + j) * g.m[0] + i] = v;
}

// Sum over the interior elements around a node of the element-wise stress column
// sigma_{.j} at line point q, for the element on side pt along j: with nk, nl the
// interior side counts along the other axes and S_k = sum over those sides of the
// derivative along k (the set of interior elements is a product of side sets),
//   sum sigma_jj = lam (nk nl d_j u_j + nl S_k u_k + nk S_l u_l) + 2 mu nk nl d_j u_j
//   sum sigma_kj = mu (nk nl d_j u_k + nl S_k u_j),  sum sigma_lj = mu (nk nl d_j u_l + nk S_l u_j)
template <int j>
__device__ __forceinline__ void interior_line_point(const Geo &g, const float *__restrict__ U, int64_t q,
                                                    const int64_t st[3], const int cq[3], int pt, const Ax ax[3],
                                                    float nk, float nl, bool all_sides, float &sj_, float &sk_,
                                                    float &sl_) {
  constexpr int k = (j + 1) % 3, l = (j + 2) % 3;
  const int64_t S = g.stride;
  const float dj_j = dst(U + j * S, q, st[j], pt);
  const float dj_k = dst(U + k * S, q, st[j], pt);
  const float dj_l = dst(U + l * S, q, st[j], pt);
  const float Sk_k = dsum(U + k * S, q, st[k], ax[k], all_sides);
  const float Sk_j = dsum(U + j * S, q, st[k], ax[k], all_sides);
  const float Sl_l = dsum(U + l * S, q, st[l], ax[l], all_sides);
  const float Sl_j = dsum(U + j * S, q, st[l], ax[l], all_sides);
  const float lam = __ldg(g.lam_n + q), mu = __ldg(g.mu_n + q);
  const float n2 = nk * nl;
  sj_ = lam * (n2 * dj_j + nl * Sk_k + nk * Sl_l) + 2.f * mu * n2 * dj_j;
  sk_ = mu * (n2 * dj_k + nl * Sk_j);
  sl_ = mu * (n2 * dj_l + nk * Sl_j);
}

// interior-element force (times 3 h^2 / (W detJ)) at a node, contribution of axis j
template <int j>
__device__ __forceinline__ void interior_force_axis(const Geo &g, const float *__restrict__ U, int64_t node,
                                                    const int c3[3], const int64_t st[3], const Ax ax[3],
                                                    bool all_sides, float f[3]) {
  constexpr int k = (j + 1) % 3, l = (j + 2) % 3;
  const float invw = (c3[j] & 1) ? 0.75f : 3.0f;
  float acc_j = 0.f, acc_k = 0.f, acc_l = 0.f;
#pragma unroll 1
  for (int sj = 0; sj < 2; sj++) {
    if (sj >= ax[j].ns) continue;
    const int t = sj == 0 ? ax[j].t0 : ax[j].t1;
    const bool rdj = sj == 0 ? ax[j].r0 : ax[j].r1;
    if (!all_sides && !rdj) continue;
    const float nk = all_sides ? (float)ax[k].ns : (float)nrd(ax[k]);
    const float nl = all_sides ? (float)ax[l].ns : (float)nrd(ax[l]);
    if (nk == 0.f || nl == 0.f) continue;
#pragma unroll 1
    for (int p = 0; p < 3; p++) {
      const float cf = line_coef(t, p);
      if (cf == 0.f) continue;
      const int off = line_off(t, p);
      int cq[3] = {c3[0], c3[1], c3[2]};
      cq[j] += off;
      float a, b, c;
      interior_line_point<j>(g, U, node + off * st[j], st, cq, point_type(p), ax, nk, nl, all_sides, a, b, c);
      acc_j += cf * a;
      acc_k += cf * b;
      acc_l += cf * c;
    }
  }
  f[j] += invw * acc_j;
  f[k] += invw * acc_k;
  f[l] += invw * acc_l;
}

// PML-element force (times 3h / (W detJ)) at a node, contribution of axis j:
// line quadrature of the j-column of Sdot Le + S Lp + Sbar Lw (forward) or of the
// same with tau(T) = mu (T + diag T) + lambda tr(T) I in place of S (adjoint).
// Lambda_jj does not depend on x_j, so it is the node's value along the whole line.
template <bool ADJ, int j>
__device__ __forceinline__ void pml_force_axis(const Geo &g, const float *__restrict__ Y, int64_t node,
                                               const int c3[3], const int64_t st[3], const Ax ax[3], const float Le[3],
                                               const float Lp[3], const float Lw[3], float f[3]) {
  constexpr int k = (j + 1) % 3, l = (j + 2) % 3;
  const int64_t S = g.stride;
  const float invw = (c3[j] & 1) ? 0.75f : 3.0f;
  const float Lv[3] = {Lw[j], Lp[j], Le[j]};  // history, value, rate levels
  float acc_j = 0.f, acc_k = 0.f, acc_l = 0.f;
#pragma unroll 1
  for (int sj = 0; sj < 2; sj++) {
    if (sj >= ax[j].ns) continue;
    const int t = sj == 0 ? ax[j].t0 : ax[j].t1;
    const bool rdj = sj == 0 ? ax[j].r0 : ax[j].r1;
    const int cpml = ax[k].ns * ax[l].ns - (rdj ? nrd(ax[k]) * nrd(ax[l]) : 0);
    if (cpml == 0) continue;
    float qj = 0.f, qk = 0.f, ql = 0.f;
#pragma unroll 1
    for (int p = 0; p < 3; p++) {
      const float cf = line_coef(t, p);
      if (cf == 0.f) continue;
      const int off = line_off(t, p);
      const int64_t q = node + off * st[j];
      float vj = 0.f, vk = 0.f, vl = 0.f;
      if (!ADJ) {
#pragma unroll
        for (int lv = 0; lv < 3; lv++) {
          const float *b = Y + (int64_t)(9 * lv + 3) * S;
          vj += Lv[lv] * __ldg(b + sym(j, j) * S + q);
          vk += Lv[lv] * __ldg(b + sym(k, j) * S + q);
          vl += Lv[lv] * __ldg(b + sym(l, j) * S + q);
        }
      } else {
        const float lam = __ldg(g.lam_n + q), mu = __ldg(g.mu_n + q);
#pragma unroll
        for (int lv = 0; lv < 3; lv++) {
          const float *b = Y + (int64_t)(9 * lv + 3) * S;
          const float tjj = __ldg(b + j * S + q), tkk = __ldg(b + k * S + q), tll = __ldg(b + l * S + q);
          vj += Lv[lv] * (2.f * mu * tjj + lam * (tjj + tkk + tll));
          vk += Lv[lv] * (mu * __ldg(b + sym(k, j) * S + q));
          vl += Lv[lv] * (mu * __ldg(b + sym(l, j) * S + q));
        }
      }
      qj += cf * vj;
      qk += cf * vk;
      ql += cf * vl;
    }
    const float w = invw * (float)cpml;
    acc_j += w * qj;
    acc_k += w * qk;
    acc_l += w * ql;
  }
  f[j] += acc_j;
  f[k] += acc_k;
  f[l] += acc_l;
}

// S rows: column j of H = sum over PML elements of the element-wise derivatives of
// udot (x Le_jj), u (x Lp_jj) and ubar (x Lw_jj) at the node
template <int j>
__device__ __forceinline__ void pml_strain_axis(const Geo &g, const float *__restrict__ Y, int64_t node,
                                                const int64_t st[3], const Ax ax[3], const float Le[3],
                                                const float Lp[3], const float Lw[3], float H[3][3]) {
  constexpr int k = (j + 1) % 3, l = (j + 2) % 3;
  const int64_t S = g.stride;
  float h0 = 0.f, h1 = 0.f, h2 = 0.f;
#pragma unroll 1
  for (int sj = 0; sj < 2; sj++) {
    if (sj >= ax[j].ns) continue;
    const int t = sj == 0 ? ax[j].t0 : ax[j].t1;
    const bool rdj = sj == 0 ? ax[j].r0 : ax[j].r1;
    const int cpml = ax[k].ns * ax[l].ns - (rdj ? nrd(ax[k]) * nrd(ax[l]) : 0);
    if (cpml == 0) continue;
    const float c = (float)cpml;
    h0 += c * (Le[j] * dst(Y + 18 * S, node, st[j], t) + Lp[j] * dst(Y + 9 * S, node, st[j], t) +
               Lw[j] * dst(Y, node, st[j], t));
    h1 += c * (Le[j] * dst(Y + 19 * S, node, st[j], t) + Lp[j] * dst(Y + 10 * S, node, st[j], t) +
               Lw[j] * dst(Y + S, node, st[j], t));
    h2 += c * (Le[j] * dst(Y + 20 * S, node, st[j], t) + Lp[j] * dst(Y + 11 * S, node, st[j], t) +
               Lw[j] * dst(Y + 2 * S, node, st[j], t));
  }
  H[0][j] = h0;
  H[1][j] = h1;
  H[2][j] = h2;
}

// per-node quantities shared by both phases of shell_kernel
struct NodeCtx {
  int64_t node;
  int c3[3];
  int64_t st[3];
  Ax ax[3];
  bool dir, pml;
  int nel, npml;
  float cb, cc, cd, inv_a, Le[3], Lp[3], Lw[3];
};

__device__ __forceinline__ NodeCtx node_ctx(const Geo &g, int I, int J, int K) {
  NodeCtx n;
  n.node = ((int64_t)K * g.n[1] + J) * g.px + I;
  n.c3[0] = I; n.c3[1] = J; n.c3[2] = K;
  n.st[0] = 1; n.st[1] = g.px; n.st[2] = (int64_t)g.px * g.n[1];
  n.ax[0] = make_ax(I, g.n[0], g.lo[0], g.hi[0]);
  n.ax[1] = make_ax(J, g.n[1], g.lo[1], g.hi[1]);
  n.ax[2] = make_ax(K, g.n[2], g.lo[2], g.hi[2]);
  n.dir = I == 0 || I == g.n[0] - 1 || J == 0 || J == g.n[1] - 1 || K == g.n[2] - 1 || (g.top_dir && K == 0);
  n.nel = n.ax[0].ns * n.ax[1].ns * n.ax[2].ns;
  n.npml = n.nel - nrd(n.ax[0]) * nrd(n.ax[1]) * nrd(n.ax[2]);
  n.pml = n.npml > 0;
  // stretch coefficients at the node (products of eps_x eps_y eps_z)
  const float alx = __ldg(g.alpha[0] + I), aly = __ldg(g.alpha[1] + J), alz = __ldg(g.alpha[2] + K);
  const float bex = __ldg(g.beta[0] + I), bey = __ldg(g.beta[1] + J), bez = __ldg(g.beta[2] + K);
  n.cb = alx * aly * bez + alx * bey * alz + bex * aly * alz;
  n.cc = alx * bey * bez + bex * aly * bez + bex * bey * alz;
  n.cd = bex * bey * bez;
  n.Le[0] = aly * alz; n.Le[1] = alx * alz; n.Le[2] = alx * aly;
  n.Lp[0] = aly * bez + bey * alz; n.Lp[1] = alx * bez + bex * alz; n.Lp[2] = alx * bey + bex * aly;
  n.Lw[0] = bey * bez; n.Lw[1] = bex * bez; n.Lw[2] = bex * bey;
  n.inv_a = __ldg(g.ialpha[0] + I) * __ldg(g.ialpha[1] + J) * __ldg(g.ialpha[2] + K);
  return n;
}

// Interface shell: nodes of the closed interior box [2lo, 2hi] (free top: from
// k = 0) outside the open box of interior_kernel, i.e. the nodes shared by
// interior and PML elements (and, without a PML, the fixed outer faces). Their
// node numbers come from a list built once per context (g.shell, g.nshell).
//
// A block owns 32 list nodes and has three warps. In the first phase warp j forms
// the axis-j terms of every sum at its nodes (the element line quadratures along j
// of the u rows, column j of H of the S rows) and leaves them in shared memory; in
// the second phase warp w writes displacement component w and stress components
// w and w + 3 of the same nodes.
constexpr int kShellNodes = 32;

struct ShellShared {
  float f[3][3][kShellNodes];  // [axis][component][node]: u-row terms s_rd fr + s_pml fp of one axis
  float H[3][3][kShellNodes];  // [i][j][node]
};

template <bool ADJ, int J>
__device__ __forceinline__ void shell_axis(const Geo &g, const StageArgs &a, const NodeCtx &n, ShellShared &sh,
                                           int lane) {
  const float *__restrict__ Y = a.Y;
  const int64_t S = g.stride;
  if (!n.dir) {
    float fr[3] = {0.f, 0.f, 0.f}, fp[3] = {0.f, 0.f, 0.f};
    interior_force_axis<J>(g, Y + 9 * S, n.node, n.c3, n.st, n.ax, false, fr);
    if (n.pml) pml_force_axis<ADJ, J>(g, Y, n.node, n.c3, n.st, n.ax, n.Le, n.Lp, n.Lw, fp);
    const float s_rd = g.inv_h * g.inv_h * (1.f / 3.f), s_pml = g.inv_h * (1.f / 3.f);
#pragma unroll
    for (int c = 0; c < 3; c++) sh.f[J][c][lane] = s_rd * fr[c] + s_pml * fp[c];
  }
  if (n.pml) {
    float H[3][3];
    pml_strain_axis<J>(g, Y, n.node, n.st, n.ax, n.Le, n.Lp, n.Lw, H);
#pragma unroll
    for (int i = 0; i < 3; i++) sh.H[i][J][lane] = H[i][J];
  }
}

// stress component c (order xx yy zz yz xz xy) of the node: its three levels
template <bool ADJ>
__device__ __forceinline__ void shell_stress(const Geo &g, const StageArgs &a, const NodeCtx &n,
                                             const ShellShared &sh, int lane, int c) {
  const int64_t S = g.stride;
  const float *__restrict__ Y = a.Y;
  const int64_t i0 = (int64_t)(3 + c) * S + n.node, i1 = (int64_t)(12 + c) * S + n.node,
                i2 = (int64_t)(21 + c) * S + n.node;
  if (!n.pml) {
    if (a.stage == 0) {
      __stcs(a.out + i0, 0.f);
      __stcs(a.out + i1, 0.f);
      __stcs(a.out + i2, 0.f);
    }
    return;
  }
  const float sc = g.inv_h / (float)n.npml;
  // P(H): diagonal H_ii, off-diagonal H_ij + H_ji
  auto P = [&](int k) {
    if (k < 3) return sc * sh.H[k][k][lane];
    const int i = k == 5 ? 0 : (k == 4 ? 0 : 1), j = k == 5 ? 1 : 2;  // xy, xz, yz
    return sc * (sh.H[i][j][lane] + sh.H[j][i][lane]);
  };
  float src = P(c);
  if (!ADJ) {  // tau(P(H)) = mu (P + diag P) + lambda tr(P) I
    const float lam = __ldg(g.lam_n + n.node), mu = __ldg(g.mu_n + n.node);
    src = c < 3 ? 2.f * mu * src + lam * (P(0) + P(1) + P(2)) : mu * src;
  }
  const float s0 = __ldg(Y + i0), s1 = __ldg(Y + i1), s2 = __ldg(Y + i2);
  __stcs(a.out + i0, stage_value(a, i0, s0, s1));
  __stcs(a.out + i1, stage_value(a, i1, s1, s2));
  __stcs(a.out + i2, stage_value(a, i2, s2, (src - n.cb * s2 - n.cc * s1 - n.cd * s0) * n.inv_a));
}

// displacement component c of the node: its three levels
__device__ __forceinline__ void shell_disp(const Geo &g, const StageArgs &a, const NodeCtx &n, const ShellShared &sh,
                                           int lane, int c) {
  const int64_t S = g.stride;
  const float *__restrict__ Y = a.Y;
  const int64_t i0 = (int64_t)c * S + n.node, i1 = (int64_t)(9 + c) * S + n.node, i2 = (int64_t)(18 + c) * S + n.node;
  if (n.dir) {
    if (a.stage == 0) {
      __stcs(a.out + i0, 0.f);
      __stcs(a.out + i1, 0.f);
      __stcs(a.out + i2, 0.f);
    }
    return;
  }
  const float fsum = sh.f[0][c][lane] + sh.f[1][c][lane] + sh.f[2][c][lane];
  const float inv_m = n.inv_a / (g.rho * (float)n.nel);
  const float u0 = __ldg(Y + i0), u1 = __ldg(Y + i1), u2 = __ldg(Y + i2);
  const float acc = -fsum * inv_m - (n.cb * u2 + n.cc * u1 + n.cd * u0) * n.inv_a;
  if (n.pml || a.stage == 0) __stcs(a.out + i0, stage_value(a, i0, u0, n.pml ? u1 : 0.f));
  const float v1 = stage_value(a, i1, u1, u2);
  __stcs(a.out + i1, v1);
  __stcs(a.out + i2, stage_value(a, i2, u2, acc));
  if (a.hist) write_hist(g, a, n.c3[0], n.c3[1], n.c3[2], c, v1);
}

#ifndef FWI_SHELL_MINB
#define FWI_SHELL_MINB 8
#endif
template <bool ADJ>
__global__ void __launch_bounds__(3 * kShellNodes, FWI_SHELL_MINB) shell_kernel(Geo g, StageArgs a0) {
  __shared__ ShellShared sh;
  const int nbs = (g.nshell + kShellNodes - 1) / kShellNodes;  // blocks per shot
  const StageArgs a = shot_args(a0, blockIdx.x / nbs);
  const int lane = threadIdx.x, w = threadIdx.y;
  const int i = (blockIdx.x % nbs) * kShellNodes + lane;
  const bool live = i < g.nshell && node_ok(g, kSiteShell, g.shell[i]);
  NodeCtx n;
  if (live) {
    const int node = g.shell[i];
    const int I = node % g.px, r = node / g.px;
    n = node_ctx(g, I, r % g.n[1], r / g.n[1]);
    if (w == 0) shell_axis<ADJ, 0>(g, a, n, sh, lane);
    else if (w == 1) shell_axis<ADJ, 1>(g, a, n, sh, lane);
    else shell_axis<ADJ, 2>(g, a, n, sh, lane);
  }
  __syncthreads();
  if (live) {
    shell_disp(g, a, n, sh, lane, w);
    shell_stress<ADJ>(g, a, n, sh, lane, w);
    shell_stress<ADJ>(g, a, n, sh, lane, w + 3);
  }
}

// ---- persistent forward sweep (see PersistArgs)

// grid-wide barrier on a global arrival count and generation; the spin gives up after
// wait_cycles and records FWI_E_TIMEOUT. False when this or an earlier barrier gave up.
__device__ bool grid_barrier(const PersistArgs &p, unsigned expected) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int ok = 1;
    volatile unsigned *gen = p.bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(p.bar, 1u) + 1u == expected) {
      atomicExch(p.bar, 0u);
      __threadfence();
      atomicAdd(p.bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g0) {
        if (clock64() - t0 > p.wait_cycles) {
          atomicExch(p.status, 6);  // FWI_E_TIMEOUT
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int *)p.status != 0) ok = 0;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// displacement component c of a node for the persistent sweep: shell_disp, plus the
// source load of the shot (forward point load, as point_kernel adds it) and the receiver
// sample after the last stage
__device__ __forceinline__ void persist_disp(const Geo &g, const StageArgs &a, const NodeCtx &n,
                                             const ShellShared &sh, int lane, int c, const PersistArgs &p, int b,
                                             int step, int stage) {
  const int64_t S = g.stride;
  const float *__restrict__ Y = a.Y;
  const int64_t i0 = (int64_t)c * S + n.node, i1 = (int64_t)(9 + c) * S + n.node, i2 = (int64_t)(18 + c) * S + n.node;
  if (n.dir) return;
  const float fsum = sh.f[0][c][lane] + sh.f[1][c][lane] + sh.f[2][c][lane];
  const float inv_m = n.inv_a / (g.rho * (float)n.nel);
  const float u0 = __ldg(Y + i0), u1 = __ldg(Y + i1), u2 = __ldg(Y + i2);
  const float acc = -fsum * inv_m - (n.cb * u2 + n.cc * u1 + n.cd * u0) * n.inv_a;
  if (n.pml) __stcs(a.out + i0, stage_value(a, i0, u0, u1));
  const float v1 = stage_value(a, i1, u1, u2);
  __stcs(a.out + i1, v1);
  float v2 = stage_value(a, i2, u2, acc);
  if (n.node == p.src_node[b]) {
    // stage times t_n, t_n + dt/2, t_n + dt/2, t_n + dt: samples 2n, 2n+1, 2n+1, 2n+2
    const float amp = p.wave[stage == 0 ? 2 * step : (stage == 3 ? 2 * step + 2 : 2 * step + 1)];
    v2 += a.cdt * amp * p.src_vec[3 * b + c];
  }
  __stcs(a.out + i2, v2);
  if (a.hist) write_hist(g, a, n.c3[0], n.c3[1], n.c3[2], c, v1);
  if (stage == 3) {
    const int r = p.rec_of[n.node];
    if (r >= 0 && guard(g.oob, kSitePersist, r, p.nrec)) p.traces[(int64_t)b * p.tstride + ((int64_t)(step + 1) * p.nrec + r) * 3 + c] = v1;
  }
}

__global__ void __launch_bounds__(3 * kShellNodes) persistent_forward_kernel(Geo g, PersistArgs p) {
  __shared__ ShellShared sh;
  const int lane = threadIdx.x, w = threadIdx.y;
  const int nch = (p.nall + kShellNodes - 1) / kShellNodes;  // node chunks per shot
  const unsigned expected = gridDim.x + (unsigned)p.extra;
  const float cdts[4] = {0.5f * p.dt, 0.5f * p.dt, p.dt, p.dt / 6.0f};
  for (int step = p.n0; step < p.n1; step++) {
    for (int s = 0; s < 4; s++) {
      StageArgs a0{};
      a0.Y = p.st[s];
      a0.X = p.st[0];
      a0.Y2 = p.st[1];
      a0.Y3 = p.st[2];
      a0.out = p.st[(s + 1) % 4];
      a0.cdt = cdts[s];
      a0.stage = s + 1;
      a0.hist = (s == 3 && p.hist) ? p.hist + (int64_t)(step + 1) * p.hstep : nullptr;
      a0.nshot = p.nshot;
      a0.sstride = p.sstride;
      a0.hstride = p.hstride;
      for (int ch = blockIdx.x; ch < nch * p.nshot; ch += gridDim.x) {
        const int b = ch / nch;
        const StageArgs a = shot_args(a0, b);
        const int i = (ch % nch) * kShellNodes + lane;
        const bool live = i < p.nall && node_ok(g, kSitePersist, p.nodes[i]);
        NodeCtx n;
        if (live) {
          const int node = p.nodes[i];
          const int I = node % g.px, r = node / g.px;
          n = node_ctx(g, I, r % g.n[1], r / g.n[1]);
          if (w == 0) shell_axis<false, 0>(g, a, n, sh, lane);
          else if (w == 1) shell_axis<false, 1>(g, a, n, sh, lane);
          else shell_axis<false, 2>(g, a, n, sh, lane);
        }
        __syncthreads();
        if (live) {
          persist_disp(g, a, n, sh, lane, w, p, b, step, s);
          shell_stress<false>(g, a, n, sh, lane, w);
          shell_stress<false>(g, a, n, sh, lane, w + 3);
        }
        __syncthreads();
      }
      if (!grid_barrier(p, expected)) return;
    }
  }
}

}  // namespace

cudaError_t launch_persistent_forward(const Geo &g, const PersistArgs &p, cudaStream_t s) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_forward_kernel, 3 * kShellNodes, 0);
  if (e != cudaSuccess) return e;
  const int chunks = (p.nall + kShellNodes - 1) / kShellNodes * p.nshot;
  const int grid = std::max(1, std::min(per_sm * nsm, chunks));
  Geo gg = g;
  PersistArgs pp = p;
  void *args[2] = {&gg, &pp};
  return cudaLaunchCooperativeKernel((const void *)persistent_forward_kernel, dim3(grid), dim3(kShellNodes, 3), args,
                                     0, s);
}

int launch_shell(const Geo &g, const StageArgs &a, bool adjoint, cudaStream_t s) {
  int n = 0;
  if (g.nshell > 0) {
    n = 1;
    const int nb = (g.nshell + kShellNodes - 1) / kShellNodes * a.nshot;
    const dim3 blk(kShellNodes, 3);
    if (adjoint)
      shell_kernel<true><<<nb, blk, 0, s>>>(g, a);
    else
      shell_kernel<false><<<nb, blk, 0, s>>>(g, a);
  }
  return n + launch_pml_face(g, a, adjoint, s);
}

}  // namespace fwi
