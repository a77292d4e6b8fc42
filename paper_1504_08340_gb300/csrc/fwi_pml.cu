// fwi_pml.cu -- RK4 stage kernel for the nodes all of whose elements are PML
// elements ("deep" PML nodes: the bulk of the PML buffer of Fig. 3).
//
// At such a node every element-level sum of (3a)/(3b) (Sec. 2 of
// arXiv:1504.08340) runs over all ns_x ns_y ns_z elements around the node, and
// with the lumped masses it collapses to symmetric one-dimensional stencils:
//  - S rows: the element-summed derivative divided by the element count is the
//    average over the sides along j of the one-sided derivatives,
//      D_j v = (v[c+1] - v[c-1]) / h                           (c odd)
//      D_j v = (v[c-2] - 4 v[c-1] + 4 v[c+1] - v[c+2]) / (2h)    (c even, two sides)
//      one-sided (-3 v0 + 4 v1 - v2)/h or (v-2 - 4 v-1 + 3 v0)/h on the outer faces;
//    H_ij = Le_jj D_j udot_i + Lp_jj D_j u_i + Lw_jj D_j ubar_i and
//    S'' = (tau(P(H)) - b S' - c S - d Sbar) / a   (adjoint: P(H) in place of tau(P(H)))
//  - u rows: (1/w_j) times the line quadrature of d phi_a/dx_j divided by the
//    element count is exactly -D_j, except on the free top face where the one-sided
//    quadrature (-3 g0 - 4 g1 + g2)/h keeps its centre term (the traction-free
//    boundary of (2b)); so
//      u'' = (sum_j D_j Q_ij) / (rho a) - (b u' + c u + d ubar) / a,
//      Q_ij = Le_jj Sdot_ij + Lp_jj S_ij + Lw_jj Sbar_ij  (adjoint: tau(T) in place of S).
// Lambda_jj does not depend on x_j, so it is the node's value along the j-line.
//
// Threads own node pairs (even x, odd x) of row segments of the PML region
// (outside the closed interior box), with 32-bit field offsets.
#include <cuda_runtime.h>

#include <type_traits>

#include "fwi_internal.h"

namespace fwi {
namespace {

enum { kSC = 0, kSLR = 1, kSR = 2, kSL = 3 };  // odd, even (both sides), first node, last node

__device__ __forceinline__ int side_kind(int c, int n) {
  return (c & 1) ? kSC : (c == 0 ? kSR : (c == n - 1 ? kSL : kSLR));
}

// averaged element-wise derivative (times h) of f at offset o, axis stride s
__device__ __forceinline__ float dav(const float *__restrict__ f, int o, int s, int kind) {
  switch (kind) {
    case kSC: return __ldg(f + o + s) - __ldg(f + o - s);
    case kSLR: return 0.5f * (__ldg(f + o - 2 * s) - 4.f * __ldg(f + o - s) + 4.f * __ldg(f + o + s) - __ldg(f + o + 2 * s));
    case kSR: return -3.f * __ldg(f + o) + 4.f * __ldg(f + o + s) - __ldg(f + o + 2 * s);
    default: return __ldg(f + o - 2 * s) - 4.f * __ldg(f + o - s) + 3.f * __ldg(f + o);
  }
}

// divergence part of the u rows (times h): +D_j for interior kinds; the free top face
// (first node along z, one element) keeps the full one-sided quadrature.
__device__ __forceinline__ float ddiv(float g_m2, float g_m1, float g0, float g_p1, float g_p2, int kind) {
  if (kind == kSC) return g_p1 - g_m1;
  if (kind == kSLR) return 0.5f * (g_m2 - 4.f * g_m1 + 4.f * g_p1 - g_p2);
  return 3.f * g0 + 4.f * g_p1 - g_p2;  // kSR on the free surface: -(-3 g0 - 4 g1 + g2)
}

__host__ __device__ constexpr int sym(int i, int j) { return i == j ? i : (i + j == 1 ? 5 : (i + j == 2 ? 4 : 3)); }

// PML boxes and their warp tasks. The node pairs of a box row are cut into nseg
// x segments of at most `per` <= 32 pairs. A warp task is one segment of R rows of
// one plane with equal y parity (J0, J0 + 2, ..., J0 + 2(R-1)): R = 32 / per for
// narrow boxes, else 1. The side kinds along y and z are then uniform across the
// warp. Tasks run segment by segment, so the warps resident at one time cover one
// x segment of many rows and planes, and the rows that their y and z stencils
// share stay in L2.
struct Region {
  int nbox;
  int lo[6][3], hi[6][3];  // inclusive node boxes
  int P[6], R[6];          // node pairs per row, rows per warp task
  int nseg[6], per[6];     // x segments per row, pairs per segment (the last may have fewer)
  int jfirst[6][2], nj[6][2], groups[6][2];  // per y-parity class: first J, row count, warp groups per plane
  int tasks_before[7];     // prefix sums of warp tasks per box
};

__device__ __forceinline__ float stage_value(const StageArgs &a, int idx, float yv, float rate) {
  if (a.stage == 0) return rate;
  if (a.stage == 1) return yv + a.cdt * rate;  // X is the stage input
  if (a.stage < 4) return __ldcs(a.X + idx) + a.cdt * rate;
  return (-__ldcs(a.X + idx) + __ldcs(a.Y2 + idx) + 2.f * __ldcs(a.Y3 + idx) + yv) * (1.f / 3.f) + a.cdt * rate;
}


// ---------------------------------------------------------------------------
// Vectorised pair path: a thread owns the nodes (I0, I0 + 1), I0 even, of a bulk
// row. Rows are padded to a multiple of 4 nodes, so every (I0, I0 + 1) pair is
// 8-byte aligned: all loads and stores are float2 and fully coalesced, and the
// arithmetic of the two nodes runs as packed f32x2 instructions (.x: the even
// node, .y: the odd node). x-window of a field: values at I0-2 .. I0+3; the even
// node's x kind is LR, the odd node's C.
__device__ __forceinline__ float2 ld2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ float2 ldcs2(const float *p) { return __ldcs(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ void st2(float *p, float2 v, bool even_ok) {
  if (even_ok)
    __stcs(reinterpret_cast<float2 *>(p), v);
  else
    __stcs(p + 1, v.y);
}

// packed two-lane FP32 arithmetic, round to nearest even (each lane as the scalar op)
#define FWI_PACKED_BINARY(name, op)                                                                   \
  __device__ __forceinline__ float2 name(float2 a, float2 b) {                                        \
    float2 d;                                                                                         \
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t" op        \
        ".rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"                                          \
        : "=f"(d.x), "=f"(d.y)                                                                        \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                                    \
    return d;                                                                                         \
  }
FWI_PACKED_BINARY(padd, "add")
FWI_PACKED_BINARY(psub, "sub")
FWI_PACKED_BINARY(pmul, "mul")
#undef FWI_PACKED_BINARY
// a * b + c, one rounding per lane
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 bc(float s) { return make_float2(s, s); }

struct XWin {
  float v[6];
};
__device__ __forceinline__ XWin xwin(const float *p) {
  const float2 a = ld2(p - 2), b = ld2(p), c = ld2(p + 2);
  XWin w;
  w.v[0] = a.x; w.v[1] = a.y; w.v[2] = b.x; w.v[3] = b.y; w.v[4] = c.x; w.v[5] = c.y;
  return w;
}
// D_x (times h) of the even (LR) and the odd (C) node
__device__ __forceinline__ float2 dx2(const XWin &w) {
  return make_float2(0.5f * (w.v[0] - w.v[4]) + 2.f * (w.v[3] - w.v[1]), w.v[4] - w.v[2]);
}

// derivative (times h) along y or z (stride s) of a field for both nodes:
// C: v[+1] - v[-1]; LR: 2 (v[+1] - v[-1]) + 0.5 (v[-2] - v[+2])
template <int KD>
__device__ __forceinline__ float2 dline(const float *p, int s) {
  const float2 m1 = ld2(p - s), p1 = ld2(p + s);
  if constexpr (KD == kSC) {
    return psub(p1, m1);
  } else {
    const float2 m2 = ld2(p - 2 * s), p2 = ld2(p + 2 * s);
    return pfma(bc(2.f), psub(p1, m1), pmul(bc(0.5f), psub(m2, p2)));
  }
}

// stretch coefficients of a pair. Level order lv = 0, 1, 2: Lambda^w, Lambda^p, Lambda^e.
// Lambda_xx does not depend on x, so it is one value for both nodes.
struct Coef2 {
  float2 ia, nb, nc, nd;  // 1/a and -b, -c, -d
  float Lx[3];
  float2 Ly[3], Lz[3];
};
__device__ __forceinline__ Coef2 coef_pair(const Geo &g, int I0, int J, int K) {
  const float2 alx = ld2(g.alpha[0] + I0), bex = ld2(g.beta[0] + I0), iax = ld2(g.ialpha[0] + I0);
  const float aly = __ldg(g.alpha[1] + J), alz = __ldg(g.alpha[2] + K);
  const float bey = __ldg(g.beta[1] + J), bez = __ldg(g.beta[2] + K);
  const float eyz = aly * alz, pyz = aly * bez + bey * alz, wyz = bey * bez;
  Coef2 c;
  c.ia = pmul(iax, bc(__ldg(g.ialpha[1] + J) * __ldg(g.ialpha[2] + K)));
  // a = ax ay az, b = ax (ay bz + by az) + bx ay az, c = ax by bz + bx (ay bz + by az), d = bx by bz
  c.nb = pfma(alx, bc(-pyz), pmul(bex, bc(-eyz)));
  c.nc = pfma(alx, bc(-wyz), pmul(bex, bc(-pyz)));
  c.nd = pmul(bex, bc(-wyz));
  c.Lx[0] = wyz; c.Lx[1] = pyz; c.Lx[2] = eyz;
  c.Ly[0] = pmul(bex, bc(bez)); c.Ly[1] = pfma(alx, bc(bez), pmul(bex, bc(alz))); c.Ly[2] = pmul(alx, bc(alz));
  c.Lz[0] = pmul(bex, bc(bey)); c.Lz[1] = pfma(alx, bc(bey), pmul(bex, bc(aly))); c.Lz[2] = pmul(alx, bc(aly));
  return c;
}

// stage output of a node pair from its own input value y and rate r; MODE 0: the
// rate, 1: stage 1 (X is the stage input, so x = y), 2: stages 2-3, 3: stage 4
template <int MODE>
__device__ __forceinline__ float2 stage2(const StageArgs &a, int idx, float2 y, float2 r) {
  if constexpr (MODE == 0) return r;
  if constexpr (MODE == 1) return pfma(bc(a.cdt), r, y);
  const float2 x = ldcs2(a.X + idx);
  if constexpr (MODE == 2) return pfma(bc(a.cdt), r, x);
  const float2 b = ldcs2(a.Y2 + idx), c = ldcs2(a.Y3 + idx);
  return pfma(bc(1.f / 3.f), padd(pfma(bc(2.f), c, psub(b, x)), y), pmul(bc(a.cdt), r));
}

// adjoint: column j of sum_lv Lambda^lv_jj tau(T^lv) at the nodes (I0, J, K) and
// (I0 + 1, J, K), whose Lambda_jj are Lj (levels 0..2), T read at offset o from the pair
template <int JAX>
__device__ __forceinline__ void tau_col2(const Geo &g, const float *__restrict__ Y, int S, int o, int node,
                                         const float2 Lj[3], float2 q[3]) {
  constexpr int KAX = (JAX + 1) % 3, LAX = (JAX + 2) % 3;
  const float2 lq = ld2(g.lam_n + node + o), muq = ld2(g.mu_n + node + o);
  const float2 mu2 = padd(muq, muq);
  q[0] = q[1] = q[2] = bc(0.f);
#pragma unroll
  for (int lv = 0; lv < 3; lv++) {
    const float *b = Y + (9 * lv + 3) * S + o;
    const float2 tjj = ld2(b + JAX * S), tkk = ld2(b + KAX * S), tll = ld2(b + LAX * S);
    const float2 vj = pfma(mu2, tjj, pmul(lq, padd(padd(tjj, tkk), tll)));
    q[0] = pfma(Lj[lv], vj, q[0]);
    q[1] = pfma(Lj[lv], pmul(muq, ld2(b + sym(KAX, JAX) * S)), q[1]);
    q[2] = pfma(Lj[lv], pmul(muq, ld2(b + sym(LAX, JAX) * S)), q[2]);
  }
}

// adjoint: y- and z-line contributions sum_j D_j Q_cj of a pair, as weighted sums over
// the line points (C: q[+1] - q[-1]; LR: 0.5 (q[-2] - 4 q[-1] + 4 q[+1] - q[+2]))
template <int KY, int KZ>
__device__ __forceinline__ void adj_yz(const Geo &g, const float *__restrict__ Yn, int S, int sy, int sz, int node,
                                       const Coef2 &cf, float2 f[3]) {
#pragma unroll 1
  for (int d = -2; d <= 2; d++) {
    if (d == 0 || (KY == kSC && (d == -2 || d == 2))) continue;
    const float2 w = bc(KY == kSC ? (float)d : (d == -2 ? 0.5f : (d == -1 ? -2.f : (d == 1 ? 2.f : -0.5f))));
    float2 q[3];
    tau_col2<1>(g, Yn, S, d * sy, node, cf.Ly, q);  // (yy, zy, xy) column
    f[1] = pfma(w, q[0], f[1]); f[2] = pfma(w, q[1], f[2]); f[0] = pfma(w, q[2], f[0]);
  }
#pragma unroll 1
  for (int d = -2; d <= 2; d++) {
    if (d == 0 || (KZ == kSC && (d == -2 || d == 2))) continue;
    const float2 w = bc(KZ == kSC ? (float)d : (d == -2 ? 0.5f : (d == -1 ? -2.f : (d == 1 ? 2.f : -0.5f))));
    float2 q[3];
    tau_col2<2>(g, Yn, S, d * sz, node, cf.Lz, q);  // (zz, xz, yz) column
    f[2] = pfma(w, q[0], f[2]); f[0] = pfma(w, q[1], f[0]); f[1] = pfma(w, q[2], f[1]);
  }
}

// PART 0: the whole pair update; 1: the stress rows only; 2: the displacement rows only
template <bool ADJ, int MODE, int KY, int KZ, int PART = 0>
__device__ void pml_pair(const Geo &g, const StageArgs &a, int I0, int J, int K, bool even_ok) {
  constexpr bool DO_S = PART != 2, DO_U = PART != 1;
  const int S = (int)g.stride;
  const int node = (K * g.n[1] + J) * g.px + I0;
  const int sy = g.px, sz = g.px * g.n[1];
  const float *__restrict__ Yn = a.Y + node;
  const Coef2 cf = coef_pair(g, I0, J, K);
  float2 f[3] = {bc(0.f), bc(0.f), bc(0.f)};  // u-row sums (times h)
  if constexpr (ADJ && DO_U) {
    // Q = sum_lv Lambda^lv_jj tau(T^lv): pointwise with the material of each line point.
    // x: Q at the points I0-2 .. I0+3 as three aligned pairs (the last point is not
    // used); even node (LR): 0.5 Q[-2] - 2 Q[-1] + 2 Q[+1] - 0.5 Q[+2], odd node (C,
    // at I0+1): Q[+2] - Q[0]
    {
      const float2 Lx[3] = {bc(cf.Lx[0]), bc(cf.Lx[1]), bc(cf.Lx[2])};
      float2 qm[3], q0[3], qp[3];  // pairs (I0-2, I0-1), (I0, I0+1), (I0+2, I0+3)
      tau_col2<0>(g, Yn, S, -2, node, Lx, qm);
      tau_col2<0>(g, Yn, S, 0, node, Lx, q0);
      tau_col2<0>(g, Yn, S, 2, node, Lx, qp);
#pragma unroll
      for (int c = 0; c < 3; c++) {  // q[0], q[1], q[2]: the xx, yx, zx entries -> components x, y, z
        const float e = 0.5f * (qm[c].x - qp[c].x) + 2.f * (q0[c].y - qm[c].y);
        const float o = qp[c].x - q0[c].x;
        f[c] = padd(f[c], make_float2(e, o));
      }
    }
    adj_yz<KY, KZ>(g, Yn, S, sy, sz, node, cf, f);
  }
  // ---- S rows: H_ij = sum_lv Lambda^lv_jj D_j u^lv_i (times h)
  float2 s[6];
  if constexpr (DO_S) {
    float2 H[3][3];  // [i][j]
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++) H[i][j] = bc(0.f);
#pragma unroll
    for (int lv = 0; lv < 3; lv++)
#pragma unroll
      for (int i = 0; i < 3; i++) {
        const float *p = Yn + (9 * lv + i) * S;
        const float2 dx = dx2(xwin(p));
        const float2 dy = dline<KY>(p, sy), dz = dline<KZ>(p, sz);
        H[i][0] = pfma(bc(cf.Lx[lv]), dx, H[i][0]);
        H[i][1] = pfma(cf.Ly[lv], dy, H[i][1]);
        H[i][2] = pfma(cf.Lz[lv], dz, H[i][2]);
      }
    s[0] = H[0][0]; s[1] = H[1][1]; s[2] = H[2][2];
    s[3] = padd(H[1][2], H[2][1]); s[4] = padd(H[0][2], H[2][0]); s[5] = padd(H[0][1], H[1][0]);
  }
  if constexpr (!ADJ && DO_S) {  // tau(P(H)) with the node's own material
    const float2 lm = ld2(g.lam_n + node), mu = ld2(g.mu_n + node);
    const float2 mu2 = padd(mu, mu);
    const float2 ltr = pmul(lm, padd(padd(s[0], s[1]), s[2]));
#pragma unroll
    for (int c = 0; c < 3; c++) s[c] = pfma(mu2, s[c], ltr);
#pragma unroll
    for (int c = 3; c < 6; c++) s[c] = pmul(mu, s[c]);
  }

  // ---- u rows (times h): f_c = sum_j D_j Q_cj; forward Q = sum_lv Lambda^lv_jj S^lv
  const float2 ih = bc(g.inv_h);
  // S components in the order xx yy zz yz xz xy; for each: (c, j) pairs it feeds
  constexpr bool PHASE_B = DO_S || !ADJ;  // the adjoint u rows need nothing from this loop
#pragma unroll
  for (int comp = 0; comp < (PHASE_B ? 6 : 0); comp++) {
    float2 sv[3];  // own values per level
#pragma unroll
    for (int lv = 0; lv < 3; lv++) {
      const float *p = Yn + (9 * lv + 3 + comp) * S;
      const bool on_x = comp == 0 || comp == 4 || comp == 5;  // xx, xz, xy
      const bool on_y = comp == 1 || comp == 3 || comp == 5;  // yy, yz, xy
      const bool on_z = comp == 2 || comp == 3 || comp == 4;  // zz, yz, xz
      if (on_x && !ADJ && DO_U) {
        const XWin w = xwin(p);
        sv[lv] = make_float2(w.v[2], w.v[3]);
        const int c = comp == 0 ? 0 : (comp == 5 ? 1 : 2);  // xx -> c 0, xy -> c 1, xz -> c 2 (j = x)
        f[c] = pfma(bc(cf.Lx[lv]), dx2(w), f[c]);
      } else if (DO_S) {
        sv[lv] = ld2(p);
      }
      if constexpr (!ADJ && DO_U) {
        if (on_y) {
          const int c = comp == 1 ? 1 : (comp == 5 ? 0 : 2);  // yy -> 1, xy -> 0, yz -> 2 (j = y)
          f[c] = pfma(cf.Ly[lv], dline<KY>(p, sy), f[c]);
        }
        if (on_z) {
          const int c = comp == 2 ? 2 : (comp == 4 ? 0 : 1);  // zz -> 2, xz -> 0, yz -> 1 (j = z)
          f[c] = pfma(cf.Lz[lv], dline<KZ>(p, sz), f[c]);
        }
      }
    }
    if constexpr (!DO_S) continue;
    // stress update of this component: S'' = (src - b S' - c S - d Sbar) / a
    const int i0 = (3 + comp) * S + node, i1 = (12 + comp) * S + node, i2 = (21 + comp) * S + node;
    const float2 acc = pmul(pfma(cf.nb, sv[2], pfma(cf.nc, sv[1], pfma(cf.nd, sv[0], pmul(s[comp], ih)))), cf.ia);
    st2(a.out + i0, stage2<MODE>(a, i0, sv[0], sv[1]), even_ok);
    st2(a.out + i1, stage2<MODE>(a, i1, sv[1], sv[2]), even_ok);
    st2(a.out + i2, stage2<MODE>(a, i2, sv[2], acc), even_ok);
  }
  // ---- displacement update: u'' = (f / h) / (rho a) - (b u' + c u + d ubar) / a
  // (own u values read again here rather than held since the S rows)
  if constexpr (!DO_U) return;
  const float2 irh = bc(g.inv_rho_h);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const int i0 = c * S + node, i1 = (9 + c) * S + node, i2 = (18 + c) * S + node;
    const float2 u0 = ld2(Yn + c * S), u1 = ld2(Yn + (9 + c) * S), u2 = ld2(Yn + (18 + c) * S);
    const float2 acc = pmul(pfma(cf.nb, u2, pfma(cf.nc, u1, pfma(cf.nd, u0, pmul(irh, f[c])))), cf.ia);
    st2(a.out + i0, stage2<MODE>(a, i0, u0, u1), even_ok);
    st2(a.out + i1, stage2<MODE>(a, i1, u1, u2), even_ok);
    st2(a.out + i2, stage2<MODE>(a, i2, u2, acc), even_ok);
  }
}

// ---------------------------------------------------------------------------
// PML nodes on the outer faces of the grid (fixed faces, and the free top face
// outside the interior), from a list built once per context, with the general
// side kinds (one-sided on the faces). A block owns 32 list nodes and has three
// warps: warp j first forms the axis-j terms (the u-row divergence along j and
// column j of H) into shared memory, then warp w writes displacement component w
// and stress components w and w + 3.
constexpr int kFaceNodes = 32;

struct FaceCtx {
  int node, st[3], kind[3];
  bool dir;
  bool flat[3];  // the line along this axis through the node lies in a fixed face
  float cb, cc, cd, inv_a, Le[3], Lp[3], Lw[3];
};

struct FaceShared {
  float f[3][3][kFaceNodes];  // [axis][component][node]: u-row divergence terms (times h)
  float H[3][3][kFaceNodes];  // [i][j][node] (times 1)
};

__device__ __forceinline__ FaceCtx face_ctx(const Geo &g, int I, int J, int K) {
  FaceCtx n;
  n.node = (K * g.n[1] + J) * g.px + I;
  n.st[0] = 1; n.st[1] = g.px; n.st[2] = g.px * g.n[1];
  n.kind[0] = side_kind(I, g.n[0]); n.kind[1] = side_kind(J, g.n[1]); n.kind[2] = side_kind(K, g.n[2]);
  const bool fx = I == 0 || I == g.n[0] - 1, fy = J == 0 || J == g.n[1] - 1,
             fz = K == g.n[2] - 1 || (g.top_dir && K == 0);
  n.dir = fx || fy || fz;
  n.flat[0] = fy || fz;
  n.flat[1] = fx || fz;
  n.flat[2] = fx || fy;
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

template <bool ADJ, int JA>
__device__ __forceinline__ void face_axis(const Geo &g, const StageArgs &a, const FaceCtx &n, int I, int J, int K,
                                          FaceShared &sh, int lane) {
  constexpr int KA = (JA + 1) % 3, LA = (JA + 2) % 3;
  const int S = (int)g.stride;
  const float *__restrict__ Y = a.Y;
  const int kd = n.kind[JA], s = n.st[JA];
  if (!n.dir) {
    // Q column JA at offsets -2..2 along JA (only the ones the kind uses)
    const float Lv[3] = {n.Lw[JA], n.Lp[JA], n.Le[JA]};
    float q[3][5];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int d = 0; d < 5; d++) q[c][d] = 0.f;
#pragma unroll
    for (int d = 0; d < 5; d++) {
      const int off = d - 2;
      const bool used = kd == kSC ? (off == -1 || off == 1) : (kd == kSLR ? off != 0 : off >= 0);
      if (!used) continue;
      const int o = n.node + off * s;
      float vj = 0.f, vk = 0.f, vl = 0.f;
      if (!ADJ) {
#pragma unroll
        for (int lv = 0; lv < 3; lv++) {
          const float *b = Y + (9 * lv + 3) * S;
          vj += Lv[lv] * __ldg(b + sym(JA, JA) * S + o);
          vk += Lv[lv] * __ldg(b + sym(KA, JA) * S + o);
          vl += Lv[lv] * __ldg(b + sym(LA, JA) * S + o);
        }
      } else {
        const float lq = __ldg(g.lam_n + o), muq = __ldg(g.mu_n + o);
#pragma unroll
        for (int lv = 0; lv < 3; lv++) {
          const float *b = Y + (9 * lv + 3) * S;
          const float tjj = __ldg(b + JA * S + o), tkk = __ldg(b + KA * S + o), tll = __ldg(b + LA * S + o);
          vj += Lv[lv] * (2.f * muq * tjj + lq * (tjj + tkk + tll));
          vk += Lv[lv] * (muq * __ldg(b + sym(KA, JA) * S + o));
          vl += Lv[lv] * (muq * __ldg(b + sym(LA, JA) * S + o));
        }
      }
      q[0][d] = vj;
      q[1][d] = vk;
      q[2][d] = vl;
    }
    sh.f[JA][JA][lane] = ddiv(q[0][0], q[0][1], q[0][2], q[0][3], q[0][4], kd);
    sh.f[JA][KA][lane] = ddiv(q[1][0], q[1][1], q[1][2], q[1][3], q[1][4], kd);
    sh.f[JA][LA][lane] = ddiv(q[2][0], q[2][1], q[2][2], q[2][3], q[2][4], kd);
  }
  // column JA of H (times h). Every displacement level is zero on a fixed face, so
  // the derivative along a line that lies in one is exactly zero.
  if (n.flat[JA]) {
#pragma unroll
    for (int i = 0; i < 3; i++) sh.H[i][JA][lane] = 0.f;
    return;
  }
#pragma unroll
  for (int i = 0; i < 3; i++)
    sh.H[i][JA][lane] = n.Le[JA] * dav(Y + (18 + i) * S, n.node, s, kd) + n.Lp[JA] * dav(Y + (9 + i) * S, n.node, s, kd) +
                        n.Lw[JA] * dav(Y + i * S, n.node, s, kd);
}

template <bool ADJ>
__device__ __forceinline__ void face_write(const Geo &g, const StageArgs &a, const FaceCtx &n, int I, int J, int K,
                                           const FaceShared &sh, int lane, int w) {
  const int S = (int)g.stride;
  const float *__restrict__ Y = a.Y;
  // ---- displacement component w
  {
    const int c = w;
    const int i0 = c * S + n.node, i1 = (9 + c) * S + n.node, i2 = (18 + c) * S + n.node;
    if (!n.dir) {
      const float f = sh.f[0][c][lane] + sh.f[1][c][lane] + sh.f[2][c][lane];
      const float u0 = __ldg(Y + i0), u1 = __ldg(Y + i1), u2 = __ldg(Y + i2);
      const float acc = (g.inv_rho_h * f - (n.cb * u2 + n.cc * u1 + n.cd * u0)) * n.inv_a;
      __stcs(a.out + i0, stage_value(a, i0, u0, u1));
      __stcs(a.out + i1, stage_value(a, i1, u1, u2));
      __stcs(a.out + i2, stage_value(a, i2, u2, acc));
    } else if (a.stage == 0) {
      __stcs(a.out + i0, 0.f);
      __stcs(a.out + i1, 0.f);
      __stcs(a.out + i2, 0.f);
    }
  }
  // ---- stress components w and w + 3: S'' = (tau(P(H)) / h - b S' - c S - d Sbar) / a
  float lam = 0.f, mu = 0.f;
  if (!ADJ) {
    lam = __ldg(g.lam_n + n.node);
    mu = __ldg(g.mu_n + n.node);
  }
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int c = w + 3 * h;
    float src;
    if (h == 0) {
      src = sh.H[w][w][lane];
      if (!ADJ) src = 2.f * mu * src + lam * (sh.H[0][0][lane] + sh.H[1][1][lane] + sh.H[2][2][lane]);
    } else {
      const int i = w == 2 ? 0 : (w == 1 ? 0 : 1), j = w == 2 ? 1 : 2;  // yz, xz, xy
      src = sh.H[i][j][lane] + sh.H[j][i][lane];
      if (!ADJ) src = mu * src;
    }
    const int i0 = (3 + c) * S + n.node, i1 = (12 + c) * S + n.node, i2 = (21 + c) * S + n.node;
    const float s0 = __ldg(Y + i0), s1 = __ldg(Y + i1), s2 = __ldg(Y + i2);
    __stcs(a.out + i0, stage_value(a, i0, s0, s1));
    __stcs(a.out + i1, stage_value(a, i1, s1, s2));
    __stcs(a.out + i2, stage_value(a, i2, s2, (g.inv_h * src - n.cb * s2 - n.cc * s1 - n.cd * s0) * n.inv_a));
  }
}

#ifndef FWI_PML_STAGE4_MINB
#define FWI_PML_STAGE4_MINB 7  // stage 4 reads three more step-start rows: 72 registers, no spills
#endif
#ifndef FWI_PML_SPLIT_MINB
#define FWI_PML_SPLIT_MINB 8
#endif
#ifndef FWI_PML_BY
#define FWI_PML_BY 4
#endif
#ifndef FWI_PML_MINB
#define FWI_PML_MINB 7
#endif
#ifndef FWI_FACE_MINB
#define FWI_FACE_MINB 10
#endif
constexpr int kBX = 32, kBY = FWI_PML_BY;

// grid.x: blocks of kBY warp tasks (see Region); tasks of a box run plane by plane.
// The boxes exclude the outer faces of the grid, so every node takes the bulk path.
// PART 3 runs the stress-row update and then the displacement-row update of the same
// pair in the same thread: each part keeps its own register footprint, and the second
// part's loads (the rows the first part just read) hit in L1/L2 instead of DRAM.
template <bool ADJ, int MODE, int KY, int KZ, int PART>
__device__ __forceinline__ void pml_task(const Geo &g, const StageArgs &a, int I0, int J, int K, bool even_ok) {
  if constexpr (PART == 3) {
    pml_pair<ADJ, MODE, KY, KZ, 1>(g, a, I0, J, K, even_ok);
    pml_pair<ADJ, MODE, KY, KZ, 2>(g, a, I0, J, K, even_ok);
  } else {
    pml_pair<ADJ, MODE, KY, KZ, PART>(g, a, I0, J, K, even_ok);
  }
}

template <bool ADJ, int MODE, int PART>
__global__ void __launch_bounds__(kBX *kBY, MODE == 3 ? FWI_PML_STAGE4_MINB : (PART == 0 ? FWI_PML_MINB : FWI_PML_SPLIT_MINB))
    pml_kernel(Geo g, StageArgs a0, Region r) {
  const int nbs = (r.tasks_before[r.nbox] + kBY - 1) / kBY;  // blocks per shot
  const StageArgs a = shot_args(a0, blockIdx.x / nbs);
  const int task = (blockIdx.x % nbs) * kBY + threadIdx.y;
  if (task >= r.tasks_before[r.nbox]) return;
  int b = 0;
  while (b + 1 < r.nbox && task >= r.tasks_before[b + 1]) b++;
  const int G = r.groups[b][0] + r.groups[b][1];
  const int per_seg = G * (r.hi[b][2] - r.lo[b][2] + 1);  // tasks of one x segment
  const int t = (task - r.tasks_before[b]) % per_seg;
  const int pb = (task - r.tasks_before[b]) / per_seg * r.per[b];  // first pair of the segment
  const int K = r.lo[b][2] + t / G;
  const int qa = t % G;
  const int P = min(r.per[b], r.P[b] - pb), R = r.R[b];  // pairs of this segment
  const int x0 = r.lo[b][0] & ~1;  // pairs start at even x
  const int kz = side_kind(K, g.n[2]);
  const int cls = qa < r.groups[b][0] ? 0 : 1;
  const int q = cls ? qa - r.groups[b][0] : qa;
  const int rr = R > 1 ? threadIdx.x / P : 0;  // row of the group handled by this lane
  const int jrow = q * R + rr;
  if (rr >= R || jrow >= r.nj[b][cls]) return;
  const int J = r.jfirst[b][cls] + 2 * jrow;
  const int ky = side_kind(r.jfirst[b][cls], g.n[1]);
  const int p = R > 1 ? threadIdx.x % P : threadIdx.x;  // pair of the segment (P <= 32)
  if (p < P) {
    const int I0 = x0 + 2 * (pb + p);
    // reach of the pair's stencils: the x window I0-2 .. I0+3 of its row, +-1 (odd) or
    // +-2 (even) rows and planes
    const int ry = ky == kSC ? 1 : 2, rz = kz == kSC ? 1 : 2;
    if (!(guard(g.oob, kSitePml, J - ry, g.n[1]) && guard(g.oob, kSitePml, J + ry, g.n[1]) &&
          guard(g.oob, kSitePml, K - rz, g.n[2]) && guard(g.oob, kSitePml, K + rz, g.n[2]) &&
          guard(g.oob, kSitePml, I0 + 3, g.px) &&
          guard(g.oob, kSitePml, ((long long)K * g.n[1] + J) * g.px + I0 - 2, (long long)g.px * g.n[1] * g.n[2])))
      return;
    // box x-ranges end at odd nodes, so the odd node of a pair is always in the box;
    // the even node of a box's first pair may not be (its results are dropped)
    const bool even_ok = I0 >= r.lo[b][0];
    if (ky == kSC) {
      if (kz == kSC) pml_task<ADJ, MODE, kSC, kSC, PART>(g, a, I0, J, K, even_ok);
      else pml_task<ADJ, MODE, kSC, kSLR, PART>(g, a, I0, J, K, even_ok);
    } else {
      if (kz == kSC) pml_task<ADJ, MODE, kSLR, kSC, PART>(g, a, I0, J, K, even_ok);
      else pml_task<ADJ, MODE, kSLR, kSLR, PART>(g, a, I0, J, K, even_ok);
    }
  }
}

template <bool ADJ>
__global__ void __launch_bounds__(3 * kFaceNodes, FWI_FACE_MINB) pml_face_kernel(Geo g, StageArgs a0) {
  __shared__ FaceShared sh;
  const int nbs = (g.nface + kFaceNodes - 1) / kFaceNodes;  // blocks per shot
  const StageArgs a = shot_args(a0, blockIdx.x / nbs);
  const int lane = threadIdx.x, w = threadIdx.y;
  const int i = (blockIdx.x % nbs) * kFaceNodes + lane;
  const bool live = i < g.nface && node_ok(g, kSiteFace, g.face[i]);
  int I = 0, J = 0, K = 0;
  FaceCtx n;
  if (live) {
    const int node = g.face[i];
    const int rr = node / g.px;
    I = node % g.px;
    J = rr % g.n[1];
    K = rr / g.n[1];
    n = face_ctx(g, I, J, K);
    if (w == 0) face_axis<ADJ, 0>(g, a, n, I, J, K, sh, lane);
    else if (w == 1) face_axis<ADJ, 1>(g, a, n, I, J, K, sh, lane);
    else face_axis<ADJ, 2>(g, a, n, I, J, K, sh, lane);
  }
  __syncthreads();
  if (live) face_write<ADJ>(g, a, n, I, J, K, sh, lane, w);
}

}  // namespace

// boxes of the nodes outside the closed interior box [2lo, 2hi] (free top: from k = 0)
static Region pml_region(const Geo &g) {
  Region r{};
  const int c0[3] = {2 * g.lo[0], 2 * g.lo[1], g.top_dir ? 2 * g.lo[2] : 0};
  const int c1[3] = {2 * g.hi[0], 2 * g.hi[1], 2 * g.hi[2]};
  auto add = [&](int x0, int x1, int y0, int y1, int z0, int z1) {
    if (x0 > x1 || y0 > y1 || z0 > z1) return;
    const int b = r.nbox++;
    r.lo[b][0] = x0; r.hi[b][0] = x1;
    r.lo[b][1] = y0; r.hi[b][1] = y1;
    r.lo[b][2] = z0; r.hi[b][2] = z1;
  };
  // boxes clipped to the grid without its outer faces (those go to pml_face_kernel)
  const int nx = g.n[0] - 2, ny = g.n[1] - 2, nz = g.n[2] - 2;
  const int z0 = c0[2] > 1 ? c0[2] : 1, y0 = c0[1] > 1 ? c0[1] : 1;
  add(1, nx, 1, ny, c1[2] + 1, nz);                       // below the interior
  add(1, nx, 1, ny, 1, c0[2] - 1);                        // above (top PML)
  add(1, nx, 1, c0[1] - 1, z0, c1[2]);                    // y- side
  add(1, nx, c1[1] + 1, ny, z0, c1[2]);                   // y+ side
  add(1, c0[0] - 1, y0, c1[1], z0, c1[2]);                // x- side
  add(c1[0] + 1, nx, y0, c1[1], z0, c1[2]);               // x+ side
  r.tasks_before[0] = 0;
  for (int b = 0; b < r.nbox; b++) {
    r.P[b] = (r.hi[b][0] - (r.lo[b][0] & ~1)) / 2 + 1;
    r.nseg[b] = (r.P[b] + g.pml_seg - 1) / g.pml_seg;
    r.per[b] = (r.P[b] + r.nseg[b] - 1) / r.nseg[b];
    r.R[b] = r.per[b] > 16 ? 1 : 32 / r.per[b];  // rows per warp task: fill the 32 lanes
    int per_plane = 0;
    for (int c = 0; c < 2; c++) {
      const int jf = r.lo[b][1] + ((r.lo[b][1] & 1) != c ? 1 : 0);  // first J of parity c
      r.jfirst[b][c] = jf;
      r.nj[b][c] = jf > r.hi[b][1] ? 0 : (r.hi[b][1] - jf) / 2 + 1;
      r.groups[b][c] = (r.nj[b][c] + r.R[b] - 1) / r.R[b];
      per_plane += r.groups[b][c];
    }
    r.tasks_before[b + 1] = r.tasks_before[b] + r.nseg[b] * per_plane * (r.hi[b][2] - r.lo[b][2] + 1);
  }
  for (int b = r.nbox; b < 6; b++) r.tasks_before[b + 1] = r.tasks_before[b];
  return r;
}

int launch_pml(const Geo &g, const StageArgs &a, bool adjoint, cudaStream_t s) {
  const Region r = pml_region(g);
  const int tasks = r.tasks_before[r.nbox];
  if (tasks == 0) return 0;
  const dim3 grd((tasks + kBY - 1) / kBY * a.nshot), blk(kBX, kBY);
  const int mode = a.stage == 0 ? 0 : (a.stage == 1 ? 1 : (a.stage < 4 ? 2 : 3));
  auto go = [&](auto part, cudaStream_t st) {
    constexpr int P = decltype(part)::value;
    if (adjoint) {
      if (mode == 0) pml_kernel<true, 0, P><<<grd, blk, 0, st>>>(g, a, r);
      else if (mode == 1) pml_kernel<true, 1, P><<<grd, blk, 0, st>>>(g, a, r);
      else if (mode == 2) pml_kernel<true, 2, P><<<grd, blk, 0, st>>>(g, a, r);
      else pml_kernel<true, 3, P><<<grd, blk, 0, st>>>(g, a, r);
    } else {
      if (mode == 0) pml_kernel<false, 0, P><<<grd, blk, 0, st>>>(g, a, r);
      else if (mode == 1) pml_kernel<false, 1, P><<<grd, blk, 0, st>>>(g, a, r);
      else if (mode == 2) pml_kernel<false, 2, P><<<grd, blk, 0, st>>>(g, a, r);
      else pml_kernel<false, 3, P><<<grd, blk, 0, st>>>(g, a, r);
    }
  };
  // one launch: per pair the stress rows, then the displacement rows (disjoint outputs, the
  // same inputs), each part with the registers of its own update
  go(std::integral_constant<int, 3>{}, s);
  return 1;
}

int launch_pml_face(const Geo &g, const StageArgs &a, bool adjoint, cudaStream_t s) {
  if (g.nface <= 0) return 0;
  const int nb = (g.nface + kFaceNodes - 1) / kFaceNodes * a.nshot;
  const dim3 blk(kFaceNodes, 3);
  if (adjoint)
    pml_face_kernel<true><<<nb, blk, 0, s>>>(g, a);
  else
    pml_face_kernel<false><<<nb, blk, 0, s>>>(g, a);
  return 1;
}

}  // namespace fwi
