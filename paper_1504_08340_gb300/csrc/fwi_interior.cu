// fwi_interior.cu -- RK4 stage kernel for the nodes all of whose elements are
// interior (regular-domain) elements: M udd = -K_RD u, plus the stage update.
//
// K_RD is the interior stiffness of (3a) (Sec. 2 of arXiv:1504.08340) with
// 27-node LGL elements. At such a node every element around it is interior,
// so the sum over elements factorises per axis (see fwi_stage.cu):
//   F_i(a) = sum_j (1/w_j) sum_{side s_j} sum_{line points q} c(q) Sigma_ij(q)
//   Sigma_jj = lam (nk nl d_j u_j + nl S_k u_k + nk S_l u_l) + 2 mu nk nl d_j u_j
//   Sigma_kj = mu (nk nl d_j u_k + nl S_k u_j), Sigma_lj = mu (nk nl d_j u_l + nk S_l u_j)
// with d_j the element-wise derivative at q inside the element on side s_j,
// S_k the sum of the element-wise derivatives along k over both k-sides
// (one 4-point stencil), nk, nl the element counts along k, l, and
// c(q) = w_q (2/h) D[q][a] the line quadrature coefficient.
//
// GB300 mapping: a block owns a 64 x 8 node tile in (x, y) and marches along
// z through a chunk of planes. u (3 components) of planes K-2 .. K+2 sits in a
// shared-memory ring (6 planes x 3 fields x 12 rows x 72 floats, 62.2 KB; rows
// start at a 16-byte aligned x and are copied in 16-byte chunks); plane K+3
// streams in with cp.async while plane K is computed. lambda and mu are read from
// global memory (L1/L2 resident). Each thread computes a pair of nodes (even x,
// odd x) of plane K.
// Side types are template parameters, so every stencil access is a shared
// load at a compile-time offset from one of five plane base registers.
#include <cuda_runtime.h>

#include "fwi_internal.h"

namespace fwi {
namespace {

constexpr int kTP = 32;             // node pairs per tile row (64 nodes)
#ifndef FWI_INT_TY
#define FWI_INT_TY 8
#endif
constexpr int kTY = FWI_INT_TY;     // rows per tile
// smem row: the tile's 64 nodes with a halo of 2 on each side, from a 16-byte aligned
// start (at most 2 nodes before the halo), copied in 16-byte chunks
constexpr int kTXS = 2 * kTP + 8;   // smem row pitch
constexpr int kCPR = kTXS / 4;      // 16-byte chunks per row
constexpr int kTYS = kTY + 4;
constexpr int kFS = kTXS * kTYS;    // floats per field and plane
constexpr int kNF = 3;              // u_x, u_y, u_z
constexpr int kPS = kNF * kFS;      // floats per plane
constexpr int kRing = 6;            // planes K-2 .. K+2 in use, K+3 in flight
constexpr int kSmem = kRing * kPS * (int)sizeof(float);

enum { kC = 0, kL = 1, kR = 2 };
// side set of a node along an axis: odd coordinate {C}, even {L, R}, top face {R}
enum { kOdd = 0, kEven = 1, kTop = 2 };

extern __shared__ float s_ring[];  // the plane ring (dynamic shared memory)

struct Tile {
  int pl[5];  // ring offsets (floats) of the planes dz = -2..2
  int o;      // offset of the node in a field slab
  const float *lam, *mu;  // material grid (when it is not in the ring)
  int mi, ms1, ms2;       // material index of the node, material row / plane strides
  template <int DX, int DY, int DZ>
  __device__ __forceinline__ float mat(int which) const {
    return __ldg((which == 0 ? lam : mu) + mi + DX + DY * ms1 + DZ * ms2);
  }
  template <int DX, int DY, int DZ>
  __device__ __forceinline__ float v(int c) const {
    return s_ring[pl[DZ + 2] + c * kFS + o + DY * kTXS + DX];
  }
};

__host__ __device__ constexpr int ex(int ax) { return ax == 0 ? 1 : 0; }
__host__ __device__ constexpr int ey(int ax) { return ax == 1 ? 1 : 0; }
__host__ __device__ constexpr int ez(int ax) { return ax == 2 ? 1 : 0; }

// element-wise derivative (times h) along AX, side type T, at offset (DX,DY,DZ)
template <int AX, int T, int DX, int DY, int DZ>
__device__ __forceinline__ float der(const Tile &t, int c) {
  constexpr int X = ex(AX), Y = ey(AX), Z = ez(AX);
  if constexpr (T == kC) {
    return t.v<DX + X, DY + Y, DZ + Z>(c) - t.v<DX - X, DY - Y, DZ - Z>(c);
  } else if constexpr (T == kL) {
    return t.v<DX - 2 * X, DY - 2 * Y, DZ - 2 * Z>(c) - 4.f * t.v<DX - X, DY - Y, DZ - Z>(c) +
           3.f * t.v<DX, DY, DZ>(c);
  } else {
    return -3.f * t.v<DX, DY, DZ>(c) + 4.f * t.v<DX + X, DY + Y, DZ + Z>(c) - t.v<DX + 2 * X, DY + 2 * Y, DZ + 2 * Z>(c);
  }
}

// sum over the node's sides along AX (side set ST) of the derivative, at offset
template <int AX, int ST, int DX, int DY, int DZ>
__device__ __forceinline__ float xsum(const Tile &t, int c) {
  constexpr int X = ex(AX), Y = ey(AX), Z = ez(AX);
  if constexpr (ST == kOdd) {
    return der<AX, kC, DX, DY, DZ>(t, c);
  } else if constexpr (ST == kEven) {
    return t.v<DX - 2 * X, DY - 2 * Y, DZ - 2 * Z>(c) - 4.f * t.v<DX - X, DY - Y, DZ - Z>(c) +
           4.f * t.v<DX + X, DY + Y, DZ + Z>(c) - t.v<DX + 2 * X, DY + 2 * Y, DZ + 2 * Z>(c);
  } else {
    return der<AX, kR, DX, DY, DZ>(t, c);
  }
}

__host__ __device__ constexpr float line_coef(int T, int P) {
  return T == kC ? (P == 0 ? 4.f : (P == 2 ? -4.f : 0.f))
                 : (T == kL ? (P == 0 ? -1.f : (P == 1 ? 4.f : 3.f)) : (P == 0 ? -3.f : (P == 1 ? -4.f : 1.f)));
}
__host__ __device__ constexpr int line_off(int T, int P) { return T == kC ? P - 1 : (T == kL ? P - 2 : P); }
__host__ __device__ constexpr int point_type(int P) { return P == 0 ? kR : (P == 1 ? kC : kL); }
__host__ __device__ constexpr float nsides(int ST) { return ST == kEven ? 2.f : 1.f; }

// contribution of line point P of the element on side T along axis J
template <int J, int T, int P, int SK, int SL>
__device__ __forceinline__ void line_point(const Tile &t, float &aj, float &ak, float &al) {
  constexpr float cf = line_coef(T, P);
  if constexpr (cf != 0.f) {
    constexpr int K = (J + 1) % 3, L = (J + 2) % 3;
    constexpr int off = line_off(T, P);
    constexpr int DX = J == 0 ? off : 0, DY = J == 1 ? off : 0, DZ = J == 2 ? off : 0;
    constexpr int PT = point_type(P);
    constexpr float nk = nsides(SK), nl = nsides(SL), n2 = nk * nl;
    const float djj = der<J, PT, DX, DY, DZ>(t, J);
    const float djk = der<J, PT, DX, DY, DZ>(t, K);
    const float djl = der<J, PT, DX, DY, DZ>(t, L);
    const float skk = xsum<K, SK, DX, DY, DZ>(t, K), skj = xsum<K, SK, DX, DY, DZ>(t, J);
    const float sll = xsum<L, SL, DX, DY, DZ>(t, L), slj = xsum<L, SL, DX, DY, DZ>(t, J);
    const float lam = t.template mat<DX, DY, DZ>(0), mu = t.template mat<DX, DY, DZ>(1);
    aj += cf * (lam * (n2 * djj + nl * skk + nk * sll) + 2.f * mu * n2 * djj);
    ak += cf * (mu * (n2 * djk + nl * skj));
    al += cf * (mu * (n2 * djl + nk * slj));
  }
}

template <int J, int SJ, int SK, int SL>
__device__ __forceinline__ void axis_force(const Tile &t, float f[3]) {
  constexpr int K = (J + 1) % 3, L = (J + 2) % 3;
  constexpr float invw = SJ == kOdd ? 0.75f : 3.0f;
  float aj = 0.f, ak = 0.f, al = 0.f;
  if constexpr (SJ == kOdd) {
    line_point<J, kC, 0, SK, SL>(t, aj, ak, al);
    line_point<J, kC, 2, SK, SL>(t, aj, ak, al);
  } else {
    if constexpr (SJ == kEven) {
      line_point<J, kL, 0, SK, SL>(t, aj, ak, al);
      line_point<J, kL, 1, SK, SL>(t, aj, ak, al);
      line_point<J, kL, 2, SK, SL>(t, aj, ak, al);
    }
    line_point<J, kR, 0, SK, SL>(t, aj, ak, al);
    line_point<J, kR, 1, SK, SL>(t, aj, ak, al);
    line_point<J, kR, 2, SK, SL>(t, aj, ak, al);
  }
  f[J] += invw * aj;
  f[K] += invw * ak;
  f[L] += invw * al;
}

// acceleration -K_RD u / M at one node, side sets SX, SY, SZ
template <int SX, int SY, int SZ>
__device__ __forceinline__ void node_accel(const Tile &t, float sc, float acc[3]) {
  float f[3] = {0.f, 0.f, 0.f};
  axis_force<0, SX, SY, SZ>(t, f);
  axis_force<1, SY, SZ, SX>(t, f);
  axis_force<2, SZ, SX, SY>(t, f);
  constexpr float nel = nsides(SX) * nsides(SY) * nsides(SZ);
  acc[0] = sc * f[0] * (1.f / nel);
  acc[1] = sc * f[1] * (1.f / nel);
  acc[2] = sc * f[2] * (1.f / nel);
}

template <int SX>
__device__ __forceinline__ void node_accel_dispatch(const Tile &t, int sy, int sz, float sc, float acc[3]) {
  if (sy == kOdd) {
    if (sz == kOdd) node_accel<SX, kOdd, kOdd>(t, sc, acc);
    else if (sz == kEven) node_accel<SX, kOdd, kEven>(t, sc, acc);
    else node_accel<SX, kOdd, kTop>(t, sc, acc);
  } else {
    if (sz == kOdd) node_accel<SX, kEven, kOdd>(t, sc, acc);
    else if (sz == kEven) node_accel<SX, kEven, kEven>(t, sc, acc);
    else node_accel<SX, kEven, kTop>(t, sc, acc);
  }
}

// the node's own stage-update operands, loaded before the stencil work so that
// their latency overlaps it
struct Own {
  float yd[3];         // u rate of the stage input
  float x1[3], x2[3];  // u and u rate at the step start
};

__device__ __forceinline__ void load_own(const Geo &g, const StageArgs &a, int64_t node, Own &o) {
  const int64_t S = g.stride;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const int64_t i1 = (int64_t)(9 + c) * S + node, i2 = (int64_t)(18 + c) * S + node;
    o.yd[c] = __ldg(a.Y + i2);
    if (a.stage >= 2) {  // in stage 1 X is the stage input
      o.x1[c] = __ldcs(a.X + i1);
      o.x2[c] = __ldcs(a.X + i2);
    }
  }
}

// RK4 stage update (see StageArgs); stage 4 reads Y2 and Y3 here
__device__ __forceinline__ float stage_value(const StageArgs &a, int64_t idx, float x, float yv, float rate) {
  if (a.stage == 0) return rate;
  if (a.stage == 1) return yv + a.cdt * rate;
  if (a.stage < 4) return x + a.cdt * rate;
  return (-x + __ldcs(a.Y2 + idx) + 2.f * __ldcs(a.Y3 + idx) + yv) * (1.f / 3.f) + a.cdt * rate;
}

// write the stage outputs of one interior node
__device__ __forceinline__ void finish_node(const Geo &g, const StageArgs &a, int I, int J, int K, const Tile &t,
                                            const Own &o, const float acc[3]) {
  const int64_t S = g.stride;
  const int64_t node = ((int64_t)K * g.n[1] + J) * g.px + I;
  const int64_t mi = ((int64_t)(K - 2 * g.lo[2]) * g.m[1] + (J - 2 * g.lo[1])) * g.m[0] + (I - 2 * g.lo[0]);
  if (!guard(g.oob, kSiteInterior, mi, g.nmat)) return;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const int64_t i1 = (int64_t)(9 + c) * S + node, i2 = (int64_t)(18 + c) * S + node;
    const float u1 = t.v<0, 0, 0>(c);
    const float v1 = stage_value(a, i1, o.x1[c], u1, o.yd[c]);
    __stcs(a.out + (i1), v1);
    __stcs(a.out + (i2), stage_value(a, i2, o.x2[c], o.yd[c], acc[c]));
    if (a.hist) a.hist[(int64_t)c * g.nmat + mi] = v1;
  }
  if (a.stage == 0) {  // history and stress do not exist on these nodes
    for (int f = 0; f < 27; f++)
      if (f % 9 >= 3 || f < 3) __stcs(a.out + ((int64_t)f * S + node), 0.f);
  }
}

// asynchronous 16-byte global -> shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async16(float *dst, const float *src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// issue the copies of plane K (u of the stage input) of the tile into dst: rows
// y0-2 .. y0+kTY+1, x from xs = (x0 - 2) rounded down to a multiple of 4. Chunks
// outside the grid (rows, planes, x < 0 or x >= px) are zero-filled; the row padding
// x in [NI, px) holds zeros in every state buffer.
__device__ __forceinline__ void load_plane(const Geo &g, const StageArgs &a, float *dst, int K, int xs, int y0) {
  const int64_t S = g.stride;
  const bool kin = K >= 0 && K < g.n[2];
  for (int idx = threadIdx.y * kTP + threadIdx.x; idx < kNF * kTYS * kCPR; idx += kTP * kTY) {
    const int f = idx / (kTYS * kCPR), r = (idx / kCPR) % kTYS, ch = idx % kCPR;
    const int gx = xs + 4 * ch, gy = y0 - 2 + r;
    const bool ok = kin && gx >= 0 && gx < g.px && gy >= 0 && gy < g.n[1];
    const float *src = ok ? a.Y + (int64_t)(9 + f) * S + ((int64_t)K * g.n[1] + gy) * g.px + gx : a.Y;
    cp_async16(dst + f * kFS + r * kTXS + 4 * ch, src, ok ? 16 : 0);
  }
}

#ifndef FWI_INT_MINB
#define FWI_INT_MINB 2
#endif
__global__ void __launch_bounds__(kTP *kTY, FWI_INT_MINB) interior_kernel(Geo g, StageArgs a0) {
  float *smem = s_ring;
  const int kc = g.int_kc;                                   // planes per block
  const int nzc = (g.box_hi[2] - g.box_lo[2] + kc) / kc;     // z chunks per shot
  const StageArgs a = shot_args(a0, blockIdx.z / nzc);
  const int bz = blockIdx.z % nzc;
  const int x0 = g.box_lo[0] - 1 + 2 * kTP * blockIdx.x;  // even: pairs (even, odd)
  const int xs = (x0 - 2) & ~3;                            // first x of the smem rows
  const int sh = x0 - 2 - xs;                              // 0 or 2
  const int y0 = g.box_lo[1] + kTY * blockIdx.y;
  const int k0 = g.box_lo[2] + kc * bz;
  const int k1 = min(k0 + kc - 1, g.box_hi[2]);
  const int IE = x0 + 2 * threadIdx.x, IO = IE + 1, J = y0 + threadIdx.y;
  const bool rowok = J <= g.box_hi[1];
  const bool even_ok = rowok && IE >= g.box_lo[0] && IE <= g.box_hi[0];
  const bool odd_ok = rowok && IO >= g.box_lo[0] && IO <= g.box_hi[0];
  const int sy = (J & 1) ? kOdd : kEven;
  const float sc = -(g.inv_h * g.inv_h * (1.f / 3.f)) / g.rho;
  for (int K = k0 - 2; K <= k0 + 2; K++) load_plane(g, a, smem + ((K + 12) % kRing) * kPS, K, xs, y0);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  for (int K = k0; K <= k1; K++) {
    // plane K+3 streams into the free ring slot while plane K is computed
    if (K + 1 <= k1) load_plane(g, a, smem + ((K + 3 + 12) % kRing) * kPS, K + 3, xs, y0);
    cp_async_commit();
    Tile t;
#pragma unroll
    for (int d = 0; d < 5; d++) t.pl[d] = ((K + d - 2 + 12) % kRing) * kPS;
    const int sz = (K & 1) ? kOdd : ((K == 0 && !g.top_dir) ? kTop : kEven);
    t.o = (threadIdx.y + 2) * kTXS + 2 + sh + 2 * threadIdx.x;
    t.lam = g.lam;
    t.mu = g.mu;
    t.ms1 = g.m[0];
    t.ms2 = g.m[0] * g.m[1];
    t.mi = ((K - 2 * g.lo[2]) * g.m[1] + (J - 2 * g.lo[1])) * g.m[0] + (IE - 2 * g.lo[0]);
    const int64_t rowbase = ((int64_t)K * g.n[1] + J) * g.px;
    const bool e_ok = even_ok && node_ok(g, kSiteInterior, rowbase + IE);
    const bool o_ok = odd_ok && node_ok(g, kSiteInterior, rowbase + IO);
    Own oe, oo;
    if (e_ok) load_own(g, a, rowbase + IE, oe);
    if (o_ok) load_own(g, a, rowbase + IO, oo);
    if (e_ok) {
      float acc[3];
      node_accel_dispatch<kEven>(t, sy, sz, sc, acc);
      finish_node(g, a, IE, J, K, t, oe, acc);
    }
    t.o += 1;
    t.mi += 1;
    if (o_ok) {
      float acc[3];
      node_accel_dispatch<kOdd>(t, sy, sz, sc, acc);
      finish_node(g, a, IO, J, K, t, oo, acc);
    }
    cp_async_wait_all();
    __syncthreads();
  }
}

}  // namespace

cudaError_t prepare_interior() {
  return cudaFuncSetAttribute(interior_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

int launch_interior(const Geo &g, const StageArgs &a, cudaStream_t s) {
  if (g.box_hi[0] < g.box_lo[0] || g.box_hi[1] < g.box_lo[1] || g.box_hi[2] < g.box_lo[2]) return 0;
  const int nx = g.box_hi[0] - (g.box_lo[0] - 1) + 1;
  const dim3 grd((nx + 2 * kTP - 1) / (2 * kTP), (g.box_hi[1] - g.box_lo[1] + kTY) / kTY,
                 (g.box_hi[2] - g.box_lo[2] + g.int_kc) / g.int_kc * a.nshot);
  interior_kernel<<<grd, dim3(kTP, kTY), kSmem, s>>>(g, a);
  return 1;
}

}  // namespace fwi
