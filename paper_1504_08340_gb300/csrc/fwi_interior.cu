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
// start at a 16-byte aligned x). Each plane arrives as one tensor copy (TMA,
// cp.async.bulk.tensor: a 72 x 12 x 1 x 3 box of the stage input, zero outside the
// grid) issued by one thread and signalled on the ring slot's mbarrier; plane K+3
// streams in while plane K is computed, and the block waits only for plane K+2
// before it computes K. Every wait is bounded (Geo::wait_cycles). lambda and mu are
// read from global memory (L1/L2 resident). Each thread computes a pair of nodes
// (even x, odd x) of plane K.
// Side types are template parameters, so every stencil access is a shared
// load at a compile-time offset from one of five plane base registers.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>

#include "fwi_internal.h"

namespace fwi {
namespace {

constexpr int kTP = 32;             // node pairs per tile row (64 nodes)
#ifndef FWI_INT_TY
#define FWI_INT_TY 8
#endif
constexpr int kTY = FWI_INT_TY;     // rows per tile
// smem row: the tile's 64 nodes with a halo of 2 on each side, from a 16-byte aligned
// start (at most 2 nodes before the halo); it is also the tensor copy's box width
constexpr int kTXS = 2 * kTP + 8;   // smem row pitch
constexpr int kTYS = kTY + 4;
constexpr int kFS = kTXS * kTYS;    // floats per field and plane
constexpr int kNF = 3;              // u_x, u_y, u_z
constexpr int kPS = kNF * kFS;      // floats per plane
constexpr int kRing = 6;            // planes K-2 .. K+2 in use, K+3 in flight
constexpr int kPlaneBytes = kPS * (int)sizeof(float);   // one tensor copy (10,368 bytes)
constexpr int kSmem = kRing * kPlaneBytes + kRing * 8;  // the ring, then one mbarrier per slot
static_assert(kPlaneBytes % 128 == 0, "tensor copies land on 128-byte aligned ring slots");
static_assert(kTXS <= 256 && kTYS <= 256, "TMA box extents");

enum { kC = 0, kL = 1, kR = 2 };
// side set of a node along an axis: odd coordinate {C}, even {L, R}, top face {R}
enum { kOdd = 0, kEven = 1, kTop = 2 };

extern __shared__ __align__(1024) float s_ring[];  // the plane ring, then the slot barriers

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

// ---- plane copies: mbarrier and TMA (PTX)
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(uint64_t *b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(b)) : "memory");
}
// the one arrival of a slot's phase, with the bytes its copy will deliver
__device__ __forceinline__ void bar_arm(uint64_t *b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_done(uint64_t *b, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return done != 0;
}
// wait for the phase of parity `parity` to complete; false after `limit` clock cycles
__device__ __forceinline__ bool bar_wait(uint64_t *b, unsigned parity, long long limit) {
  if (bar_done(b, parity)) return true;
  const long long t0 = clock64();
  while (!bar_done(b, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
// box (x .. x+71, y .. y+11, plane z, fields f .. f+2) of the tensor map into dst
__device__ __forceinline__ void copy_plane(float *dst, const CUtensorMap *tm, int x, int y, int z, int f, uint64_t *b) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(f), "r"(smem_u32(b))
      : "memory");
}

#ifndef FWI_INT_MINB
#define FWI_INT_MINB 2
#endif
// tm: the u fields of the stage input of the batch (see plane_map); the copies of a plane
// are numbered from k0 - 2: copy q lands in ring slot q % kRing, and is that slot's
// (q / kRing)-th phase
__global__ void __launch_bounds__(kTP *kTY, FWI_INT_MINB)
    interior_kernel(const __grid_constant__ CUtensorMap tm, Geo g, StageArgs a0) {
  float *smem = s_ring;
  uint64_t *bar = reinterpret_cast<uint64_t *>(s_ring + kRing * kPS);
  const int kc = g.int_kc;                                   // planes per block
  const int nzc = (g.box_hi[2] - g.box_lo[2] + kc) / kc;     // z chunks per shot
  const int shot = blockIdx.z / nzc;
  const StageArgs a = shot_args(a0, shot);
  const int bz = blockIdx.z % nzc;
  const int x0 = g.box_lo[0] - 1 + 2 * kTP * blockIdx.x;  // even: pairs (even, odd)
  const int xs = (x0 - 2) & ~3;                            // first x of the smem rows (16-byte aligned)
  const int sh = x0 - 2 - xs;                              // 0 or 2
  const int y0 = g.box_lo[1] + kTY * blockIdx.y;
  const int k0 = g.box_lo[2] + kc * bz;
  const int k1 = min(k0 + kc - 1, g.box_hi[2]);
  const int q0 = k0 - 2;                                   // plane of copy 0
  const int f0 = kFields * shot + 9;                       // the shot's u_x field in the map
  const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
  const unsigned bytes = kPlaneBytes + (unsigned)g.copy_extra;
  auto issue = [&](int K) {
    uint64_t *b = &bar[(K - q0) % kRing];
    bar_arm(b, bytes);
    copy_plane(smem + ((K - q0) % kRing) * kPS, &tm, xs, y0 - 2, K, f0, b);
  };
  auto landed = [&](int K) { return bar_wait(&bar[(K - q0) % kRing], ((K - q0) / kRing) & 1, g.wait_cycles); };
  // after a wait of this call gave up, later launches do nothing until the host has read
  // it (one thread reads the word, so the whole block takes the same branch)
  if (__syncthreads_or(lead && *(volatile int *)g.status != 0)) return;
  if (lead) {
    for (int s = 0; s < kRing; s++) bar_init(&bar[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int K = k0 - 2; K <= k0 + 2; K++) issue(K);
  }
  __syncthreads();
  const int IE = x0 + 2 * threadIdx.x, IO = IE + 1, J = y0 + threadIdx.y;
  const bool rowok = J <= g.box_hi[1];
  const bool even_ok = rowok && IE >= g.box_lo[0] && IE <= g.box_hi[0];
  const bool odd_ok = rowok && IO >= g.box_lo[0] && IO <= g.box_hi[0];
  const int sy = (J & 1) ? kOdd : kEven;
  const float sc = -(g.inv_h * g.inv_h * (1.f / 3.f)) / g.rho;
  int K = k0;
  bool ok = true;
  for (; K <= k1; K++) {
    // plane K+3 goes to the slot of plane K-3, which every thread finished with before the
    // barrier that ended the previous plane
    if (lead && K + 1 <= k1) issue(K + 3);
    bool got = true;
    if (K == k0)
      for (int q = k0 - 2; q <= k0 + 1 && got; q++) got = landed(q);
    got = got && landed(K + 2);
    if (!got) atomicExch(g.status, 6);  // FWI_E_TIMEOUT
    Tile t;
#pragma unroll
    for (int d = 0; d < 5; d++) t.pl[d] = ((K + d - 2 - q0) % kRing) * kPS;
    const int sz = (K & 1) ? kOdd : ((K == 0 && !g.top_dir) ? kTop : kEven);
    t.o = (threadIdx.y + 2) * kTXS + 2 + sh + 2 * threadIdx.x;
    t.lam = g.lam;
    t.mu = g.mu;
    t.ms1 = g.m[0];
    t.ms2 = g.m[0] * g.m[1];
    t.mi = ((K - 2 * g.lo[2]) * g.m[1] + (J - 2 * g.lo[1])) * g.m[0] + (IE - 2 * g.lo[0]);
    const int64_t rowbase = ((int64_t)K * g.n[1] + J) * g.px;
    const bool e_ok = got && even_ok && node_ok(g, kSiteInterior, rowbase + IE);
    const bool o_ok = got && odd_ok && node_ok(g, kSiteInterior, rowbase + IO);
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
    if (__syncthreads_or(!got)) {
      ok = false;
      break;
    }
  }
  if (!ok && lead) {
    // a wait gave up: before the block's shared memory is released, wait (bounded) for the
    // copies it may still have in flight, the last kRing issued
    const int last = max(k0 + 2, min(K + 3, k1 + 2));
    for (int q = max(q0, last - kRing + 1); q <= last; q++) landed(q);
  }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static const EncodeTiled fn = []() -> EncodeTiled {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// tensor map of the stage input Y of nshot shots as a 4-D FP32 tensor: x (the row pitch px),
// y (NJ rows), z (NK planes), f (27 nshot fields, `stride` floats apart; shot b's field c is
// 27 b + c, as the shots' state sets are 27 stride floats apart). Boxes are 72 x 12 x 1 x 3;
// elements outside the tensor read as zero (the row padding x >= NI holds zeros in every
// state buffer, so a box reads zero wherever the node grid ends).
bool plane_map(const Geo &g, const StageArgs &a, CUtensorMap *tm) {
  const EncodeTiled enc = encode_tiled();
  if (!enc || ((uintptr_t)a.Y & 15) != 0 || (a.nshot > 1 && a.sstride != (int64_t)kFields * g.stride)) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.px, (cuuint64_t)g.n[1], (cuuint64_t)g.n[2],
                              (cuuint64_t)kFields * (cuuint64_t)a.nshot};
  const cuuint64_t pitch[3] = {(cuuint64_t)g.px * 4, (cuuint64_t)g.px * g.n[1] * 4, (cuuint64_t)g.stride * 4};
  const cuuint32_t box[4] = {(cuuint32_t)kTXS, (cuuint32_t)kTYS, 1, (cuuint32_t)kNF};
  const cuuint32_t step[4] = {1, 1, 1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(a.Y), dims, pitch, box, step,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
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
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  if (!plane_map(g, a, &tm)) return -1;
  interior_kernel<<<grd, dim3(kTP, kTY), kSmem, s>>>(tm, g, a);
  return 1;
}

}  // namespace fwi
