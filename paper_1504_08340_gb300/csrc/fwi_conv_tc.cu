// fwi_conv_tc.cu -- the forward 3x3x3 convolution of the learned preconditioner on the
// fifth-generation tensor cores (tcgen05, sm_103a), as an implicit GEMM:
//
//   D[p][co] = sum_k A[p][k] B[co][k],  A[p][t Cp + ci] = x[ci][p + off(t)],
//                                       B[co][t Cp + ci] = w[co][ci][t],
//
// p a voxel, t one of the 27 taps (kz, ky, kx; kx fastest), ci an input channel (Cp =
// cin rounded up to 8, the extra channels zero), out-of-grid taps reading zero. Products
// of BF16 values are exact and the sums run in FP32 in tensor memory (TMEM).
//
// A block (8 warps) owns 128 consecutive voxels (the GEMM's M) and a tile of up to 256
// output channels (N, a multiple of 16). K runs in chunks of 64 (four MMAs of K = 16)
// through two shared-memory buffers:
//   - the weight chunk is a contiguous image (packed once per call by pack_kernel in
//     the layout the MMA reads) and arrives by one bulk asynchronous copy that completes
//     on the buffer's "loaded" mbarrier;
//   - the im2col chunk is gathered by the threads from a channels-last copy of x
//     (xcl[p][Cp], made once per call by to_channels_last): a thread owns a voxel and
//     four core columns, each 8 channels of one tap, i.e. one 16-byte load and one
//     16-byte store;
//   - one thread issues the four tcgen05.mma and commits them to the buffer's "done"
//     mbarrier, which the gather of chunk c + 2 waits for before it reuses the buffer.
// Operands use the no-swizzle K-major canonical layout: a core matrix is 8 rows of 16
// bytes (8 BF16 along K) stored contiguously; core (kg, mg) of a chunk sits at
// kg * LBO + mg * 128 bytes. After the last commit the accumulator goes TMEM -> registers
// (tcgen05.ld, a warp reads the 32 lanes = voxels of its quarter) -> bias, ReLU, BF16 ->
// y[co][p], coalesced across the voxels.
//
// Every mbarrier wait is bounded (about a second). A wait that gives up marks the block
// failed: it waits (bounded) for the MMAs it issued, writes NaN to its outputs (so the
// caller's loss turns non-finite) and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fwi_conv_tc.h"

namespace fwi_tc {
namespace {

constexpr int kM = 128;          // voxels per block (MMA M)
constexpr int kKC = 64;          // K per chunk: 8 core columns, 4 MMAs of K = 16
constexpr int kThreads = 256;    // 8 warps
constexpr int kMaxN = 256;       // output channels per block (MMA N <= 256)
constexpr int kABytes = kM * kKC * 2;     // 16 KB im2col chunk
constexpr int kBBytes = kMaxN * kKC * 2;  // <= 32 KB weight chunk
constexpr int kLboA = (kM / 8) * 128;     // between core columns of the A chunk (2 KB)
// shared memory: A[2], B[2] (2 x N x 128 bytes), then the barriers and the TMEM slots
constexpr int kOffB = 2 * kABytes;
constexpr int kSmemMax = kOffB + 2 * kBBytes + 64;
constexpr int kSmPerSM = 233472;  // shared memory of an SM (228 KB); 1 KB more is reserved per block
constexpr int kMinBlocks = 4;     // blocks per SM the register budget allows (64 registers)
constexpr long long kWaitCycles = 2000000000LL;  // about a second

__device__ __forceinline__ unsigned su32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1 (bit 46)
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B
// (bits 7-9, 10-12 = 1), both K-major, N / 8 at bit 17, M / 16 at bit 24
__host__ __device__ constexpr uint32_t instr_desc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void bar_init(uint64_t *b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool bar_done(uint64_t *b, unsigned parity) {
  unsigned d;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(d)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return d != 0;
}
__device__ __forceinline__ bool bar_wait(uint64_t *b, unsigned parity) {
  if (bar_done(b, parity)) return true;
  const long long t0 = clock64();
  while (!bar_done(b, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

// xcl[p][c] = x[c][p] for c < cin, zero for cin <= c < cp: thread per voxel and 8 channels
__global__ void to_channels_last(const uint16_t *__restrict__ x, int64_t nv, int cin, int cp, uint16_t *__restrict__ xcl) {
  const int groups = cp / 8;
  const int64_t total = nv * groups;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i % nv;
    const int c0 = (int)(i / nv) * 8;
    uint32_t v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int e = 0; e < 8; e++)
      if (c0 + e < cin) v[e >> 1] |= (uint32_t)__ldg(x + (int64_t)(c0 + e) * nv + p) << (16 * (e & 1));
    *reinterpret_cast<uint4 *>(xcl + p * cp + c0) = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

// packed weights: for output-channel tile nt and chunk c, the Nt x 64 chunk image in the
// layout above (core (kg, ng) at kg * (Nt / 8) * 128 + ng * 128, row n % 8, 8 k each).
// Row n of B is an output channel of the GEMM (co forward, ci backward); column k = t cpa
// + c' reads source channel c' of tap t, whose weight channel is c' % cgrp (the source of
// the backward pass holds three BF16 parts of each gradient channel, cgrp apart).
__global__ void pack_kernel(const uint16_t *__restrict__ w, int n_rows, int n_red, int cgrp, int cpa, bool bwd,
                            int nt_n, int nchunk, int ntiles, uint16_t *__restrict__ out) {
  const int64_t total = (int64_t)ntiles * nchunk * nt_n * kKC;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(i % 8), row = (int)(i / 8 % 8);
    const int64_t r = i / 64;
    const int ng = (int)(r % (nt_n / 8)), kg = (int)(r / (nt_n / 8) % 8);
    const int64_t tc = r / (nt_n / 8) / 8;  // tile * nchunk + chunk
    const int c = (int)(tc % nchunk), nt = (int)(tc / nchunk);
    const int n = nt * nt_n + ng * 8 + row;
    const int64_t k = (int64_t)c * kKC + kg * 8 + kk;
    const int t = (int)(k / cpa), cc = (int)(k % cpa) % cgrp;
    uint16_t v = 0;
    if (n < n_rows && cc < n_red && t < 27)
      v = w[(bwd ? (int64_t)cc * n_rows + n : (int64_t)n * n_red + cc) * 27 + t];
    out[i] = v;
  }
}

// src[p][s cop + co] = part s of dy[co][p] (s = 0, 1, 2: hi, lo, lo2 with hi + lo + lo2 =
// dy to within 2^-24 relative; each part the BF16 rounding of what the earlier parts left),
// zero for cout <= co < cop: thread per voxel and 8 channels
__global__ void split_channels_last(const float *__restrict__ dy, int64_t nv, int cout, int cop,
                                    uint16_t *__restrict__ src) {
  const int cpa = 3 * cop, groups = cpa / 8;
  const int64_t total = nv * groups;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i % nv;
    const int g0 = (int)(i / nv) * 8;
    const int part = g0 / cop, co0 = g0 % cop;
    uint32_t v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int e = 0; e < 8; e++) {
      if (co0 + e >= cout) continue;
      float r = __ldg(dy + (int64_t)(co0 + e) * nv + p);
      uint16_t h = 0;
      for (int q = 0; q <= part; q++) {
        h = __bfloat16_as_ushort(__float2bfloat16_rn(r));
        r -= __uint_as_float((uint32_t)h << 16);
      }
      v[e >> 1] |= (uint32_t)h << (16 * (e & 1));
    }
    *reinterpret_cast<uint4 *>(src + p * cpa + g0) = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

// BWD = false: y = BF16 [n_out][nv] of act(bias + D) with taps at p + off(t) (forward);
// BWD = true: y = FP32 [n_out][nv] of D with taps at p - off(t) (backward data)
template <bool BWD>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    igemm_kernel(const uint16_t *__restrict__ xcl, const uint16_t *__restrict__ wpack, const float *__restrict__ bias,
                 int cout, int cp, int nt_n, int tmem_cols, int nchunk, int D, int H, int W, int relu,
                 void *__restrict__ yout) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int b_bytes = nt_n * kKC * 2;
  uint64_t *loaded = reinterpret_cast<uint64_t *>(sm + kOffB + 2 * b_bytes);  // [2]
  uint64_t *done = loaded + 2;                                      // [2]
  unsigned *tslot = reinterpret_cast<unsigned *>(done + 2);  // TMEM address, then the committed count
  int *abort_flag = reinterpret_cast<int *>(tslot + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nv = (int64_t)D * H * W;
  const int64_t p0 = (int64_t)blockIdx.x * kM;
  const int nt = blockIdx.y;
  const unsigned lbo_b = (unsigned)(nt_n / 8) * 128u;
  const uint16_t *wtile = wpack + (int64_t)nt * nchunk * nt_n * kKC;

  // the thread's voxel (gather) and its half of each chunk's 8 core columns
  const int m = tid & (kM - 1), half = tid >> 7;
  const int64_t p = p0 + m;
  const bool pin = p < nv;
  const int vx = (int)(p % W), vy = (int)(p / W % H), vz = (int)(p / W / H);

  if (tid == 0) {
    for (int i = 0; i < 2; i++) {
      bar_init(&loaded[i]);
      bar_init(&done[i]);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tslot;
  const uint32_t idesc = instr_desc(nt_n);

  int issued = 0;        // chunks whose MMAs thread 0 committed
  int copy_pending = -1;  // thread 0: the chunk whose weight copy it has not yet waited for
  bool ok = true;
  for (int c = 0; c < nchunk; c++) {
    const int s = c & 1;
    unsigned char *sa = sm + s * kABytes;
    unsigned char *sb = sm + kOffB + s * b_bytes;
    // the MMAs of chunk c - 2 read this buffer
    if (c >= 2 && !bar_wait(&done[s], ((c - 2) >> 1) & 1)) atomicExch(abort_flag, 1);
    if (tid == 0 && *(volatile int *)abort_flag == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&loaded[s])), "r"(b_bytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(sb)),
          "l"(wtile + (int64_t)c * nt_n * kKC), "r"(b_bytes), "r"(su32(&loaded[s]))
          : "memory");
      copy_pending = c;
    }
    // im2col: core columns 4 half .. 4 half + 3 of the chunk, each 8 channels of one tap
    uint4 v[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int k0 = c * kKC + (4 * half + j) * 8;
      const int t = k0 / cp, ci0 = k0 % cp;
      v[j] = make_uint4(0u, 0u, 0u, 0u);
      if (pin && t < 27) {
        constexpr int sg = BWD ? -1 : 1;
        const int qx = vx + sg * (t % 3 - 1), qy = vy + sg * (t / 3 % 3 - 1), qz = vz + sg * (t / 9 - 1);
        if (qx >= 0 && qx < W && qy >= 0 && qy < H && qz >= 0 && qz < D)
          v[j] = __ldg(reinterpret_cast<const uint4 *>(xcl + (((int64_t)qz * H + qy) * W + qx) * cp + ci0));
      }
    }
#pragma unroll
    for (int j = 0; j < 4; j++)
      *reinterpret_cast<uint4 *>(sa + (4 * half + j) * kLboA + (m >> 3) * 128 + (m & 7) * 16) = v[j];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (*(volatile int *)abort_flag != 0) {
      ok = false;
      break;
    }
    if (tid == 0) {
      if (!bar_wait(&loaded[s], (c >> 1) & 1)) {
        atomicExch(abort_flag, 1);
      } else {
        copy_pending = -1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int ks = 0; ks < kKC / 16; ks++) {
          const uint64_t da = smem_desc(su32(sa) + 2 * ks * kLboA, kLboA, 128);
          const uint64_t db = smem_desc(su32(sb) + 2 * ks * lbo_b, lbo_b, 128);
          const unsigned acc = (c > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         su32(&done[s]))
                     : "memory");
        issued = c + 1;
      }
    }
  }
  // a weight copy still in flight lands before the block's shared memory is released
  if (tid == 0 && copy_pending >= 0) bar_wait(&loaded[copy_pending & 1], (copy_pending >> 1) & 1);
  // every thread learns the count of committed chunks from thread 0
  __syncthreads();
  if (tid == 0) tslot[1] = (unsigned)issued;
  __syncthreads();
  issued = (int)tslot[1];
  if (*(volatile int *)abort_flag != 0) ok = false;
  // the last commit covers every MMA issued before it
  if (issued > 0 && !bar_wait(&done[(issued - 1) & 1], ((issued - 1) >> 1) & 1)) ok = false;
  ok = __syncthreads_and(ok) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its voxels), columns of its half
  const int q = warp & 3, chalf = warp >> 2;
  const int64_t pe = p0 + q * 32 + lane;
  const int cols_half = nt_n / 2;  // a multiple of 8
  for (int c0 = chalf * cols_half; c0 < (chalf + 1) * cols_half; c0 += 8) {
    uint32_t r[8];
    const unsigned ta = tmem + ((unsigned)(q * 32) << 16) + (unsigned)c0;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (pe < nv) {
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int co = nt * nt_n + c0 + j;
        if (co >= cout) continue;
        if constexpr (BWD) {
          static_cast<float *>(yout)[(int64_t)co * nv + pe] = ok ? __uint_as_float(r[j]) : __uint_as_float(0x7FC00000u);
        } else {
          float v = __uint_as_float(r[j]) + (bias ? __ldg(bias + co) : 0.f);
          if (relu) v = fmaxf(v, 0.f);
          const uint16_t o = ok ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : (uint16_t)0x7FC0;
          static_cast<uint16_t *>(yout)[(int64_t)co * nv + pe] = o;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

}  // namespace

namespace {

// ---- weight gradient: dW[m][co] = sum_p A[p][m] dy[co][p], m = t Cp + ci (tap t, input
// channel ci) and one more row m = 27 Cp of ones (the bias gradient), over a slice of
// kSlice voxels per block; then the slices summed in order.
//   - A is the im2col matrix of x in MN-major layout: a core matrix is 8 voxels (along K)
//     of 16 bytes along M (8 channels of one tap), so a row is one 16-byte load from the
//     channels-last copy; core (mg, kg) at mg * 1024 + kg * 128 (LBO = 128 along K, SBO =
//     1024 along M);
//   - B is the gradient in K-major layout, three BF16 parts per channel: a core row is 8
//     consecutive voxels of one channel and part (16 bytes of the split copy), core (kg, ng)
//     at kg * (N / 8) * 128 + ng * 128; each chunk runs 3 x 4 MMAs into one accumulator.
constexpr int kSlice = 2048;          // voxels per block (K per block before the split)
constexpr int kWgSbo = 1024;          // A: bytes between cores along M (8 cores along K)
constexpr int kWgABytes = 16 * kWgSbo;  // 128 rows x 64 voxels

// dys[s][co][p] = part s of dy[co][p] (as split_channels_last), zero for co >= cout or
// p >= nv: rows of nvp = nv rounded up to kSlice voxels
__global__ void split_channels_first(const float *__restrict__ dy, int64_t nv, int64_t nvp, int cout, int cop,
                                     uint16_t *__restrict__ dys) {
  const int64_t total = (int64_t)cop * nvp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i % nvp;
    const int co = (int)(i / nvp);
    float r = (co < cout && p < nv) ? __ldg(dy + (int64_t)co * nv + p) : 0.f;
#pragma unroll
    for (int part = 0; part < 3; part++) {
      const uint16_t h = __bfloat16_as_ushort(__float2bfloat16_rn(r));
      dys[((int64_t)part * cop + co) * nvp + p] = h;
      r -= __uint_as_float((uint32_t)h << 16);
    }
  }
}

__global__ void __launch_bounds__(kThreads, kMinBlocks)
    wgrad_kernel(const uint16_t *__restrict__ xcl, const uint16_t *__restrict__ dys, int cp, int cop, int nt_n,
                 int tmem_cols, int mrows, int D, int H, int W, int64_t nvp, float *__restrict__ part) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int bpart = nt_n * kKC * 2;  // one part's B chunk
  const int bbuf = 3 * bpart;
  uint64_t *done = reinterpret_cast<uint64_t *>(sm + 2 * kWgABytes + 2 * bbuf);  // [2]
  unsigned *tslot = reinterpret_cast<unsigned *>(done + 2);
  int *abort_flag = reinterpret_cast<int *>(tslot + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nv = (int64_t)D * H * W;
  // the row tiles of a slice are neighbours in the grid, so they read its voxels while L2
  // still holds them
  const int mt = blockIdx.x, slice = blockIdx.y, nt = blockIdx.z;
  const int64_t v0 = (int64_t)slice * kSlice;
  const unsigned lbo_b = (unsigned)(nt_n / 8) * 128u;
  const int nchunk = kSlice / kKC;
  if (tid == 0) {
    bar_init(&done[0]);
    bar_init(&done[1]);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tslot;
  const uint32_t idesc = instr_desc(nt_n) | (1u << 15);  // A MN-major

  int issued = 0;
  bool ok = true;
  for (int c = 0; c < nchunk; c++) {
    const int s = c & 1;
    unsigned char *sa = sm + s * kWgABytes;
    unsigned char *sb = sm + 2 * kWgABytes + s * bbuf;
    if (c >= 2 && !bar_wait(&done[s], ((c - 2) >> 1) & 1)) atomicExch(abort_flag, 1);
    const int64_t pc = v0 + (int64_t)c * kKC;  // first voxel of the chunk
    // A: 16 x 8 cores of 8 rows (voxels): 1024 rows, 4 per thread
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int r = tid + j * kThreads;  // row id: (mg, kg, row)
      const int mg = r >> 6, kg = (r >> 3) & 7, rw = r & 7;
      const int m0 = mt * 128 + mg * 8;
      const int t = m0 / cp, ci0 = m0 % cp;
      const int64_t p = pc + kg * 8 + rw;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (p < nv && m0 < mrows) {
        if (t < 27) {
          const int vx = (int)(p % W), vy = (int)(p / W % H), vz = (int)(p / W / H);
          const int qx = vx + t % 3 - 1, qy = vy + t / 3 % 3 - 1, qz = vz + t / 9 - 1;
          if (qx >= 0 && qx < W && qy >= 0 && qy < H && qz >= 0 && qz < D)
            v = __ldg(reinterpret_cast<const uint4 *>(xcl + (((int64_t)qz * H + qy) * W + qx) * cp + ci0));
        } else {
          v.x = 0x3F80u;  // the ones row: BF16 1.0 in its first element
        }
      }
      *reinterpret_cast<uint4 *>(sa + mg * kWgSbo + kg * 128 + rw * 16) = v;
    }
    // B: three parts of nt_n channels x 8 cores of 8 voxels
    for (int r = tid; r < 3 * nt_n * 8; r += kThreads) {
      const int part_i = r / (nt_n * 8), rr = r % (nt_n * 8);
      const int n = rr >> 3, kg = rr & 7;
      const int co = nt * nt_n + n;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (co < cop)
        v = __ldg(reinterpret_cast<const uint4 *>(dys + ((int64_t)part_i * cop + co) * nvp + pc + kg * 8));
      *reinterpret_cast<uint4 *>(sb + part_i * bpart + kg * lbo_b + (n >> 3) * 128 + (n & 7) * 16) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (*(volatile int *)abort_flag != 0) {
      ok = false;
      break;
    }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int pi = 0; pi < 3; pi++)
#pragma unroll
        for (int ks = 0; ks < kKC / 16; ks++) {
          const uint64_t da = smem_desc(su32(sa) + ks * 256, 128, kWgSbo);
          const uint64_t db = smem_desc(su32(sb) + pi * bpart + 2 * ks * lbo_b, lbo_b, 128);
          const unsigned acc = (c > 0 || pi > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(idesc), "r"(acc)
              : "memory");
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&done[s]))
                   : "memory");
    }
    issued = c + 1;  // every thread counts the chunks thread 0 committed
  }
  if (*(volatile int *)abort_flag != 0) ok = false;
  if (issued > 0 && !bar_wait(&done[(issued - 1) & 1], ((issued - 1) >> 1) & 1)) ok = false;
  ok = __syncthreads_and(ok) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // partial sums of this slice: part[slice][co][m], lanes = consecutive m
  const int q = warp & 3, chalf = warp >> 2;
  const int m = mt * 128 + q * 32 + lane;
  const int cols_half = nt_n / 2;
  const int mpad = gridDim.x * 128;
  for (int c0 = chalf * cols_half; c0 < (chalf + 1) * cols_half; c0 += 8) {
    uint32_t r[8];
    const unsigned ta = tmem + ((unsigned)(q * 32) << 16) + (unsigned)c0;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int co = nt * nt_n + c0 + j;
      part[((int64_t)slice * (gridDim.z * nt_n) + co) * mpad + m] = ok ? __uint_as_float(r[j]) : __uint_as_float(0x7FC00000u);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// dw[co][ci][t] and db[co]: the slices' partial sums added in slice order
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int nslice, int ncol, int mpad, int cin, int cout,
                                    int cp, float *__restrict__ dw, float *__restrict__ db) {
  const int64_t total = (int64_t)cout * (cin * 27 + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int co = (int)(i / (cin * 27 + 1)), j = (int)(i % (cin * 27 + 1));
    const bool bias = j == cin * 27;
    const int ci = bias ? 0 : j / 27, t = bias ? 0 : j % 27;
    const int m = bias ? 27 * cp : t * cp + ci;
    float acc = 0.f;
    for (int sl = 0; sl < nslice; sl++) acc += part[((int64_t)sl * ncol + co) * mpad + m];
    if (bias) {
      if (db) db[co] = acc;
    } else {
      dw[((int64_t)co * cin + ci) * 27 + t] = acc;
    }
  }
}

}  // namespace

// floats of partial sums conv3d_backward_weight_tc needs
int64_t conv3d_backward_weight_tc_work(int cin, int cout, int D, int H, int W) {
  const int cp = (cin + 7) / 8 * 8;
  const int64_t nv = (int64_t)D * H * W;
  const int64_t nslice = (nv + kSlice - 1) / kSlice;
  const int64_t mpad = ((int64_t)27 * cp + 1 + 127) / 128 * 128;
  const int n16 = (cout + 15) / 16 * 16;
  const int nt_n = n16 < kMaxN ? n16 : kMaxN;
  const int64_t ncol = (int64_t)((cout + nt_n - 1) / nt_n) * nt_n;
  return nslice * ncol * mpad;
}

cudaError_t conv3d_backward_weight_tc(const float *dy, const uint16_t *x, int cin, int cout, int D, int H, int W,
                                      float *dw, float *db, float *work, cudaStream_t s) {
  const int cp = (cin + 7) / 8 * 8;
  const int cop = (cout + 7) / 8 * 8;
  const int64_t nv = (int64_t)D * H * W;
  const int64_t nslice = (nv + kSlice - 1) / kSlice;
  const int64_t nvp = nslice * kSlice;
  const int mrows = 27 * cp + 1;
  const int mtiles = (mrows + 127) / 128;
  const int n16 = (cout + 15) / 16 * 16;
  const int nt_n = n16 < kMaxN ? n16 : kMaxN;
  const int ntiles = (cout + nt_n - 1) / nt_n;
  if (nslice > 65535 || ntiles > 65535) return cudaErrorInvalidValue;
  int tmem_cols = 32;
  while (tmem_cols < nt_n) tmem_cols *= 2;
  const int max_blocks = 512 / tmem_cols;
  int smem = 2 * kWgABytes + 2 * 3 * nt_n * kKC * 2 + 64;
  const int floor_smem = kSmPerSM / (max_blocks + 1) - 1024 + 16;
  if (smem < floor_smem) smem = floor_smem;
  if (smem > 232448) return cudaErrorInvalidValue;  // more than a block's shared memory
  cudaError_t e = cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  uint16_t *xcl = nullptr, *dys = nullptr;
  e = cudaMallocAsync(reinterpret_cast<void **>(&xcl), (size_t)nv * cp * sizeof(uint16_t), s);
  if (e != cudaSuccess) return e;
  e = cudaMallocAsync(reinterpret_cast<void **>(&dys), (size_t)3 * cop * nvp * sizeof(uint16_t), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(xcl, s);
    return e;
  }
  const int64_t xb = (nv * (cp / 8) + 255) / 256, yb = ((int64_t)cop * nvp + 255) / 256;
  to_channels_last<<<(unsigned)(xb < 65536 ? xb : 65536), 256, 0, s>>>(x, nv, cin, cp, xcl);
  split_channels_first<<<(unsigned)(yb < 65536 ? yb : 65536), 256, 0, s>>>(dy, nv, nvp, cout, cop, dys);
  wgrad_kernel<<<dim3((unsigned)mtiles, (unsigned)nslice, (unsigned)ntiles), kThreads, smem, s>>>(
      xcl, dys, cp, cop, nt_n, tmem_cols, mrows, D, H, W, nvp, work);
  const int64_t nout = (int64_t)cout * (cin * 27 + 1);
  wgrad_reduce_kernel<<<(unsigned)((nout + 255) / 256 < 65536 ? (nout + 255) / 256 : 65536), 256, 0, s>>>(
      work, (int)nslice, ntiles * nt_n, mtiles * 128, cin, cout, cp, dw, db);
  e = cudaGetLastError();
  const cudaError_t f1 = cudaFreeAsync(dys, s), f2 = cudaFreeAsync(xcl, s);
  return e != cudaSuccess ? e : (f1 != cudaSuccess ? f1 : f2);
}

namespace {

// the GEMM over n_out output rows (tiles of up to 256) with reduce channels cpa per tap;
// src: the channels-last source the caller's `prepare` fills (nv x cpa BF16)
template <bool BWD, class Prepare>
cudaError_t run_igemm(const uint16_t *w, const float *b, int n_out, int n_red, int cgrp, int cpa, int D, int H, int W,
                      int relu, void *y, cudaStream_t s, Prepare prepare) {
  const cudaError_t attr =
      cudaFuncSetAttribute(igemm_kernel<BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax);
  if (attr != cudaSuccess) return attr;
  const int64_t kpad = ((int64_t)27 * cpa + kKC - 1) / kKC * kKC;
  const int64_t nv = (int64_t)D * H * W;
  const int64_t nblk = (nv + kM - 1) / kM;
  if (nblk > 0x7fffffff || kpad / kKC > 0x7fffffff) return cudaErrorInvalidValue;
  const int nchunk = (int)(kpad / kKC);
  const int n16 = (n_out + 15) / 16 * 16;
  const int nt_n = n16 < kMaxN ? n16 : kMaxN;
  const int ntiles = (n_out + nt_n - 1) / nt_n;
  int tmem_cols = 32;
  while (tmem_cols < nt_n) tmem_cols *= 2;
  // shared memory per block: the buffers, raised where needed so that the blocks one SM
  // can hold never ask for more than its 512 TMEM columns (an allocation would wait)
  const int max_blocks = 512 / tmem_cols;
  int smem = kOffB + 2 * nt_n * kKC * 2 + 64;
  const int floor_smem = kSmPerSM / (max_blocks + 1) - 1024 + 16;
  if (smem < floor_smem) smem = floor_smem;
  if (smem > kSmemMax) smem = kSmemMax;
  const size_t pack_elems = (size_t)ntiles * nchunk * nt_n * kKC;
  uint16_t *wp = nullptr, *src = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&wp), pack_elems * sizeof(uint16_t), s);
  if (e != cudaSuccess) return e;
  e = cudaMallocAsync(reinterpret_cast<void **>(&src), (size_t)nv * cpa * sizeof(uint16_t), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(wp, s);
    return e;
  }
  const int64_t pblocks = ((int64_t)pack_elems + 255) / 256;
  pack_kernel<<<(unsigned)(pblocks < 4096 ? pblocks : 4096), 256, 0, s>>>(w, n_out, n_red, cgrp, cpa, BWD, nt_n,
                                                                           nchunk, ntiles, wp);
  const int64_t xblocks = (nv * (cpa / 8) + 255) / 256;
  prepare(src, (unsigned)(xblocks < 65536 ? xblocks : 65536));
  igemm_kernel<BWD><<<dim3((unsigned)nblk, (unsigned)ntiles), kThreads, smem, s>>>(
      src, wp, b, n_out, cpa, nt_n, tmem_cols, nchunk, D, H, W, relu, y);
  e = cudaGetLastError();
  const cudaError_t f1 = cudaFreeAsync(src, s), f2 = cudaFreeAsync(wp, s);
  return e != cudaSuccess ? e : (f1 != cudaSuccess ? f1 : f2);
}

}  // namespace

cudaError_t conv3d_forward_tc(const uint16_t *x, const uint16_t *w, const float *b, int cin, int cout, int D, int H,
                              int W, int relu, uint16_t *y, cudaStream_t s) {
  const int cp = (cin + 7) / 8 * 8;
  const int64_t nv = (int64_t)D * H * W;
  return run_igemm<false>(w, b, cout, cin, cp, cp, D, H, W, relu, y, s, [&](uint16_t *src, unsigned blocks) {
    to_channels_last<<<blocks, 256, 0, s>>>(x, nv, cin, cp, src);
  });
}

cudaError_t conv3d_backward_data_tc(const float *dy, const uint16_t *w, int cin, int cout, int D, int H, int W,
                                    float *dx, cudaStream_t s) {
  const int cop = (cout + 7) / 8 * 8;
  const int64_t nv = (int64_t)D * H * W;
  return run_igemm<true>(w, nullptr, cin, cout, cop, 3 * cop, D, H, W, 0, dx, s, [&](uint16_t *src, unsigned blocks) {
    split_channels_last<<<blocks, 256, 0, s>>>(dy, nv, cout, cop, src);
  });
}

}  // namespace fwi_tc
