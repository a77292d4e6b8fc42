// fwi_conv_tc.cu -- the 3x3x3 convolutions of the learned preconditioner on the
// fifth-generation tensor cores (tcgen05, sm_103a), as implicit GEMMs with BF16 operands
// in shared memory and FP32 accumulators in tensor memory (TMEM):
//
//   forward         y[co][p]  = act(b[co] + sum_t sum_ci w[co][ci][t] x[ci][p + off(t)])
//   backward data   dx[ci][p] = sum_t sum_co w[co][ci][t] dy[co][p - off(t)]
//   weight gradient dw[co][ci][t] = sum_p dy[co][p] x[ci][p + off(t)], db[co] = sum_p dy[co][p]
//
// t one of the 27 taps (kz, ky, kx; kx fastest), out-of-grid taps reading zero. Products
// of BF16 values are exact; the FP32 gradients of the backward passes enter as three BF16
// parts (hi, lo, lo2 with hi + lo + lo2 = dy to 2^-24), so their products stay exact too.
// Operands use the no-swizzle canonical layouts: a core matrix is 8 rows of 16 bytes
// stored contiguously; LBO is the byte stride between core matrices along K and SBO along
// M (or N), in both K-major and MN-major operands. One thread issues the tcgen05.mma and
// commits them to an mbarrier; the epilogue reads the accumulator with tcgen05.ld.
//
// The forward and backward-data passes use the tile form (tile_conv_kernel): a TMA box of
// the input with its halo, and the 27 taps as shifted MMA views of it. The weight gradient
// (wgrad_kernel) gathers im2col rows from a channels-last copy into an MN-major operand.
//
// Every mbarrier wait is bounded (about a second). A block whose wait gives up waits
// (bounded) for what it issued, writes NaN to its outputs (so the caller's loss turns
// non-finite) and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "fwi_conv_tc.h"

namespace fwi_tc {
namespace {

constexpr int kM = 128;          // MMA M: voxels (forward, backward data) or tap-channel rows
constexpr int kKC = 64;          // K per chunk of the weight gradient: 4 MMAs of K = 16
constexpr int kThreads = 256;    // threads of a weight-gradient block
constexpr int kMaxN = 256;       // output channels per block (MMA N <= 256)
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
// (bits 7-9, 10-12 = 1), N / 8 at bit 17, M / 16 at bit 24; both operands K-major (a caller
// sets bit 15 for an MN-major A)
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

// ---- tile form of the forward and backward-data convolutions. The source is a
// channel-group-major copy src[g][z][y][x][8] (G groups of 8 channels, zero past the real
// ones). A block owns an output tile of 8 (x) x 16 (y) voxels of one plane (MMA M = 128,
// m = 8 y + x) and up to 256 GEMM output channels (N). Per pass of Gp groups one TMA box
// (10 voxels x 8 channels as one 160-byte row, 18 rows, 3 planes, Gp groups) brings the tile with its halo into shared
// memory as [g][z][y][x][8], zero outside the grid. The A operand of tap t and group pair
// (2j, 2j + 1) is then a view of that box: core matrix y = the 8 x-voxels of row y (16 bytes
// each, contiguous), start at the tap's shifted voxel, SBO = one staged row (160 bytes),
// LBO = one staged group (8640 bytes). No thread gathers anything.
// Weights stream per (pass, tap) chunk (N x Gp x 8 BF16, K-major, packed once per call by
// tile_pack_kernel) through a ring of 4 buffers by bulk copies. One thread drives the copies
// and the MMAs; all threads run the epilogue.
constexpr int kTX = 8, kTY = 16;                // output tile (x, y)
constexpr int kBX = kTX + 2, kBY = kTY + 2;     // staged box with the halo
constexpr int kGroupBytes = kBX * kBY * 3 * 16;  // one staged group: 8640 bytes
constexpr int kRowBytes = kBX * 16;             // one staged row: 160 bytes
constexpr int kRingB = 4;                       // weight chunks in flight
constexpr int kTileThreads = 128;

// src[g][p][e] = x[8 g + e][p] (zero for channels >= cin)
__global__ void to_group_major(const uint16_t *__restrict__ x, int64_t nv, int cin, int G, uint16_t *__restrict__ src) {
  const int64_t total = nv * G;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i % nv;
    const int g = (int)(i / nv);
    uint32_t v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int e = 0; e < 8; e++)
      if (8 * g + e < cin) v[e >> 1] |= (uint32_t)__ldg(x + (int64_t)(8 * g + e) * nv + p) << (16 * (e & 1));
    *reinterpret_cast<uint4 *>(src + ((int64_t)g * nv + p) * 8) = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

// src[g][p][e] = part s of dy[co][p] for channel 8 g + e = s cop + co (three BF16 parts,
// as split_channels_last), zero for co >= cout and for channels past 3 cop
__global__ void split_group_major(const float *__restrict__ dy, int64_t nv, int cout, int cop, int G,
                                  uint16_t *__restrict__ src) {
  const int64_t total = nv * G;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i % nv;
    const int g = (int)(i / nv);
    uint32_t v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int e = 0; e < 8; e++) {
      const int c = 8 * g + e, part = c / cop, co = c % cop;
      if (part >= 3 || co >= cout) continue;
      float r = __ldg(dy + (int64_t)co * nv + p);
      uint16_t h = 0;
      for (int q = 0; q <= part; q++) {
        h = __bfloat16_as_ushort(__float2bfloat16_rn(r));
        r -= __uint_as_float((uint32_t)h << 16);
      }
      v[e >> 1] |= (uint32_t)h << (16 * (e & 1));
    }
    *reinterpret_cast<uint4 *>(src + ((int64_t)g * nv + p) * 8) = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

// weight chunks: for N tile nt, pass ps, tap t: N x (Gp x 8) K-major, core (kg, ng) at
// kg * (N / 8) * 128 + ng * 128. Source channel c = 8 (ps Gp + kg) + kk; forward: w[n][c][t];
// backward: c = s cop + co, w[co][n][t]
__global__ void tile_pack_kernel(const uint16_t *__restrict__ w, int n_rows, int n_red, int cop, bool bwd, int nt_n,
                                 int gp, int npass, int ntiles, uint16_t *__restrict__ out) {
  const int64_t chunk = (int64_t)nt_n * gp * 8;
  const int64_t total = (int64_t)ntiles * npass * 27 * chunk;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int kk = (int)(i % 8), row = (int)(i / 8 % 8);
    const int64_t r = i / 64;
    const int ng = (int)(r % (nt_n / 8)), kg = (int)(r / (nt_n / 8) % gp);
    const int64_t q = r / (nt_n / 8) / gp;  // (tile, pass, tap)
    const int t = (int)(q % 27), ps = (int)(q / 27 % npass), nt = (int)(q / 27 / npass);
    const int n = nt * nt_n + ng * 8 + row;
    const int c = 8 * (ps * gp + kg) + kk;
    uint16_t v = 0;
    if (n < n_rows) {
      if (!bwd) {
        if (c < n_red) v = w[((int64_t)n * n_red + c) * 27 + t];
      } else {
        const int part = c / cop, co = c % cop;
        if (part < 3 && co < n_red) v = w[((int64_t)co * n_rows + n) * 27 + t];
      }
    }
    out[i] = v;
  }
}

// the halo box of a tile: x and the 8 channels of a group form one row of 80 elements (the
// inner coordinate 8 (x0 - 1) is a multiple of 16 bytes), then y, z and the groups
__device__ __forceinline__ void tma_box(void *dst, const CUtensorMap *tm, int x0, int y0, int z0, int g0, uint64_t *b) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(8 * (x0 - 1)), "r"(y0 - 1), "r"(z0 - 1), "r"(g0), "r"(su32(b))
      : "memory");
}
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, uint64_t *b) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(b))
               : "memory");
}

template <bool BWD>
__global__ void __launch_bounds__(kTileThreads)
    tile_conv_kernel(const __grid_constant__ CUtensorMap tm, const uint16_t *__restrict__ wpack,
                     const float *__restrict__ bias, int n_out, int nt_n, int tmem_cols, int gp, int npass, int D, int H,
                     int W, int relu, void *__restrict__ yout) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int a_bytes = kGroupBytes * gp;
  const int b_bytes = nt_n * gp * 16;  // one chunk
  unsigned char *sa = sm;
  unsigned char *sb = sm + (a_bytes + 127) / 128 * 128;
  uint64_t *loaded = reinterpret_cast<uint64_t *>(sb + kRingB * b_bytes);  // [kRingB]
  uint64_t *done = loaded + kRingB;                                        // [kRingB]
  uint64_t *a_full = done + kRingB;
  unsigned *tslot = reinterpret_cast<unsigned *>(a_full + 1);
  int *okslot = reinterpret_cast<int *>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntx = (W + kTX - 1) / kTX;
  const int x0 = (blockIdx.x % ntx) * kTX, y0 = (blockIdx.x / ntx) * kTY, z0 = blockIdx.y;
  const int nt = blockIdx.z;
  const unsigned lbo_b = (unsigned)(nt_n / 8) * 128u;
  const int nch = npass * 27;
  const uint16_t *wt = wpack + (int64_t)nt * nch * nt_n * gp * 8;

  if (tid == 0) {
    for (int i = 0; i < kRingB; i++) {
      bar_init(&loaded[i]);
      bar_init(&done[i]);
    }
    bar_init(a_full);
    *okslot = 1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

  if (tid == 0) {
    const uint32_t idesc = instr_desc(nt_n);
    bool ok = true;
    int copies = 0, committed = 0;  // weight chunks issued / chunks whose MMAs are committed
    int a_pending = -1;  // the pass whose box copy has not been waited for
    auto chunk_src = [&](int c) { return wt + (int64_t)c * nt_n * gp * 8; };
    for (; copies < kRingB && copies < nch; copies++) bulk_copy(sb + copies * b_bytes, chunk_src(copies), b_bytes, &loaded[copies]);
    for (int c = 0; c < nch && ok; c++) {
      const int ps = c / 27, t = c % 27, s = c % kRingB;
      if (t == 0) {
        // a new pass: the previous pass's MMAs read the box, so they finish first
        if (c > 0 && !bar_wait(&done[(c - 1) % kRingB], ((c - 1) / kRingB) & 1)) {
          ok = false;
          break;
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(a_full)), "r"(a_bytes)
                     : "memory");
        tma_box(sa, &tm, x0, y0, z0, ps * gp, a_full);
        a_pending = ps;
        if (!bar_wait(a_full, ps & 1)) {
          ok = false;
          break;
        }
        a_pending = -1;
      }
      if (!bar_wait(&loaded[s], (c / kRingB) & 1)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // the tap's shift (mirrored for the backward pass), as a staged voxel offset
      const int dx = t % 3 - 1, dy = t / 3 % 3 - 1, dz = t / 9 - 1;
      const int sx = BWD ? 1 - dx : 1 + dx, sy = BWD ? 1 - dy : 1 + dy, sz = BWD ? 1 - dz : 1 + dz;
      const unsigned a0 = su32(sa) + (unsigned)(((sz * kBY) + sy) * kBX + sx) * 16u;
      const unsigned b0 = su32(sb + s * b_bytes);
      for (int j = 0; j < gp / 2; j++) {
        const uint64_t da = smem_desc(a0 + 2 * j * kGroupBytes, kGroupBytes, kRowBytes);
        const uint64_t db = smem_desc(b0 + 2 * j * lbo_b, lbo_b, 128);
        const unsigned acc = (c > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&done[s]))
                   : "memory");
      committed = c + 1;
      // refill the buffer of chunk c - 1 (its MMAs ran before this chunk's) with chunk c + 3
      if (c >= 1 && copies < nch) {
        const int sp = (c - 1) % kRingB;
        if (!bar_wait(&done[sp], ((c - 1) / kRingB) & 1)) {
          ok = false;
          break;
        }
        bulk_copy(sb + sp * b_bytes, chunk_src(copies), b_bytes, &loaded[sp]);
        copies++;
      }
    }
    // copies still in flight land before the shared memory is released
    if (a_pending >= 0) bar_wait(a_full, a_pending & 1);
    for (int c = committed; c < copies; c++) bar_wait(&loaded[c % kRingB], (c / kRingB) & 1);
    if (committed > 0 && !bar_wait(&done[(committed - 1) % kRingB], ((committed - 1) / kRingB) & 1)) ok = false;
    if (committed < nch) ok = false;
    *okslot = ok ? 1 : 0;
  }
  __syncthreads();
  const bool ok = *(volatile int *)okslot != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warp q reads TMEM lanes 32 q .. 32 q + 31 (tile rows 4 q .. 4 q + 3)
  const int m = warp * 32 + lane;
  const int ox = x0 + (m & 7), oy = y0 + (m >> 3);
  const bool in = ox < W && oy < H;
  const int64_t nv = (int64_t)D * H * W;
  const int64_t pe = ((int64_t)z0 * H + oy) * W + ox;
  for (int c0 = 0; c0 < nt_n; c0 += 8) {
    uint32_t r[8];
    const unsigned ta = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (in) {
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int co = nt * nt_n + c0 + j;
        if (co >= n_out) continue;
        if constexpr (BWD) {
          static_cast<float *>(yout)[(int64_t)co * nv + pe] = ok ? __uint_as_float(r[j]) : __uint_as_float(0x7FC00000u);
        } else {
          float v = __uint_as_float(r[j]) + (bias ? __ldg(bias + co) : 0.f);
          if (relu) v = fmaxf(v, 0.f);
          static_cast<uint16_t *>(yout)[(int64_t)co * nv + pe] =
              ok ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : (uint16_t)0x7FC0;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
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

// the tile form over a group-major source of G groups (G a multiple of 4) that `prepare`
// fills; n_rows GEMM output channels, n_red real source channels (forward: cin; backward:
// cout, with cop = the part stride)
template <bool BWD, class Prepare>
cudaError_t run_tile(const uint16_t *w, const float *b, int n_rows, int n_red, int cop, int G, int D, int H, int W,
                     int relu, void *y, cudaStream_t s, Prepare prepare) {
  const EncodeTiled enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const int n16 = (n_rows + 15) / 16 * 16;
  const int nt_n = n16 < kMaxN ? n16 : kMaxN;
  const int ntiles = (n_rows + nt_n - 1) / nt_n;
  int tmem_cols = 32;
  while (tmem_cols < nt_n) tmem_cols *= 2;
  // groups per pass: the largest of 12, 8, 4 that divides G and fits shared memory
  int gp = 0, smem = 0;
  for (int cand : {12, 8, 4}) {
    if (G % cand) continue;
    const int need = (kGroupBytes * cand + 127) / 128 * 128 + kRingB * nt_n * cand * 16 + 2 * kRingB * 8 + 32;
    if (need <= 200 * 1024) {
      gp = cand;
      smem = need;
      break;
    }
  }
  if (gp == 0) return cudaErrorInvalidValue;
  const int npass = G / gp;
  const int max_blocks = 512 / tmem_cols;
  const int floor_smem = kSmPerSM / (max_blocks + 1) - 1024 + 16;
  if (smem < floor_smem) smem = floor_smem;
  const int64_t nv = (int64_t)D * H * W;
  const int64_t tiles_xy = (int64_t)((W + kTX - 1) / kTX) * ((H + kTY - 1) / kTY);
  if (tiles_xy > 0x7fffffff || D > 65535 || ntiles > 65535) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(tile_conv_kernel<BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const size_t pack_elems = (size_t)ntiles * npass * 27 * nt_n * gp * 8;
  uint16_t *wp = nullptr, *src = nullptr;
  e = cudaMallocAsync(reinterpret_cast<void **>(&wp), pack_elems * sizeof(uint16_t), s);
  if (e != cudaSuccess) return e;
  e = cudaMallocAsync(reinterpret_cast<void **>(&src), (size_t)G * nv * 8 * sizeof(uint16_t), s);
  if (e != cudaSuccess) {
    cudaFreeAsync(wp, s);
    return e;
  }
  // tensor map of src as (x and 8 channels: 8 W, H, D, G) BF16; boxes (80, 18, 3, gp), zero
  // outside the grid
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  const cuuint64_t dims[4] = {(cuuint64_t)W * 8, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)G};
  const cuuint64_t pitch[3] = {(cuuint64_t)W * 16, (cuuint64_t)W * H * 16, (cuuint64_t)nv * 16};
  const cuuint32_t box[4] = {kBX * 8, kBY, 3, (cuuint32_t)gp};
  const cuuint32_t step[4] = {1, 1, 1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, src, dims, pitch, box, step, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS) {
    cudaFreeAsync(src, s);
    cudaFreeAsync(wp, s);
    return cudaErrorInvalidValue;
  }
  const int64_t pblocks = ((int64_t)pack_elems + 255) / 256;
  tile_pack_kernel<<<(unsigned)(pblocks < 4096 ? pblocks : 4096), 256, 0, s>>>(w, n_rows, n_red, cop, BWD, nt_n, gp,
                                                                               npass, ntiles, wp);
  const int64_t xblocks = (nv * G + 255) / 256;
  prepare(src, (unsigned)(xblocks < 65536 ? xblocks : 65536));
  tile_conv_kernel<BWD><<<dim3((unsigned)tiles_xy, (unsigned)D, (unsigned)ntiles), kTileThreads, smem, s>>>(
      tm, wp, b, n_rows, nt_n, tmem_cols, gp, npass, D, H, W, relu, y);
  e = cudaGetLastError();
  const cudaError_t f1 = cudaFreeAsync(src, s), f2 = cudaFreeAsync(wp, s);
  return e != cudaSuccess ? e : (f1 != cudaSuccess ? f1 : f2);
}

}  // namespace


cudaError_t conv3d_forward_tc(const uint16_t *x, const uint16_t *w, const float *b, int cin, int cout, int D, int H,
                              int W, int relu, uint16_t *y, cudaStream_t s) {
  const int G = (cin + 31) / 32 * 4;  // groups of 8 channels, a multiple of 4
  const int64_t nv = (int64_t)D * H * W;
  return run_tile<false>(w, b, cout, cin, 0, G, D, H, W, relu, y, s, [&](uint16_t *src, unsigned blocks) {
    to_group_major<<<blocks, 256, 0, s>>>(x, nv, cin, G, src);
  });
}

cudaError_t conv3d_backward_data_tc(const float *dy, const uint16_t *w, int cin, int cout, int D, int H, int W,
                                    float *dx, cudaStream_t s) {
  const int cop = (cout + 7) / 8 * 8;
  const int G = (3 * cop / 8 + 3) / 4 * 4;
  const int64_t nv = (int64_t)D * H * W;
  return run_tile<true>(w, nullptr, cin, cout, cop, G, D, H, W, 0, dx, s, [&](uint16_t *src, unsigned blocks) {
    split_group_major<<<blocks, 256, 0, s>>>(dy, nv, cout, cop, G, src);
  });
}

}  // namespace fwi_tc
