// fwi_internal.h -- shared declarations between the C-ABI host code (fwi_api.cu)
// and the CUDA kernels (fwi_kernels.cu). Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fwi {

constexpr int kFields = 27;  // 3 levels x (3 displacement + 6 stress components)
constexpr int kLevelFields = 9;

// Mesh geometry and per-node coefficient sources, passed by value to kernels.
// ---- bounds-checked build (-DFWI_BOUNDS_CHECK)
// Every node number read from a list (shell, face, source and receiver points, snapshot
// and sweep lists) and every node a structured kernel derives from its tile is checked
// before any access: a failed check records (site << 48) | (index & (2^48 - 1)) in the
// context's error word (the first one wins) and the thread skips that node, so nothing out
// of range is read or written; the call then returns FWI_E_BOUNDS. In the normal build
// guard() is the constant true and the checks compile away.
enum BoundsSite {
  kSiteShell = 1, kSiteFace = 2, kSitePml = 3, kSiteInterior = 4, kSitePoint = 5, kSiteSample = 6,
  kSiteGradient = 7, kSiteSnapshot = 8, kSitePersist = 9
};
#ifdef FWI_BOUNDS_CHECK
__device__ __forceinline__ bool guard(unsigned long long *err, int site, long long idx, long long n) {
  if (idx >= 0 && idx < n) return true;
  if (err) atomicCAS(err, 0ull, ((unsigned long long)site << 48) | ((unsigned long long)idx & 0xffffffffffffull));
  return false;
}
#else
__device__ __forceinline__ bool guard(unsigned long long *, int, long long, long long) { return true; }
#endif

struct Geo {
  int n[3];         // nodes per axis (NI, NJ, NK)
  int px;           // row pitch: node (i, j, k) is at (k * NJ + j) * px + i; px = NI rounded up to 4
  int lo[3], hi[3]; // interior element range per axis, [lo, hi)
  int m[3];         // material-grid nodes per axis (2nx+1, 2ny+1, 2nz+1)
  int top_dir;      // 1: displacement fixed on k = 0 (top PML)
  int box_lo[3], box_hi[3];  // inclusive node box whose elements are all interior (no fixed faces)
  int64_t stride;   // floats per state field (>= node count, padded)
  int64_t nnode, nmat;
  float inv_h;      // 1 / h
  float rho;
  float inv_rho_h;  // 1 / (rho h)
  float wdetj;      // (h/2)^3
  const float *alpha[3];  // stretch alpha_s at each node coordinate, per axis
  const float *ialpha[3]; // 1 / alpha_s (rounded from FP64)
  const float *beta[3];   // stretch beta_s, 1/s
  const float *lam, *mu;  // interior material grid [k][j][i]
  const float *lam_n, *mu_n;  // lambda, mu at every node in the state layout (PML: clamped interface value)
  const int *shell;       // node numbers of the interface shell (see shell_kernel)
  int nshell;
  const int *face;        // node numbers of the PML nodes on the grid's outer faces
  int nface;
  unsigned long long *oob;  // error word of the bounds-checked build (else null)
  // bounded waits of interior_kernel on its plane copies: after wait_cycles clock cycles a
  // wait gives up, sets *status to FWI_E_TIMEOUT (6) and the block returns; copy_extra > 0
  // makes every plane barrier expect that many bytes more than the copy delivers (tests of
  // the timeout path only)
  int *status;
  long long wait_cycles;
  int copy_extra;
  // launch shapes (fwi_tune_tiles; they change no node's arithmetic)
  int int_kc;             // planes per block of interior_kernel
  int pml_seg;            // node pairs per x segment of a pml_kernel warp task (<= 32)
};

// One RK4 stage over every node (see fwi_kernels.cu).
//  stage 0: out = rate(Y)                   (fwi_rhs)
//  stage 1..3: out = X + cdt * rate(Y)   (stage 1: X must be Y; the kernels read Y only)
//  stage 4: out = (-X + Y2 + 2 Y3 + Y)/3 + cdt * rate(Y)   (out may alias X)
struct StageArgs {
  const float *Y;    // stage input
  const float *X;    // step start
  const float *Y2, *Y3;
  float *out;
  float cdt;
  int stage;
  float *hist;       // stage 4: interior displacement written here as [3][nmat], or null
  // a batch of nshot shots: shot b's buffers start sstride floats (history: hstride)
  // after shot b-1's; one launch of each stage kernel advances every shot of the batch
  int nshot;
  int64_t sstride, hstride;
};

// the buffers of shot `shot` of the batch
__host__ __device__ inline StageArgs shot_args(StageArgs a, int shot) {
  const int64_t o = (int64_t)shot * a.sstride;
  a.Y += o;
  if (a.X) a.X += o;
  if (a.Y2) a.Y2 += o;
  if (a.Y3) a.Y3 += o;
  a.out += o;
  if (a.hist) a.hist += (int64_t)shot * a.hstride;
  return a;
}

// a node number of the state layout: inside the grid and not in a row's padding
__device__ __forceinline__ bool node_ok(const Geo &g, int site, long long node) {
  return guard(g.oob, site, node, (long long)g.px * g.n[1] * g.n[2]) && guard(g.oob, site, node % g.px, g.n[0]);
}

// One RK4 stage is four kernels writing disjoint node sets; they read the same
// input and may run concurrently on different streams. Each launcher returns the
// number of kernels it launched:
//  launch_interior: nodes all of whose elements are interior (fwi_interior.cu); -1 if
//                   the tensor map of the stage input could not be encoded (Y not
//                   16-byte aligned, or the driver entry point missing);
//  launch_pml:      nodes all of whose elements are PML, off the outer faces (fwi_pml.cu);
//  launch_shell:    the interface shell (fwi_stage.cu) and the PML nodes on the
//                   outer faces of the grid (launch_pml_face, fwi_pml.cu).
int launch_interior(const Geo &g, const StageArgs &a, cudaStream_t s);
int launch_pml(const Geo &g, const StageArgs &a, bool adjoint, cudaStream_t s);
int launch_pml_face(const Geo &g, const StageArgs &a, bool adjoint, cudaStream_t s);
int launch_shell(const Geo &g, const StageArgs &a, bool adjoint, cudaStream_t s);
// raises the interior kernel's shared-memory limit on the current device
cudaError_t prepare_interior();

// A whole forward sweep (steps n0 .. n1 - 1) of nshot shots in one cooperative launch
// (fwi_stage.cu): every node takes the general per-node formulas of the shell kernel, the
// four stages of a step are separated by grid-wide barriers, and the source loads, the
// receiver samples and the displacement history are written by the threads that own the
// nodes. Each barrier's spin gives up after wait_cycles clock cycles and sets *status to
// FWI_E_TIMEOUT; the kernel then returns. A barrier waits for gridDim.x + extra arrivals
// (extra > 0 only to exercise that path).
struct PersistArgs {
  float *st[4];               // X, Y2, Y3, Y4 of the batch's first shot (shot b at + b sstride)
  int nshot;
  int64_t sstride;
  int n0, n1;                 // steps t_n -> t_{n+1} of the sweep
  float dt;
  const int *nodes;           // every node of the grid, (k, j, i) order
  int nall;
  const int64_t *src_node;    // shot b's source node and load vector (dir / M) at src_node[b], src_vec[3 b]
  const float *src_vec;
  const float *wave;          // wavelet samples every dt / 2
  const int *rec_of;          // node -> receiver index, or -1
  float *traces;              // shot b's traces at traces + b tstride, [n][nrec][3]
  int64_t tstride;
  int nrec;
  float *hist;                // displacement history, level n at hist + n hstep (shot b at + b hstride), or null
  int64_t hstep, hstride;
  unsigned *bar;              // [2]: arrival count and generation, zero before the launch
  int extra;
  long long wait_cycles;
  int *status;
};
cudaError_t launch_persistent_forward(const Geo &g, const PersistArgs &p, cudaStream_t s);

// Point loads on level-2 displacement rows of buffer `buf`:
// buf[9*2 + c][node[p]] += cdt * amp_p * vec[p][c], where
//   mode 0 (sources): amp_p = wave[widx0] (or 0.5*(wave[widx0]+wave[widx1]))
//   mode 1 (receiver residuals): amp_p = 1 and vec = minv * (resid[t0][p] (+ resid[t1][p])/2)
struct PointArgs {
  float *buf;
  int64_t stride;
  int npts;
  const int64_t *node;
  const float *vec;      // [npts][3]: dir * Minv (sources) or Minv replicated (receivers)
  const float *table;    // sources: wavelet samples at t = j dt/2; receivers: residual [nt][npts][3]
  int i0, i1;            // sample indices (i1 < 0: single sample)
  float cdt;
  int mode;
  // batch: shot b adds into buf + b * sstride; sources: its point is node[b], vec[b];
  // receivers: its residuals start at table + b * tstride
  int nshot;
  int64_t sstride, tstride;
  int64_t nnode_pad;          // valid node numbers: [0, nnode_pad) (bounds-checked build)
  unsigned long long *oob;    // error word of the bounds-checked build (else null)
};
void launch_point(const PointArgs &p, cudaStream_t s);

// traces[b][r][c] = buf[b * sstride + (9 + c) * stride + node[r]] for the nshot shots of a
// batch (trace of shot b at traces + b * tstride)
void launch_sample(const float *buf, int64_t stride, int nrec, const int64_t *node, float *traces,
                   cudaStream_t s, int nshot = 1, int64_t sstride = 0, int64_t tstride = 0,
                   unsigned long long *oob = nullptr);

// Gradient integrand of (C.1f)/(C.1g) at one time level, accumulated in FP64:
// gl[i] -= wdt * sum_e W detJ (div w)(div u), gm[i] -= wdt * sum_e W detJ 2 eps(w):eps(u),
// for the shots b = 0 .. nshot - 1 in order (adjoint state at w_state + b sstride, history
// level at u_hist + b hstride).
void launch_gradient(const Geo &g, const float *w_state, const float *u_hist, double wdt, double *gl,
                     double *gm, cudaStream_t s, int nshot = 1, int64_t sstride = 0, int64_t hstride = 0);

// resid = traces - observed (n values); partial sums of w_n dt e^2 / 2 per block into part;
// flag set to 1 on a non-finite trace value.
int misfit_blocks(int64_t n);
void launch_residual(const float *traces, const float *observed, float *resid, int64_t n,
                     int64_t per_step, int nsteps, double dt, double *part, int *flag, cudaStream_t s);
void launch_sum(const double *part, int nblocks, double *out, cudaStream_t s);

// Compact snapshot of nshot RK4 state sets (shot b at state + b sstride) into snap (shot b
// at snap + b snap_stride), or back (pack = false): u and udot (fields 9-11, 18-20) over
// all `stride` entries, then the other 21 fields at the npml PML nodes of `list`, each in
// a slot of npad >= npml floats (npad a multiple of 64). The restored state's other
// entries of those 21 fields must already be zero (no stage kernel writes them).
void launch_snapshot(float *state, float *snap, const int *list, int64_t npml, int64_t npad, int64_t stride,
                     int nshot, int64_t sstride, int64_t snap_stride, bool pack, cudaStream_t s,
                     unsigned long long *oob = nullptr);

// flag = 1 if any value of x (n doubles) is not finite.
void launch_check_finite(const double *x, int64_t n, int *flag, cudaStream_t s);
// g.lam_n / g.mu_n from the material grid (run whenever lam or mu change)
void launch_extend_material(const Geo &g, float *lam_n, float *mu_n, cudaStream_t s);

// reduced-space update helpers (fwi_opt.cu); vectors hold (lambda, mu) halves of nmat values
void opt_wdot(const double *a, const double *b, const double *w, int64_t nmat, double *part, double *out,
              cudaStream_t s);
void opt_axpby(double *y, double a, const double *x, double b, int64_t n, cudaStream_t s);
void opt_riesz(const double *gl, const double *gm, const double *mt, double *g, int64_t nmat, int mask,
               cudaStream_t s);
// plain dot product of n values (fixed-order reduction), part: >= 1024 doubles
void opt_dot(const double *a, const double *b, int64_t n, double *part, double *out, cudaStream_t s);
// regularisation term (8)/(9) of a field on the material grid (m nodes per axis):
// gradient (C.1b)-(C.1e) into g, functional into *value (device), part: >= 1024 doubles
void opt_regularization(const float *f, const int m[3], double h, bool tv, double eps, double *g, double *part,
                        double *value, cudaStream_t s);
void opt_trial(const double *m, const double *d, double alpha, float *lam, float *mu, int64_t nmat, unsigned *flags,
               cudaStream_t s);
void opt_pack(const float *lam, const float *mu, double *m, int64_t nmat, cudaStream_t s);
void opt_absmax(const double *x, int64_t n, unsigned long long *out, cudaStream_t s);

}  // namespace fwi
