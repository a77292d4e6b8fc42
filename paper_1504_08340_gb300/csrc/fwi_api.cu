// fwi_api.cu -- host side of the C ABI declared in include/fwi.h.
//
// The host code validates arguments, owns the device buffers, builds the
// small per-axis tables (PML stretch functions, wavelet samples, lumped-mass
// inverses at the loaded nodes) in FP64 and drives the time loops; every step
// of the wavefield, misfit and gradient arithmetic runs in the kernels of
// fwi_kernels.cu on the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/fwi.h"
#include "fwi_internal.h"

struct fwi_ctx {
  fwi_config cfg{};
  fwi::Geo geo{};
  cudaStream_t stream = nullptr;
  cudaStream_t side[2] = {nullptr, nullptr};  // the stage's kernels fork onto these and join back
  cudaStream_t cap = nullptr;  // sweeps are recorded on this stream (the caller's may be the legacy one)
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  bool cuda_failed = false;
  std::string err;
  int64_t nelem = 0, npml_nodes = 0;

  float *state[4] = {nullptr, nullptr, nullptr, nullptr};  // X, Y2, Y3, Y4; each [batch][27][stride]
  int batch = 1;  // shots advanced together by one launch of each stage kernel (fwi_set_shot_batch)
  float *d_alpha[3] = {nullptr, nullptr, nullptr};
  float *d_beta[3] = {nullptr, nullptr, nullptr};
  float *d_ialpha[3] = {nullptr, nullptr, nullptr};
  std::vector<double> h_alpha[3], h_beta[3];
  float *d_lam = nullptr, *d_mu = nullptr;
  float *d_lam_n = nullptr, *d_mu_n = nullptr;  // the material in the state layout (Geo::lam_n)
  int *d_shell = nullptr, *d_face = nullptr;
  bool have_material = false;

  int nshots = 0;
  std::vector<int64_t> src_node;
  std::vector<double> src_dir;
  int wavelet = 0;
  double wparams[3] = {0, 0, 0};
  float *d_wave = nullptr;
  int64_t *d_src_node = nullptr;
  float *d_src_vec = nullptr;

  int nrec = 0;
  std::vector<int64_t> rec_node;
  int64_t *d_rec_node = nullptr;
  float *d_rec_vec = nullptr;

  float *d_traces = nullptr, *d_obs = nullptr, *d_resid = nullptr;
  double *d_part = nullptr, *d_J = nullptr;
  int d_J_cap = 0;
  int *d_flag = nullptr;
  float *d_hist = nullptr;
  size_t hist_cap = 0;  // history slots (levels) d_hist holds
  double *d_gl = nullptr, *d_gm = nullptr;

  // forward-state checkpointing of the adjoint sweep (fwi_set_checkpointing)
  int ckpt = 0;                 // 0: full displacement history; > 0: snapshot interval; < 0: ceil(sqrt(N))
  float *rstate[4] = {nullptr, nullptr, nullptr, nullptr};  // RK4 state set of the forward recompute
  float *d_snap = nullptr;      // compact snapshots of X (snap_floats each), [shot][segment]
  size_t snap_cap = 0;          // snapshots d_snap holds
  int *d_pml_list = nullptr;    // the PML nodes (nodes of at least one PML element), (k, j, i) order
  unsigned long long *d_oob = nullptr;  // error word of the bounds-checked build (see fwi::guard)

  // reduced-space update (fwi_step): model, gradient, direction, L-BFGS pairs (FP64)
  int lb_cap = 0, lb_count = 0, lb_head = 0;
  bool lb_have_prev = false;
  std::vector<double> lb_rho;
  double *d_mt = nullptr, *d_m = nullptr, *d_mprev = nullptr, *d_g = nullptr, *d_gprev = nullptr;
  double *d_dir = nullptr, *d_S = nullptr, *d_Yv = nullptr, *d_opart = nullptr, *d_oscal = nullptr;
  unsigned *d_oflags = nullptr;
  unsigned long long *d_omax = nullptr;
  // regularisation (fwi_regularization): gradients, block partials, functional values
  double *d_rg = nullptr, *d_rpart = nullptr, *d_rval = nullptr;

  // recorded sweeps (fwi_set_graphs): kind 0 forward sweep, 1 adjoint sweep over the stored
  // history, 2 one checkpoint segment (recompute and adjoint); a, b, g identify the shots
  // and the segment
  struct Graph {
    int kind, a, b, g;
    const float *st;
    uint64_t gen;
    cudaGraphExec_t exec;
    int64_t launches[4];
  };
  bool graphs = false;
  std::vector<Graph> gcache;

  // persistent forward sweeps (fwi_set_persistent)
  bool persistent = false;
  double wait_ms = 1000.0;
  int bar_extra = 0;
  int *d_all = nullptr, *d_rec_of = nullptr;  // every node; node -> receiver index
  unsigned *d_bar = nullptr;
  int *d_status = nullptr;                    // FWI_E_TIMEOUT when a bounded device wait gave up

  bool timing = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
  std::vector<int> ev_class;
  double t_ms[4] = {0, 0, 0, 0};
  int64_t t_launch[4] = {0, 0, 0, 0};
};

namespace {

fwi_status fail(fwi_ctx *c, fwi_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) {
    c->err = buf;
    if (s == FWI_E_CUDA) c->cuda_failed = true;
  }
  return s;
}

#define CUDA_TRY(ctx, call)                                                                          \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? FWI_E_NOMEM : FWI_E_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                                \
  } while (0)

#define TRY(expr)                     \
  do {                                \
    fwi_status s_ = (expr);           \
    if (s_ != FWI_OK) return s_;      \
  } while (0)

// bumped by every device allocation and free: a recorded CUDA graph holds raw pointers, so
// a cached graph is replayed only while no buffer has changed since it was recorded
std::atomic<uint64_t> g_alloc_gen{0};

template <class T>
fwi_status dalloc(fwi_ctx *c, T **p, size_t n) {
  if (*p) return FWI_OK;
  g_alloc_gen++;
  cudaError_t e = cudaMalloc((void **)p, n * sizeof(T) + 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, FWI_E_NOMEM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
  }
  return FWI_OK;
}

template <class T>
void dfree(T *&p) {
  if (p) {
    g_alloc_gen++;
    cudaFree((void *)p);
  }
  p = nullptr;
}

// floats of one shot's RK4 state set, of one shot's traces (or residuals), of one history level
size_t set_floats(const fwi_ctx *c) { return (size_t)fwi::kFields * c->geo.stride; }
size_t trace_floats(const fwi_ctx *c) { return (size_t)(c->cfg.nsteps + 1) * c->nrec * 3; }
size_t level_floats(const fwi_ctx *c) { return (size_t)3 * c->geo.nmat; }
// floats of one shot's compact snapshot: u and udot everywhere, the other 21 fields at the
// PML nodes (see fwi::launch_snapshot), each PML slot padded to a multiple of 64 floats
int64_t pml_pad(const fwi_ctx *c) { return (c->npml_nodes + 63) / 64 * 64; }
size_t snap_floats(const fwi_ctx *c) { return (size_t)6 * c->geo.stride + (size_t)21 * pml_pad(c); }

bool is_dirichlet(const fwi_ctx *c, int i, int j, int k) {
  const int *n = c->geo.n;
  return i == 0 || i == n[0] - 1 || j == 0 || j == n[1] - 1 || k == n[2] - 1 || (c->geo.top_dir && k == 0);
}

// number of elements containing node coordinate cc along axis ax
int elems_along(const fwi_ctx *c, int ax, int cc) {
  if (cc & 1) return 1;
  return (cc >= 2) + (cc <= c->geo.n[ax] - 3);
}

// lumped u-row mass rho * a(x) * W * detJ * (elements around the node) -- (3a)
double mass_u(const fwi_ctx *c, int i, int j, int k) {
  const int cc[3] = {i, j, k};
  double w = 1.0, nel = 1.0, a = 1.0, hh = 0.5 * c->cfg.h;
  for (int ax = 0; ax < 3; ax++) {
    w *= (cc[ax] & 1) ? 4.0 / 3.0 : 1.0 / 3.0;
    nel *= elems_along(c, ax, cc[ax]);
    a *= c->h_alpha[ax][cc[ax]];
  }
  return c->cfg.rho * a * w * hh * hh * hh * nel;
}

fwi_status check_stream(fwi_ctx *c) {
  if (c->cuda_failed) return fail(c, FWI_E_CUDA, "context unusable after an earlier CUDA error: %s", c->err.c_str());
  return FWI_OK;
}

void drop_graphs(fwi_ctx *c) {
  for (auto &e : c->gcache) cudaGraphExecDestroy(e.exec);
  c->gcache.clear();
}

// Runs body() (stream work on the context's stream and its side streams) directly, or, with
// graphs on (and kernel timing off), replays it as a CUDA graph: the first call with a
// given key records body() by stream capture; later calls with the same key and no device
// allocation in between launch the recorded graph, which issues the same kernels with the
// same arguments in the same order.
template <class F>
fwi_status graphed(fwi_ctx *c, int kind, int a, int b, int g, F body) {
  if (!c->graphs || c->timing || c->persistent) return body();
  const uint64_t gen = g_alloc_gen.load();
  for (const auto &e : c->gcache)
    if (e.gen != gen) {
      drop_graphs(c);
      break;
    }
  for (const auto &e : c->gcache)
    if (e.kind == kind && e.a == a && e.b == b && e.g == g && e.st == c->state[0]) {
      CUDA_TRY(c, cudaGraphLaunch(e.exec, c->stream));
      for (int i = 0; i < 4; i++) c->t_launch[i] += e.launches[i];
      return FWI_OK;
    }
  if (c->gcache.size() >= 512) drop_graphs(c);
  int64_t before[4];
  for (int i = 0; i < 4; i++) before[i] = c->t_launch[i];
  // record on the library's own stream (nothing runs while recording); the graph is then
  // launched on the context's stream, after the work already queued there
  const cudaStream_t user = c->stream;
  CUDA_TRY(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  c->stream = c->cap;
  const fwi_status st = body();
  c->stream = user;
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(c->cap, &graph);
  if (st != FWI_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ee != cudaSuccess) return fail(c, FWI_E_CUDA, "stream capture of a sweep failed: %s", cudaGetErrorString(ee));
  fwi_ctx::Graph e{kind, a, b, g, c->state[0], gen, nullptr, {0, 0, 0, 0}};
  const cudaError_t ei = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return fail(c, FWI_E_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
  for (int i = 0; i < 4; i++) e.launches[i] = c->t_launch[i] - before[i];
  c->gcache.push_back(e);
  CUDA_TRY(c, cudaGraphLaunch(e.exec, c->stream));
  return FWI_OK;
}

// ---- timing of kernel classes
void time_begin(fwi_ctx *c, cudaEvent_t *e0) {
  *e0 = nullptr;
  if (!c->timing) return;
  if (c->ev_free.size() < 2) {
    for (int i = 0; i < 256; i++) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) break;
      c->ev_free.push_back(e);
    }
  }
  if (c->ev_free.empty()) return;
  *e0 = c->ev_free.back();
  c->ev_free.pop_back();
  cudaEventRecord(*e0, c->stream);
}

void time_end(fwi_ctx *c, cudaEvent_t e0, int cls) {
  c->t_launch[cls]++;
  c->t_launch[3]++;
  if (!c->timing || !e0) return;
  if (c->ev_free.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    c->ev_free.push_back(e);
  }
  cudaEvent_t e1 = c->ev_free.back();
  c->ev_free.pop_back();
  cudaEventRecord(e1, c->stream);
  c->ev_pending.push_back({e0, e1});
  c->ev_class.push_back(cls);
}

fwi_status time_flush(fwi_ctx *c) {
  if (c->ev_pending.empty()) return FWI_OK;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < c->ev_pending.size(); i++) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev_pending[i].first, c->ev_pending[i].second);
    c->t_ms[c->ev_class[i]] += ms;
    c->ev_free.push_back(c->ev_pending[i].first);
    c->ev_free.push_back(c->ev_pending[i].second);
  }
  c->ev_pending.clear();
  c->ev_class.clear();
  return FWI_OK;
}

// FWI_E_BOUNDS if a guarded index was out of range (bounds-checked build), FWI_E_TIMEOUT
// if a bounded device wait gave up, since the last check (synchronises)
fwi_status check_status(fwi_ctx *c) {
  if (c->d_oob) {
    unsigned long long w = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&w, c->d_oob, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (w != 0) {
      CUDA_TRY(c, cudaMemsetAsync(c->d_oob, 0, sizeof(w), c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      return fail(c, FWI_E_BOUNDS, "index %lld out of range at check site %d", (long long)(w & 0xffffffffffffull),
                  (int)(w >> 48));
    }
  }
  if (!c->d_status) return FWI_OK;
  int st = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (st != 0) {
    CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return fail(c, FWI_E_TIMEOUT, "a bounded device wait gave up (a grid barrier of the persistent sweep, or a "
                                  "plane copy of the interior kernel)");
  }
  return FWI_OK;
}

fwi_status stage(fwi_ctx *c, bool adj, const fwi::StageArgs &a) {
  cudaEvent_t e0;
  time_begin(c, &e0);
  // fork: interior and interface/face kernels on the side streams, bulk PML here
  CUDA_TRY(c, cudaEventRecord(c->ev_fork, c->stream));
  for (int i = 0; i < 2; i++) CUDA_TRY(c, cudaStreamWaitEvent(c->side[i], c->ev_fork, 0));
  const int ni = fwi::launch_interior(c->geo, a, c->side[0]);
  if (ni < 0) return fail(c, FWI_E_CUDA, "no tensor map for the stage input (not 16-byte aligned, or no driver entry)");
  const int nk = ni + fwi::launch_shell(c->geo, a, adj, c->side[1]) + fwi::launch_pml(c->geo, a, adj, c->stream);
  for (int i = 0; i < 2; i++) {
    CUDA_TRY(c, cudaEventRecord(c->ev_join[i], c->side[i]));
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_join[i], 0));
  }
  time_end(c, e0, 0);
  c->t_launch[3] += nk - 1;  // time_end counted the stage once; count its kernels
  CUDA_TRY(c, cudaGetLastError());
  if (c->ev_pending.size() > 400000) TRY(time_flush(c));
  return FWI_OK;
}

fwi_status point(fwi_ctx *c, const fwi::PointArgs &p) {
  fwi::launch_point(p, c->stream);
  c->t_launch[2]++;
  c->t_launch[3]++;
  CUDA_TRY(c, cudaGetLastError());
  return FWI_OK;
}

fwi_status zero_state(fwi_ctx *c) {
  const size_t bytes = sizeof(float) * set_floats(c) * c->batch;
  for (int b = 0; b < 4; b++) CUDA_TRY(c, cudaMemsetAsync(c->state[b], 0, bytes, c->stream));
  return FWI_OK;
}

// One RK4 step (4 fused stage kernels) of the forward (adj = false) or the
// reversed-time adjoint (adj = true) system, with the point loads of the step (source
// samples, or receiver residuals). Both run the forward stage kernels (see below); the
// transposed kernels serve fwi_rhs's adjoint rate.
// nb shots (shot0 .. shot0 + nb - 1 for the sources) advance together; shot b's history
// level goes to hist_slot + b * hstride
fwi_status rk4_step(fwi_ctx *c, bool adj, int n, int shot0, int nb, float *hist_slot, int64_t hstride) {
  const float dt = (float)c->cfg.dt;
  float *X = c->state[0], *Y2 = c->state[1], *Y3 = c->state[2], *Y4 = c->state[3];
  const float *ins[4] = {X, Y2, Y3, Y4};
  float *outs[4] = {Y2, Y3, Y4, X};
  const float cdt[4] = {0.5f * dt, 0.5f * dt, dt, dt / 6.0f};
  const int N = c->cfg.nsteps;
  for (int s = 0; s < 4; s++) {
    fwi::StageArgs a{};
    a.Y = ins[s];
    a.X = X;
    a.Y2 = Y2;
    a.Y3 = Y3;
    a.out = outs[s];
    a.cdt = cdt[s];
    a.stage = s + 1;
    a.hist = (s == 3) ? hist_slot : nullptr;
    a.nshot = nb;
    a.sstride = (int64_t)set_floats(c);
    a.hstride = hstride;
    // The adjoint sweep advances (w, W = tau(T)) rather than (w, T): tau is linear,
    // node-local and constant in time, so applied to the transposed system's stress rows it
    // gives exactly the forward system's form (tau on P(H) in the S rows, the plain stress
    // columns in the u rows), and the forward stage kernels advance it. The displacement w,
    // all the gradient reads, is the same; the stress slots hold tau(T).
    TRY(stage(c, false, a));
    fwi::PointArgs p{};
    p.nnode_pad = (int64_t)c->geo.px * c->geo.n[1] * c->geo.n[2];
    p.oob = c->geo.oob;
    p.buf = outs[s];
    p.stride = c->geo.stride;
    p.cdt = cdt[s];
    p.nshot = nb;
    p.sstride = (int64_t)set_floats(c);
    p.tstride = (int64_t)trace_floats(c);
    if (!adj) {
      // stage times t_n, t_n + dt/2, t_n + dt/2, t_n + dt; wavelet sampled every dt/2
      p.mode = 0;
      p.npts = 1;
      p.node = c->d_src_node + shot0;
      p.vec = c->d_src_vec + 3 * shot0;
      p.table = c->d_wave;
      p.i0 = (s == 0) ? 2 * n : (s == 3 ? 2 * n + 2 : 2 * n + 1);
      p.i1 = -1;
    } else {
      // reversed time: s_m <-> t_{N-m}; half steps use the mean of the two samples
      p.mode = 1;
      p.npts = c->nrec;
      p.node = c->d_rec_node;
      p.vec = c->d_rec_vec;
      p.table = c->d_resid;
      p.i0 = (s == 3) ? N - n - 1 : N - n;
      p.i1 = (s == 1 || s == 2) ? N - n - 1 : -1;
    }
    TRY(point(c, p));
  }
  return FWI_OK;
}

fwi_status require_ready(fwi_ctx *c, int shot0, int nshots) {
  TRY(check_stream(c));
  if (!c->state[0]) return fail(c, FWI_E_STATE, "no RK4 state buffers (a shot batch allocation failed)");
  if (!c->have_material) return fail(c, FWI_E_STATE, "material not set");
  if (c->nshots <= 0) return fail(c, FWI_E_STATE, "sources not set");
  if (c->nrec <= 0) return fail(c, FWI_E_STATE, "receivers not set");
  if (shot0 < 0 || nshots < 1 || shot0 + nshots > c->nshots)
    return fail(c, FWI_E_INVAL, "shot range [%d, %d) outside [0, %d)", shot0, shot0 + nshots, c->nshots);
  return FWI_OK;
}

fwi_status ensure_trace_buffers(fwi_ctx *c) {
  const size_t nt = trace_floats(c) * c->batch;
  TRY(dalloc(c, &c->d_traces, nt));
  TRY(dalloc(c, &c->d_obs, nt));
  TRY(dalloc(c, &c->d_resid, nt));
  TRY(dalloc(c, &c->d_part, 1024));
  TRY(dalloc(c, &c->d_flag, 4));
  return FWI_OK;
}

// the PML node list of the compact snapshots, built on first use
fwi_status ensure_pml_list(fwi_ctx *c) {
  if (c->d_pml_list) return FWI_OK;
  const fwi::Geo &g = c->geo;
  std::vector<char> all_rd[3];  // per axis: every element along it around the coordinate is interior
  for (int ax = 0; ax < 3; ax++) {
    all_rd[ax].assign(g.n[ax], 0);
    for (int cc = 0; cc < g.n[ax]; cc++) {
      bool all = true;
      if (cc & 1) {
        const int e = (cc - 1) / 2;
        all = e >= g.lo[ax] && e < g.hi[ax];
      } else {
        if (cc >= 2) all = all && (cc / 2 - 1 >= g.lo[ax] && cc / 2 - 1 < g.hi[ax]);
        if (cc <= g.n[ax] - 3) all = all && (cc / 2 >= g.lo[ax] && cc / 2 < g.hi[ax]);
      }
      all_rd[ax][cc] = all;
    }
  }
  std::vector<int> list;
  list.reserve((size_t)c->npml_nodes);
  for (int k = 0; k < g.n[2]; k++)
    for (int j = 0; j < g.n[1]; j++)
      for (int i = 0; i < g.n[0]; i++)
        if (!(all_rd[0][i] && all_rd[1][j] && all_rd[2][k])) list.push_back((k * g.n[1] + j) * g.px + i);
  if ((int64_t)list.size() != c->npml_nodes) return fail(c, FWI_E_CUDA, "PML node list size mismatch");
  if (list.empty()) list.push_back(0);  // a PML-free box: slots of zero length, one valid entry
  TRY(dalloc(c, &c->d_pml_list, list.size()));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_pml_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FWI_OK;
}

// compact snapshot g of the nb step-start states X (shot b's at (b * nseg + g) * snap_floats)
fwi_status take_snapshot(fwi_ctx *c, float *snap, int g, int nseg, int nb) {
  const size_t sf = snap_floats(c);
  fwi::launch_snapshot(c->state[0], snap + (size_t)g * sf, c->d_pml_list, c->npml_nodes, pml_pad(c), c->geo.stride,
                       nb, (int64_t)set_floats(c), (int64_t)(nseg * sf), true, c->stream, c->geo.oob);
  c->t_launch[3]++;
  CUDA_TRY(c, cudaGetLastError());
  return FWI_OK;
}

// forward sweep of shots shot0 .. shot0 + nb - 1 into d_traces (shot b at b * trace_floats);
// hist: optional displacement history (shot b at b * hstride); snap: optional snapshots of
// the step-start state X every `every` steps (shot b's segment g at (b * nseg + g) * set)
fwi_status forward_sweep_body(fwi_ctx *c, int shot0, int nb, float *hist, int64_t hstride, float *snap, int every,
                              int nseg) {
  TRY(zero_state(c));
  const int64_t per_step = (int64_t)c->nrec * 3;
  const size_t hstep = level_floats(c);
  const size_t sfloats = set_floats(c);
  const int64_t tf = (int64_t)trace_floats(c);
  if (hist)
    for (int b = 0; b < nb; b++)
      CUDA_TRY(c, cudaMemsetAsync(hist + b * hstride, 0, sizeof(float) * hstep, c->stream));
  fwi::launch_sample(c->state[0], c->geo.stride, c->nrec, c->d_rec_node, c->d_traces, c->stream, nb,
                     (int64_t)sfloats, tf, c->geo.oob);
  if (c->persistent) {
    if (!c->d_rec_of) {
      std::vector<int> rec_of((size_t)c->geo.stride, -1);
      for (int r = 0; r < c->nrec; r++) rec_of[(size_t)c->rec_node[r]] = r;
      TRY(dalloc(c, &c->d_rec_of, rec_of.size()));
      CUDA_TRY(c, cudaMemcpyAsync(c->d_rec_of, rec_of.data(), sizeof(int) * rec_of.size(), cudaMemcpyHostToDevice,
                                  c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    // one cooperative launch per checkpoint segment (the whole sweep without snapshots)
    fwi::PersistArgs p{};
    for (int b = 0; b < 4; b++) p.st[b] = c->state[b];
    p.nshot = nb;
    p.sstride = (int64_t)sfloats;
    p.dt = (float)c->cfg.dt;
    p.nodes = c->d_all;
    p.nall = (int)c->geo.nnode;
    p.src_node = c->d_src_node + shot0;
    p.src_vec = c->d_src_vec + 3 * shot0;
    p.wave = c->d_wave;
    p.rec_of = c->d_rec_of;
    p.traces = c->d_traces;
    p.tstride = tf;
    p.nrec = c->nrec;
    p.hist = hist;
    p.hstep = (int64_t)hstep;
    p.hstride = hstride;
    p.bar = c->d_bar;
    p.extra = c->bar_extra;
    p.wait_cycles = (long long)(c->wait_ms * 1e-3 * 2.2e9);
    p.status = c->d_status;
    const int seg = snap ? every : c->cfg.nsteps;
    for (int n0 = 0; n0 < c->cfg.nsteps; n0 += seg) {
      if (snap) TRY(take_snapshot(c, snap, n0 / every, nseg, nb));
      p.n0 = n0;
      p.n1 = std::min(n0 + seg, c->cfg.nsteps);
      CUDA_TRY(c, cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), c->stream));
      CUDA_TRY(c, fwi::launch_persistent_forward(c->geo, p, c->stream));
      c->t_launch[0] += 4 * (p.n1 - p.n0);  // stage updates done by the launch
      c->t_launch[3]++;
    }
    return FWI_OK;
  }
  for (int n = 0; n < c->cfg.nsteps; n++) {
    if (snap && n % every == 0) TRY(take_snapshot(c, snap, n / every, nseg, nb));
    TRY(rk4_step(c, false, n, shot0, nb, hist ? hist + (size_t)(n + 1) * hstep : nullptr, hstride));
    fwi::launch_sample(c->state[0], c->geo.stride, c->nrec, c->d_rec_node, c->d_traces + (n + 1) * per_step,
                       c->stream, nb, (int64_t)sfloats, tf, c->geo.oob);
    c->t_launch[2]++;
    c->t_launch[3]++;
  }
  CUDA_TRY(c, cudaGetLastError());
  return FWI_OK;
}

fwi_status forward_sweep(fwi_ctx *c, int shot0, int nb, float *hist, int64_t hstride, float *snap = nullptr,
                         int every = 0, int nseg = 0) {
  // hist, snap and their strides follow from the context's buffers and checkpointing mode
  return graphed(c, 0, shot0, nb, hist ? 1 : (snap ? 2 + every : 0),
                 [&] { return forward_sweep_body(c, shot0, nb, hist, hstride, snap, every, nseg); });
}

// residual and misfit of the traces of batch shot b against observed (device) -> d_J[slot]
fwi_status misfit_of_traces(fwi_ctx *c, int b, const float *obs_dev, int slot) {
  const int64_t per_step = (int64_t)c->nrec * 3;
  const int64_t n = per_step * (c->cfg.nsteps + 1);
  fwi::launch_residual(c->d_traces + b * n, obs_dev, c->d_resid + b * n, n, per_step, c->cfg.nsteps, c->cfg.dt,
                       c->d_part, c->d_flag, c->stream);
  fwi::launch_sum(c->d_part, fwi::misfit_blocks(n), c->d_J + slot, c->stream);
  c->t_launch[3] += 2;
  CUDA_TRY(c, cudaGetLastError());
  return FWI_OK;
}

fwi_status ensure_J(fwi_ctx *c, int n) {
  if (c->d_J_cap < n) {
    dfree(c->d_J);
    TRY(dalloc(c, &c->d_J, (size_t)n));
    c->d_J_cap = n;
  }
  return FWI_OK;
}

// observed traces of shot s (counted from the call's first shot) on the device; host data
// go through the batch slot b of d_obs
const float *observed_for_shot(fwi_ctx *c, const float *observed, int on_device, int s, int b, fwi_status *st) {
  const size_t nt = trace_floats(c);
  *st = FWI_OK;
  if (on_device) return observed + (size_t)s * nt;
  cudaError_t e = cudaMemcpyAsync(c->d_obs + (size_t)b * nt, observed + (size_t)s * nt, nt * sizeof(float),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) {
    *st = fail(c, FWI_E_CUDA, "observed upload: %s", cudaGetErrorString(e));
    return nullptr;
  }
  return c->d_obs + (size_t)b * nt;
}

fwi_status finish_J(fwi_ctx *c, int nshots, double *J) {
  std::vector<double> hJ(nshots);
  int flag = 0;
  CUDA_TRY(c, cudaMemcpyAsync(hJ.data(), c->d_J, sizeof(double) * nshots, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  TRY(check_status(c));
  if (flag) return fail(c, FWI_E_NONFINITE, "non-finite value in the computed traces");
  double s = 0.0;
  for (int i = 0; i < nshots; i++) s += hJ[i];
  if (!std::isfinite(s)) return fail(c, FWI_E_NONFINITE, "non-finite misfit");
  if (J) *J = s;
  return FWI_OK;
}

}  // namespace

extern "C" {

const char *fwi_status_string(fwi_status s) {
  switch (s) {
    case FWI_OK: return "ok";
    case FWI_E_INVAL: return "invalid argument";
    case FWI_E_NOMEM: return "out of memory";
    case FWI_E_CUDA: return "CUDA error";
    case FWI_E_UNSTABLE: return "time step above the RK4 stability estimate";
    case FWI_E_NONFINITE: return "non-finite value";
    case FWI_E_TIMEOUT: return "bounded device wait gave up";
    case FWI_E_STATE: return "call out of order";
    case FWI_E_BOUNDS: return "device index out of range";
  }
  return "unknown status";
}

const char *fwi_last_error(const fwi_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int fwi_bounds_checked(void) {
#ifdef FWI_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

fwi_status fwi_create(const fwi_config *cfg, fwi_ctx **out) {
  if (!cfg || !out) return FWI_E_INVAL;
  *out = nullptr;
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || cfg->npml < 0 || !(cfg->h > 0) || !(cfg->rho > 0) ||
      !(cfg->dt > 0) || cfg->nsteps < 1 || cfg->pml_m < 0 || !(cfg->pml_alpha0 >= 0) || !(cfg->pml_beta0 >= 0))
    return FWI_E_INVAL;
  if (cfg->npml == 0 && cfg->top_pml) return FWI_E_INVAL;
  const int64_t nI = 2LL * (cfg->nx + 2LL * cfg->npml) + 1, nJ = 2LL * (cfg->ny + 2LL * cfg->npml) + 1,
                nK = 2LL * (cfg->nz + cfg->npml + (cfg->top_pml ? cfg->npml : 0)) + 1;
  // the PML stage kernel addresses the 27 state fields with 32-bit offsets
  const int64_t px = (nI + 3) / 4 * 4;
  if (27 * (px * nJ * nK + 64) >= (1LL << 31)) return FWI_E_INVAL;
  fwi_ctx *c = new (std::nothrow) fwi_ctx();
  if (!c) return FWI_E_NOMEM;
  c->cfg = *cfg;
  c->stream = (cudaStream_t)cfg->cuda_stream;
  fwi::Geo &g = c->geo;
  g.n[0] = (int)nI;
  g.n[1] = (int)nJ;
  g.px = (int)px;
  g.n[2] = (int)nK;
  g.lo[0] = cfg->npml;
  g.lo[1] = cfg->npml;
  g.lo[2] = cfg->top_pml ? cfg->npml : 0;
  g.hi[0] = g.lo[0] + cfg->nx;
  g.hi[1] = g.lo[1] + cfg->ny;
  g.hi[2] = g.lo[2] + cfg->nz;
  g.m[0] = 2 * cfg->nx + 1;
  g.m[1] = 2 * cfg->ny + 1;
  g.m[2] = 2 * cfg->nz + 1;
  g.top_dir = cfg->top_pml ? 1 : 0;
  for (int ax = 0; ax < 3; ax++) {
    // coordinates all of whose elements along this axis are interior, minus fixed faces
    const int Nax = (g.n[ax] - 1) / 2;
    int lo_c = 2 * g.lo[ax] + (g.lo[ax] > 0 ? 1 : 0);
    int hi_c = 2 * g.hi[ax] - (g.hi[ax] < Nax ? 1 : 0);
    const int first_free = (ax == 2 && !g.top_dir) ? 0 : 1;
    g.box_lo[ax] = lo_c > first_free ? lo_c : first_free;
    g.box_hi[ax] = hi_c < g.n[ax] - 2 ? hi_c : g.n[ax] - 2;
  }
  g.nnode = nI * nJ * nK;
  g.nmat = (int64_t)g.m[0] * g.m[1] * g.m[2];
  g.stride = (px * nJ * nK + 63) / 64 * 64;
  g.inv_h = (float)(1.0 / cfg->h);
  g.rho = (float)cfg->rho;
  g.int_kc = 8;
  g.pml_seg = 32;
  g.inv_rho_h = (float)(1.0 / (cfg->rho * cfg->h));
  g.wdetj = (float)(0.125 * cfg->h * cfg->h * cfg->h);
  c->nelem = (int64_t)(nI / 2) * (nJ / 2) * (nK / 2);
  {
    // PML nodes: nodes of at least one PML element
    int64_t rd_only = 1;
    for (int ax = 0; ax < 3; ax++) {
      // coordinates whose every element along this axis is interior
      int64_t cnt = 0;
      for (int cc = 0; cc < g.n[ax]; cc++) {
        bool all = true;
        if (cc & 1) {
          int e = (cc - 1) / 2;
          all = e >= g.lo[ax] && e < g.hi[ax];
        } else {
          if (cc >= 2) all = all && (cc / 2 - 1 >= g.lo[ax] && cc / 2 - 1 < g.hi[ax]);
          if (cc <= g.n[ax] - 3) all = all && (cc / 2 >= g.lo[ax] && cc / 2 < g.hi[ax]);
        }
        cnt += all;
      }
      rd_only *= cnt;
    }
    c->npml_nodes = g.nnode - rd_only;
  }
  // PML stretch functions per axis, FP64 on the host (reading of [13]):
  // alpha = 1 + alpha0 (l/L)^m, beta = beta0 (l/L)^m, l = depth into the layer
  const double L = cfg->npml * cfg->h;
  for (int ax = 0; ax < 3; ax++) {
    c->h_alpha[ax].resize(g.n[ax]);
    c->h_beta[ax].resize(g.n[ax]);
    const int a0 = 2 * g.lo[ax], b0 = 2 * g.hi[ax];
    for (int cc = 0; cc < g.n[ax]; cc++) {
      double l = cc < a0 ? (a0 - cc) * 0.5 * cfg->h : (cc > b0 ? (cc - b0) * 0.5 * cfg->h : 0.0);
      double r = (L > 0 && l > 0) ? std::pow(l / L, (double)cfg->pml_m) : 0.0;
      c->h_alpha[ax][cc] = 1.0 + cfg->pml_alpha0 * r;
      c->h_beta[ax][cc] = cfg->pml_beta0 * r;
    }
  }
  fwi_status st = FWI_OK;
  for (int i = 0; i < 2 && st == FWI_OK; i++)
    if (cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming) != cudaSuccess)
      st = fail(c, FWI_E_CUDA, "stream setup failed");
  if (st == FWI_OK && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    st = fail(c, FWI_E_CUDA, "event setup failed");
  if (st == FWI_OK && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
    st = fail(c, FWI_E_CUDA, "stream setup failed");
  const size_t sbytes = (size_t)fwi::kFields * g.stride;
  for (int b = 0; b < 4 && st == FWI_OK; b++) st = dalloc(c, &c->state[b], sbytes);
  for (int ax = 0; ax < 3 && st == FWI_OK; ax++) {
    st = dalloc(c, &c->d_alpha[ax], g.n[ax]);
    if (st == FWI_OK) st = dalloc(c, &c->d_beta[ax], g.n[ax]);
    if (st == FWI_OK) st = dalloc(c, &c->d_ialpha[ax], g.n[ax]);
    if (st != FWI_OK) break;
    std::vector<float> fa(g.n[ax]), fb(g.n[ax]), fi(g.n[ax]);
    for (int i = 0; i < g.n[ax]; i++) {
      fa[i] = (float)c->h_alpha[ax][i];
      fb[i] = (float)c->h_beta[ax][i];
      fi[i] = (float)(1.0 / c->h_alpha[ax][i]);
    }
    if (cudaMemcpy(c->d_alpha[ax], fa.data(), sizeof(float) * g.n[ax], cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_beta[ax], fb.data(), sizeof(float) * g.n[ax], cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_ialpha[ax], fi.data(), sizeof(float) * g.n[ax], cudaMemcpyHostToDevice) != cudaSuccess)
      st = fail(c, FWI_E_CUDA, "stretch table upload failed");
    g.alpha[ax] = c->d_alpha[ax];
    g.beta[ax] = c->d_beta[ax];
    g.ialpha[ax] = c->d_ialpha[ax];
  }
  if (st == FWI_OK && fwi::prepare_interior() != cudaSuccess) st = fail(c, FWI_E_CUDA, "kernel attribute setup failed");
  if (st == FWI_OK) {
    // interface shell: closed interior box minus the open box of the interior kernel
    std::vector<int> shell;
    const int c0[3] = {2 * g.lo[0], 2 * g.lo[1], g.top_dir ? 2 * g.lo[2] : 0};
    const int c1[3] = {2 * g.hi[0], 2 * g.hi[1], 2 * g.hi[2]};
    for (int k = c0[2]; k <= c1[2]; k++)
      for (int j = c0[1]; j <= c1[1]; j++)
        for (int i = c0[0]; i <= c1[0]; i++) {
          const bool in_open = i >= g.box_lo[0] && i <= g.box_hi[0] && j >= g.box_lo[1] && j <= g.box_hi[1] &&
                               k >= g.box_lo[2] && k <= g.box_hi[2];
          if (!in_open) shell.push_back((k * g.n[1] + j) * g.px + i);
        }
    // PML nodes on the outer faces of the grid: outside the closed box, on a face
    std::vector<int> face;
    for (int k = 0; k < g.n[2]; k++)
      for (int j = 0; j < g.n[1]; j++)
        for (int i = 0; i < g.n[0]; i++) {
          const bool on_face = i == 0 || i == g.n[0] - 1 || j == 0 || j == g.n[1] - 1 || k == 0 || k == g.n[2] - 1;
          if (!on_face) continue;
          const bool in_closed = i >= c0[0] && i <= c1[0] && j >= c0[1] && j <= c1[1] && k >= c0[2] && k <= c1[2];
          if (!in_closed) face.push_back((k * g.n[1] + j) * g.px + i);
        }
    // both lists stay in (k, j, i) order: the nodes of a warp are neighbours in memory,
    // and their stencil rows are shared
    g.nface = (int)face.size();
    if (g.nface > 0) {
      st = dalloc(c, &c->d_face, face.size());
      if (st == FWI_OK &&
          cudaMemcpy(c->d_face, face.data(), sizeof(int) * face.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        st = fail(c, FWI_E_CUDA, "face list upload failed");
      g.face = c->d_face;
    }
    g.nshell = (int)shell.size();
    if (g.nshell > 0) {
      st = dalloc(c, &c->d_shell, shell.size());
      if (st == FWI_OK &&
          cudaMemcpy(c->d_shell, shell.data(), sizeof(int) * shell.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        st = fail(c, FWI_E_CUDA, "shell list upload failed");
      g.shell = c->d_shell;
    }
  }
  if (st == FWI_OK) st = dalloc(c, &c->d_lam, (size_t)g.nmat);
  if (st == FWI_OK) st = dalloc(c, &c->d_mu, (size_t)g.nmat);
  if (st == FWI_OK) st = dalloc(c, &c->d_lam_n, (size_t)g.stride);
  if (st == FWI_OK) st = dalloc(c, &c->d_mu_n, (size_t)g.stride);
#ifdef FWI_BOUNDS_CHECK
  if (st == FWI_OK) st = dalloc(c, &c->d_oob, 1);
  if (st == FWI_OK && cudaMemset(c->d_oob, 0, sizeof(unsigned long long)) != cudaSuccess)
    st = fail(c, FWI_E_CUDA, "error word clear failed");
#endif
  g.oob = c->d_oob;
  if (st == FWI_OK) st = dalloc(c, &c->d_status, 1);
  if (st == FWI_OK && cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess)
    st = fail(c, FWI_E_CUDA, "status word clear failed");
  g.status = c->d_status;
  g.wait_cycles = (long long)(1000.0 * 1e-3 * 2.2e9);  // about a second
  g.copy_extra = 0;
  if (st == FWI_OK) {
    g.lam = c->d_lam;
    g.mu = c->d_mu;
    g.lam_n = c->d_lam_n;
    g.mu_n = c->d_mu_n;
    for (int b = 0; b < 4 && st == FWI_OK; b++)
      if (cudaMemset(c->state[b], 0, sizeof(float) * sbytes) != cudaSuccess)
        st = fail(c, FWI_E_CUDA, "state clear failed");
  }
  if (st != FWI_OK) {
    fwi_destroy(c);
    return st;
  }
  *out = c;
  return FWI_OK;
}

void fwi_destroy(fwi_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (int b = 0; b < 4; b++) {
    dfree(c->state[b]);
    dfree(c->rstate[b]);
  }
  dfree(c->d_snap);
  for (int ax = 0; ax < 3; ax++) {
    dfree(c->d_alpha[ax]);
    dfree(c->d_beta[ax]);
    dfree(c->d_ialpha[ax]);
  }
  dfree(c->d_lam);
  dfree(c->d_mu);
  dfree(c->d_lam_n);
  dfree(c->d_mu_n);
  drop_graphs(c);
  dfree(c->d_all);
  dfree(c->d_pml_list);
  dfree(c->d_oob);
  dfree(c->d_rec_of);
  dfree(c->d_bar);
  dfree(c->d_status);
  dfree(c->d_shell);
  dfree(c->d_face);
  dfree(c->d_wave);
  dfree(c->d_src_node);
  dfree(c->d_src_vec);
  dfree(c->d_rec_node);
  dfree(c->d_rec_vec);
  dfree(c->d_traces);
  dfree(c->d_obs);
  dfree(c->d_resid);
  dfree(c->d_part);
  dfree(c->d_J);
  dfree(c->d_flag);
  dfree(c->d_hist);
  dfree(c->d_gl);
  dfree(c->d_gm);
  for (double **p : {&c->d_mt, &c->d_m, &c->d_mprev, &c->d_g, &c->d_gprev, &c->d_dir, &c->d_S, &c->d_Yv,
                     &c->d_opart, &c->d_oscal, &c->d_rg, &c->d_rpart, &c->d_rval})
    dfree(*p);
  dfree(c->d_oflags);
  dfree(c->d_omax);
  for (int i = 0; i < 2; i++) {
    if (c->side[i]) {
      cudaStreamSynchronize(c->side[i]);
      cudaStreamDestroy(c->side[i]);
    }
    if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (auto e : c->ev_free) cudaEventDestroy(e);
  for (auto &p : c->ev_pending) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  delete c;
}

fwi_status fwi_get_dims(const fwi_ctx *c, int64_t dims[9]) {
  if (!c || !dims) return FWI_E_INVAL;
  dims[0] = c->geo.n[0];
  dims[1] = c->geo.n[1];
  dims[2] = c->geo.n[2];
  dims[3] = c->geo.nnode;
  dims[4] = c->geo.nmat;
  dims[5] = c->geo.stride;
  dims[6] = c->nelem;
  dims[7] = c->npml_nodes;
  dims[8] = c->geo.px;
  return FWI_OK;
}

fwi_status fwi_set_material(fwi_ctx *c, const float *lambda, const float *mu, int on_device) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  if (!lambda || !mu) return fail(c, FWI_E_INVAL, "null material pointer");
  const size_t n = (size_t)c->geo.nmat;
  std::vector<float> hl(n), hm(n);
  if (on_device) {
    CUDA_TRY(c, cudaMemcpyAsync(hl.data(), lambda, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(hm.data(), mu, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  } else {
    std::memcpy(hl.data(), lambda, n * sizeof(float));
    std::memcpy(hm.data(), mu, n * sizeof(float));
  }
  double vmax = 0.0;
  for (size_t i = 0; i < n; i++) {
    if (!std::isfinite(hl[i]) || !std::isfinite(hm[i]))
      return fail(c, FWI_E_NONFINITE, "non-finite material value at node %zu", i);
    if (!(hm[i] > 0.f) || !(hl[i] + 2.f * hm[i] > 0.f))
      return fail(c, FWI_E_INVAL, "material at node %zu violates mu > 0, lambda + 2 mu > 0", i);
    vmax = std::fmax(vmax, std::sqrt(((double)hl[i] + 2.0 * hm[i]) / c->cfg.rho));
  }
  const double cfl = c->cfg.dt * vmax / (0.5 * c->cfg.h);
  if (cfl > 0.66)
    return fail(c, FWI_E_UNSTABLE, "dt * vp_max / (h/2) = %.3f above the RK4 limit estimate 0.66", cfl);
  CUDA_TRY(c, cudaMemcpyAsync(c->d_lam, hl.data(), n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_mu, hm.data(), n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  fwi::launch_extend_material(c->geo, c->d_lam_n, c->d_mu_n, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->have_material = true;
  return FWI_OK;
}

fwi_status fwi_set_sources(fwi_ctx *c, int nshots, const int *node_ijk, const double *dir, int wavelet,
                           const double *wparams) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  if (nshots < 1 || !node_ijk || !dir || !wparams) return fail(c, FWI_E_INVAL, "bad source arguments");
  if (wavelet != FWI_WAVELET_RICKER && wavelet != FWI_WAVELET_GAUSS)
    return fail(c, FWI_E_INVAL, "unknown wavelet %d", wavelet);
  if (wavelet == FWI_WAVELET_GAUSS && !(wparams[1] > 0)) return fail(c, FWI_E_INVAL, "gauss sigma must be > 0");
  std::vector<int64_t> nodes(nshots);
  std::vector<float> vec(3 * (size_t)nshots);
  for (int s = 0; s < nshots; s++) {
    const int i = node_ijk[3 * s], j = node_ijk[3 * s + 1], k = node_ijk[3 * s + 2];
    if (i < 0 || j < 0 || k < 0 || i >= c->geo.n[0] || j >= c->geo.n[1] || k >= c->geo.n[2])
      return fail(c, FWI_E_INVAL, "source %d node (%d,%d,%d) outside the mesh", s, i, j, k);
    if (is_dirichlet(c, i, j, k)) return fail(c, FWI_E_INVAL, "source %d on a fixed (Dirichlet) face", s);
    nodes[s] = ((int64_t)k * c->geo.n[1] + j) * c->geo.px + i;
    const double minv = 1.0 / mass_u(c, i, j, k);
    for (int d = 0; d < 3; d++) {
      if (!std::isfinite(dir[3 * s + d])) return fail(c, FWI_E_NONFINITE, "non-finite source direction");
      vec[3 * s + d] = (float)(dir[3 * s + d] * minv);
    }
  }
  // wavelet samples at t = j dt / 2, j = 0 .. 2 nsteps (RK4 stage times), FP64 -> FP32
  const int nw = 2 * c->cfg.nsteps + 1;
  std::vector<float> wave(nw);
  for (int j = 0; j < nw; j++) {
    const double t = 0.5 * j * c->cfg.dt;
    double r;
    if (wavelet == FWI_WAVELET_RICKER) {
      const double a = M_PI * wparams[0] * (t - wparams[1]);
      r = wparams[2] * (1.0 - 2.0 * a * a) * std::exp(-a * a);
    } else {
      const double x = t - wparams[0];
      r = wparams[2] * std::exp(-x * x / wparams[1]);
    }
    wave[j] = (float)r;
  }
  dfree(c->d_src_node);
  dfree(c->d_src_vec);
  dfree(c->d_wave);
  TRY(dalloc(c, &c->d_src_node, (size_t)nshots));
  TRY(dalloc(c, &c->d_src_vec, 3 * (size_t)nshots));
  TRY(dalloc(c, &c->d_wave, (size_t)nw));
  CUDA_TRY(c, cudaMemcpy(c->d_src_node, nodes.data(), sizeof(int64_t) * nshots, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->d_src_vec, vec.data(), sizeof(float) * 3 * nshots, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->d_wave, wave.data(), sizeof(float) * nw, cudaMemcpyHostToDevice));
  c->nshots = nshots;
  c->src_node = nodes;
  c->src_dir.assign(dir, dir + 3 * (size_t)nshots);
  c->wavelet = wavelet;
  std::memcpy(c->wparams, wparams, sizeof c->wparams);
  return FWI_OK;
}

fwi_status fwi_set_receivers(fwi_ctx *c, int nrec, const int *node_ijk) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  if (nrec < 1 || !node_ijk) return fail(c, FWI_E_INVAL, "bad receiver arguments");
  std::vector<int64_t> nodes(nrec);
  std::vector<float> vec(3 * (size_t)nrec);
  for (int r = 0; r < nrec; r++) {
    const int i = node_ijk[3 * r], j = node_ijk[3 * r + 1], k = node_ijk[3 * r + 2];
    if (i < 0 || j < 0 || k < 0 || i >= c->geo.n[0] || j >= c->geo.n[1] || k >= c->geo.n[2])
      return fail(c, FWI_E_INVAL, "receiver %d node (%d,%d,%d) outside the mesh", r, i, j, k);
    if (is_dirichlet(c, i, j, k)) return fail(c, FWI_E_INVAL, "receiver %d on a fixed (Dirichlet) face", r);
    nodes[r] = ((int64_t)k * c->geo.n[1] + j) * c->geo.px + i;
    const float minv = (float)(1.0 / mass_u(c, i, j, k));
    vec[3 * r] = vec[3 * r + 1] = vec[3 * r + 2] = minv;
  }
  {
    std::vector<int64_t> sorted = nodes;
    std::sort(sorted.begin(), sorted.end());
    for (int r = 1; r < nrec; r++)
      if (sorted[r] == sorted[r - 1]) return fail(c, FWI_E_INVAL, "receivers must be distinct nodes");
  }
  dfree(c->d_rec_node);
  dfree(c->d_rec_vec);
  dfree(c->d_traces);
  dfree(c->d_obs);
  dfree(c->d_resid);
  TRY(dalloc(c, &c->d_rec_node, (size_t)nrec));
  TRY(dalloc(c, &c->d_rec_vec, 3 * (size_t)nrec));
  CUDA_TRY(c, cudaMemcpy(c->d_rec_node, nodes.data(), sizeof(int64_t) * nrec, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->d_rec_vec, vec.data(), sizeof(float) * 3 * nrec, cudaMemcpyHostToDevice));
  c->nrec = nrec;
  c->rec_node = nodes;
  dfree(c->d_rec_of);  // rebuilt by the next persistent sweep
  return FWI_OK;
}

fwi_status fwi_forward(fwi_ctx *c, int shot0, int nshots, float *traces, int on_device) {
  if (!c) return FWI_E_INVAL;
  TRY(require_ready(c, shot0, nshots));
  if (!traces) return fail(c, FWI_E_INVAL, "null traces");
  TRY(ensure_trace_buffers(c));
  CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  const size_t nt = trace_floats(c);
  for (int s0 = 0; s0 < nshots; s0 += c->batch) {
    const int nb = std::min(c->batch, nshots - s0);
    TRY(forward_sweep(c, shot0 + s0, nb, nullptr, 0));
    CUDA_TRY(c, cudaMemcpyAsync(traces + s0 * nt, c->d_traces, nb * nt * sizeof(float),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return check_status(c);
}

namespace {

// misfit (7) of shots [shot0, shot0 + nshots) at the current material
fwi_status run_misfit(fwi_ctx *c, int shot0, int nshots, const float *observed, int on_device, double *J) {
  TRY(ensure_trace_buffers(c));
  TRY(ensure_J(c, nshots));
  CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  for (int s0 = 0; s0 < nshots; s0 += c->batch) {
    const int nb = std::min(c->batch, nshots - s0);
    TRY(forward_sweep(c, shot0 + s0, nb, nullptr, 0));
    for (int b = 0; b < nb; b++) {
      fwi_status st;
      const float *obs = observed_for_shot(c, observed, on_device, s0 + b, b, &st);
      if (!obs) return st;
      TRY(misfit_of_traces(c, b, obs, s0 + b));
    }
  }
  return finish_J(c, nshots, J);
}

// misfit and g_mis (dJ/dlambda_i, dJ/dmu_i) into d_gl / d_gm
// (re)allocate the displacement history for `slots` levels
// history slots (levels) per shot of the batch; shot b's levels start at b * slots levels
fwi_status ensure_hist(fwi_ctx *c, size_t slots) {
  if (c->hist_cap >= slots * c->batch) return FWI_OK;
  dfree(c->d_hist);
  c->hist_cap = 0;
  TRY(dalloc(c, &c->d_hist, slots * c->batch * level_floats(c)));
  c->hist_cap = slots * c->batch;
  return FWI_OK;
}

// the adjoint step that yields w(t_lvl) for the nb shots of the batch, and the gradient
// integrand at that level from their displacement history slots (shot b at hist_lvl + b hstride)
fwi_status adjoint_level(fwi_ctx *c, int lvl, const float *hist_lvl, int nb, int64_t hstride) {
  const int N = c->cfg.nsteps;
  TRY(rk4_step(c, true, N - lvl - 1, 0, nb, nullptr, 0));
  if (lvl > 0) {
    const double wn = (lvl == N) ? 0.5 : 1.0;
    cudaEvent_t e0;
    time_begin(c, &e0);
    fwi::launch_gradient(c->geo, c->state[0], hist_lvl, wn * c->cfg.dt, c->d_gl, c->d_gm, c->stream, nb,
                         (int64_t)set_floats(c), hstride);
    time_end(c, e0, 1);
    CUDA_TRY(c, cudaGetLastError());
  }
  return FWI_OK;
}

fwi_status run_gradient(fwi_ctx *c, int shot0, int nshots, const float *observed, int on_device, double *J) {
  TRY(ensure_trace_buffers(c));
  TRY(ensure_J(c, nshots));
  const size_t nmat = (size_t)c->geo.nmat;
  const int N = c->cfg.nsteps;
  const size_t hstep = level_floats(c);
  // checkpoint interval: 0 keeps every level of the displacement history
  int every = c->ckpt < 0 ? (int)std::ceil(std::sqrt((double)N)) : c->ckpt;
  if (every >= N) every = 0;
  const int nseg = every > 0 ? (N + every - 1) / every : 0;
  const size_t sfloats = set_floats(c);
  const size_t slots = every > 0 ? (size_t)every + 1 : (size_t)N + 1;
  const int64_t hstride = (int64_t)(slots * hstep);  // one shot's history levels
  TRY(ensure_hist(c, slots));
  if (every > 0) {
    TRY(ensure_pml_list(c));
    const size_t nsnap = (size_t)nseg * c->batch;
    if (c->snap_cap < nsnap) {
      dfree(c->d_snap);
      c->snap_cap = 0;
      TRY(dalloc(c, &c->d_snap, nsnap * snap_floats(c)));
      c->snap_cap = nsnap;
    }
    for (int b = 0; b < 4; b++) {
      if (c->rstate[b]) continue;
      TRY(dalloc(c, &c->rstate[b], sfloats * c->batch));
      // entries that no stage writes (history and stress off the PML, fixed faces, padding) stay zero
      CUDA_TRY(c, cudaMemsetAsync(c->rstate[b], 0, sfloats * c->batch * sizeof(float), c->stream));
    }
  }
  TRY(dalloc(c, &c->d_gl, nmat));
  TRY(dalloc(c, &c->d_gm, nmat));
  CUDA_TRY(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_gl, 0, sizeof(double) * nmat, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_gm, 0, sizeof(double) * nmat, c->stream));
  for (int s0 = 0; s0 < nshots; s0 += c->batch) {
    const int nb = std::min(c->batch, nshots - s0);
    TRY(forward_sweep(c, shot0 + s0, nb, every > 0 ? nullptr : c->d_hist, hstride, every > 0 ? c->d_snap : nullptr,
                      every, nseg));
    for (int b = 0; b < nb; b++) {
      fwi_status st;
      const float *obs = observed_for_shot(c, observed, on_device, s0 + b, b, &st);
      if (!obs) return st;
      TRY(misfit_of_traces(c, b, obs, s0 + b));
    }
    // adjoint sweep in reversed time with the gradient time integral (C.1f)/(C.1g)
    if (every == 0) {
      TRY(graphed(c, 1, 0, nb, 0, [&]() -> fwi_status {
        TRY(zero_state(c));
        for (int lvl = N - 1; lvl >= 0; lvl--)
          TRY(adjoint_level(c, lvl, c->d_hist + (size_t)lvl * hstep, nb, hstride));
        return FWI_OK;
      }));
      continue;
    }
    TRY(zero_state(c));
    // checkpointed: segment g holds the steps [g every, min((g+1) every, N)). Its forward
    // steps are recomputed from snapshot g in the second state set, writing the history
    // levels g every + 1 .. of the segment; then the adjoint runs through those levels.
    // The recomputed steps repeat the forward sweep's arithmetic exactly, so the
    // gradient equals the one from the stored history bit for bit.
    for (int g = nseg - 1; g >= 0; g--) {
      TRY(graphed(c, 2, shot0 + s0, nb, g * 65536 + every, [&]() -> fwi_status {
        const int L0 = g * every, L1 = std::min(L0 + every, N);
        std::swap(c->state, c->rstate);
        fwi_status rs = FWI_OK;
        const size_t sf = snap_floats(c);
        fwi::launch_snapshot(c->state[0], c->d_snap + (size_t)g * sf, c->d_pml_list, c->npml_nodes, pml_pad(c),
                             c->geo.stride, nb, (int64_t)sfloats, (int64_t)(nseg * sf), false, c->stream,
                             c->geo.oob);
        c->t_launch[3]++;
        if (cudaGetLastError() != cudaSuccess) rs = fail(c, FWI_E_CUDA, "snapshot restore failed");
        for (int n = L0; n < L1 && rs == FWI_OK; n++)
          rs = rk4_step(c, false, n, shot0 + s0, nb, c->d_hist + (size_t)(n + 1 - L0) * hstep, hstride);
        std::swap(c->state, c->rstate);
        TRY(rs);
        for (int lvl = std::min(L1, N - 1); lvl > L0; lvl--)
          TRY(adjoint_level(c, lvl, c->d_hist + (size_t)(lvl - L0) * hstep, nb, hstride));
        return FWI_OK;
      }));
    }
  }
  fwi::launch_check_finite(c->d_gl, (int64_t)nmat, c->d_flag, c->stream);
  fwi::launch_check_finite(c->d_gm, (int64_t)nmat, c->d_flag, c->stream);
  c->t_launch[3] += 2;
  return finish_J(c, nshots, J);
}

}  // namespace

fwi_status fwi_misfit(fwi_ctx *c, int shot0, int nshots, const float *observed, int on_device, double *J) {
  if (!c) return FWI_E_INVAL;
  TRY(require_ready(c, shot0, nshots));
  if (!observed || !J) return fail(c, FWI_E_INVAL, "null argument");
  return run_misfit(c, shot0, nshots, observed, on_device, J);
}

fwi_status fwi_adjoint_gradient(fwi_ctx *c, int shot0, int nshots, const float *observed, int on_device,
                                double *J, double *g_lambda, double *g_mu) {
  if (!c) return FWI_E_INVAL;
  TRY(require_ready(c, shot0, nshots));
  if (!observed || !g_lambda || !g_mu) return fail(c, FWI_E_INVAL, "null argument");
  double Jv = 0.0;
  TRY(run_gradient(c, shot0, nshots, observed, on_device, &Jv));
  // the outputs are written only after the finite check in run_gradient passed
  const size_t nmat = (size_t)c->geo.nmat;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(c, cudaMemcpyAsync(g_lambda, c->d_gl, sizeof(double) * nmat, kind, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(g_mu, c->d_gm, sizeof(double) * nmat, kind, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (J) *J = Jv;
  return FWI_OK;
}


namespace {

// <a, b> in the Mtilde inner product over both halves, returned on the host
fwi_status wdot(fwi_ctx *c, const double *a, const double *b, double *out) {
  fwi::opt_wdot(a, b, c->d_mt, c->geo.nmat, c->d_opart, c->d_oscal, c->stream);
  CUDA_TRY(c, cudaMemcpyAsync(out, c->d_oscal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FWI_OK;
}

fwi_status dot(fwi_ctx *c, const double *a, const double *b, int64_t n, double *out) {
  fwi::opt_dot(a, b, n, c->d_opart, c->d_oscal, c->stream);
  CUDA_TRY(c, cudaMemcpyAsync(out, c->d_oscal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FWI_OK;
}

// regularisation terms (8)/(9) of the context's lambda and mu into Rf[2]; with g, their
// gradients into g (lambda half, then mu half)
fwi_status reg_terms(fwi_ctx *c, int kind, double eps, double Rf[2], double *g) {
  const size_t nmat = (size_t)c->geo.nmat;
  TRY(dalloc(c, &c->d_rg, 2 * nmat));
  TRY(dalloc(c, &c->d_rpart, 1024));
  TRY(dalloc(c, &c->d_rval, 2));
  const float *f[2] = {c->d_lam, c->d_mu};
  for (int p = 0; p < 2; p++)
    fwi::opt_regularization(f[p], c->geo.m, c->cfg.h, kind == FWI_REG_TV, eps, g ? g + p * nmat : c->d_rg + p * nmat,
                            c->d_rpart, c->d_rval + p, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(Rf, c->d_rval, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FWI_OK;
}

fwi_status absmax(fwi_ctx *c, const double *x, double *out) {
  CUDA_TRY(c, cudaMemsetAsync(c->d_omax, 0, sizeof(unsigned long long), c->stream));
  fwi::opt_absmax(x, 2 * c->geo.nmat, c->d_omax, c->stream);
  unsigned long long bits = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&bits, c->d_omax, sizeof bits, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  std::memcpy(out, &bits, sizeof(double));
  return FWI_OK;
}

// material m + alpha d into the context; *ok = 0 when it is inadmissible
fwi_status set_trial(fwi_ctx *c, double alpha, const double *d, int *ok) {
  CUDA_TRY(c, cudaMemsetAsync(c->d_oflags, 0, 2 * sizeof(unsigned), c->stream));
  fwi::opt_trial(c->d_m, d, alpha, c->d_lam, c->d_mu, c->geo.nmat, c->d_oflags, c->stream);
  fwi::launch_extend_material(c->geo, c->d_lam_n, c->d_mu_n, c->stream);
  unsigned fl[2] = {0, 0};
  CUDA_TRY(c, cudaMemcpyAsync(fl, c->d_oflags, sizeof fl, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  float pmax;
  std::memcpy(&pmax, &fl[1], sizeof pmax);
  const double cfl = c->cfg.dt * std::sqrt((double)pmax / c->cfg.rho) / (0.5 * c->cfg.h);
  *ok = (fl[0] == 0 && cfl <= 0.66) ? 1 : 0;
  return FWI_OK;
}

}  // namespace

fwi_status fwi_step_reset(fwi_ctx *c) {
  if (!c) return FWI_E_INVAL;
  c->lb_count = c->lb_head = 0;
  c->lb_have_prev = false;
  return FWI_OK;
}

fwi_status fwi_get_material(fwi_ctx *c, float *lambda, float *mu, int on_device) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  if (!c->have_material) return fail(c, FWI_E_STATE, "material not set");
  if (!lambda || !mu) return fail(c, FWI_E_INVAL, "null argument");
  const size_t n = (size_t)c->geo.nmat;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(c, cudaMemcpyAsync(lambda, c->d_lam, n * sizeof(float), kind, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(mu, c->d_mu, n * sizeof(float), kind, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FWI_OK;
}

fwi_status fwi_step(fwi_ctx *c, const float *observed, int on_device, const fwi_step_opts *o, fwi_step_info *info) {
  if (!c) return FWI_E_INVAL;
  if (!o || !observed || !info) return fail(c, FWI_E_INVAL, "null argument");
  TRY(require_ready(c, o->shot0, o->nshots));
  if (o->invert < 1 || o->invert > 3 || o->lbfgs_m < 0 || o->lbfgs_m > 1000 || !(o->c1 > 0 && o->c1 < 1) ||
      !(o->rho > 0 && o->rho < 1) || o->max_backtracks < 1 || !(o->first_step > 0) || o->reg < -1 ||
      o->reg > 1 || (o->reg == FWI_REG_TV && !(o->reg_eps > 0)) || !(o->reg_wp >= 0) ||
      !(o->bias_w >= 0 && o->bias_w <= 1))
    return fail(c, FWI_E_INVAL, "invalid step options");
  const int64_t nmat = c->geo.nmat, n2 = 2 * nmat;
  // device vectors (allocated once; the pair store grows with lbfgs_m)
  if (!c->d_mt) {
    TRY(dalloc(c, &c->d_mt, (size_t)nmat));
    std::vector<double> mt(nmat);
    TRY(fwi_get_mass_tilde(c, mt.data()));
    CUDA_TRY(c, cudaMemcpy(c->d_mt, mt.data(), sizeof(double) * nmat, cudaMemcpyHostToDevice));
  }
  for (double **p : {&c->d_m, &c->d_mprev, &c->d_g, &c->d_gprev, &c->d_dir}) TRY(dalloc(c, p, (size_t)n2));
  TRY(dalloc(c, &c->d_opart, 1024));
  TRY(dalloc(c, &c->d_oscal, 1));
  TRY(dalloc(c, &c->d_oflags, 2));
  TRY(dalloc(c, &c->d_omax, 1));
  if (o->lbfgs_m != c->lb_cap) {
    dfree(c->d_S);
    dfree(c->d_Yv);
    c->lb_cap = o->lbfgs_m;
    c->lb_rho.assign(c->lb_cap, 0.0);
    c->lb_count = c->lb_head = 0;
    if (c->lb_cap > 0) {
      TRY(dalloc(c, &c->d_S, (size_t)n2 * c->lb_cap));
      TRY(dalloc(c, &c->d_Yv, (size_t)n2 * c->lb_cap));
    }
  }
  // 1. misfit and gradient at the current material (Algorithm 2, lines 6-8)
  double J0 = 0.0;
  TRY(run_gradient(c, o->shot0, o->nshots, observed, on_device, &J0));
  const double Jmis0 = J0;
  double Rp[2] = {0.0, 0.0};  // regularisation factors R_lambda, R_mu of this iteration
  if (o->reg >= 0) {
    // (18): M g = R g_reg + g_mis with R_p = wp |g_mis,p| / |g_reg,p| (24)
    double Rf[2];
    TRY(reg_terms(c, o->reg, o->reg_eps, Rf, nullptr));
    double *gmis[2] = {c->d_gl, c->d_gm};
    for (int p = 0; p < 2; p++) {
      if (!(o->invert & (1 << p))) continue;
      double mm = 0.0, rr = 0.0;
      TRY(dot(c, gmis[p], gmis[p], nmat, &mm));
      TRY(dot(c, c->d_rg + p * nmat, c->d_rg + p * nmat, nmat, &rr));
      Rp[p] = rr > 0.0 ? o->reg_wp * std::sqrt(mm) / std::sqrt(rr) : 0.0;
      fwi::opt_axpby(gmis[p], Rp[p], c->d_rg + p * nmat, 1.0, nmat, c->stream);
      J0 += Rp[p] * Rf[p];
    }
    CUDA_TRY(c, cudaGetLastError());
  }
  fwi::opt_pack(c->d_lam, c->d_mu, c->d_m, nmat, c->stream);
  fwi::opt_riesz(c->d_gl, c->d_gm, c->d_mt, c->d_g, nmat, o->invert, c->stream);
  CUDA_TRY(c, cudaGetLastError());
  // 2. new L-BFGS pair s = m_k - m_{k-1}, y = g_k - g_{k-1}, kept when <s, y> > 0
  if (c->lb_have_prev && c->lb_cap > 0) {
    double *S = c->d_S + (size_t)c->lb_head * n2, *Yv = c->d_Yv + (size_t)c->lb_head * n2;
    CUDA_TRY(c, cudaMemcpyAsync(S, c->d_m, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->stream));
    fwi::opt_axpby(S, -1.0, c->d_mprev, 1.0, n2, c->stream);
    CUDA_TRY(c, cudaMemcpyAsync(Yv, c->d_g, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->stream));
    fwi::opt_axpby(Yv, -1.0, c->d_gprev, 1.0, n2, c->stream);
    double sy = 0.0;
    TRY(wdot(c, S, Yv, &sy));
    if (sy > 0.0 && std::isfinite(sy)) {
      c->lb_rho[c->lb_head] = 1.0 / sy;
      c->lb_head = (c->lb_head + 1) % c->lb_cap;
      c->lb_count = std::min(c->lb_count + 1, c->lb_cap);
    }
  }
  // 3. search direction: two-loop recursion, d = -H g
  double gtd = 0.0;
  for (int attempt = 0; attempt < 2; attempt++) {
    CUDA_TRY(c, cudaMemcpyAsync(c->d_dir, c->d_g, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->stream));
    std::vector<double> al(c->lb_count);
    for (int t = 0; t < c->lb_count; t++) {  // newest to oldest
      const int i = (c->lb_head - 1 - t + c->lb_cap) % c->lb_cap;
      double sq = 0.0;
      TRY(wdot(c, c->d_S + (size_t)i * n2, c->d_dir, &sq));
      al[t] = c->lb_rho[i] * sq;
      fwi::opt_axpby(c->d_dir, -al[t], c->d_Yv + (size_t)i * n2, 1.0, n2, c->stream);
    }
    if (c->lb_count > 0) {  // H0 = <s, y> / <y, y> of the newest pair
      const int i = (c->lb_head - 1 + c->lb_cap) % c->lb_cap;
      double yy = 0.0;
      TRY(wdot(c, c->d_Yv + (size_t)i * n2, c->d_Yv + (size_t)i * n2, &yy));
      const double gamma = (1.0 / c->lb_rho[i]) / yy;
      fwi::opt_axpby(c->d_dir, 0.0, c->d_dir, gamma, n2, c->stream);
      for (int t = c->lb_count - 1; t >= 0; t--) {  // oldest to newest
        const int j = (c->lb_head - 1 - t + c->lb_cap) % c->lb_cap;
        double yr = 0.0;
        TRY(wdot(c, c->d_Yv + (size_t)j * n2, c->d_dir, &yr));
        const double beta = c->lb_rho[j] * yr;
        fwi::opt_axpby(c->d_dir, al[t] - beta, c->d_S + (size_t)j * n2, 1.0, n2, c->stream);
      }
    } else {  // no curvature yet: steepest descent sized to first_step * max|m|
      double gmax = 0.0, mmax = 0.0;
      TRY(absmax(c, c->d_g, &gmax));
      TRY(absmax(c, c->d_m, &mmax));
      if (!(gmax > 0.0)) return fail(c, FWI_E_NONFINITE, "zero or non-finite gradient");
      fwi::opt_axpby(c->d_dir, 0.0, c->d_dir, o->first_step * mmax / gmax, n2, c->stream);
    }
    fwi::opt_axpby(c->d_dir, 0.0, c->d_dir, -1.0, n2, c->stream);
    CUDA_TRY(c, cudaGetLastError());
    TRY(wdot(c, c->d_g, c->d_dir, &gtd));
    if (o->bias_w > 0.0 && o->invert == 3 && gtd < 0.0 && std::isfinite(gtd)) {
      // (25): d_l <- |d_l| (W d_m / |d_m| + (1 - W) d_l / |d_l|), kept only if still a descent direction
      double ll = 0.0, mm = 0.0;
      TRY(dot(c, c->d_dir, c->d_dir, nmat, &ll));
      TRY(dot(c, c->d_dir + nmat, c->d_dir + nmat, nmat, &mm));
      if (ll > 0.0 && mm > 0.0) {
        TRY(dalloc(c, &c->d_rg, 2 * nmat));
        CUDA_TRY(c, cudaMemcpyAsync(c->d_rg, c->d_dir, sizeof(double) * nmat, cudaMemcpyDeviceToDevice, c->stream));
        fwi::opt_axpby(c->d_dir, o->bias_w * std::sqrt(ll) / std::sqrt(mm), c->d_dir + nmat, 1.0 - o->bias_w, nmat,
                       c->stream);
        double gtb = 0.0;
        TRY(wdot(c, c->d_g, c->d_dir, &gtb));
        if (gtb < 0.0 && std::isfinite(gtb))
          gtd = gtb;
        else  // not a descent direction: back to the unbiased one
          CUDA_TRY(c, cudaMemcpyAsync(c->d_dir, c->d_rg, sizeof(double) * nmat, cudaMemcpyDeviceToDevice, c->stream));
      }
    }
    if (gtd < 0.0 && std::isfinite(gtd)) break;
    c->lb_count = c->lb_head = 0;  // not a descent direction: drop the memory, steepest descent
    if (attempt == 1) return fail(c, FWI_E_NONFINITE, "no descent direction");
  }
  // 4. Armijo backtracking (Algorithm 1) and update (19)
  double alpha = 1.0, J1 = J0, Jmis1 = Jmis0;
  int trials = 0, accepted = 0;
  for (int b = 0; b <= o->max_backtracks; b++, alpha *= o->rho) {
    int ok = 0;
    TRY(set_trial(c, alpha, c->d_dir, &ok));
    if (!ok) continue;
    double Jt = 0.0;
    trials++;
    fwi_status st = run_misfit(c, o->shot0, o->nshots, observed, on_device, &Jt);
    if (st == FWI_E_NONFINITE) continue;
    TRY(st);
    const double Jmis_t = Jt;
    if (o->reg >= 0) {
      double Rf[2];
      TRY(reg_terms(c, o->reg, o->reg_eps, Rf, nullptr));
      Jt += Rp[0] * Rf[0] + Rp[1] * Rf[1];
    }
    if (Jt < J0 + o->c1 * alpha * gtd) {
      J1 = Jt;
      Jmis1 = Jmis_t;
      accepted = 1;
      break;
    }
  }
  if (!accepted) {  // restore the material and forget the curvature pairs
    int ok = 0;
    TRY(set_trial(c, 0.0, c->d_dir, &ok));
    c->lb_count = c->lb_head = 0;
    c->lb_have_prev = false;
  } else {
    CUDA_TRY(c, cudaMemcpyAsync(c->d_mprev, c->d_m, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_gprev, c->d_g, sizeof(double) * n2, cudaMemcpyDeviceToDevice, c->stream));
    c->lb_have_prev = true;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  info->J_old = J0;
  info->J_new = J1;
  info->alpha = accepted ? alpha : 0.0;
  info->gtd = gtd;
  info->trials = trials;
  info->accepted = accepted;
  info->pairs = c->lb_count;
  info->R_lambda = Rp[0];
  info->R_mu = Rp[1];
  info->Jmis_old = Jmis0;
  info->Jmis_new = Jmis1;
  return FWI_OK;
}

fwi_status fwi_get_mass_tilde(fwi_ctx *c, double *mtilde) {
  if (!c || !mtilde) return FWI_E_INVAL;
  // (C.1a) with LGL quadrature: sum over the interior elements around node i of W_i detJ
  const fwi::Geo &g = c->geo;
  const double hh = 0.5 * c->cfg.h, wd = hh * hh * hh;
  for (int k = 0; k < g.m[2]; k++)
    for (int j = 0; j < g.m[1]; j++)
      for (int i = 0; i < g.m[0]; i++) {
        const int cc[3] = {i, j, k};
        double w = wd, nel = 1.0;
        for (int ax = 0; ax < 3; ax++) {
          w *= (cc[ax] & 1) ? 4.0 / 3.0 : 1.0 / 3.0;
          nel *= (cc[ax] & 1) ? 1 : ((cc[ax] >= 2) + (cc[ax] <= g.m[ax] - 3));
        }
        mtilde[((int64_t)k * g.m[1] + j) * g.m[0] + i] = w * nel;
      }
  return FWI_OK;
}

fwi_status fwi_rhs(fwi_ctx *c, int adjoint, const float *state, float *rate, int on_device) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  if (!c->have_material) return fail(c, FWI_E_STATE, "material not set");
  if (!state || !rate) return fail(c, FWI_E_INVAL, "null argument");
  if (on_device && ((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(rate)) & 15) != 0)
    return fail(c, FWI_E_INVAL, "device state and rate must be 16-byte aligned");
  if (!c->state[0]) return fail(c, FWI_E_STATE, "no RK4 state buffers (a shot batch allocation failed)");
  const size_t n = (size_t)fwi::kFields * c->geo.stride;
  const float *in = state;
  float *out = rate;
  if (!on_device) {
    CUDA_TRY(c, cudaMemcpyAsync(c->state[1], state, n * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    in = c->state[1];
    out = c->state[2];
  }
  fwi::StageArgs a{};
  a.Y = in;
  a.X = in;
  a.out = out;
  a.stage = 0;
  a.nshot = 1;
  TRY(stage(c, adjoint != 0, a));
  if (!on_device)
    CUDA_TRY(c, cudaMemcpyAsync(rate, c->state[2], n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (!on_device) {
    CUDA_TRY(c, cudaMemsetAsync(c->state[1], 0, n * sizeof(float), c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->state[2], 0, n * sizeof(float), c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  return check_status(c);
}

fwi_status fwi_get_state(fwi_ctx *c, float *state, int on_device) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  if (!state) return fail(c, FWI_E_INVAL, "null argument");
  if (!c->state[0]) return fail(c, FWI_E_STATE, "no RK4 state buffers (a shot batch allocation failed)");
  const size_t n = set_floats(c);
  CUDA_TRY(c, cudaMemcpyAsync(state, c->state[0], n * sizeof(float),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FWI_OK;
}

fwi_status fwi_regularization(fwi_ctx *c, int kind, double eps, double *R, double *g_lambda, double *g_mu,
                              int on_device) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  if (!c->have_material) return fail(c, FWI_E_STATE, "material not set");
  if (kind != FWI_REG_TN && kind != FWI_REG_TV) return fail(c, FWI_E_INVAL, "unknown regularisation %d", kind);
  if (kind == FWI_REG_TV && !(eps > 0)) return fail(c, FWI_E_INVAL, "total variation needs eps > 0");
  if (!R) return fail(c, FWI_E_INVAL, "null R");
  const size_t nmat = (size_t)c->geo.nmat;
  TRY(dalloc(c, &c->d_rg, 2 * nmat));
  TRY(dalloc(c, &c->d_rpart, 1024));
  TRY(dalloc(c, &c->d_rval, 2));
  const float *f[2] = {c->d_lam, c->d_mu};
  double *out[2] = {g_lambda, g_mu};
  for (int p = 0; p < 2; p++) {
    double *g = (on_device && out[p]) ? out[p] : c->d_rg + p * nmat;
    fwi::opt_regularization(f[p], c->geo.m, c->cfg.h, kind == FWI_REG_TV, eps, g, c->d_rpart, c->d_rval + p,
                            c->stream);
    CUDA_TRY(c, cudaGetLastError());
    if (!on_device && out[p])
      CUDA_TRY(c, cudaMemcpyAsync(out[p], g, nmat * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  CUDA_TRY(c, cudaMemcpyAsync(R, c->d_rval, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FWI_OK;
}

namespace {

// drop every buffer sized by the shot batch and allocate the RK4 state sets for B shots;
// on failure the context falls back to B = 1 (or, if even that fails, holds no state
// sets, which require_ready reports)
fwi_status resize_batch(fwi_ctx *c, int batch) {
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int b = 0; b < 4; b++) {
    dfree(c->state[b]);
    dfree(c->rstate[b]);
  }
  for (float **p : {&c->d_snap, &c->d_hist, &c->d_traces, &c->d_obs, &c->d_resid}) dfree(*p);
  c->snap_cap = c->hist_cap = 0;
  fwi_status st = FWI_OK;
  for (int attempt = 0; attempt < 2; attempt++) {
    c->batch = attempt == 0 ? batch : 1;
    const size_t n = set_floats(c) * c->batch;
    st = FWI_OK;
    for (int b = 0; b < 4 && st == FWI_OK; b++) {
      st = dalloc(c, &c->state[b], n);
      if (st == FWI_OK && cudaMemsetAsync(c->state[b], 0, n * sizeof(float), c->stream) != cudaSuccess)
        st = fail(c, FWI_E_CUDA, "state clear failed");
    }
    if (st == FWI_OK) break;
    for (int b = 0; b < 4; b++) dfree(c->state[b]);
  }
  if (st == FWI_OK && c->batch != batch) st = fail(c, FWI_E_NOMEM, "no memory for a batch of %d shots", batch);
  const cudaError_t e = cudaStreamSynchronize(c->stream);
  if (st == FWI_OK && e != cudaSuccess) st = fail(c, FWI_E_CUDA, "%s", cudaGetErrorString(e));
  return st;
}

// device bytes one shot of a batch needs for a gradient evaluation in the current
// checkpointing mode: RK4 state sets, history, snapshots and recompute sets, traces
size_t bytes_per_shot(const fwi_ctx *c) {
  const int N = c->cfg.nsteps;
  int every = c->ckpt < 0 ? (int)std::ceil(std::sqrt((double)N)) : c->ckpt;
  if (every >= N) every = 0;
  size_t f = 4 * set_floats(c) + 3 * trace_floats(c);
  if (every == 0)
    f += (size_t)(N + 1) * level_floats(c);
  else
    f += (size_t)(every + 1) * level_floats(c) + (size_t)((N + every - 1) / every) * snap_floats(c) +
         (size_t)4 * set_floats(c);
  return f * sizeof(float);
}

}  // namespace

fwi_status fwi_set_shot_batch(fwi_ctx *c, int batch) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  if (batch < 1 || batch > 1024) return fail(c, FWI_E_INVAL, "shot batch %d outside [1, 1024]", batch);
  if (batch == c->batch && c->state[0]) return FWI_OK;
  return resize_batch(c, batch);
}

fwi_status fwi_tune_shot_batch(fwi_ctx *c, int shot0, int nshots, int max_batch, int steps, double mem_fraction,
                               int *chosen) {
  if (!c) return FWI_E_INVAL;
  TRY(require_ready(c, shot0, nshots));
  if (!chosen || max_batch < 1 || steps < 1 || steps >= c->cfg.nsteps || !(mem_fraction > 0 && mem_fraction <= 1))
    return fail(c, FWI_E_INVAL, "invalid tuning arguments");
  // memory cap: what is free plus what this context's per-shot buffers hold now
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(c, cudaMemGetInfo(&free_b, &total_b));
  size_t held = (size_t)4 * set_floats(c) * c->batch + c->hist_cap * level_floats(c) + c->snap_cap * snap_floats(c);
  if (c->rstate[0]) held += (size_t)4 * set_floats(c) * c->batch;
  if (c->d_traces) held += (size_t)3 * trace_floats(c) * c->batch;
  held *= sizeof(float);
  const double avail = mem_fraction * (double)(free_b + held);
  int bmax = (int)std::min<double>(avail / (double)bytes_per_shot(c), 1024.0);
  bmax = std::min(std::min(bmax, max_batch), nshots);
  if (bmax < 1) bmax = 1;
  std::vector<int> cand;
  for (int b = 1; b < bmax; b *= 2) cand.push_back(b);
  cand.push_back(bmax);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(c, FWI_E_CUDA, "event creation failed");
  }
  int best = 1;
  double best_rate = -1.0;
  fwi_status st = FWI_OK;
  for (size_t q = 0; q < cand.size() && st == FWI_OK; q++) {
    const int B = cand[q];
    st = resize_batch(c, B);
    // one untimed step, then `steps` timed forward RK4 steps of shots shot0 .. shot0 + B - 1
    if (st == FWI_OK) st = rk4_step(c, false, 0, shot0, B, nullptr, 0);
    if (st == FWI_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) st = fail(c, FWI_E_CUDA, "event record failed");
    for (int n = 1; n <= steps && st == FWI_OK; n++) st = rk4_step(c, false, n, shot0, B, nullptr, 0);
    float ms = 0.f;
    if (st == FWI_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = fail(c, FWI_E_CUDA, "tuning timing failed");
    if (st != FWI_OK) break;
    // shot-steps per second; a larger batch has to be 2 % faster to be kept (memory)
    const double rate = (double)B * steps / (ms * 1e-3);
    if (rate > 1.02 * best_rate) {
      best = B;
      best_rate = rate;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TRY(st);
  TRY(resize_batch(c, best));
  *chosen = best;
  return FWI_OK;
}

fwi_status fwi_tune_tiles(fwi_ctx *c, int shot0, int nshots, int steps, int chosen[2]) {
  if (!c) return FWI_E_INVAL;
  TRY(require_ready(c, shot0, nshots));
  if (!chosen || steps < 1 || steps >= c->cfg.nsteps) return fail(c, FWI_E_INVAL, "invalid tuning arguments");
  const int nb = std::min(nshots, c->batch);
  static const int kcs[4] = {4, 8, 16, 32}, segs[2] = {16, 32};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(c, FWI_E_CUDA, "event creation failed");
  }
  drop_graphs(c);  // recorded sweeps hold the launch shapes they were recorded with
  const fwi::Geo saved = c->geo;
  int best[2] = {saved.int_kc, saved.pml_seg};
  float best_ms = -1.f;
  fwi_status st = FWI_OK;
  for (int i = 0; i < 4 && st == FWI_OK; i++)
    for (int j = 0; j < 2 && st == FWI_OK; j++) {
      c->geo.int_kc = kcs[i];
      c->geo.pml_seg = segs[j];
      // one untimed step, then `steps` timed forward RK4 steps of the first batch of shots
      st = rk4_step(c, false, 0, shot0, nb, nullptr, 0);
      if (st == FWI_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) st = fail(c, FWI_E_CUDA, "event record failed");
      for (int n = 1; n <= steps && st == FWI_OK; n++) st = rk4_step(c, false, n, shot0, nb, nullptr, 0);
      float ms = 0.f;
      if (st == FWI_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        st = fail(c, FWI_E_CUDA, "tuning timing failed");
      if (st == FWI_OK && (best_ms < 0.f || ms < best_ms)) {
        best_ms = ms;
        best[0] = kcs[i];
        best[1] = segs[j];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->geo = saved;
  TRY(st);
  c->geo.int_kc = best[0];
  c->geo.pml_seg = best[1];
  chosen[0] = best[0];
  chosen[1] = best[1];
  return FWI_OK;
}

fwi_status fwi_set_checkpointing(fwi_ctx *c, int interval) {
  if (!c) return FWI_E_INVAL;
  c->ckpt = interval;
  return FWI_OK;
}

fwi_status fwi_set_persistent(fwi_ctx *c, int enable, double wait_ms, int test_extra_arrivals) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  if (enable && !(wait_ms > 0.0 && wait_ms <= 60000.0)) return fail(c, FWI_E_INVAL, "wait_ms outside (0, 60000]");
  if (test_extra_arrivals < 0) return fail(c, FWI_E_INVAL, "negative test_extra_arrivals");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (enable) {
    if (!c->d_all) {
      std::vector<int> all((size_t)c->geo.nnode);
      size_t q = 0;
      for (int k = 0; k < c->geo.n[2]; k++)
        for (int j = 0; j < c->geo.n[1]; j++)
          for (int i = 0; i < c->geo.n[0]; i++) all[q++] = (k * c->geo.n[1] + j) * c->geo.px + i;
      TRY(dalloc(c, &c->d_all, all.size()));
      CUDA_TRY(c, cudaMemcpy(c->d_all, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice));
    }
    TRY(dalloc(c, &c->d_bar, 2));
    TRY(dalloc(c, &c->d_status, 1));
    CUDA_TRY(c, cudaMemset(c->d_status, 0, sizeof(int)));
    c->wait_ms = wait_ms;
    c->bar_extra = test_extra_arrivals;
  }
  c->persistent = enable != 0;
  return FWI_OK;
}

fwi_status fwi_set_copy_wait(fwi_ctx *c, double wait_ms, int test_extra_bytes) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  if (!(wait_ms > 0.0 && wait_ms <= 60000.0)) return fail(c, FWI_E_INVAL, "wait_ms outside (0, 60000]");
  if (test_extra_bytes < 0 || test_extra_bytes > 65536)
    return fail(c, FWI_E_INVAL, "test_extra_bytes outside [0, 65536]");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->geo.wait_cycles = (long long)(wait_ms * 1e-3 * 2.2e9);
  c->geo.copy_extra = test_extra_bytes;
  drop_graphs(c);  // recorded sweeps hold the wait limits they were recorded with
  return FWI_OK;
}

fwi_status fwi_set_graphs(fwi_ctx *c, int enable) {
  if (!c) return FWI_E_INVAL;
  TRY(check_stream(c));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->graphs = enable != 0;
  if (!c->graphs) drop_graphs(c);
  return FWI_OK;
}

fwi_status fwi_set_timing(fwi_ctx *c, int enable) {
  if (!c) return FWI_E_INVAL;
  c->timing = enable != 0;
  return FWI_OK;
}

fwi_status fwi_get_timing(fwi_ctx *c, int which, double *ms, int64_t *launches) {
  if (!c || which < 0 || which > 3) return FWI_E_INVAL;
  TRY(time_flush(c));
  if (ms) *ms = c->t_ms[which];
  if (launches) *launches = c->t_launch[which];
  return FWI_OK;
}

fwi_status fwi_reset_timing(fwi_ctx *c) {
  if (!c) return FWI_E_INVAL;
  TRY(time_flush(c));
  for (int i = 0; i < 4; i++) {
    c->t_ms[i] = 0;
    c->t_launch[i] = 0;
  }
  return FWI_OK;
}

}  // extern "C"
