/*
 * fwi.h -- C ABI of the GB300 per-shot material-gradient library for
 * time-domain elastic full-waveform inversion in PML-truncated 3D media
 * (Fathi, Kallivokas & Poursartip, arXiv:1504.08340).
 *
 * The library evaluates, for a trial distribution of the Lame parameters
 * lambda(x), mu(x), the misfit (7) between computed and observed receiver
 * displacements and its gradients dJ/dlambda_i, dJ/dmu_i (the misfit parts
 * g_mis of (18), Appendix C (C.1f)/(C.1g)). One evaluation runs
 *   - the state problem: the semi-discrete system (5) of the hybrid
 *     spectral-element discretisation (displacement-only interior, displacement-
 *     stress PML, 27-node LGL hexahedra) as the first-order system (6),
 *     integrated by classic RK4 (Sec. 2);
 *   - the adjoint problem (14)/(15) with the transposed system matrices,
 *     integrated by the reverse RK4 of Appendix B, driven by the receiver
 *     residuals (13a);
 *   - the time integrals (C.1f)/(C.1g) over the interior domain, in FP64.
 * All wavefield arithmetic runs in CUDA kernels on the GPU of the context's
 * stream, in FP32 with FP64 accumulation of J and of the gradients.
 *
 * Mesh. A structured box of 27-node hexahedra of edge h: nx*ny*nz interior
 * ("regular domain") elements, wrapped by npml PML elements on the faces
 * x-, x+, y-, y+ and the bottom (and the top when top_pml = 1; the paper's
 * configuration, top_pml = 0, has a traction-free ground surface, Eq. (2a)).
 * Nodes are indexed (i, j, k), 0 <= i <= 2(nx + 2 npml), 0 <= j <= 2(ny + 2 npml),
 * 0 <= k <= 2(nz + npml [+ npml]), i along x, j along y, k along depth, k = 0 at
 * the top. Node number n = (k * NJ + j) * NI + i with NI, NJ the node counts
 * along x and y. Displacements vanish on the outer PML faces (2c).
 *
 * Material. lambda and mu are nodal (quadratic) on the interior nodes only,
 * FP32 arrays of (2nz+1)(2ny+1)(2nx+1) values ordered [k][j][i] (i fastest),
 * in Pa; they are extended into the PML by the value at the nearest interface
 * node (Sec. 4.1: "extended into the PML"). rho is constant.
 *
 * Conventions for every call:
 *   - the caller owns every array it passes; the library keeps no caller
 *     pointer beyond the call;
 *   - on_device = 1: the array arguments marked "host or device" are device
 *     pointers usable on the context's stream; on_device = 0: host pointers;
 *   - every call returns an fwi_status; fwi_last_error() gives detail;
 *   - on an error the outputs are left untouched; the context stays usable
 *     except after FWI_E_CUDA, which is sticky;
 *   - calls are synchronous with respect to their outputs: they wait for the
 *     context's stream before returning.
 */
#ifndef FWI_H
#define FWI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fwi_ctx fwi_ctx; /* opaque, owned by the library */

typedef enum {
  FWI_OK = 0,
  FWI_E_INVAL = 1,     /* invalid argument or size */
  FWI_E_NOMEM = 2,     /* device or host allocation failed */
  FWI_E_CUDA = 3,      /* a CUDA call failed; sticky */
  FWI_E_UNSTABLE = 4,  /* time step above the RK4 stability estimate */
  FWI_E_NONFINITE = 5, /* NaN or Inf in material, traces or gradients */
  FWI_E_TIMEOUT = 6,   /* a bounded device wait gave up */
  FWI_E_STATE = 7,     /* call out of order (e.g. no material or receivers yet) */
  FWI_E_BOUNDS = 8     /* bounds-checked build only: a device index was out of range */
} fwi_status;

enum { FWI_WAVELET_RICKER = 0, FWI_WAVELET_GAUSS = 1 };
enum { FWI_REG_TN = 0, FWI_REG_TV = 1 };  /* regularisation schemes, Eqs. (8) and (9) */

typedef struct {
  int nx, ny, nz;   /* interior elements per axis (>= 1) */
  int npml;         /* PML elements on each truncated face (>= 0) */
  int top_pml;      /* 0: free ground surface (paper); 1: PML on the top face too */
  double h;         /* element edge, m */
  double rho;       /* mass density, kg/m^3 */
  double pml_alpha0;/* PML stretch amplitude alpha_o (Sec. 4.1 uses 5) */
  double pml_beta0; /* PML attenuation amplitude beta_o, 1/s (Sec. 4.1 uses 400) */
  int pml_m;        /* PML profile exponent m (Sec. 4.1 uses 2) */
  double dt;        /* RK4 step, s */
  int nsteps;       /* number of steps; traces have nsteps + 1 samples t_n = n dt */
  void *cuda_stream;/* cudaStream_t for all work, or NULL for the legacy default stream */
} fwi_config;

/* Create a context for one mesh (Sec. 2 / Fig. 3 domain layout). Allocates the
 * device state (four RK4 stage buffers of 27 FP32 fields per node) on the
 * current CUDA device. Errors: FWI_E_INVAL (sizes), FWI_E_NOMEM, FWI_E_CUDA. */
fwi_status fwi_create(const fwi_config *cfg, fwi_ctx **out);

/* Release the context and all its device memory. NULL is accepted. */
void fwi_destroy(fwi_ctx *ctx);

/* Last error message of this context (never NULL; "" when none). */
const char *fwi_last_error(const fwi_ctx *ctx);

/* 1 if this library was compiled with -DFWI_BOUNDS_CHECK, else 0 (host only; no
 * context, no device work). In that build every node number a kernel reads from a list
 * (interface shell, outer faces, source and receiver points, snapshot and sweep node
 * lists) and every node a structured kernel derives from its tile, with the reach of
 * its stencils, is checked before any access; an index out of range is skipped and
 * recorded, and the next synchronising call (fwi_forward, fwi_misfit,
 * fwi_adjoint_gradient, fwi_rhs, fwi_step) returns FWI_E_BOUNDS with the index and the
 * check site in fwi_last_error(). The results of the two builds are otherwise the same. */
int fwi_bounds_checked(void);

/* Static description of a status code. */
const char *fwi_status_string(fwi_status s);

/* Sizes: dims[0..2] nodes per axis (NI, NJ, NK), dims[3] node count,
 * dims[4] interior (material) node count, dims[5] field stride in floats of the
 * state layout used by fwi_rhs, dims[6] number of elements, dims[7] number of
 * PML nodes, dims[8] row pitch PX of that layout (NI rounded up to 4). */
fwi_status fwi_get_dims(const fwi_ctx *ctx, int64_t dims[9]);

/* Set the trial Lame parameters (D4: nodal values on the interior nodes,
 * [k][j][i], Pa; host or device). Checks finiteness, mu > 0, lambda + 2 mu > 0
 * (FWI_E_NONFINITE / FWI_E_INVAL) and the RK4 time-step limit estimated as
 * dt * vp_max / (h/2) <= 0.66 (FWI_E_UNSTABLE). */
fwi_status fwi_set_material(fwi_ctx *ctx, const float *lambda, const float *mu, int on_device);

/* Point-load sources (the right side of (3a) for a nodal load): shot s loads
 * node node_ijk[3s..3s+2] (host) with force dir[3s..3s+2] * r(t) (host), where
 * r is the wavelet: FWI_WAVELET_RICKER, wparams = {f0 [Hz], t0 [s], amplitude [N]},
 * r = A (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2);
 * FWI_WAVELET_GAUSS (Table 1 pulse, read as A exp(-(t - mu)^2 / sigma)),
 * wparams = {mu [s], sigma [s^2], amplitude [N]}. The node must not lie on a
 * Dirichlet face. Errors: FWI_E_INVAL. */
fwi_status fwi_set_sources(fwi_ctx *ctx, int nshots, const int *node_ijk, const double *dir,
                           int wavelet, const double *wparams);

/* Receivers (delta(x - x_j) of (7)): nrec distinct nodes node_ijk[3r..3r+2]
 * (host), not on a Dirichlet face. Errors: FWI_E_INVAL. */
fwi_status fwi_set_receivers(fwi_ctx *ctx, int nrec, const int *node_ijk);

/* State problem (6) for shots shot0 .. shot0+nshots-1; writes the receiver
 * displacements traces[s][n][r][c] = u_c(x_r, t_n), n = 0..nsteps, FP32
 * (host or device, caller-owned, nshots*(nsteps+1)*nrec*3 floats).
 * Errors: FWI_E_STATE (no material / sources / receivers), FWI_E_INVAL,
 * FWI_E_NONFINITE, FWI_E_TIMEOUT (a bounded device wait gave up: a grid barrier of the
 * persistent sweep, or a plane copy of the interior kernel; the context stays usable),
 * FWI_E_BOUNDS (bounds-checked build only), FWI_E_CUDA. */
fwi_status fwi_forward(fwi_ctx *ctx, int shot0, int nshots, float *traces, int on_device);

/* Misfit (7) without regularisation, summed over the shots, with the trapezoid
 * rule in time: J = 1/2 sum_s sum_r sum_n w_n dt |u - u_m|^2 (w_0 = w_N = 1/2).
 * observed: same layout as fwi_forward's traces (host or device). *J: host. */
fwi_status fwi_misfit(fwi_ctx *ctx, int shot0, int nshots, const float *observed, int on_device,
                      double *J);

/* Misfit and its gradients for shots shot0 .. shot0+nshots-1 (Algorithm 2,
 * lines 6-8): state solve (6), adjoint solve (15)/Appendix B, and
 *   g_lambda[i] = -int_0^T int_RD chi_i (div w)(div u)            (C.1f)
 *   g_mu[i]     = -int_0^T int_RD chi_i 2 eps(w):eps(u)           (C.1g)
 * i.e. g_mis = dJ/dlambda_i, dJ/dmu_i on the interior nodes ([k][j][i], FP64,
 * summed over the shots; host or device per on_device). The full gradient of
 * (18) with R = 0 is g = Mtilde^-1 g_mis, see fwi_get_mass_tilde. *J: host.
 * Device memory for the forward displacement history, nsteps+1 copies of the
 * interior displacement field (12 bytes per interior node per step), is
 * allocated on the first call and kept. Errors as fwi_forward. */
fwi_status fwi_adjoint_gradient(fwi_ctx *ctx, int shot0, int nshots, const float *observed,
                                int on_device, double *J, double *g_lambda, double *g_mu);

/* Options of one inversion iteration (fwi_step). */
typedef struct {
  int shot0, nshots;  /* shots whose summed misfit is minimised */
  int invert;         /* 1: lambda only, 2: mu only, 3: both (simultaneous inversion) */
  int lbfgs_m;        /* L-BFGS pairs kept (Sec. 3.2 keeps 15); 0: steepest descent */
  double c1;          /* Armijo sufficient-decrease constant (Algorithm 1: 1e-4) */
  double rho;         /* backtracking factor (Algorithm 1: 0.5) */
  int max_backtracks; /* trial steps before the iteration gives up */
  double first_step;  /* first trial update (no L-BFGS pairs yet): max|alpha d| = first_step * max|m| */
  int reg;            /* regularisation of (7): -1 none (R = 0), FWI_REG_TN (8) or FWI_REG_TV (9) */
  double reg_eps;     /* eps of (9) */
  double reg_wp;      /* wp of (23c): each iteration R_p = wp |g_mis,p| / |g_reg,p| (24), p = lambda, mu */
  double bias_w;      /* W of (25): the lambda search direction is biased toward mu's (0: no biasing) */
} fwi_step_opts;

typedef struct {
  double J_old, J_new; /* misfit before and after the iteration */
  double alpha;        /* accepted step length (alpha^lambda = alpha^mu, Algorithm 1) */
  double gtd;          /* directional derivative of J along the search direction */
  int trials;          /* misfit evaluations of the line search */
  int accepted;        /* 1 when the Armijo condition held and the material moved */
  int pairs;           /* L-BFGS pairs held after the iteration */
  double R_lambda, R_mu; /* regularisation factors of the iteration (24) (0 without regularisation) */
  double Jmis_old, Jmis_new; /* misfit parts of J_old, J_new */
} fwi_step_info;

/* One iteration of Algorithm 2 (lines 6-11) at the current material:
 * gradient (state (6), adjoint (15), g = Mtilde^-1 (R g_reg + g_mis) of (18); with
 * opts->reg >= 0 the factors R_lambda, R_mu follow (24) from opts->reg_wp at the
 * current material, and J_old, J_new are the misfit plus R_p times the terms of
 * fwi_regularization: the objective (7) that the line search tests),
 * L-BFGS search direction (two-loop recursion in the Mtilde inner product,
 * <a, b> = sum_i a_i Mtilde_i b_i, so that <g, d> = g_mis . d is the exact
 * directional derivative), Armijo backtracking of Algorithm 1 (alpha^lambda =
 * alpha^mu, halved together) and the update (19), which becomes the context's
 * material. Trial materials that violate mu > 0, lambda + 2 mu > 0 or the time-step
 * limit count as failed trials. The L-BFGS pairs live on the device (FP64, 2 *
 * lbfgs_m vectors of 2 * dims[4] values) and persist between calls; a pair is kept
 * only when <s, y> > 0. With opts->bias_w = W > 0 and invert = 3, the lambda part
 * of the direction becomes |d_l| (W d_m / |d_m| + (1 - W) d_l / |d_l|) (25)
 * (Euclidean norms; the unbiased direction is kept when the biased one is not a
 * descent direction). observed: as fwi_misfit (host or device); info: host.
 * When no trial satisfies Armijo the material is restored, info->accepted = 0 and
 * the memory is cleared. Errors: as fwi_adjoint_gradient, FWI_E_INVAL (options:
 * also reg outside -1..1, TV with reg_eps <= 0, reg_wp < 0, bias_w outside [0, 1]). */
fwi_status fwi_step(fwi_ctx *ctx, const float *observed, int on_device, const fwi_step_opts *opts,
                    fwi_step_info *info);

/* Forget the L-BFGS pairs (e.g. when the source wavelet changes, Sec. 3.3.2). */
fwi_status fwi_step_reset(fwi_ctx *ctx);

/* Regularisation term of the objective (7) at the context's material, Sec. 3.1:
 * Tikhonov (kind FWI_REG_TN, Eq. (8)) or total variation (FWI_REG_TV, Eq. (9)),
 * for lambda and for mu, without the factors R_lambda, R_mu:
 *   R[0], R[1] (host): int |grad f|^2 / 2 (TN) or int (|grad f|^2 + eps)^(1/2) (TV)
 *     over the interior domain, f = lambda, mu, by the LGL quadrature of the mesh;
 *   g_lambda, g_mu (FP64, dims[4] values on the interior nodes, host or device per
 *     on_device; either may be null): their gradients, g_reg of (18), as in
 *     (C.1b)-(C.1e).
 * The TV functional is the one whose derivative is (17a)/(C.1d): (9) without
 * its factor 1/2. Errors: FWI_E_STATE (no material), FWI_E_INVAL (unknown kind,
 * eps <= 0 for TV, null R). */
fwi_status fwi_regularization(fwi_ctx *ctx, int kind, double eps, double *R, double *g_lambda, double *g_mu,
                              int on_device);

/* How fwi_adjoint_gradient and fwi_step give the adjoint sweep the forward
 * displacement u(t_n) that the gradient integrals (C.1f)/(C.1g) need at every step:
 *   interval = 0 (default): the forward sweep stores u at every step
 *     ((nsteps + 1) * 3 * dims[4] floats of device memory);
 *   interval > 0: the forward sweep stores its full RK4 state every `interval`
 *     steps (ceil(nsteps / interval) snapshots of 27 * dims[5] floats). The adjoint
 *     sweep then walks the segments backwards and recomputes each segment's forward
 *     steps from its snapshot, in a second state set, into an (interval + 1)-level
 *     history, before running the adjoint steps of that segment;
 *   interval < 0: interval = ceil(sqrt(nsteps)), the sqrt(T) checkpointing scheme.
 * Checkpointing costs one more forward sweep. The recomputed steps repeat the
 * forward arithmetic exactly, so J and the gradients are bit-identical to those of
 * interval 0. The paper does not say how u(t) reaches the gradient. Memory is
 * allocated by the next gradient call. Errors: FWI_E_INVAL (null context). */
fwi_status fwi_set_checkpointing(fwi_ctx *ctx, int interval);

/* Number of shots B that one launch of each stage kernel advances together
 * (default 1). The shots of a fwi_forward, fwi_misfit, fwi_adjoint_gradient or
 * fwi_step call (each shot an independent wave problem on the same material,
 * Sec. 3: the misfit and the gradient are sums over the shots) run in groups of
 * B: the RK4 state sets, traces, residuals, observed-trace slots, displacement
 * history and snapshots hold B shots each, shot b of a group at b times one
 * shot's size. Results are those of B = 1: traces bitwise, J and the gradients
 * up to the order of the FP64 sums over the shots. Device memory grows about B
 * times. Reallocates those buffers (synchronising the context's stream) when B
 * changes. Errors: FWI_E_INVAL (B outside [1, 1024]), FWI_E_NOMEM. */
fwi_status fwi_set_shot_batch(fwi_ctx *ctx, int batch);

/* Picks the shot batch B by measurement and leaves the context at it (as
 * fwi_set_shot_batch). Candidates are B = 1, 2, 4, ... below, and equal to, the
 * largest B that is at most max_batch and nshots and whose per-shot buffers for a
 * gradient evaluation (RK4 state sets, traces, and the history, snapshots and
 * recompute sets of the current checkpointing mode) fit in mem_fraction of the
 * device memory that is free or held by this context's per-shot buffers. Each
 * candidate runs one untimed and `steps` timed forward RK4 steps of the shots
 * shot0 .. shot0 + B - 1 (CUDA events on the context's stream); a larger B is kept
 * only if it advances at least 2 % more shot-steps per second.
 *   chosen (host): the B picked.
 * The context's RK4 state is cleared. Errors: FWI_E_STATE (material, sources or
 * receivers not set), FWI_E_INVAL (shot range, max_batch < 1, steps outside
 * [1, nsteps), mem_fraction outside (0, 1], null chosen), FWI_E_NOMEM, FWI_E_CUDA. */
fwi_status fwi_tune_shot_batch(fwi_ctx *ctx, int shot0, int nshots, int max_batch, int steps, double mem_fraction,
                               int *chosen);

/* Picks the launch shapes of the stage kernels by measurement: for each candidate (planes
 * per block of the interior kernel: 4, 8, 16, 32; node pairs per x segment of a PML warp
 * task: 16, 32) it times `steps` forward RK4 steps (1 <= steps < nsteps) of the first
 * shot batch of shots [shot0, shot0 + nshots), keeps the fastest for later calls and
 * returns it in chosen[0] (planes) and chosen[1] (pairs). The shapes change no node's
 * arithmetic: every result is bitwise the same with any of them. Not in the paper.
 * Errors: FWI_E_INVAL, FWI_E_STATE, FWI_E_CUDA. */
fwi_status fwi_tune_tiles(fwi_ctx *ctx, int shot0, int nshots, int steps, int chosen[2]);

/* Current material ([k][j][i] as in fwi_set_material; host or device). */
fwi_status fwi_get_material(fwi_ctx *ctx, float *lambda, float *mu, int on_device);

/* Diagonal of the lumped mass-like matrix Mtilde of (C.1a), FP64, on the
 * interior nodes (host array of dims[4] values). */
fwi_status fwi_get_mass_tilde(fwi_ctx *ctx, double *mtilde);

/* Right side of the first-order system at one state (no loads):
 * adjoint = 0: Eq. (6), rate = (x1|PML, x2, M^-1(-G x0 - K x1 - C x2));
 * adjoint = 1: the adjoint system in reversed time s = T - t,
 *   M z'' + C' z' + K' z + G' zbar = 0 with C' = D C^T D, K' = D K^T D,
 *   G' = D G^T D, D = diag(I on displacements, -I on stresses); with
 *   z = D y1(T - s), z' = -D y2(T - s), zbar = -D y0(T - s) this is (15).
 * state and rate: 27 fields of dims[5] floats each (host or device); field
 * 9*l + c holds level l (0: history, 1: value, 2: rate) and component c
 * (0..2 displacement x,y,z; 3..8 stress xx,yy,zz,yz,xz,xy) of every node;
 * node (i, j, k) sits at offset (k * NJ + j) * PX + i of a field (PX = dims[8];
 * the padding entries i >= NI must be zero).
 * Displacement fields must be zero on the Dirichlet faces and history / stress
 * fields zero off the PML nodes. Device buffers (on_device = 1) must start on a
 * 16-byte boundary (the stage kernels read the state with 16-byte and tensor copies).
 * Errors: FWI_E_INVAL (null or unaligned), FWI_E_STATE (no material), FWI_E_TIMEOUT,
 * FWI_E_CUDA. */
fwi_status fwi_rhs(fwi_ctx *ctx, int adjoint, const float *state, float *rate, int on_device);

/* The RK4 state at the end of the most recent sweep, in the layout of fwi_rhs
 * (27 fields of dims[5] floats, host or device): after fwi_forward(ctx, s, 1, ...)
 * it is shot s's state x(t_N) of (6) (displacement, rate and history levels, the
 * PML stresses). A diagnostic accessor, e.g. for energy checks. After a gradient
 * evaluation it holds the reversed-time adjoint state at its end instead, with
 * tau(T) = mu (T + diag T) + lambda tr(T) I of the adjoint stress T in the stress slots
 * (the adjoint sweep advances (w, tau(T)), which has the forward system's form).
 * Caller-owned output; synchronous.
 * Errors: FWI_E_INVAL (null), FWI_E_STATE (no state buffers), FWI_E_CUDA. */
fwi_status fwi_get_state(fwi_ctx *ctx, float *state, int on_device);

/* Persistent forward sweeps: with enable = 1, every later forward sweep (fwi_forward, and
 * the forward part of fwi_misfit, fwi_adjoint_gradient and fwi_step) of a group of shots
 * runs as one cooperative kernel launch (one per checkpoint segment) instead of about
 * 20 launches per RK4 step. All nodes take the general per-node formulas of (3a)/(3b);
 * the four stages of a step are separated by grid-wide barriers, and source loads,
 * receiver samples and the displacement history are written by the threads that own
 * the nodes. Meant for small meshes, where a step is dominated by launch latency; the
 * results agree with the class-specialised kernels to rounding. Every barrier waits at
 * most wait_ms milliseconds (0 < wait_ms <= 60000): a barrier that gives up makes the
 * kernel return, and the call that ran the sweep returns FWI_E_TIMEOUT (the context stays
 * usable). test_extra_arrivals > 0 makes every barrier wait for that many blocks more
 * than the launch has, so that the timeout path can be exercised; use 0 otherwise.
 * The adjoint sweep always uses the specialised kernels. Not in the paper.
 * Errors: FWI_E_INVAL, FWI_E_NOMEM, FWI_E_CUDA. */
fwi_status fwi_set_persistent(fwi_ctx *ctx, int enable, double wait_ms, int test_extra_arrivals);

/* Bounded waits of the interior stage kernel: each plane of the stage input reaches the
 * kernel's shared-memory ring as one tensor copy (TMA) that completes on an mbarrier, and
 * every wait for one gives up after wait_ms milliseconds (0 < wait_ms <= 60000; 1000 when
 * the context is created). A wait that gives up makes its thread block wait (again
 * bounded) for its copies in flight and return; the call that ran the sweep returns
 * FWI_E_TIMEOUT and the context stays usable. test_extra_bytes > 0 (at most 65536) makes
 * every plane barrier expect that many bytes more than its copy delivers, so that the
 * timeout path can be exercised; use 0 otherwise. Drops recorded graphs. Not in the
 * paper. Errors: FWI_E_INVAL, FWI_E_CUDA. */
fwi_status fwi_set_copy_wait(fwi_ctx *ctx, double wait_ms, int test_extra_bytes);

/* CUDA graphs for the time loops: with enable = 1, each sweep of a later call (a forward
 * sweep, the adjoint sweep over the stored history, one checkpoint segment) is recorded by
 * stream capture the first time it runs with a given shot group and replayed as one
 * graph launch afterwards. A replay issues the same kernels with the same arguments in
 * the same order as the direct launches, so results are bitwise the same; it saves the
 * host launch work and the gaps between kernels. Recorded graphs are dropped when any
 * device buffer of the library is allocated or freed (they hold raw pointers), when
 * graphs are turned off, and at fwi_destroy. Kernel timing (fwi_set_timing) runs the
 * sweeps directly. Not in the paper. Errors: FWI_E_INVAL, FWI_E_CUDA. */
fwi_status fwi_set_graphs(fwi_ctx *ctx, int enable);

/* Kernel timing: with enable = 1 every stage-kernel launch of later calls is
 * bracketed by CUDA events on the context's stream; fwi_get_timing returns the
 * summed device time (ms) and launch count of kernel class `which`
 * (0: RK stage kernels, 1: gradient kernel, 2: point-load / sampling kernels,
 * 3: all kernels launched, time unset) since the last reset. */
fwi_status fwi_set_timing(fwi_ctx *ctx, int enable);
fwi_status fwi_get_timing(fwi_ctx *ctx, int which, double *ms, int64_t *launches);
fwi_status fwi_reset_timing(fwi_ctx *ctx);

/* Misfit of traces that are already on the GPU, for callers that cannot allocate
 * device memory (code running where cudaMalloc is not allowed or where the host
 * application owns the whole device-memory budget). No counterpart in the paper:
 * it computes the same J as fwi_misfit's reduction, from caller-supplied traces.
 * traces, observed: device arrays of (nsteps+1)*nrec*3 floats ([n][r][c]);
 * J: host. The call allocates nothing: its scratch is a fixed 512 KiB device
 * array inside the library, which every GPU that loads the library keeps until
 * the process exits. Each call looks up that array's address in the current
 * context. The call is synchronous (it waits on cuda_stream before returning),
 * so it must not be issued on a stream that is being captured. Calls share the
 * array, so calls that overlap on the GPU race. Errors: FWI_E_INVAL (null
 * pointers, nrec < 1, dt <= 0, or nsteps + 1 > 65536, the scratch limit),
 * FWI_E_NONFINITE (a trace or observed value is NaN/Inf, or the sum overflows),
 * FWI_E_CUDA. */
fwi_status fwi_trace_misfit_noalloc(const float *traces, const float *observed, int nsteps, int nrec,
                                    double dt, void *cuda_stream, double *J);

#ifdef __cplusplus
}
#endif

#endif /* FWI_H */
