"""Thin Python binding of the C ABI in include/fwi.h (argument marshalling only).

Every operation runs in the CUDA library ``libfwi.so``; there is no fallback.
Arrays are either torch CUDA tensors (passed as device pointers on the
context's stream) or numpy arrays (passed as host pointers).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfwi.so")

STATUS = {0: "FWI_OK", 1: "FWI_E_INVAL", 2: "FWI_E_NOMEM", 3: "FWI_E_CUDA", 4: "FWI_E_UNSTABLE",
          5: "FWI_E_NONFINITE", 6: "FWI_E_TIMEOUT", 7: "FWI_E_STATE", 8: "FWI_E_BOUNDS"}
WAVELETS = {"ricker": 0, "gauss": 1}


class FWIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class _Config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("npml", C.c_int),
                ("top_pml", C.c_int), ("h", C.c_double), ("rho", C.c_double),
                ("pml_alpha0", C.c_double), ("pml_beta0", C.c_double), ("pml_m", C.c_int),
                ("dt", C.c_double), ("nsteps", C.c_int), ("cuda_stream", C.c_void_p)]


class StepOpts(C.Structure):
    """fwi_step_opts: one iteration of Algorithm 2 (L-BFGS + Armijo backtracking)."""
    _fields_ = [("shot0", C.c_int), ("nshots", C.c_int), ("invert", C.c_int), ("lbfgs_m", C.c_int),
                ("c1", C.c_double), ("rho", C.c_double), ("max_backtracks", C.c_int),
                ("first_step", C.c_double), ("reg", C.c_int), ("reg_eps", C.c_double), ("reg_wp", C.c_double),
                ("bias_w", C.c_double)]


class StepInfo(C.Structure):
    _fields_ = [("J_old", C.c_double), ("J_new", C.c_double), ("alpha", C.c_double), ("gtd", C.c_double),
                ("trials", C.c_int), ("accepted", C.c_int), ("pairs", C.c_int), ("R_lambda", C.c_double),
                ("R_mu", C.c_double), ("Jmis_old", C.c_double), ("Jmis_new", C.c_double)]


# every symbol the header declares; the CPU test checks the library exports them all
EXPORTS = ("fwi_create", "fwi_destroy", "fwi_last_error", "fwi_status_string", "fwi_bounds_checked", "fwi_get_dims",
           "fwi_set_material", "fwi_set_sources", "fwi_set_receivers", "fwi_forward", "fwi_misfit",
           "fwi_adjoint_gradient", "fwi_get_mass_tilde", "fwi_rhs", "fwi_get_state", "fwi_set_graphs", "fwi_set_persistent", "fwi_set_copy_wait",
           "fwi_set_timing",
           "fwi_get_timing", "fwi_reset_timing", "fwi_trace_misfit_noalloc", "fwi_step",
           "fwi_step_reset", "fwi_get_material", "fwi_set_checkpointing", "fwi_regularization",
           "fwi_set_shot_batch", "fwi_tune_shot_batch", "fwi_tune_tiles",
           # include/fwi_precond.h: the learned preconditioner's kernels
           "fwi_nn_conv3d_forward", "fwi_nn_conv3d_backward_data", "fwi_nn_conv3d_backward_weight_work",
           "fwi_nn_conv3d_backward_weight", "fwi_nn_relu_backward", "fwi_nn_mse", "fwi_nn_adam", "fwi_nn_pool2_forward",
           "fwi_nn_pool2_backward", "fwi_nn_upsample2_forward", "fwi_nn_upsample2_backward", "fwi_nn_to_bf16",
           "fwi_nn_from_bf16")

_lib = None


def load_library(path: str = None):
    """Load libfwi.so (or the library FWI_LIBRARY names, e.g. the bounds-checked build
    libfwi_check.so); raises ImportError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("FWI_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1504_08340_gb300.build.build() "
                          "(or __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(path)
    P, I, D, F = C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_float)
    I64 = C.POINTER(C.c_int64)
    lib.fwi_create.argtypes = [C.POINTER(_Config), C.POINTER(P)]
    lib.fwi_destroy.argtypes = [P]
    lib.fwi_destroy.restype = None
    lib.fwi_last_error.argtypes = [P]
    lib.fwi_bounds_checked.argtypes = []
    lib.fwi_last_error.restype = C.c_char_p
    lib.fwi_status_string.argtypes = [I]
    lib.fwi_status_string.restype = C.c_char_p
    lib.fwi_get_dims.argtypes = [P, I64]
    lib.fwi_set_material.argtypes = [P, P, P, I]
    lib.fwi_set_sources.argtypes = [P, I, C.POINTER(C.c_int), D, I, D]
    lib.fwi_set_receivers.argtypes = [P, I, C.POINTER(C.c_int)]
    lib.fwi_forward.argtypes = [P, I, I, P, I]
    lib.fwi_misfit.argtypes = [P, I, I, P, I, D]
    lib.fwi_adjoint_gradient.argtypes = [P, I, I, P, I, D, P, P]
    lib.fwi_get_mass_tilde.argtypes = [P, D]
    lib.fwi_rhs.argtypes = [P, I, P, P, I]
    lib.fwi_get_state.argtypes = [P, P, I]
    lib.fwi_set_graphs.argtypes = [P, I]
    lib.fwi_set_persistent.argtypes = [P, I, C.c_double, I]
    lib.fwi_set_copy_wait.argtypes = [P, C.c_double, I]
    lib.fwi_set_timing.argtypes = [P, I]
    lib.fwi_get_timing.argtypes = [P, I, D, I64]
    lib.fwi_reset_timing.argtypes = [P]
    lib.fwi_trace_misfit_noalloc.argtypes = [P, P, I, I, C.c_double, P, D]
    lib.fwi_step.argtypes = [P, P, I, C.POINTER(StepOpts), C.POINTER(StepInfo)]
    lib.fwi_step_reset.argtypes = [P]
    lib.fwi_get_material.argtypes = [P, P, P, I]
    lib.fwi_set_checkpointing.argtypes = [P, I]
    lib.fwi_set_shot_batch.argtypes = [P, I]
    lib.fwi_tune_shot_batch.argtypes = [P, I, I, I, I, C.c_double, C.POINTER(I)]
    lib.fwi_tune_tiles.argtypes = [P, I, I, I, C.POINTER(I)]
    lib.fwi_regularization.argtypes = [P, I, C.c_double, D, P, P, I]
    L, Fl = C.c_int64, C.c_float
    lib.fwi_nn_conv3d_forward.argtypes = [P, P, P, I, I, I, I, I, I, P, P]
    lib.fwi_nn_conv3d_backward_data.argtypes = [P, P, I, I, I, I, I, P, P]
    lib.fwi_nn_conv3d_backward_weight_work.argtypes = [I, I, I, I, I]
    lib.fwi_nn_conv3d_backward_weight.argtypes = [P, P, I, I, I, I, I, P, P, P, P]
    lib.fwi_nn_relu_backward.argtypes = [P, P, L, P, P]
    lib.fwi_nn_mse.argtypes = [P, P, L, P, P, P, P]
    lib.fwi_nn_adam.argtypes = [P, P, P, P, P, L, Fl, Fl, Fl, Fl, I, P]
    lib.fwi_nn_pool2_forward.argtypes = [P, I, I, I, I, P, P]
    lib.fwi_nn_pool2_backward.argtypes = [P, I, I, I, I, I, P, P]
    lib.fwi_nn_upsample2_forward.argtypes = [P, I, I, I, I, P, P]
    lib.fwi_nn_upsample2_backward.argtypes = [P, I, I, I, I, I, P, P]
    lib.fwi_nn_to_bf16.argtypes = [P, L, P, P]
    lib.fwi_nn_from_bf16.argtypes = [P, L, P, P]
    for name in EXPORTS:
        if name not in ("fwi_destroy", "fwi_last_error", "fwi_status_string"):
            getattr(lib, name).restype = I
    lib.fwi_nn_conv3d_backward_weight_work.restype = L
    _lib = lib
    return lib


def bounds_checked() -> bool:
    """True when the loaded library is the -DFWI_BOUNDS_CHECK build (fwi_bounds_checked)."""
    return bool(load_library().fwi_bounds_checked())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, on_device) for a torch CUDA tensor or a numpy array of the given dtype."""
    if _is_torch(x):
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        if not x.is_cuda:
            raise TypeError("torch tensors must live on the GPU; pass numpy arrays for host data")
        return C.c_void_p(x.data_ptr()), 1
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    return C.c_void_p(x.ctypes.data), 0


class Context:
    """One mesh, its material, sources and receivers (fwi_ctx)."""

    def __init__(self, nx, ny, nz, npml, h, dt, nsteps, rho=2000.0, alpha0=5.0, beta0=400.0,
                 pml_m=2, top_pml=False, stream=None):
        self.lib = load_library()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
            except Exception:  # pragma: no cover
                stream = None
        self.cfg = _Config(nx, ny, nz, npml, int(top_pml), h, rho, alpha0, beta0, pml_m, dt, nsteps,
                           C.c_void_p(stream) if stream else None)
        self.ptr = C.c_void_p()
        st = self.lib.fwi_create(C.byref(self.cfg), C.byref(self.ptr))
        if st != 0:
            raise FWIError(st, "fwi_create failed")
        dims = (C.c_int64 * 9)()
        self._check(self.lib.fwi_get_dims(self.ptr, dims))
        self.nn = tuple(dims[0:3])
        self.nnode, self.nmat, self.stride, self.nelem, self.npml_nodes, self.px = (
            dims[3], dims[4], dims[5], dims[6], dims[7], dims[8])
        self.nsteps, self.dt = nsteps, dt
        self.nrec = 0
        self.nshots = 0

    def _check(self, st):
        if st != 0:
            raise FWIError(st, self.lib.fwi_last_error(self.ptr).decode())

    def close(self):
        if getattr(self, "ptr", None) and self.ptr.value:
            self.lib.fwi_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def mat_shape(self):
        nx, ny, nz = self.cfg.nx, self.cfg.ny, self.cfg.nz
        return (2 * nz + 1, 2 * ny + 1, 2 * nx + 1)

    def set_material(self, lam, mu):
        pl, dl = _ptr(lam, np.float32)
        pm, dm = _ptr(mu, np.float32)
        if dl != dm:
            raise TypeError("lambda and mu must both be host or both be device arrays")
        self._check(self.lib.fwi_set_material(self.ptr, pl, pm, dl))

    def set_sources(self, nodes_ijk, dirs, wavelet="ricker", params=(10.0, 0.15, 1e3)):
        n = np.ascontiguousarray(nodes_ijk, dtype=np.int32).reshape(-1, 3)
        d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        p = np.ascontiguousarray(params, dtype=np.float64)
        self._check(self.lib.fwi_set_sources(self.ptr, n.shape[0], n.ctypes.data_as(C.POINTER(C.c_int)),
                                             d.ctypes.data_as(C.POINTER(C.c_double)), WAVELETS[wavelet],
                                             p.ctypes.data_as(C.POINTER(C.c_double))))
        self.nshots = n.shape[0]

    def set_receivers(self, nodes_ijk):
        n = np.ascontiguousarray(nodes_ijk, dtype=np.int32).reshape(-1, 3)
        self._check(self.lib.fwi_set_receivers(self.ptr, n.shape[0], n.ctypes.data_as(C.POINTER(C.c_int))))
        self.nrec = n.shape[0]

    def trace_shape(self, nshots=1):
        return (nshots, self.nsteps + 1, self.nrec, 3)

    def forward(self, shot0=0, nshots=1, out=None):
        if out is None:
            out = np.zeros(self.trace_shape(nshots), dtype=np.float32)
        p, dev = _ptr(out, np.float32)
        self._check(self.lib.fwi_forward(self.ptr, shot0, nshots, p, dev))
        return out

    def misfit(self, observed, shot0=0, nshots=1):
        p, dev = _ptr(observed, np.float32)
        J = C.c_double()
        self._check(self.lib.fwi_misfit(self.ptr, shot0, nshots, p, dev, C.byref(J)))
        return J.value

    def adjoint_gradient(self, observed, shot0=0, nshots=1, g_lambda=None, g_mu=None):
        """(J, g_lambda, g_mu): misfit (7) and dJ/dlambda_i, dJ/dmu_i (FP64) on the interior nodes."""
        p, dev = _ptr(observed, np.float32)
        if g_lambda is None:
            if dev:
                import torch
                g_lambda = torch.empty(self.mat_shape(), dtype=torch.float64, device=observed.device)
                g_mu = torch.empty(self.mat_shape(), dtype=torch.float64, device=observed.device)
            else:
                g_lambda = np.empty(self.mat_shape())
                g_mu = np.empty(self.mat_shape())
        pl, dl = _ptr(g_lambda, np.float64)
        pm, dm = _ptr(g_mu, np.float64)
        if not (dl == dm == dev):
            raise TypeError("observed and gradient outputs must all be host or all be device arrays")
        J = C.c_double()
        self._check(self.lib.fwi_adjoint_gradient(self.ptr, shot0, nshots, p, dev, C.byref(J), pl, pm))
        return J.value, g_lambda, g_mu

    def step(self, observed, shot0=0, nshots=1, invert=3, lbfgs_m=15, c1=1e-4, rho=0.5, max_backtracks=20,
             first_step=0.05, reg=None, reg_eps=0.0, reg_wp=0.5, bias_w=0.0):
        """One iteration of Algorithm 2; returns the StepInfo (J_old, J_new, alpha, ...).
        reg: None, "tn" or "tv" (objective (7) with (8) or (9), factors from (24) with wp = reg_wp);
        bias_w: W of the lambda search-direction biasing (25)."""
        p, dev = _ptr(observed, np.float32)
        opts = StepOpts(shot0, nshots, invert, lbfgs_m, c1, rho, max_backtracks, first_step,
                        {None: -1, "tn": 0, "tv": 1}[reg], reg_eps, reg_wp, bias_w)
        info = StepInfo()
        self._check(self.lib.fwi_step(self.ptr, p, dev, C.byref(opts), C.byref(info)))
        return info

    def step_reset(self):
        self._check(self.lib.fwi_step_reset(self.ptr))

    def get_material(self):
        lam = np.empty(self.mat_shape(), dtype=np.float32)
        mu = np.empty(self.mat_shape(), dtype=np.float32)
        self._check(self.lib.fwi_get_material(self.ptr, C.c_void_p(lam.ctypes.data), C.c_void_p(mu.ctypes.data), 0))
        return lam, mu

    def mass_tilde(self):
        out = np.empty(self.mat_shape())
        self._check(self.lib.fwi_get_mass_tilde(self.ptr, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def state_index(self):
        """Offsets, inside one field of the state layout, of the nodes in natural order
        ((k * NJ + j) * NI + i): the layout pads every row to the pitch px."""
        ni, nj, nk = self.nn
        k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
        return ((k * nj + j) * self.px + i).ravel()

    def rhs(self, state, adjoint=False, out=None):
        """Right side of the first-order system; state/out: [27, stride] float32."""
        if out is None:
            out = np.zeros_like(state) if not _is_torch(state) else state.new_zeros(state.shape)
        ps, ds = _ptr(state, np.float32)
        po, do = _ptr(out, np.float32)
        if ds != do:
            raise TypeError("state and rate must both be host or both be device arrays")
        self._check(self.lib.fwi_rhs(self.ptr, int(adjoint), ps, po, ds))
        return out

    def state(self, out=None):
        """The RK4 state at the end of the last sweep ([27, stride] float32; fwi_get_state)."""
        if out is None:
            out = np.zeros((27, self.stride), dtype=np.float32)
        p, dev = _ptr(out, np.float32)
        self._check(self.lib.fwi_get_state(self.ptr, p, dev))
        return out

    def regularization(self, kind="tn", eps=0.0, device=False):
        """(R, g_lambda, g_mu): the TN (8) or TV (9) term of the current lambda and mu
        (R = [R_lambda_term, R_mu_term], without the factors) and its gradients (C.1b)-(C.1e),
        FP64 on the interior nodes (numpy, or torch CUDA tensors with device=True)."""
        R = (C.c_double * 2)()
        if device:
            import torch
            gl = torch.empty(self.mat_shape(), dtype=torch.float64, device="cuda")
            gm = torch.empty_like(gl)
        else:
            gl = np.empty(self.mat_shape())
            gm = np.empty(self.mat_shape())
        pl, dl = _ptr(gl, np.float64)
        pm, _ = _ptr(gm, np.float64)
        self._check(self.lib.fwi_regularization(self.ptr, {"tn": 0, "tv": 1}[kind], float(eps), R, pl, pm, dl))
        return [R[0], R[1]], gl, gm

    def set_shot_batch(self, batch):
        """Shots advanced together by one launch of each stage kernel (fwi_set_shot_batch)."""
        self._check(self.lib.fwi_set_shot_batch(self.ptr, int(batch)))

    def tune_shot_batch(self, shot0=0, nshots=None, max_batch=64, steps=10, mem_fraction=0.8):
        """Pick the shot batch by timing forward steps per candidate (fwi_tune_shot_batch); returns it."""
        if nshots is None:
            nshots = self.nshots - shot0
        b = C.c_int()
        self._check(self.lib.fwi_tune_shot_batch(self.ptr, int(shot0), int(nshots), int(max_batch), int(steps),
                                                 float(mem_fraction), C.byref(b)))
        return b.value

    def tune_tiles(self, shot0=0, nshots=None, steps=5):
        """Pick the stage kernels' launch shapes by timing forward steps (fwi_tune_tiles);
        returns (interior planes per block, PML pairs per segment)."""
        if nshots is None:
            nshots = self.nshots - shot0
        out = (C.c_int * 2)()
        self._check(self.lib.fwi_tune_tiles(self.ptr, int(shot0), int(nshots), int(steps), out))
        return out[0], out[1]

    def set_checkpointing(self, interval):
        """0: store u at every step; k > 0: snapshot every k steps and recompute;
        k < 0: every ceil(sqrt(nsteps)) steps (fwi_set_checkpointing)."""
        self._check(self.lib.fwi_set_checkpointing(self.ptr, int(interval)))

    def set_persistent(self, enable=True, wait_ms=1000.0, test_extra_arrivals=0):
        """Forward sweeps as one cooperative launch with bounded grid barriers (fwi_set_persistent)."""
        self._check(self.lib.fwi_set_persistent(self.ptr, int(enable), float(wait_ms), int(test_extra_arrivals)))

    def set_copy_wait(self, wait_ms=1000.0, test_extra_bytes=0):
        """Limit of the interior kernel's bounded waits on its plane copies (fwi_set_copy_wait)."""
        self._check(self.lib.fwi_set_copy_wait(self.ptr, float(wait_ms), int(test_extra_bytes)))

    def set_graphs(self, enable=True):
        """Record each sweep once as a CUDA graph and replay it (fwi_set_graphs)."""
        self._check(self.lib.fwi_set_graphs(self.ptr, int(enable)))

    def set_timing(self, enable=True):
        self._check(self.lib.fwi_set_timing(self.ptr, int(enable)))

    def timing(self, which):
        ms = C.c_double()
        n = C.c_int64()
        self._check(self.lib.fwi_get_timing(self.ptr, which, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def reset_timing(self):
        self._check(self.lib.fwi_reset_timing(self.ptr))
