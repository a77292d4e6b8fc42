"""FP64 CPU oracle for the per-shot material gradient (arXiv:1504.08340).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import
this package. The CUDA library and its Python binding never import it.

The arithmetic lives in ``fwi_oracle.c`` (plain C, FP64, element-by-element
quadrature of the weak form (3a)/(3b), classic RK4 on (6), the reverse RK4 of
Appendix B with the transposed operators of (15), gradients (C.1f)/(C.1g)).
This module only compiles and marshals it.

Parity unpinned: the absolute Table 2 values (the paper does not give the trial
model, the PML details of its companion paper, or the data mesh).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fwi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NV = 9  # per node: u_x, u_y, u_z, S_xx, S_yy, S_zz, S_yz, S_xz, S_xy


def build(force: bool = False) -> str:
    """Compile ``fwi_oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        D = C.POINTER(C.c_double)
        L = C.POINTER(C.c_long)
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [C.c_int] * 5 + [C.c_double] * 4 + [C.c_int]
        lib.orc_destroy.argtypes = [P]
        lib.orc_set_threads.argtypes = [P, C.c_int]
        lib.orc_dims.argtypes = [P, L]
        lib.orc_set_material.argtypes = [P, D, D]
        lib.orc_get_diag.argtypes = [P, C.c_int, D]
        lib.orc_get_masks.argtypes = [P, C.c_char_p, C.c_char_p]
        lib.orc_get_stretch.argtypes = [P, C.c_int, D, D]
        for name in ("orc_apply_A", "orc_apply_At", "orc_apply_B", "orc_apply_Bt"):
            getattr(lib, name).argtypes = [P, C.c_int, D, D]
        lib.orc_apply_KRD.argtypes = [P, D, D]
        lib.orc_rhs.argtypes = [P, C.c_int, D, D, D]
        lib.orc_wavelet.restype = C.c_double
        lib.orc_wavelet.argtypes = [C.c_int, D, C.c_double]
        lib.orc_forward.argtypes = [P, C.c_double, C.c_int, C.c_int, L, D, C.c_int, D, C.c_int, L, D, D]
        lib.orc_rk4_step.argtypes = [P, D, C.c_double]
        lib.orc_misfit.restype = C.c_double
        lib.orc_misfit.argtypes = [C.c_int, C.c_int, C.c_double, D, D]
        lib.orc_adjoint_gradient.argtypes = [P, C.c_double, C.c_int, C.c_int, L, D, D, D, D]
        lib.orc_gradient_term.argtypes = [P, D, D, C.c_double, D, D]
        lib.orc_energy.argtypes = [P, D, D]
        lib.orc_regularization.argtypes = [P, C.c_int, C.c_double, D, D]
        lib.orc_regularization.restype = C.c_double
        _lib = lib
        return lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _l(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_long))


WAVELETS = {"ricker": 0, "gauss": 1}


class Oracle:
    """One mesh of the oracle: interior nx*ny*nz elements of size h, npml PML
    elements on the four sides and the bottom (and the top when top_pml)."""

    def __init__(self, nx, ny, nz, npml, h=1.0, rho=2000.0, alpha0=5.0, beta0=400.0,
                 pml_m=2, top_pml=False, threads=None):
        self.lib = _load()
        self.ptr = self.lib.orc_create(nx, ny, nz, npml, int(top_pml), h, rho, alpha0, beta0, pml_m)
        if not self.ptr:
            raise ValueError("invalid mesh parameters")
        dims = np.zeros(14, dtype=np.int64)
        self.lib.orc_dims(self.ptr, _l(dims))
        self.nn = tuple(int(x) for x in dims[0:3])      # nodes per axis (x, y, z)
        self.N = tuple(int(x) for x in dims[3:6])       # elements per axis
        self.nnode = int(dims[6])
        self.nmat = int(dims[7])
        self.lo = tuple(int(x) for x in dims[8:11])
        self.hi = tuple(int(x) for x in dims[11:14])
        self.nel = (nx, ny, nz)
        self.h, self.rho = h, rho
        self.set_threads(threads or os.cpu_count() or 1)

    def __del__(self):
        if getattr(self, "ptr", None):
            self.lib.orc_destroy(self.ptr)
            self.ptr = None

    def set_threads(self, n: int):
        self.threads = int(n)
        self.lib.orc_set_threads(self.ptr, self.threads)

    # ---- mesh data
    def node_id(self, i, j, k):
        return (k * self.nn[1] + j) * self.nn[0] + i

    def mat_shape(self):
        """(z, y, x) shape of the interior material grid."""
        nx, ny, nz = self.nel
        return (2 * nz + 1, 2 * ny + 1, 2 * nx + 1)

    def set_material(self, lam: np.ndarray, mu: np.ndarray):
        lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
        mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(-1)
        assert lam.size == self.nmat and mu.size == self.nmat
        self.lib.orc_set_material(self.ptr, _d(lam), _d(mu))

    def diag(self, which: str) -> np.ndarray:
        names = ["Mu", "Cu", "Ku", "Gu", "Ms", "Cs", "Ks", "Gs", "Mtilde"]
        idx = names.index(which)
        out = np.zeros(self.nmat if idx == 8 else self.nnode)
        self.lib.orc_get_diag(self.ptr, idx, _d(out))
        return out

    def masks(self):
        pml = np.zeros(self.nnode, dtype=np.uint8)
        dirn = np.zeros(self.nnode, dtype=np.uint8)
        self.lib.orc_get_masks(self.ptr, pml.ctypes.data_as(C.c_char_p), dirn.ctypes.data_as(C.c_char_p))
        return pml.astype(bool), dirn.astype(bool)

    def stretch(self, axis: int):
        n = self.nn[axis]
        a = np.zeros(n)
        b = np.zeros(n)
        self.lib.orc_get_stretch(self.ptr, axis, _d(a), _d(b))
        return a, b

    # ---- operators (out += op(in))
    def apply(self, name: str, which_L: int | None, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        if name == "KRD":
            out = np.zeros((self.nnode, 3))
            self.lib.orc_apply_KRD(self.ptr, _d(x), _d(out))
            return out
        out_cols = {"A": 3, "At": 6, "B": 6, "Bt": 3}[name]
        out = np.zeros((self.nnode, out_cols))
        getattr(self.lib, "orc_apply_" + name)(self.ptr, which_L, _d(x), _d(out))
        return out

    def rhs(self, Y: np.ndarray, fext: np.ndarray | None = None, adjoint=False) -> np.ndarray:
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        assert Y.shape == (3, self.nnode, NV)
        dY = np.zeros_like(Y)
        f = None
        if fext is not None:
            f = np.ascontiguousarray(fext, dtype=np.float64)
            assert f.shape == (self.nnode, 3)
        self.lib.orc_rhs(self.ptr, int(adjoint), _d(Y), _d(f) if f is not None else None, _d(dY))
        return dY

    def rk4_step(self, Y: np.ndarray, dt: float) -> np.ndarray:
        Y = np.array(Y, dtype=np.float64, order="C")
        self.lib.orc_rk4_step(self.ptr, _d(Y), dt)
        return Y

    def energy(self, Y: np.ndarray):
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        out = np.zeros(2)
        self.lib.orc_energy(self.ptr, _d(Y), _d(out))
        return out

    # ---- sweeps
    def forward(self, dt, nsteps, src_nodes, src_dirs, wavelet="ricker", wparams=(15.0, 0.1, 1e3),
                rec_nodes=(), keep_history=False):
        src_nodes = np.ascontiguousarray(src_nodes, dtype=np.int64).reshape(-1)
        src_dirs = np.ascontiguousarray(src_dirs, dtype=np.float64).reshape(-1)
        rec_nodes = np.ascontiguousarray(rec_nodes, dtype=np.int64).reshape(-1)
        wp = np.ascontiguousarray(wparams, dtype=np.float64)
        nrec = rec_nodes.size
        traces = np.zeros((nsteps + 1, max(nrec, 1), 3))
        hist = np.zeros((nsteps + 1, self.nnode, 3)) if keep_history else None
        self.lib.orc_forward(self.ptr, dt, nsteps, src_nodes.size, _l(src_nodes), _d(src_dirs),
                             WAVELETS[wavelet], _d(wp), nrec, _l(rec_nodes) if nrec else None,
                             _d(traces), _d(hist) if hist is not None else None)
        traces = traces[:, :nrec, :]
        return (traces, hist) if keep_history else traces

    @staticmethod
    def misfit(dt, traces, observed) -> float:
        t = np.ascontiguousarray(traces, dtype=np.float64)
        o = np.ascontiguousarray(observed, dtype=np.float64)
        assert t.shape == o.shape
        return float(_load().orc_misfit(t.shape[0] - 1, t.shape[1], dt, _d(t), _d(o)))

    def adjoint_gradient(self, dt, nsteps, rec_nodes, resid, uhist):
        rec_nodes = np.ascontiguousarray(rec_nodes, dtype=np.int64).reshape(-1)
        resid = np.ascontiguousarray(resid, dtype=np.float64)
        uhist = np.ascontiguousarray(uhist, dtype=np.float64)
        assert resid.shape == (nsteps + 1, rec_nodes.size, 3)
        assert uhist.shape == (nsteps + 1, self.nnode, 3)
        gl = np.zeros(self.nmat)
        gm = np.zeros(self.nmat)
        self.lib.orc_adjoint_gradient(self.ptr, dt, nsteps, rec_nodes.size, _l(rec_nodes),
                                      _d(resid), _d(uhist), _d(gl), _d(gm))
        return gl, gm

    def gradient_term(self, u, w, wdt):
        gl = np.zeros(self.nmat)
        gm = np.zeros(self.nmat)
        self.lib.orc_gradient_term(self.ptr, _d(np.ascontiguousarray(u, dtype=np.float64)),
                                   _d(np.ascontiguousarray(w, dtype=np.float64)), wdt, _d(gl), _d(gm))
        return gl, gm

    def regularization(self, f, kind="tn", eps=0.0):
        """(R, g): the TN (8) or TV (9) term of a field on the interior nodes and its
        gradient (C.1b)-(C.1e), without the regularisation factor."""
        f = np.ascontiguousarray(f, dtype=np.float64).ravel()
        if f.size != self.nmat:
            raise ValueError("field must have one value per interior node")
        g = np.zeros(self.nmat)
        R = self.lib.orc_regularization(self.ptr, {"tn": 0, "tv": 1}[kind], float(eps), _d(f), _d(g))
        return R, g

    def misfit_and_gradient(self, dt, nsteps, src_nodes, src_dirs, rec_nodes, observed,
                            wavelet="ricker", wparams=(15.0, 0.1, 1e3)):
        """Forward, misfit (7) and the adjoint gradient (g_mis of (18), dJ/dlambda_i)."""
        traces, hist = self.forward(dt, nsteps, src_nodes, src_dirs, wavelet, wparams,
                                    rec_nodes, keep_history=True)
        J = self.misfit(dt, traces, observed)
        gl, gm = self.adjoint_gradient(dt, nsteps, rec_nodes, traces - observed, hist)
        return J, gl, gm, traces


def wavelet(kind: str, params, t: float) -> float:
    p = np.ascontiguousarray(params, dtype=np.float64)
    return float(_load().orc_wavelet(WAVELETS[kind], _d(p), t))
