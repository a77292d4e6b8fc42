"""fwi_trace_misfit_noalloc: the misfit of device-resident traces for callers that
cannot allocate device memory (it uses a fixed scratch array inside the library).

Its result must match fwi_misfit, the allocating entry point, on the same traces,
on two calls in a row (the scratch is shared by every call and keeps the last
call's contents). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import fwi_inputs as fi

pytestmark = pytest.mark.gpu


def test_noalloc_misfit_matches_fwi_misfit():
    torch = pytest.importorskip("torch")
    from paper_1504_08340_gb300 import Context, load_library
    from paper_1504_08340_gb300.fwi import FWIError

    lib = load_library()
    fn = lib.fwi_trace_misfit_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=50, f0=30.0, nrec_side=3)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho, stream=stream) as ctx:
        lam, mu = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "trial"))
        ctx.set_material(lam, mu)
        ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
        ctx.set_receivers(w.receivers())
        traces = torch.zeros(ctx.trace_shape(1), dtype=torch.float32, device=dev)
        ctx.forward(out=traces)
        for seed in (1, 2):  # two calls in a row, different observed data
            scale = float(traces.abs().max())
            obs = torch.tensor(fi.synthetic_traces(w.nsteps, ctx.nrec, seed, scale)[None].astype(np.float32),
                               device=dev).contiguous()
            J_ref = ctx.misfit(obs)
            J = ctypes.c_double()
            st = fn(ctypes.c_void_p(traces.data_ptr()), ctypes.c_void_p(obs.data_ptr()), w.nsteps, ctx.nrec,
                    w.dt, ctypes.c_void_p(stream), ctypes.byref(J))
            assert st == 0
            assert J_ref > 0
            assert abs(J.value - J_ref) <= 1e-12 * J_ref, (J.value, J_ref)
        # sizes beyond the scratch are rejected with FWI_E_INVAL before any work
        J = ctypes.c_double(-1.0)
        st = fn(ctypes.c_void_p(traces.data_ptr()), ctypes.c_void_p(obs.data_ptr()), 70000, ctx.nrec, w.dt,
                ctypes.c_void_p(stream), ctypes.byref(J))
        assert st == 1 and J.value == -1.0
        # a NaN in either input is reported as FWI_E_NONFINITE, J untouched; fwi_misfit agrees
        for which in ("traces", "observed"):
            bad_t, bad_o = traces.clone(), obs.clone()
            (bad_t if which == "traces" else bad_o)[0, w.nsteps // 2, 0, 1] = float("nan")
            J = ctypes.c_double(-1.0)
            st = fn(ctypes.c_void_p(bad_t.data_ptr()), ctypes.c_void_p(bad_o.data_ptr()), w.nsteps, ctx.nrec,
                    w.dt, ctypes.c_void_p(stream), ctypes.byref(J))
            assert st == 5 and J.value == -1.0, (which, st)
            if which == "observed":
                with pytest.raises(FWIError) as err:
                    ctx.misfit(bad_o)
                assert err.value.code == 5
        # the flag of the failed call does not leak into the next one
        J = ctypes.c_double()
        st = fn(ctypes.c_void_p(traces.data_ptr()), ctypes.c_void_p(obs.data_ptr()), w.nsteps, ctx.nrec, w.dt,
                ctypes.c_void_p(stream), ctypes.byref(J))
        assert st == 0 and abs(J.value - ctx.misfit(obs)) <= 1e-12 * J.value
        # nsteps = 0: one sample with trapezoid weight 1/2
        e = (traces[0, 0].double() - obs[0, 0].double()).cpu().numpy()
        J = ctypes.c_double()
        st = fn(ctypes.c_void_p(traces.data_ptr()), ctypes.c_void_p(obs.data_ptr()), 0, ctx.nrec, w.dt,
                ctypes.c_void_p(stream), ctypes.byref(J))
        expect = 0.5 * w.dt * 0.5 * float((e * e).sum())
        assert st == 0 and abs(J.value - expect) <= 1e-12 * max(expect, 1e-300), (J.value, expect)
