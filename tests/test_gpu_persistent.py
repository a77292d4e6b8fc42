"""Persistent forward sweeps (fwi_set_persistent): one cooperative launch per sweep with
grid-wide barriers between the RK4 stages, every node on the general per-node formulas.

Traces match the FP64 oracle to 1e-5 and the class-specialised kernels to rounding; a
gradient evaluation that takes its forward history from the persistent sweep matches the
oracle to 1e-4 (with and without checkpointing). The barriers' bounded wait is exercised
by asking them to wait for one block more than the launch has: the sweep returns
FWI_E_TIMEOUT after the wait limit instead of hanging, and the context stays usable."""
import numpy as np
import pytest

import fwi_inputs as fi
from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MESHES = [dict(nx=3, ny=3, nz=2, npml=2, top=False), dict(nx=2, ny=3, nz=2, npml=1, top=True),
          dict(nx=2, ny=2, nz=3, npml=0, top=False)]


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _setup(w, top=False, nshots=1):
    from paper_1504_08340_gb300 import Context

    ctx = Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho, top_pml=top)
    lam, mu = (_f32(a) for a in fi.medium(w, "trial"))
    rng = np.random.default_rng(3)
    lam = _f32(lam * (1 + 0.1 * rng.random(lam.shape)))
    mu = _f32(mu * (1 + 0.1 * rng.random(mu.shape)))
    ctx.set_material(lam, mu)
    c = (2 * w.npml + w.nx, 2 * w.npml + w.ny)
    k0 = 2 * w.npml if top else 0
    src = np.array([[c[0], c[1], k0], [c[0] + 1, c[1] - 1, k0 + 1], [c[0] - 1, c[1], k0 + 2]][:nshots], dtype=np.int64)
    dirs = np.array([[0.0, 0.0, 1.0], [0.3, -0.2, 0.9], [0.0, 0.5, 0.5]][:nshots])
    # distinct surface nodes of the interior (on the top of the interior with a top PML,
    # whose k = 0 face is fixed)
    p = w.npml
    nn = w.nodes
    rec = np.array([(2 * p + i, 2 * p + j, k0) for i, j in ((1, 1), (2, 3), (3, 2), (1, 4), (4, 4), (0, 2))
                    if 0 < 2 * p + i < nn[0] - 1 and 0 < 2 * p + j < nn[1] - 1], dtype=np.int64)
    ctx.set_sources(src, dirs, "ricker", w.ricker())
    ctx.set_receivers(rec)
    return ctx, (lam, mu), src, dirs, rec


@pytest.mark.parametrize("mesh", MESHES, ids=lambda m: f"{m['nx']}x{m['ny']}x{m['nz']}+{m['npml']}{'t' if m['top'] else ''}")
def test_persistent_forward_matches_oracle_and_kernels(oracle_mod, mesh):
    w = fi.tiny(nx=mesh["nx"], ny=mesh["ny"], nz=mesh["nz"], npml=mesh["npml"], nsteps=60, f0=30.0, nrec_side=3)
    ctx, (lam, mu), src, dirs, rec = _setup(w, mesh["top"], nshots=3)
    with ctx:
        ctx.set_shot_batch(2)
        ref_k = ctx.forward(0, 3)
        ctx.set_persistent(True)
        tr = ctx.forward(0, 3)
        assert np.abs(tr).max() > 0
        assert rel_l2(tr, ref_k) < 1e-6
        o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho, top_pml=mesh["top"], threads=4)
        o.set_material(lam.astype(np.float64), mu.astype(np.float64))
        rn = [o.node_id(*r) for r in rec]
        for s in range(3):
            ref = o.forward(w.dt, w.nsteps, [o.node_id(*src[s])], dirs[s:s + 1], "ricker", w.ricker(), rn)
            assert rel_l2(tr[s], ref) < 1e-5, (s, rel_l2(tr[s], ref))


@pytest.mark.parametrize("ckpt", [0, 7])
def test_persistent_forward_in_gradient_evaluation(oracle_mod, ckpt):
    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=60, f0=30.0, nrec_side=3)
    ctx, (lam, mu), src, dirs, rec = _setup(w)
    obs = _f32(fi.synthetic_traces(w.nsteps, len(rec), 5, 1e-9)[None])
    with ctx:
        ctx.set_checkpointing(ckpt)
        ctx.set_persistent(True)
        J, gl, gm = ctx.adjoint_gradient(obs)
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho, threads=4)
    o.set_material(lam.astype(np.float64), mu.astype(np.float64))
    J_o, gl_o, gm_o, _ = o.misfit_and_gradient(w.dt, w.nsteps, [o.node_id(*src[0])], dirs, [o.node_id(*r) for r in rec],
                                                obs[0].astype(np.float64), "ricker", w.ricker())
    assert abs(J - J_o) <= 2e-5 * J_o
    assert rel_l2(gl, gl_o) < 1e-4 and rel_l2(gm, gm_o) < 1e-4


def test_grid_barrier_gives_up_with_timeout():
    from paper_1504_08340_gb300 import FWIError

    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=20, f0=30.0, nrec_side=3)
    ctx, _, _, _, _ = _setup(w)
    with ctx:
        ctx.set_persistent(True)
        good = ctx.forward()
        # every barrier now waits for one block more than the launch has: nothing can
        # complete it, and each block gives up after 20 ms
        ctx.set_persistent(True, wait_ms=20.0, test_extra_arrivals=1)
        with pytest.raises(FWIError) as err:
            ctx.forward()
        assert err.value.name == "FWI_E_TIMEOUT"
        # the context stays usable
        ctx.set_persistent(True, wait_ms=1000.0, test_extra_arrivals=0)
        assert np.array_equal(ctx.forward(), good)
        ctx.set_persistent(False)
        assert rel_l2(ctx.forward(), good) < 1e-6
