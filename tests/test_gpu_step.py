"""fwi_step (one iteration of Algorithm 2) against the oracle-driven reference."""
import numpy as np
import pytest

import fwi_inputs as fi
from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


@pytest.mark.parametrize("invert", [3, 2])
def test_step_matches_reference(oracle_mod, invert):
    from oracle import inversion
    from paper_1504_08340_gb300 import Context

    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=40, f0=30.0, nrec_side=3)
    lt, mt = (_f32(a) for a in fi.medium(w, "true"))
    l0, m0 = (_f32(a) for a in fi.medium(w, "trial"))
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
    src = [o.node_id(*s) for s in w.sources()]
    rec = [o.node_id(*r) for r in w.receivers()]
    o.set_material(lt.astype(np.float64), mt.astype(np.float64))
    obs = o.forward(w.dt, w.nsteps, src, w.source_dirs(), "ricker", w.ricker(), rec)
    ref = inversion.Inversion(o, w.dt, w.nsteps, src, w.source_dirs(), rec, obs, "ricker", w.ricker(),
                              invert=invert)
    m = np.concatenate([l0.ravel(), m0.ravel()]).astype(np.float64)
    with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho) as ctx:
        ctx.set_material(l0, m0)
        ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
        ctx.set_receivers(w.receivers())
        obs_h = _f32(obs[None])
        for it in range(3):
            info = ctx.step(obs_h, invert=invert)
            m, r = ref.step(m)
            assert info.accepted == r["accepted"] == 1
            assert info.alpha == r["alpha"] and info.trials == r["trials"]
            assert info.J_old == pytest.approx(r["J_old"], rel=2e-5)
            assert info.J_new == pytest.approx(r["J_new"], rel=2e-5)
            assert info.gtd == pytest.approx(r["gtd"], rel=1e-4)
            assert info.pairs == len(ref.pairs)
        lam, mu = ctx.get_material()
        n = lam.size
        assert rel_l2(lam.ravel() - l0.ravel(), m[:n] - l0.ravel()) < 1e-3 or invert == 2
        assert rel_l2(mu.ravel() - m0.ravel(), m[n:] - m0.ravel()) < 1e-3
        if invert == 2:
            assert np.array_equal(lam, l0)  # lambda frozen
        ctx.step_reset()
        assert ctx.step(obs_h, invert=invert).pairs == 0


@pytest.mark.parametrize("reg,eps,bias", [("tn", 0.0, 0.0), ("tv", 0.01, 0.5)])
def test_regularized_step_matches_reference(oracle_mod, reg, eps, bias):
    """fwi_step with the regularised objective (8)/(9), factors (24) and lambda biasing
    (25) against the oracle-driven reference."""
    from oracle import inversion
    from paper_1504_08340_gb300 import Context

    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=40, f0=30.0, nrec_side=3)
    lt, mt = (_f32(a) for a in fi.medium(w, "true"))
    l0, m0 = (_f32(a) for a in fi.medium(w, "trial"))
    rng = np.random.default_rng(9)
    l0 = _f32(l0 * (1 + 0.05 * rng.standard_normal(l0.shape)))
    m0 = _f32(m0 * (1 + 0.05 * rng.standard_normal(m0.shape)))
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
    src = [o.node_id(*s) for s in w.sources()]
    rec = [o.node_id(*r) for r in w.receivers()]
    o.set_material(lt.astype(np.float64), mt.astype(np.float64))
    obs = o.forward(w.dt, w.nsteps, src, w.source_dirs(), "ricker", w.ricker(), rec)
    ref = inversion.Inversion(o, w.dt, w.nsteps, src, w.source_dirs(), rec, obs, "ricker", w.ricker(),
                              reg=reg, reg_eps=eps, reg_wp=0.5, bias_w=bias)
    m = np.concatenate([l0.ravel(), m0.ravel()]).astype(np.float64)
    with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho) as ctx:
        ctx.set_material(l0, m0)
        ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
        ctx.set_receivers(w.receivers())
        obs_h = _f32(obs[None])
        for it in range(2):
            info = ctx.step(obs_h, reg=reg, reg_eps=eps, reg_wp=0.5, bias_w=bias)
            m, r = ref.step(m)
            assert info.accepted == r["accepted"] == 1
            assert info.alpha == r["alpha"] and info.trials == r["trials"]
            assert info.R_lambda == pytest.approx(r["R"][0], rel=1e-4)
            assert info.R_mu == pytest.approx(r["R"][1], rel=1e-4)
            assert info.Jmis_old == pytest.approx(r["Jmis_old"], rel=2e-5)
            assert info.J_old == pytest.approx(r["J_old"], rel=2e-5)
            assert info.J_new == pytest.approx(r["J_new"], rel=2e-5)
            assert info.gtd == pytest.approx(r["gtd"], rel=1e-4)
        lam, mu = ctx.get_material()
        n = lam.size
        assert rel_l2(lam.ravel() - l0.ravel(), m[:n] - l0.ravel()) < 1e-3
        assert rel_l2(mu.ravel() - m0.ravel(), m[n:] - m0.ravel()) < 1e-3
