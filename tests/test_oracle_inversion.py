"""Pins of the reference inversion iteration (Algorithm 1/2, L-BFGS) on the CPU."""
import numpy as np
import pytest

import fwi_inputs as fi
from oracle import inversion


def test_two_loop_equals_dense_inverse_bfgs():
    """The two-loop recursion is the BFGS inverse-Hessian recursion applied to g,
    here with a diagonal (Mtilde-like) metric."""
    rng = np.random.default_rng(0)
    n = 7
    w = rng.uniform(0.5, 2.0, n)
    A = rng.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)  # curvature pairs of a convex quadratic: y = W^-1 A s
    pairs = []
    for _ in range(4):
        s = rng.standard_normal(n)
        pairs.append((s, np.linalg.solve(np.diag(w), A @ s)))
    g = rng.standard_normal(n)
    d = inversion.two_loop(g, pairs, w)
    H = inversion.dense_inverse_bfgs(pairs, w)
    assert np.allclose(d, -H @ g, rtol=1e-12, atol=1e-12 * np.abs(d).max())


def test_two_loop_satisfies_secant_condition():
    """H y_k = s_k for the newest pair (the defining property of a BFGS update)."""
    rng = np.random.default_rng(1)
    n = 6
    w = rng.uniform(0.5, 2.0, n)
    pairs = [(rng.standard_normal(n), None) for _ in range(3)]
    A = np.diag(rng.uniform(1.0, 3.0, n))
    pairs = [(s, A @ s) for s, _ in pairs]
    s, y = pairs[-1]
    assert np.allclose(-inversion.two_loop(y, pairs, w), s, rtol=1e-12, atol=1e-12)


@pytest.mark.slow
def test_inversion_decreases_the_misfit(oracle_mod):
    """Three iterations of Algorithm 2 on a small box: J decreases monotonically
    (Armijo) and each accepted step satisfies the sufficient-decrease condition."""
    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=40, f0=30.0, nrec_side=3)
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
    lt, mt = (np.asarray(a, dtype=np.float32).astype(np.float64) for a in fi.medium(w, "true"))
    l0, m0 = (np.asarray(a, dtype=np.float32).astype(np.float64) for a in fi.medium(w, "trial"))
    src = [o.node_id(*s) for s in w.sources()]
    rec = [o.node_id(*r) for r in w.receivers()]
    o.set_material(lt, mt)
    obs = o.forward(w.dt, w.nsteps, src, w.source_dirs(), "ricker", w.ricker(), rec)
    inv = inversion.Inversion(o, w.dt, w.nsteps, src, w.source_dirs(), rec, obs, "ricker", w.ricker())
    m = np.concatenate([l0.ravel(), m0.ravel()])
    Js = []
    for _ in range(3):
        m, info = inv.step(m)
        assert info["accepted"] == 1
        assert info["J_new"] < info["J_old"] + 1e-4 * info["alpha"] * info["gtd"]
        Js.append((info["J_old"], info["J_new"]))
    assert Js[0][1] < Js[0][0] and Js[-1][1] < Js[0][0]
    assert all(b[0] == pytest.approx(a[1], rel=1e-12) for a, b in zip(Js, Js[1:]))
