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


def test_bias_direction_limits():
    """(25): W = 0 leaves the direction alone; W = 1 points the lambda part along the
    mu part with the lambda part's length; the mu part never changes."""
    rng = np.random.default_rng(2)
    n = 5
    d = rng.standard_normal(2 * n)
    assert np.allclose(inversion.bias_direction(d, n, 0.0), d, rtol=1e-14, atol=0)
    d1 = inversion.bias_direction(d, n, 1.0)
    assert np.allclose(d1[:n], np.linalg.norm(d[:n]) * d[n:] / np.linalg.norm(d[n:]), rtol=1e-14)
    assert np.array_equal(d1[n:], d[n:])
    dh = inversion.bias_direction(d, n, 0.5)
    assert np.allclose(dh[:n], 0.5 * d1[:n] + 0.5 * d[:n], rtol=1e-14)


@pytest.mark.slow
@pytest.mark.parametrize("reg,eps", [("tn", 0.0), ("tv", 0.01)])
def test_regularized_inversion_decreases_the_objective(oracle_mod, reg, eps):
    """Algorithm 2 with the regularised objective, R from (24) and lambda biasing (25):
    every accepted step satisfies Armijo on J + R_l R^l + R_m R^m, and R_p is wp times
    the ratio of the gradient norms (so the regularisation part is wp times the misfit part)."""
    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=40, f0=30.0, nrec_side=3)
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
    lt, mt = (np.asarray(a, dtype=np.float32).astype(np.float64) for a in fi.medium(w, "true"))
    l0, m0 = (np.asarray(a, dtype=np.float32).astype(np.float64) for a in fi.medium(w, "trial"))
    src = [o.node_id(*s) for s in w.sources()]
    rec = [o.node_id(*r) for r in w.receivers()]
    o.set_material(lt, mt)
    obs = o.forward(w.dt, w.nsteps, src, w.source_dirs(), "ricker", w.ricker(), rec)
    # a trial model with structure, so that g_reg is not zero
    rng = np.random.default_rng(9)
    l0 = (l0.ravel() * (1 + 0.05 * rng.standard_normal(l0.size))).astype(np.float32).astype(np.float64)
    m0 = (m0.ravel() * (1 + 0.05 * rng.standard_normal(m0.size))).astype(np.float32).astype(np.float64)
    inv = inversion.Inversion(o, w.dt, w.nsteps, src, w.source_dirs(), rec, obs, "ricker", w.ricker(),
                              reg=reg, reg_eps=eps, reg_wp=0.5, bias_w=0.5)
    m = np.concatenate([l0, m0])
    for _ in range(2):
        mk = m.copy()
        m, info = inv.step(m)
        assert info["accepted"] == 1
        assert info["J_new"] < info["J_old"] + 1e-4 * info["alpha"] * info["gtd"]
        assert all(r > 0 for r in info["R"])
        # the regularisation part of J_old is R_p times the terms at the start model
        n = mk.size // 2
        reg_part = sum(info["R"][p] * o.regularization(mk[p * n:(p + 1) * n], reg, eps)[0] for p in range(2))
        assert info["J_old"] == pytest.approx(info["Jmis_old"] + reg_part, rel=1e-12)
