"""Pins of the oracle's spatial operators against what the mathematics fixes (CPU only)."""
import numpy as np
import pytest

import fwi_inputs as fi
from helpers import homogeneous, node_coords


@pytest.fixture(scope="module")
def small(oracle_mod):
    o = oracle_mod.Oracle(3, 2, 2, 2, h=1.0, threads=2)
    rng = np.random.default_rng(1)
    shape = o.mat_shape()
    lam = 1.6e8 * (1 + 0.2 * rng.standard_normal(shape))
    mu = 0.8e8 * (1 + 0.2 * rng.standard_normal(shape))
    o.set_material(lam, mu)
    return o


def test_gll_rule_exactness():
    """Three-point LGL rule on [-1,1] (nodes -1,0,1, weights 1/3,4/3,1/3) integrates
    cubics exactly; the derivative matrix differentiates quadratics exactly."""
    x = np.array([-1.0, 0.0, 1.0])
    w = np.array([1, 4, 1]) / 3.0
    for p in range(4):
        assert w @ x ** p == pytest.approx((1 - (-1) ** (p + 1)) / (p + 1))
    D = np.array([[-1.5, 2.0, -0.5], [-0.5, 0.0, 0.5], [0.5, -2.0, 1.5]])
    for p in range(3):
        assert np.allclose(D @ x ** p, p * x ** max(p - 1, 0) if p else 0 * x)


def test_interior_stiffness_symmetric(small):
    rng = np.random.default_rng(2)
    u, v = rng.standard_normal((2, small.nnode, 3))
    a = v.ravel() @ small.apply("KRD", None, u).ravel()
    b = u.ravel() @ small.apply("KRD", None, v).ravel()
    assert a == pytest.approx(b, rel=1e-13)
    assert u.ravel() @ small.apply("KRD", None, u).ravel() > 0


def test_interior_stiffness_rigid_modes(small):
    """K_e annihilates the 6 rigid-body modes (zero strain)."""
    x, y, z = node_coords(small)
    one = np.ones_like(x)
    zero = np.zeros_like(x)
    modes = [np.stack(m, 1) for m in ((one, zero, zero), (zero, one, zero), (zero, zero, one),
                                      (-y, x, zero), (zero, -z, y), (z, zero, -x))]
    scale = np.abs(small.apply("KRD", None, np.stack((x * x, zero, zero), 1))).max()
    for u in modes:
        assert np.abs(small.apply("KRD", None, u)).max() < 1e-12 * scale


@pytest.mark.parametrize("case", ["uxx", "uyy", "uxy"])
def test_interior_stiffness_quadratic_patch(oracle_mod, case):
    """For a quadratic displacement the stress is linear, LGL quadrature is exact and
    K u = -div(sigma) * int(phi_a) at nodes inside the interior domain:
    u_x = x^2 -> f_x = -2(lam+2mu) V_a;  u_x = y^2 -> f_x = -2 mu V_a;
    u_x = x y -> f_y = -(lam+mu) V_a, f_x = 0."""
    o = oracle_mod.Oracle(4, 4, 4, 1, h=0.5, threads=2)
    lam, mu = 1.3e8, 0.7e8
    o.set_material(*homogeneous(o, lam, mu))
    x, y, z = node_coords(o)
    zero = np.zeros_like(x)
    u = {"uxx": (x * x, zero, zero), "uyy": (y * y, zero, zero), "uxy": (x * y, zero, zero)}[case]
    f = o.apply("KRD", None, np.stack(u, 1))
    V = o.diag("Mu") / 2000.0
    n = np.arange(o.nnode)
    i, j, k = n % o.nn[0], (n // o.nn[0]) % o.nn[1], n // (o.nn[0] * o.nn[1])
    lo, hi = 2 * np.array(o.lo), 2 * np.array(o.hi)
    inside = (i > lo[0]) & (i < hi[0]) & (j > lo[1]) & (j < hi[1]) & (k > lo[2]) & (k < hi[2])
    expect = np.zeros((o.nnode, 3))
    if case == "uxx":
        expect[:, 0] = -2 * (lam + 2 * mu) * V
    elif case == "uyy":
        expect[:, 0] = -2 * mu * V
    else:
        expect[:, 1] = -(lam + mu) * V
    scale = np.abs(expect[inside]).max()
    assert np.abs(f[inside] - expect[inside]).max() < 1e-12 * scale


@pytest.mark.parametrize("which", [0, 1, 2])
def test_pml_coupling_transposes(small, which):
    """<A S, w> = <S, A^T w> and <B u, T> = <u, B^T T> (dot-product test) for
    Lambda_e, Lambda_p, Lambda_w."""
    rng = np.random.default_rng(3 + which)
    pml, dirn = small.masks()
    S, T = rng.standard_normal((2, small.nnode, 6))
    S[~pml] = 0
    T[~pml] = 0
    u, w = rng.standard_normal((2, small.nnode, 3))
    u[dirn] = 0
    w[dirn] = 0
    a = w.ravel() @ small.apply("A", which, S).ravel()
    b = S.ravel() @ small.apply("At", which, w).ravel()
    assert a == pytest.approx(b, rel=1e-12)
    c = T.ravel() @ small.apply("B", which, u).ravel()
    d = u.ravel() @ small.apply("Bt", which, T).ravel()
    assert c == pytest.approx(d, rel=1e-12)


@pytest.mark.parametrize("level", [0, 1, 2])
def test_adjoint_system_is_transpose(small, level):
    """The adjoint right side of (15) uses G^T, K^T, C^T of the forward (6):
    <y, M x2'(x)> = -s_l <M y2'(y), x> with x, y on level l only and
    s = (+1, -1, +1) for (G, K, C) -- checked through the full first-order rate."""
    pml, dirn = small.masks()
    X = fi.random_state(small.nnode, pml, dirn, 10 + level, scale=1.0)
    Y = fi.random_state(small.nnode, pml, dirn, 20 + level, scale=1.0)
    for l in range(3):
        if l != level:
            X[l] = 0
            Y[l] = 0
    if level == 0:  # history lives on PML nodes only
        X[0][~pml] = 0
        Y[0][~pml] = 0
    dX = small.rhs(X)
    dY = small.rhs(Y, adjoint=True)
    M = np.concatenate([np.repeat(small.diag("Mu")[:, None], 3, 1),
                        np.repeat(small.diag("Ms")[:, None], 6, 1)], 1)
    lhs = (Y[level] * M * dX[2]).sum()
    s = (1.0, -1.0, 1.0)[level]
    rhs = -s * (M * dY[2] * X[level]).sum()
    assert lhs == pytest.approx(rhs, rel=1e-11)
