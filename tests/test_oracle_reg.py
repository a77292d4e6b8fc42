"""Pins of the oracle's regularisation terms, Eqs. (8)/(9) with the gradients
(C.1b)-(C.1e), against closed forms, invariants and finite differences."""
import numpy as np
import pytest


def _oracle(oracle_mod, nx=3, ny=2, nz=2, h=0.5):
    return oracle_mod.Oracle(nx, ny, nz, 2, h=h, rho=2000.0)


def _coords(o, h):
    nk, nj, ni = o.mat_shape()
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    return (0.5 * h * i).ravel(), (0.5 * h * j).ravel(), (0.5 * h * k).ravel()


def _interior_mask(o):
    nk, nj, ni = o.mat_shape()
    m = np.zeros((nk, nj, ni), dtype=bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m.ravel()


@pytest.mark.parametrize("kind,eps", [("tn", 0.0), ("tv", 0.3)])
def test_linear_field_closed_form(oracle_mod, kind, eps):
    """grad f is the constant c on every element: R = V |c|^2 / 2 (TN) or
    V (|c|^2 + eps)^(1/2) (TV), V = nx ny nz h^3, and the gradient, the flux of a
    constant vector, vanishes at every node off the boundary of the interior domain."""
    h = 0.5
    o = _oracle(oracle_mod, h=h)
    x, y, z = _coords(o, h)
    c = np.array([1.5, -0.7, 0.4])
    f = c[0] * x + c[1] * y + c[2] * z + 3.0
    R, g = o.regularization(f, kind, eps)
    V = 3 * 2 * 2 * h ** 3
    want = 0.5 * V * c @ c if kind == "tn" else V * np.sqrt(c @ c + eps)
    assert R == pytest.approx(want, rel=1e-13)
    inner = _interior_mask(o)
    assert np.abs(g[inner]).max() < 1e-12 * np.abs(g).max()
    assert np.abs(g).max() > 0
    assert abs(g.sum()) < 1e-12 * np.abs(g).sum()  # the boundary fluxes cancel


@pytest.mark.parametrize("kind,eps", [("tn", 0.0), ("tv", 0.05), ("tv", 5.0)])
def test_gradient_is_the_derivative(oracle_mod, kind, eps):
    """Central differences of R along random directions equal g . d (exact for the
    quadratic TN term, O(step^2) for TV)."""
    o = _oracle(oracle_mod)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(o.nmat)
    _, g = o.regularization(f, kind, eps)
    for _ in range(3):
        d = rng.standard_normal(o.nmat)
        st = 1e-3 if kind == "tn" else 1e-5
        fd = (o.regularization(f + st * d, kind, eps)[0] - o.regularization(f - st * d, kind, eps)[0]) / (2 * st)
        assert fd == pytest.approx(g @ d, rel=1e-8 if kind == "tn" else 1e-6)


def test_tikhonov_operator_is_symmetric_with_constants_in_its_null_space(oracle_mod):
    """g_TN = K f with K = int grad chi grad chi^T: symmetric, K 1 = 0, so 1 . K f = 0,
    and f . K f = 2 R >= 0."""
    o = _oracle(oracle_mod)
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal(o.nmat), rng.standard_normal(o.nmat)
    Ru, gu = o.regularization(u, "tn")
    _, gv = o.regularization(v, "tn")
    assert gu @ v == pytest.approx(gv @ u, rel=1e-12)
    assert abs(gu.sum()) < 1e-12 * np.abs(gu).sum()
    assert np.abs(o.regularization(np.full(o.nmat, 7.0), "tn")[1]).max() == 0.0
    assert u @ gu == pytest.approx(2 * Ru, rel=1e-12) and Ru > 0


def test_total_variation_tends_to_scaled_tikhonov(oracle_mod):
    """For eps >> |grad f|^2, (|grad f|^2 + eps)^(-1/2) -> eps^(-1/2): g_TV sqrt(eps) -> g_TN."""
    o = _oracle(oracle_mod)
    f = np.random.default_rng(5).standard_normal(o.nmat)
    _, gt = o.regularization(f, "tn")
    eps = 1e10
    _, gv = o.regularization(f, "tv", eps)
    assert np.allclose(gv * np.sqrt(eps), gt, rtol=1e-6, atol=1e-9 * np.abs(gt).max())
