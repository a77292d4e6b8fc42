"""Pins of the oracle's misfit and adjoint gradient (CPU only).

The gradient is the optimize-then-discretize gradient of Sec. 3 / Appendix C; the
paper verifies it against directional finite differences of the discrete misfit
(Eqs. 26-27, Table 2: 3 to 5 matching digits). Here the same check is made, and in
addition the gap between the two is shown to vanish as dt^2.
"""
import numpy as np
import pytest

import fwi_inputs as fi


def _setup(oracle_mod, w, threads=8):
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho, threads=threads)
    src = [o.node_id(*s) for s in w.sources()]
    rec = [o.node_id(*r) for r in w.receivers()]
    lt, mt = fi.medium(w, "true")
    o.set_material(lt, mt)
    obs = o.forward(w.dt, w.nsteps, src, w.source_dirs(), "ricker", w.ricker(), rec)
    l0, m0 = fi.medium(w, "trial")
    o.set_material(l0, m0)
    return o, src, rec, obs, l0, m0


def _J(o, w, src, rec, obs, lam, mu):
    o.set_material(lam, mu)
    tr = o.forward(w.dt, w.nsteps, src, w.source_dirs(), "ricker", w.ricker(), rec)
    return o.misfit(w.dt, tr, obs)


def test_zero_residual_gives_zero_misfit_and_gradient(oracle_mod):
    w = fi.tiny(nsteps=30)
    o, src, rec, _, l0, m0 = _setup(oracle_mod, w)
    own = o.forward(w.dt, w.nsteps, src, w.source_dirs(), "ricker", w.ricker(), rec)
    J, gl, gm, _ = o.misfit_and_gradient(w.dt, w.nsteps, src, w.source_dirs(), rec, own, "ricker", w.ricker())
    assert J == 0.0
    assert np.all(gl == 0.0) and np.all(gm == 0.0)


def test_gradient_is_linear_in_the_residual(oracle_mod):
    """The adjoint (15) is linear in its forcing and (C.1f)/(C.1g) are linear in w."""
    w = fi.tiny(nsteps=30)
    o, src, rec, obs, l0, m0 = _setup(oracle_mod, w)
    tr, hist = o.forward(w.dt, w.nsteps, src, w.source_dirs(), "ricker", w.ricker(), rec, keep_history=True)
    g1 = o.adjoint_gradient(w.dt, w.nsteps, rec, tr - obs, hist)
    g3 = o.adjoint_gradient(w.dt, w.nsteps, rec, 3.0 * (tr - obs), hist)
    assert np.abs(g3[0] - 3 * g1[0]).max() <= 1e-13 * np.abs(g1[0]).max()
    assert np.abs(g3[1] - 3 * g1[1]).max() <= 1e-13 * np.abs(g1[1]).max()
    assert np.abs(g1[0]).max() > 0 and np.abs(g1[1]).max() > 0


def test_misfit_trapezoid_weights(oracle_mod):
    """J = 1/2 sum_n w_n dt |e_n|^2 with w_0 = w_N = 1/2: a residual that is 1 only at
    the first sample gives dt/4, only at an inner sample dt/2."""
    e = np.zeros((5, 2, 3))
    e[0, 1, 2] = 1.0
    assert oracle_mod.Oracle.misfit(0.1, e, np.zeros_like(e)) == pytest.approx(0.025)
    e[:] = 0
    e[2, 0, 0] = 1.0
    assert oracle_mod.Oracle.misfit(0.1, e, np.zeros_like(e)) == pytest.approx(0.05)


@pytest.mark.slow
def test_directional_fd_matches_adjoint_gradient(oracle_mod):
    """d_fd of (26) (central differences, relative step 1e-4) against d_co of (27) at a
    surface node and a buried node far from the PML: three digits, as in Table 2."""
    w = fi.tiny(nx=5, ny=5, nz=4, npml=2, nsteps=120, f0=30.0, nrec_side=5)
    o, src, rec, obs, l0, m0 = _setup(oracle_mod, w)
    J, gl, gm, _ = o.misfit_and_gradient(w.dt, w.nsteps, src, w.source_dirs(), rec, obs, "ricker", w.ricker())
    shape = o.mat_shape()
    h = 1e-4
    for kji, which in (((0, 5, 5), "lam"), ((4, 5, 5), "mu")):
        idx = np.ravel_multi_index(kji, shape)
        base = l0 if which == "lam" else m0
        d = np.zeros(shape)
        d.flat[idx] = h * base.flat[idx]
        if which == "lam":
            fd = (_J(o, w, src, rec, obs, l0 + d, m0) - _J(o, w, src, rec, obs, l0 - d, m0)) / (2 * d.flat[idx])
            co = gl[idx]
        else:
            fd = (_J(o, w, src, rec, obs, l0, m0 + d) - _J(o, w, src, rec, obs, l0, m0 - d)) / (2 * d.flat[idx])
            co = gm[idx]
        assert co != 0.0
        assert abs(fd - co) <= 2e-3 * abs(co), (kji, which, fd, co)


@pytest.mark.slow
def test_fd_gap_is_second_order_in_dt(oracle_mod):
    """The optimize-then-discretize gradient differs from the derivative of the discrete
    misfit by a time-discretisation error: halving dt cuts the gap by about 4."""
    gaps = []
    for fac in (1, 2):
        w = fi.tiny(nx=5, ny=5, nz=4, npml=2, nsteps=120 * fac, f0=30.0, nrec_side=5)
        w.dt = w.dt / fac
        o, src, rec, obs, l0, m0 = _setup(oracle_mod, w)
        J, gl, gm, _ = o.misfit_and_gradient(w.dt, w.nsteps, src, w.source_dirs(), rec, obs, "ricker",
                                             w.ricker())
        idx = np.ravel_multi_index((0, 5, 5), o.mat_shape())
        d = np.zeros(o.mat_shape())
        d.flat[idx] = 1e-4 * m0.flat[idx]
        fd = (_J(o, w, src, rec, obs, l0, m0 + d) - _J(o, w, src, rec, obs, l0, m0 - d)) / (2 * d.flat[idx])
        gaps.append(abs(fd - gm[idx]) / abs(gm[idx]))
    assert gaps[1] < gaps[0] / 3.0, gaps
