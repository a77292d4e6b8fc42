"""Pins of the oracle's PML coupling operators (orc_apply_A, orc_apply_B and the lumped
a, b, c, d diagonals), of the source wavelet (orc_wavelet) and of the forward sweep's
trivial cases, against what the mathematics fixes (CPU only).

The PML of Sec. 2 is elastodynamics in complex-stretched coordinates: with the Laplace
variable s, x_j is stretched by eps_j(s) = alpha_j + beta_j / s, so d/dx~_j = (1/eps_j) d/dx_j.
For real s > 0 every eps_j is real. Multiplying div~ sigma = rho s^2 u and
sigma = C : grad~ u by eps_x eps_y eps_z gives, term by term, the Laplace transform of
(1b)/(1c) with zero initial state, S-hat = sigma / s. Two exact discrete consequences
follow, checked here at real s without any time stepping:

  S rows: (B_e + B_p / s + B_w / s^2) u / (M_S a + M_S b / s + ...) at a node equals the
          stress of u in the stretched coordinates, C : (grad u diag(1/eps)), whenever
          grad u is continuous there (u a global quadratic: exact LGL quadrature);
  u rows: (A_e + A_p / s + A_w / s^2) sigma at a node off the grid boundary whose elements
          are all PML equals -V (eps_x eps_y eps_z) div~ sigma for a linear nodal sigma
          (V the node's lumped volume), because Lambda_jj is constant along x_j.

A mistake in where Lambda sits (row against column index), in a product of the stretch
functions, or in a, b, c, d breaks these identities.
"""
import math

import numpy as np
import pytest

import fwi_inputs as fi
from helpers import homogeneous, node_coords, rel_l2

SYM = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))  # xx yy zz yz xz xy
LAM, MU = 1.3e8, 0.7e8  # distinct, so a lambda / mu swap is visible


def _mesh(oracle_mod, top_pml):
    o = oracle_mod.Oracle(3, 2, 2, 2, h=1.0, top_pml=top_pml, threads=2)
    o.set_material(*homogeneous(o, LAM, MU))
    return o


def _quadratic(o, seed, hessian=False):
    """A global quadratic displacement u, its exact gradient G[n, i, j] = du_i/dx_j and
    (optionally) its constant second derivatives H[i, j, k] = d^2 u_i / dx_j dx_k."""
    x, y, z = node_coords(o)
    one, zero = np.ones_like(x), np.zeros_like(x)
    mono = np.stack([one, x, y, z, x * x, y * y, z * z, x * y, y * z, x * z], 1)
    dmono = [np.stack([zero, one, zero, zero, 2 * x, zero, zero, y, zero, z], 1),
             np.stack([zero, zero, one, zero, zero, 2 * y, zero, x, z, zero], 1),
             np.stack([zero, zero, zero, one, zero, zero, 2 * z, zero, y, x], 1)]
    C = np.random.default_rng(seed).standard_normal((10, 3))
    u = mono @ C
    G = np.stack([d @ C for d in dmono], 2)  # [n][i][j]
    if not hessian:
        return u, G
    H = np.zeros((3, 3, 3))
    for i in range(3):
        H[i] = [[2 * C[4, i], C[7, i], C[9, i]], [C[7, i], 2 * C[5, i], C[8, i]], [C[9, i], C[8, i], 2 * C[6, i]]]
    return u, G, H


def _eps(o, s):
    """eps_j(s) = alpha_j + beta_j / s at every node, [n][3]."""
    n = np.arange(o.nnode)
    idx = (n % o.nn[0], (n // o.nn[0]) % o.nn[1], n // (o.nn[0] * o.nn[1]))
    out = np.empty((o.nnode, 3))
    for a in range(3):
        al, be = o.stretch(a)
        out[:, a] = al[idx[a]] + be[idx[a]] / s
    return out


def _node_ijk(o):
    n = np.arange(o.nnode)
    return n % o.nn[0], (n // o.nn[0]) % o.nn[1], n // (o.nn[0] * o.nn[1])


def _deep_pml(o):
    """Nodes off the grid boundary all of whose elements are PML elements."""
    c = _node_ijk(o)
    off_boundary = np.ones(o.nnode, bool)
    touches_interior = np.ones(o.nnode, bool)
    for a in range(3):
        off_boundary &= (c[a] > 0) & (c[a] < o.nn[a] - 1)
        touches_interior &= (c[a] >= 2 * o.lo[a]) & (c[a] <= 2 * o.hi[a])
    return off_boundary & ~touches_interior


def _lumped_volume(o):
    """int phi_a: (h/2)^3 times, per axis, 4/3 at an element centre and 2/3 at a shared
    end node (off the grid boundary)."""
    c = _node_ijk(o)
    v = np.full(o.nnode, (0.5 * o.h) ** 3)
    for a in range(3):
        v *= np.where(c[a] % 2 == 1, 4.0 / 3.0, 2.0 / 3.0)
    return v


@pytest.mark.parametrize("top_pml", [False, True])
@pytest.mark.parametrize("s", [25.0, 400.0, 6000.0])
def test_stress_rows_are_the_stretched_coordinate_stress(oracle_mod, top_pml, s):
    """Pins orc_apply_B (all three Lambda's) and the S-row diagonals M_S, C_S, K_S, G_S."""
    o = _mesh(oracle_mod, top_pml)
    u, G = _quadratic(o, 11)
    num = o.apply("B", 0, u) + o.apply("B", 1, u) / s + o.apply("B", 2, u) / s ** 2
    den = o.diag("Ms") + o.diag("Cs") / s + o.diag("Ks") / s ** 2 + o.diag("Gs") / s ** 3
    pml, _ = o.masks()
    Gt = G / _eps(o, s)[:, None, :]  # grad~ u: d u_i / d x~_j
    tr = Gt[:, 0, 0] + Gt[:, 1, 1] + Gt[:, 2, 2]
    expect = np.stack([MU * (Gt[:, i, j] + Gt[:, j, i]) + (LAM * tr if i == j else 0.0) for i, j in SYM], 1)
    got = num[pml] / den[pml][:, None]
    assert np.abs(got - expect[pml]).max() < 1e-11 * np.abs(expect[pml]).max()
    # the identity is not empty: the stretching changes the stress by O(1)
    plain = np.stack([MU * (G[:, i, j] + G[:, j, i]) + (LAM * np.trace(G, axis1=1, axis2=2) if i == j else 0.0)
                      for i, j in SYM], 1)
    assert rel_l2(expect[pml], plain[pml]) > 0.1


@pytest.mark.parametrize("top_pml", [False, True])
@pytest.mark.parametrize("s", [25.0, 400.0, 6000.0])
def test_displacement_rows_are_the_stretched_divergence(oracle_mod, top_pml, s):
    """Pins orc_apply_A (all three Lambda's): for a linear symmetric nodal stress,
    (A_e + A_p/s + A_w/s^2) sigma = -V eps_x eps_y eps_z div~ sigma at deep PML nodes."""
    o = _mesh(oracle_mod, top_pml)
    x, y, z = node_coords(o)
    rng = np.random.default_rng(12)
    base, gx, gy, gz = (rng.standard_normal(6) for _ in range(4))
    S = base[None] + x[:, None] * gx[None] + y[:, None] * gy[None] + z[:, None] * gz[None]
    pml, _ = o.masks()
    S[~pml] = 0.0
    got = o.apply("A", 0, S) + o.apply("A", 1, S) / s + o.apply("A", 2, S) / s ** 2
    grad = (gx, gy, gz)  # d sigma_c / d x_j, c in SYM order
    comp = {(i, j): c for c, (i, j) in enumerate(SYM)}
    comp.update({(j, i): c for (i, j), c in list(comp.items())})
    eps = _eps(o, s)
    a = eps.prod(1)
    div = np.stack([sum(grad[j][comp[(i, j)]] / eps[:, j] for j in range(3)) for i in range(3)], 1)
    expect = -_lumped_volume(o)[:, None] * a[:, None] * div
    deep = _deep_pml(o)
    assert deep.sum() > 50
    assert np.abs(got[deep] - expect[deep]).max() < 1e-11 * np.abs(expect[deep]).max()


def test_identity_stretch_patch_test_across_the_interface(oracle_mod):
    """alpha0 = beta0 = 0 (Lambda_e = I, a = 1, every other coefficient 0): a PML element is
    then plain elastic, with Sdot the Cauchy stress (Sec. 2). For a global quadratic u with
    stress sigma(u) on the PML nodes, the u-row force -(K_RD u + A_e sigma) of the full rate
    equals V div sigma at every node off the grid boundary, interface nodes included; the
    S-row rate of a displacement rate u is sigma(u) on every PML node."""
    o = oracle_mod.Oracle(3, 2, 2, 2, h=1.0, alpha0=0.0, beta0=0.0, threads=2)
    o.set_material(*homogeneous(o, LAM, MU))
    u, G, H = _quadratic(o, 13, hessian=True)
    tr = np.trace(G, axis1=1, axis2=2)
    sig = np.stack([MU * (G[:, i, j] + G[:, j, i]) + (LAM * tr if i == j else 0.0) for i, j in SYM], 1)
    pml, dirn = o.masks()
    Y = np.zeros((3, o.nnode, 9))
    Y[1, :, :3] = u          # displacement (values on the fixed faces are read, not updated)
    Y[2, :, :3] = u          # displacement rate, drives the S rows
    Y[2, :, 3:] = np.where(pml[:, None], sig, 0.0)  # Sdot = sigma(u)
    dY = o.rhs(Y)
    c = _node_ijk(o)
    inside = np.ones(o.nnode, bool)
    for a in range(3):
        inside &= (c[a] > 0) & (c[a] < o.nn[a] - 1)
    divs = np.array([sum(MU * (H[i, j, j] + H[j, i, j]) + (LAM * np.trace(H[:, :, j]) if i == j else 0.0)
                         for j in range(3)) for i in range(3)])
    force = dY[2, :, :3] * o.diag("Mu")[:, None]
    expect = _lumped_volume(o)[:, None] * divs[None, :]
    assert np.abs(force[inside] - expect[inside]).max() < 1e-10 * np.abs(divs).max()
    # S rows: rate of Sdot = sigma(udot)
    assert np.abs(dY[2, pml, 3:] - sig[pml]).max() < 1e-11 * np.abs(sig).max()


def test_ricker_closed_form(oracle_mod):
    """orc_wavelet kind 0: A at t0, symmetric about t0, zeros at t0 +- 1/(pi f0 sqrt 2),
    minima -2A e^{-3/2} at t0 +- sqrt(3/2)/(pi f0), amplitude spectrum peaking at f0."""
    f0, t0, A = 15.0, 0.1, 1.0e3
    w = lambda t: oracle_mod.wavelet("ricker", (f0, t0, A), t)  # noqa: E731
    assert w(t0) == A
    tz = 1.0 / (math.pi * f0 * math.sqrt(2.0))
    tm = math.sqrt(1.5) / (math.pi * f0)
    for sgn in (-1, 1):
        assert abs(w(t0 + sgn * tz)) < 1e-12 * A
        assert w(t0 + sgn * tm) == pytest.approx(-2 * A * math.exp(-1.5), rel=1e-13)
        assert w(t0 + sgn * 0.9 * tm) > w(t0 + sgn * tm) < w(t0 + sgn * 1.1 * tm)
    for tau in (0.003, 0.01, 0.05):
        assert w(t0 + tau) == pytest.approx(w(t0 - tau), rel=1e-12, abs=1e-300)
    dt = 1e-4
    t = np.arange(0, 4096) * dt
    sig = np.array([w(ti) for ti in t])
    spec = np.abs(np.fft.rfft(sig, n=1 << 17))
    f = np.fft.rfftfreq(1 << 17, dt)
    assert f[np.argmax(spec)] == pytest.approx(f0, abs=0.1)


def test_gaussian_pulse_closed_form(oracle_mod):
    """orc_wavelet kind 1, A exp(-(t - mu)^2 / sigma): A at mu and A/e at mu +- sqrt(sigma)."""
    mu, sigma, A = 0.2, 0.0014, 2.5
    w = lambda t: oracle_mod.wavelet("gauss", (mu, sigma, A), t)  # noqa: E731
    assert w(mu) == A
    for sgn in (-1, 1):
        assert w(mu + sgn * math.sqrt(sigma)) == pytest.approx(A / math.e, rel=1e-13)


def _small_forward(o, amp, src_nodes, dirs, rec_nodes, nsteps=40, f0=40.0):
    dt = 0.5 * 0.5 / 400.0
    return o.forward(dt, nsteps, src_nodes, dirs, "ricker", (f0, 1.5 / f0, amp), rec_nodes)


def test_forward_zero_source_and_linearity(oracle_mod):
    """Zero load gives identically zero traces; traces are linear in the load amplitude
    and superpose over sources."""
    o = oracle_mod.Oracle(3, 3, 2, 2, h=1.0, threads=2)
    rng = np.random.default_rng(4)
    o.set_material(1.6e8 * (1 + 0.1 * rng.random(o.mat_shape())), 0.8e8 * (1 + 0.1 * rng.random(o.mat_shape())))
    rec = [o.node_id(i, j, 0) for i in (4, 6, 8) for j in (4, 6, 8)] + [o.node_id(5, 6, 3)]
    s1, s2 = [o.node_id(6, 6, 0)], [o.node_id(5, 7, 2)]
    d1, d2 = [[0.0, 0.0, 1.0]], [[0.3, -0.4, 0.5]]
    assert np.all(_small_forward(o, 0.0, s1, d1, rec) == 0.0)
    t1 = _small_forward(o, 1.0e3, s1, d1, rec)
    t3 = _small_forward(o, 3.0e3, s1, d1, rec)
    assert np.abs(t1).max() > 0
    assert np.abs(t3 - 3 * t1).max() < 1e-13 * np.abs(t3).max()
    t2 = _small_forward(o, 1.0e3, s2, d2, rec)
    both = _small_forward(o, 1.0e3, s1 + s2, d1 + d2, rec)
    assert np.abs(both - (t1 + t2)).max() < 1e-13 * np.abs(both).max()


def test_forward_mirror_symmetry(oracle_mod):
    """Homogeneous medium, square mesh, vertical load at the surface centre: traces at
    receivers mirrored in x = x_c flip u_x and keep u_y, u_z; traces at receivers swapped
    by the diagonal x <-> y swap u_x and u_y."""
    o = oracle_mod.Oracle(4, 4, 2, 2, h=1.0, threads=2)
    o.set_material(*homogeneous(o))
    c = o.nn[0] // 2
    pts = [(c + 1, c + 3), (c + 2, c - 1), (c + 4, c + 4), (c, c + 2)]
    rec = []
    for i, j in pts:
        rec += [o.node_id(i, j, 0), o.node_id(2 * c - i, j, 0), o.node_id(j, i, 0)]
    tr = _small_forward(o, 1.0e3, [o.node_id(c, c, 0)], [[0.0, 0.0, 1.0]], rec, nsteps=60)
    scale = np.abs(tr).max()
    assert scale > 0
    for p in range(len(pts)):
        a, m, t = tr[:, 3 * p], tr[:, 3 * p + 1], tr[:, 3 * p + 2]
        assert np.abs(m[:, 0] + a[:, 0]).max() < 1e-12 * scale
        assert np.abs(m[:, 1:] - a[:, 1:]).max() < 1e-12 * scale
        assert np.abs(t[:, 0] - a[:, 1]).max() < 1e-12 * scale
        assert np.abs(t[:, 1] - a[:, 0]).max() < 1e-12 * scale
        assert np.abs(t[:, 2] - a[:, 2]).max() < 1e-12 * scale


@pytest.mark.slow
def test_pml_reflection_against_a_wider_domain(oracle_mod):
    """The 8x8x4 + 3 PML box (the tiny gradient box's mesh) against the same medium on a
    domain three times as wide and deep: surface traces over the first 100 steps, which end
    before anything reflected at the wide domain's boundary returns, agree to < 1e-3
    relative L2. With the PML replaced by fixed faces the same comparison is off by more
    than 30 times as much: the window does hold the small box's boundary reflections."""
    f0, dt, nsteps = 30.0, 0.5 * 0.5 / 400.0, 100

    def traces(n, nz, p):
        o = oracle_mod.Oracle(n, n, nz, p, h=1.0, threads=8)
        o.set_material(*homogeneous(o))
        c = 2 * p + n
        rec = [o.node_id(c + di, c + dj, 0) for dj in range(-8, 9, 4) for di in range(-8, 9, 4)]
        return o.forward(dt, nsteps, [o.node_id(c, c, 0)], [[0.0, 0.0, 1.0]], "ricker", (f0, 1.5 / f0, 1e3), rec)

    wide = traces(24, 12, 3)
    err_pml = rel_l2(traces(8, 4, 3), wide)
    err_fixed = rel_l2(traces(8, 4, 0), wide)
    assert err_pml < 1e-3
    assert err_fixed > 30 * err_pml


def _stokes(x, t, f0, t0, amp, rho, vp, vs):
    """Displacement at offset x (m) of a point force amp * Ricker(t) along z at the origin of
    a homogeneous full space: Stokes' solution (Aki & Richards, Quantitative Seismology,
    Eq. 4.23), the near-field integral int_{r/vp}^{r/vs} tau X0(t - tau) dtau by
    400-point Gauss-Legendre quadrature."""
    r = float(np.linalg.norm(x))
    g = np.asarray(x, dtype=np.float64) / r

    def X0(tt):
        a = np.pi * f0 * (tt - t0)
        return amp * (1 - 2 * a * a) * np.exp(-a * a)

    xg, wg = np.polynomial.legendre.leggauss(400)
    ta, tb = r / vp, r / vs
    tau = 0.5 * (tb - ta) * xg + 0.5 * (tb + ta)
    near = (tau[None, :] * X0(t[:, None] - tau[None, :])) @ (0.5 * (tb - ta) * wg)
    u = np.zeros((t.size, 3))
    for i in range(3):
        dij = 1.0 if i == 2 else 0.0
        u[:, i] = ((3 * g[i] * g[2] - dij) / r ** 3 * near / (4 * np.pi * rho)
                   + g[i] * g[2] / r * X0(t - r / vp) / (4 * np.pi * rho * vp ** 2)
                   - (g[i] * g[2] - dij) / r * X0(t - r / vs) / (4 * np.pi * rho * vs ** 2))
    return u


@pytest.mark.slow
def test_homogeneous_point_force_matches_stokes_solution(oracle_mod):
    """Buried vertical point force in a homogeneous medium with the PML on all six faces
    (a full space), Ricker f0 = 20 Hz: traces 3-4.5 m from the source (axial, diagonal and
    oblique offsets, near-, intermediate- and far-field terms all present) against Stokes'
    closed form, over 1.5 Ricker periods after the pulse. Relative L2 <= 3e-2 at h = 1 m,
    and at least 3 times smaller than at h = 2 m over the same physical box."""
    rho, vs, vp, f0, amp = 2000.0, 200.0, 400.0, 20.0, 1.0e3
    offsets_m = [(3, 0, 0), (0, 0, 3), (2, 2, 0), (2, 0, 2), (0, 3, 2), (4, 0, 0), (0, 0, 4)]

    def error(h, n, p):
        o = oracle_mod.Oracle(n, n, n, p, h=h, top_pml=True, threads=8)
        lam, mu = fi.lame_from_velocities(vs, vp, rho)
        o.set_material(*homogeneous(o, lam, mu))
        c = 2 * p + n
        dt = 0.5 * 0.5 * h / vp
        nsteps = int(round(3.0 / f0 / dt))
        offs = [tuple(int(round(v / (0.5 * h))) for v in off) for off in offsets_m]
        rec = [o.node_id(c + a, c + b, c + d) for a, b, d in offs]
        tr = o.forward(dt, nsteps, [o.node_id(c, c, c)], [[0.0, 0.0, 1.0]], "ricker", (f0, 1.5 / f0, amp), rec)
        t = np.arange(nsteps + 1) * dt
        ref = np.stack([_stokes(np.array(off, dtype=np.float64) * 0.5 * h, t, f0, 1.5 / f0, amp, rho, vp, vs)
                        for off in offs], 1)
        return rel_l2(tr, ref)

    coarse = error(2.0, 6, 2)
    fine = error(1.0, 12, 3)
    assert fine <= 3e-2
    assert coarse >= 3 * fine
