"""Pins of the oracle's time integration: classic RK4 on (6) (CPU only)."""
import numpy as np
import pytest

from helpers import homogeneous


def _pml_off(oracle_mod):
    o = oracle_mod.Oracle(2, 2, 2, 0, h=1.0, threads=2)
    rng = np.random.default_rng(7)
    shape = o.mat_shape()
    o.set_material(1.6e8 * (1 + 0.1 * rng.random(shape)), 0.8e8 * (1 + 0.1 * rng.random(shape)))
    return o


def _dense_stiffness(o):
    _, dirn = o.masks()
    free = np.flatnonzero(~dirn)
    dofs = [(g, c) for g in free for c in range(3)]
    K = np.zeros((len(dofs), len(dofs)))
    for a, (g, c) in enumerate(dofs):
        u = np.zeros((o.nnode, 3))
        u[g, c] = 1.0
        f = o.apply("KRD", None, u)
        K[:, a] = [f[g2, c2] for g2, c2 in dofs]
    M = np.array([o.diag("Mu")[g] for g, _ in dofs])
    return dofs, K, M


def test_rk4_matches_exact_amplification_of_an_eigenmode(oracle_mod):
    """Start from an eigenvector v of K v = w^2 M v at rest; after n classic RK4 steps
    u_n = Re(R^n) v and du_n = -w Im(R^n) v with R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, z = i w dt."""
    o = _pml_off(oracle_mod)
    dofs, K, M = _dense_stiffness(o)
    assert np.allclose(K, K.T, rtol=0, atol=1e-6 * np.abs(K).max())
    Mi = 1 / np.sqrt(M)
    lam, V = np.linalg.eigh(Mi[:, None] * K * Mi[None, :])
    w_max = np.sqrt(lam.max())
    dt = 1.5 / w_max
    for idx in (len(lam) - 1, len(lam) // 2):
        w = np.sqrt(lam[idx])
        v = Mi * V[:, idx]
        Y = np.zeros((3, o.nnode, 9))
        for a, (g, c) in enumerate(dofs):
            Y[1, g, c] = v[a]
        n = 12
        for _ in range(n):
            Y = o.rk4_step(Y, dt)
        z = 1j * w * dt
        R = (1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24) ** n
        u = np.array([Y[1, g, c] for g, c in dofs])
        du = np.array([Y[2, g, c] for g, c in dofs])
        assert np.abs(u - R.real * v).max() < 1e-11 * np.abs(v).max()
        assert np.abs(du + w * R.imag * v).max() < 1e-11 * w * np.abs(v).max()


def test_energy_non_increasing_pml_off(oracle_mod):
    """Free vibration without PML: E = 1/2 du^T M du + 1/2 u^T K u never grows under RK4
    (|R(i y)|^2 = 1 - y^6/72 + y^8/576 <= 1 for y <= 2 sqrt 2) and loses at most that factor."""
    o = _pml_off(oracle_mod)
    pml, dirn = o.masks()
    _, K, M = _dense_stiffness(o)
    w_max = np.sqrt(np.linalg.eigvalsh(K / np.sqrt(M)[:, None] / np.sqrt(M)[None, :]).max())
    dt = 1.2 / w_max
    rng = np.random.default_rng(3)
    Y = np.zeros((3, o.nnode, 9))
    Y[1, :, :3] = rng.standard_normal((o.nnode, 3))
    Y[1, dirn, :3] = 0
    E = [o.energy(Y).sum()]
    for _ in range(40):
        Y = o.rk4_step(Y, dt)
        E.append(o.energy(Y).sum())
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-12 * E[0])
    y = w_max * dt
    assert E[-1] >= E[0] * (1 - y ** 6 / 72 + y ** 8 / 576) ** 40 * (1 - 1e-9)


@pytest.mark.slow
def test_energy_decays_with_pml(oracle_mod):
    """With the PML on, the energy of a surface pulse leaves the box (the paper picks T
    as the time the total energy dies out, Sec. 4.3 footnote 12): kinetic + interior
    strain energy falls below 1e-3 of its peak within 1000 steps."""
    o = oracle_mod.Oracle(4, 4, 3, 3, h=1.0, threads=8)
    o.set_material(*homogeneous(o))
    dt = 0.5 * 0.5 / 400.0
    node = o.node_id(o.nn[0] // 2, o.nn[1] // 2, 0)
    f0 = 60.0
    Y = np.zeros((3, o.nnode, 9))
    Es = []
    for n in range(1000):
        Y = _rk4_forced(o, Y, dt, n * dt, node, f0)
        if n % 10 == 9:
            Es.append(o.energy(Y).sum())
    Es = np.array(Es)
    assert np.all(np.isfinite(Es))
    assert Es[-1] < 1e-3 * Es.max()


def _rk4_forced(o, Y, dt, t, node, f0):
    def force(tt):
        a = np.pi * f0 * (tt - 1.5 / f0)
        f = np.zeros((o.nnode, 3))
        f[node, 2] = 1e3 * (1 - 2 * a * a) * np.exp(-a * a)
        return f
    k1 = o.rhs(Y, force(t))
    k2 = o.rhs(Y + 0.5 * dt * k1, force(t + 0.5 * dt))
    k3 = o.rhs(Y + 0.5 * dt * k2, force(t + 0.5 * dt))
    k4 = o.rhs(Y + dt * k3, force(t + dt))
    return Y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
