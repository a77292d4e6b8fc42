"""Pins of the oracle's mesh, DOF layout and PML coefficients (CPU only)."""
import os

import numpy as np
import pytest

from helpers import homogeneous

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "state_counts.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows.append(tuple(int(x) for x in f[:6]))
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_state_and_material_counts_match_paper(oracle_mod, row):
    """Sec. 4.2 / 4.5 print the number of state unknowns and material parameters.
    State = 3 per non-Dirichlet node (u) + 6 per PML node (symmetric S, reading R2)."""
    nx, ny, nz, p, n_state, n_mat = row
    o = oracle_mod.Oracle(nx, ny, nz, p, h=1.25, threads=1)
    pml, dirn = o.masks()
    assert 3 * int((~dirn).sum()) + 6 * int(pml.sum()) == n_state
    assert 2 * o.nmat == n_mat


def test_stretch_profile(oracle_mod):
    """alpha = 1 + alpha0 (l/L)^m, beta = beta0 (l/L)^m (Sec. 4.1 parameters), zero depth inside."""
    o = oracle_mod.Oracle(2, 2, 2, 3, h=2.0, threads=1)
    al, be = o.stretch(0)
    L = 3 * 2.0
    for c in range(o.nn[0]):
        lo, hi = 2 * 3, 2 * (3 + 2)
        l = (lo - c) * 1.0 if c < lo else ((c - hi) * 1.0 if c > hi else 0.0)
        assert al[c] == pytest.approx(1 + 5.0 * (l / L) ** 2, rel=1e-15)
        assert be[c] == pytest.approx(400.0 * (l / L) ** 2, rel=1e-15)
    al, be = o.stretch(2)
    assert al[0] == 1.0 and be[0] == 0.0  # free surface: no layer above
    assert al[-1] == pytest.approx(6.0) and be[-1] == pytest.approx(400.0)


def test_pml_coefficients_are_products_of_stretches(oracle_mod):
    """a + b s + c s^2 + d s^3 = prod_i (alpha_i + beta_i s) (reading R1), checked on the
    lumped diagonals: Mu : Cu : Ku : Gu = a : b : c : d at every PML node."""
    o = oracle_mod.Oracle(2, 2, 1, 2, h=1.0, threads=1)
    lam, mu = homogeneous(o)
    o.set_material(lam, mu)
    Mu, Cu, Ku, Gu = (o.diag(n) for n in ("Mu", "Cu", "Ku", "Gu"))
    Ms, Cs, Ks, Gs = (o.diag(n) for n in ("Ms", "Cs", "Ks", "Gs"))
    pml, _ = o.masks()
    st = [o.stretch(a) for a in range(3)]
    rng = np.random.default_rng(0)
    for g in rng.choice(np.flatnonzero(pml), 40, replace=False):
        i, j, k = g % o.nn[0], (g // o.nn[0]) % o.nn[1], g // (o.nn[0] * o.nn[1])
        poly = np.array([1.0])
        for a, c in zip(range(3), (i, j, k)):
            poly = np.polymul(poly, [st[a][1][c], st[a][0][c]])  # beta s + alpha
        poly = np.concatenate([np.zeros(4 - poly.size), poly])
        d, c, b, a = poly  # highest power first
        vol = Ms[g] / a
        assert Cs[g] == pytest.approx(b * vol, rel=1e-12, abs=1e-300)
        assert Ks[g] == pytest.approx(c * vol, rel=1e-12, abs=1e-300)
        assert Gs[g] == pytest.approx(d * vol, rel=1e-12, abs=1e-300)
        # u rows carry rho and the whole lumped volume (interior elements have a = 1, b = c = d = 0)
        assert Cu[g] * a == pytest.approx(Mu[g] * b, rel=1e-12, abs=1e-300)
        assert Gu[g] * a == pytest.approx(Mu[g] * d, rel=1e-12, abs=1e-300)


def test_lumped_volume_sums_to_domain_volume(oracle_mod):
    """The LGL-lumped M_uu / rho sums to the volume; Mtilde (C.1a) to the interior volume."""
    o = oracle_mod.Oracle(3, 2, 2, 2, h=1.5, alpha0=0.0, beta0=0.0, threads=1)
    N = o.N
    assert o.diag("Mu").sum() / 2000.0 == pytest.approx(N[0] * N[1] * N[2] * 1.5 ** 3, rel=1e-13)
    assert o.diag("Mtilde").sum() == pytest.approx(3 * 2 * 2 * 1.5 ** 3, rel=1e-13)
    # with alpha0 = beta0 = 0 the PML reduces to identity stretching: b = c = d = 0
    assert np.all(o.diag("Cu") == 0) and np.all(o.diag("Gs") == 0)
