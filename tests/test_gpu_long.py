"""Long-run parity, energy decay and finite-difference checks of the CUDA path.

- 2000 RK4 steps (the single-shot configuration's dt, f0, PML and medium recipe on a
  16x16x8 box): traces, J and gradients against the FP64 oracle's values written by
  tests/golden/make_long_run.py (which calls only the oracle);
- the energy of the GPU wavefield with the PML on decays once the source has ended
  (Sec. 4.3 takes T as the time at which the energy dies out);
- directional finite differences (26)/(27) of J computed on the GPU against the
  GPU's adjoint gradient, as the paper checks its gradient (Sec. 4.1, Table 2).
"""
import os

import numpy as np
import pytest

import fwi_inputs as fi
from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "long_run_grf_16x16x8.npz")


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _context(w, nsteps=None):
    from paper_1504_08340_gb300 import Context

    return Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, nsteps or w.nsteps, rho=w.rho)


def test_long_run_2000_steps_against_oracle():
    """Traces <= 1e-5 relative L2 (and every sample within 2e-5 of the largest), J <= 2e-5,
    gradients <= 1e-4 after 2000 FP32 RK4 steps forward and 2000 adjoint steps."""
    gold = np.load(GOLDEN)
    w = fi.grf_16x16x8()
    assert int(gold["nsteps"]) == w.nsteps and float(gold["dt"]) == w.dt
    l0, m0 = (_f32(a) for a in fi.medium(w, "trial"))
    with _context(w) as ctx:
        ctx.set_material(l0, m0)
        ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
        ctx.set_receivers(w.receivers())
        tr = ctx.forward()[0]
        obs = torch.tensor(gold["observed"][None], device="cuda:0").contiguous()
        J, gl, gm = ctx.adjoint_gradient(obs)
        gl, gm = gl.cpu().numpy().ravel(), gm.cpu().numpy().ravel()
    ref = gold["traces"].astype(np.float64)
    assert rel_l2(tr, ref) < 1e-5, rel_l2(tr, ref)
    assert np.abs(tr - ref).max() < 2e-5 * np.abs(ref).max()
    assert abs(J - float(gold["J"])) <= 2e-5 * float(gold["J"])
    assert rel_l2(gl, gold["g_lambda"]) < 1e-4, rel_l2(gl, gold["g_lambda"])
    assert rel_l2(gm, gold["g_mu"]) < 1e-4, rel_l2(gm, gold["g_mu"])


def test_energy_decays_with_the_pml_on(oracle_mod):
    """Kinetic plus interior strain energy of the GPU state (evaluated in FP64 by the
    oracle's energy routine) on the grf_16x16x8 box: after the Ricker has ended it falls
    below 1e-3 of its peak within 2000 steps, and it never rises by more than 1e-3 of the
    peak from one sample to the next."""
    w = fi.grf_16x16x8()
    lt, mt = (_f32(a) for a in fi.medium(w, "true"))
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
    o.set_material(lt.astype(np.float64), mt.astype(np.float64))
    t_end = 2 * 1.5 / w.f0  # the Ricker is below 1e-7 of its peak after 2 t0
    steps = list(range(100, 2001, 100))
    energy = []
    for n in steps:
        with _context(w, nsteps=n) as ctx:
            ctx.set_material(lt, mt)
            ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
            ctx.set_receivers(w.receivers())
            ctx.forward()
            idx = ctx.state_index()
            st = ctx.state()
        Y = np.zeros((3, o.nnode, 9))
        for lv in range(3):
            for c in range(9):
                Y[lv, :, c] = st[9 * lv + c, idx]
        energy.append(o.energy(Y).sum())
    E = np.array(energy)
    assert np.all(np.isfinite(E)) and E.max() > 0
    after = np.array([n * w.dt > t_end for n in steps])
    Ea = E[after]
    assert Ea[-1] < 1e-3 * E.max(), (Ea[-1] / E.max())
    assert np.all(np.diff(Ea) <= 1e-3 * E.max()), np.diff(Ea) / E.max()


def test_directional_finite_differences_of_the_gpu_gradient():
    """(26)/(27): for smooth perturbations of lambda and of mu inside the interior (away
    from the PML, whose material the gradient leaves out, Sec. 3.1.3), the central
    difference (J(m + h dm) - J(m - h dm)) / 2h at relative steps h = 1e-3, 1e-4, 1e-5
    agrees with g_mis . dm to three digits for the best h (Table 2 pattern)."""
    w = fi.box_8x8x4()
    lt, mt = (_f32(a) for a in fi.medium(w, "true"))
    l0, m0 = (_f32(a) for a in fi.medium(w, "trial"))
    Z, Y, X = np.meshgrid(*[np.arange(n) * 0.5 * w.h for n in w.mat_shape], indexing="ij")
    cx, cy, cz = 0.5 * w.nx * w.h + 0.7, 0.5 * w.ny * w.h - 0.4, 1.5
    bump = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) / (2 * 0.5 ** 2))
    edge = np.ones(bump.shape, bool)
    edge[:-1, 1:-1, 1:-1] = False  # interface with the PML: the sides and the bottom (not the free top)
    assert bump[edge].max() < 1e-5
    with _context(w) as ctx:
        ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
        ctx.set_receivers(w.receivers())
        ctx.set_material(lt, mt)
        obs = ctx.forward()
        ctx.set_material(l0, m0)
        J, gl, gm = ctx.adjoint_gradient(obs)
        assert J > 0
        for which, base, g in (("lambda", l0, gl), ("mu", m0, gm)):
            dm = bump * base.astype(np.float64)
            errs = []
            for h in (1e-3, 1e-4, 1e-5):
                plus, minus = _f32(base + h * dm), _f32(base - h * dm)
                # the perturbation the FP32 material actually carries
                d_co = float((g * (plus.astype(np.float64) - minus.astype(np.float64))).sum()) / (2 * h)
                Js = []
                for pert in (plus, minus):
                    if which == "lambda":
                        ctx.set_material(pert, m0)
                    else:
                        ctx.set_material(l0, pert)
                    Js.append(ctx.misfit(obs))
                d_fd = (Js[0] - Js[1]) / (2 * h)
                errs.append(abs(d_fd - d_co) / abs(d_co))
            ctx.set_material(l0, m0)
            assert min(errs) <= 2e-3, (which, errs)
