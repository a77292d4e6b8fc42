"""fwi_regularization (Eqs. (8)/(9), gradients (C.1b)-(C.1e)) against the FP64 oracle."""
import numpy as np
import pytest

import fwi_inputs as fi
from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


@pytest.mark.parametrize("make", [lambda: fi.tiny(nx=4, ny=3, nz=2, npml=2, nsteps=10),
                                  lambda: fi.box_8x8x4(), lambda: fi.grf_64x64x32()],
                         ids=["tiny", "box_8x8x4", "grf_64x64x32"])
@pytest.mark.parametrize("kind,eps", [("tn", 0.0), ("tv", 0.01), ("tv", 1e14)])
def test_regularization_matches_oracle(oracle_mod, make, kind, eps):
    from paper_1504_08340_gb300 import Context

    w = make()
    lam, mu = (_f32(a) for a in fi.medium(w, "true"))
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
    with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho) as ctx:
        ctx.set_material(lam, mu)
        R, gl, gm = ctx.regularization(kind, eps)
        Rd, gld, gmd = ctx.regularization(kind, eps, device=True)
    for f, Rg, g, gd in ((lam, R[0], gl, gld), (mu, R[1], gm, gmd)):
        Ro, go = o.regularization(f.astype(np.float64), kind, eps)
        assert Rg == pytest.approx(Ro, rel=1e-10)
        assert rel_l2(g.ravel(), go) < 1e-9
        assert np.array_equal(gd.cpu().numpy(), g)  # host and device outputs: same kernels


def test_regularization_errors():
    from paper_1504_08340_gb300 import Context, FWIError

    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=10)
    with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho) as ctx:
        with pytest.raises(FWIError):
            ctx.regularization("tn")  # no material yet
        lam, mu = (_f32(a) for a in fi.medium(w, "true"))
        ctx.set_material(lam, mu)
        with pytest.raises(FWIError):
            ctx.regularization("tv", 0.0)
