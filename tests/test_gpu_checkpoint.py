"""sqrt(T) checkpointing of the adjoint sweep and the torch.autograd wrapper.

Checkpointing recomputes the forward steps of each segment from a snapshot, so the
displacement history, and hence J and the gradients, must equal the stored-history
path bit for bit. The autograd wrapper must hand back exactly what
fwi_adjoint_gradient returns, and the gradient must match the FP64 oracle."""
import numpy as np
import pytest

import fwi_inputs as fi
from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _setup(w):
    from paper_1504_08340_gb300 import Context

    ctx = Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho)
    lt, mt = (_f32(a) for a in fi.medium(w, "true"))
    l0, m0 = (_f32(a) for a in fi.medium(w, "trial"))
    ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
    ctx.set_receivers(w.receivers())
    ctx.set_material(lt, mt)
    obs = torch.zeros(ctx.trace_shape(1), dtype=torch.float32, device="cuda")
    ctx.forward(out=obs)
    ctx.set_material(l0, m0)
    return ctx, obs, l0, m0


@pytest.mark.parametrize("nsteps", [60, 61])
def test_checkpointed_gradient_is_bit_identical(nsteps):
    w = fi.tiny(nx=4, ny=3, nz=2, npml=2, nsteps=nsteps, f0=30.0, nrec_side=3)
    ctx, obs, _, _ = _setup(w)
    with ctx:
        J0, gl0, gm0 = ctx.adjoint_gradient(obs)
        for every in (1, 7, 8, -1, nsteps - 1, nsteps, 10 * nsteps):
            ctx.set_checkpointing(every)
            J, gl, gm = ctx.adjoint_gradient(obs)
            assert J == J0, every
            assert torch.equal(gl, gl0) and torch.equal(gm, gm0), every
        ctx.set_checkpointing(0)
        J, gl, gm = ctx.adjoint_gradient(obs)
        assert J == J0 and torch.equal(gl, gl0) and torch.equal(gm, gm0)


def test_autograd_returns_the_adjoint_gradient(oracle_mod):
    from paper_1504_08340_gb300.autograd import misfit

    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=40, f0=30.0, nrec_side=3)
    ctx, obs, l0, m0 = _setup(w)
    with ctx:
        ctx.set_checkpointing(-1)
        lam = torch.tensor(l0, device="cuda", requires_grad=True)
        mu = torch.tensor(m0, device="cuda", requires_grad=True)
        J = misfit(ctx, lam, mu, obs)
        J.backward()
        ctx.set_checkpointing(0)
        ctx.set_material(l0, m0)
        J_ref, gl, gm = ctx.adjoint_gradient(obs)
        assert J.item() == J_ref
        assert torch.equal(lam.grad, gl.to(torch.float32)) and torch.equal(mu.grad, gm.to(torch.float32))
        # a scaled output gradient scales the result
        lam.grad = None
        mu.grad = None
        (3.0 * misfit(ctx, lam, mu, obs)).backward()
        assert torch.equal(lam.grad, (3.0 * gl).to(torch.float32))

        # and the gradient is the oracle's (FP64) to the parity tolerance
        o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
        src = [o.node_id(*s) for s in w.sources()]
        rec = [o.node_id(*r) for r in w.receivers()]
        o.set_material(l0.astype(np.float64), m0.astype(np.float64))
        Jo, glo, gmo, _ = o.misfit_and_gradient(w.dt, w.nsteps, src, w.source_dirs(), rec,
                                                obs.cpu().numpy()[0].astype(np.float64), "ricker", w.ricker())
        assert J.item() == pytest.approx(Jo, rel=2e-5)
        assert rel_l2(gl.cpu().numpy().ravel(), glo.ravel()) < 1e-4
        assert rel_l2(gm.cpu().numpy().ravel(), gmo.ravel()) < 1e-4
