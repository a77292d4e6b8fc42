"""sqrt(T) checkpointing of the adjoint sweep and the torch.autograd wrapper.

Checkpointing recomputes the forward steps of each segment from a compact snapshot, so
the displacement history, and hence J and the gradients, must equal the stored-history
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


@pytest.mark.parametrize("npml,top", [(2, False), (2, True), (0, False)])
def test_compact_snapshots_batched_bit_identical(npml, top):
    """Snapshots keep u and udot everywhere and the other 21 fields on the PML nodes only;
    restoring them must give the stored-history gradients bit for bit for a batch of two
    with a ragged last group (three shots), with a top PML and on a PML-free box."""
    from paper_1504_08340_gb300 import Context

    w = fi.tiny(nx=4, ny=3, nz=2, npml=npml, nsteps=41, f0=30.0, nrec_side=3)
    p, kz = npml, (2 * npml if top else 0)  # the interior's top surface
    src = np.array([(2 * p + 2, 2 * p + 2, kz), (2 * p + 4, 2 * p + 3, kz), (2 * p + 6, 2 * p + 4, kz)])
    rec = np.array([(2 * p + i, 2 * p + j, kz) for j in (1, 3, 5) for i in (1, 4, 7)])
    dirs = np.tile([0.0, 0.0, 1.0], (3, 1))
    obs = torch.tensor(np.stack([fi.synthetic_traces(w.nsteps, len(rec), 40 + s, scale=1e-7) for s in range(3)]),
                       dtype=torch.float32, device="cuda").contiguous()
    with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho, top_pml=top) as ctx:
        l0, m0 = (_f32(a) for a in fi.medium(w, "trial"))
        ctx.set_material(l0, m0)
        ctx.set_sources(src, dirs, "ricker", w.ricker())
        ctx.set_receivers(rec)
        ctx.set_shot_batch(2)
        J0, gl0, gm0 = ctx.adjoint_gradient(obs, 0, 3)
        assert J0 > 0 and float(gl0.abs().max()) > 0
        for every in (1, 5, -1, 40):
            ctx.set_checkpointing(every)
            J, gl, gm = ctx.adjoint_gradient(obs, 0, 3)
            assert J == J0, every
            assert torch.equal(gl, gl0) and torch.equal(gm, gm0), every


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
