"""The large inversion workload at full size (160x160x80 interior + 12-element PML, 3.11 M
elements, 25.2 M nodes), on a 12-step window of its first two shots: properties that hold
at any size, in the launch configuration the large bench line uses.

- Traces of a shot batch of two equal those of one shot at a time, bit for bit.
- The gradient from compact sqrt(T)-style snapshots (every 4 steps) equals the one from
  the stored displacement history, bit for bit, and is nonzero and finite.
"""
import numpy as np
import pytest

import fwi_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NSTEPS = 12


def test_large_mesh_window_batch_and_checkpoint_identities():
    from paper_1504_08340_gb300 import Context

    w = fi.large_160x160x80()
    dev = torch.device("cuda", 0)
    with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, NSTEPS, rho=w.rho) as ctx:
        assert ctx.nnode == 25_189_785 and ctx.nelem == 3_114_752
        ctx.set_sources(w.sources(), w.source_dirs(), "ricker", (w.f0, 0.0, 1e3))  # pulse peak at t = 0
        ctx.set_receivers(w.receivers())
        lt, mt = (torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev) for a in fi.medium(w, "true"))
        ctx.set_material(lt, mt)
        one = torch.empty(ctx.trace_shape(2), dtype=torch.float32, device=dev)
        for s in range(2):
            ctx.forward(s, 1, out=one[s:s + 1])
        ctx.set_shot_batch(2)
        two = torch.empty_like(one)
        ctx.forward(0, 2, out=two)
        assert torch.equal(one, two)
        assert float(one.abs().max()) > 0
        obs = torch.tensor(np.stack([fi.synthetic_traces(NSTEPS, len(w.receivers()), 300 + s, scale=1e-9)
                                     for s in range(2)]), dtype=torch.float32, device=dev).contiguous()
        l0, m0 = (torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev) for a in fi.medium(w, "trial"))
        ctx.set_material(l0, m0)
        J0, gl0, gm0 = ctx.adjoint_gradient(obs, 0, 2)
        ctx.set_checkpointing(4)
        J1, gl1, gm1 = ctx.adjoint_gradient(obs, 0, 2)
        assert J1 == J0 and J0 > 0
        assert torch.equal(gl1, gl0) and torch.equal(gm1, gm0)
        assert bool(torch.isfinite(gl0).all()) and float(gl0.abs().max()) > 0
