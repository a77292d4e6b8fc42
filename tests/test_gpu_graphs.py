"""CUDA-graph replay of the sweeps (fwi_set_graphs): the recorded graphs issue the same
kernels with the same arguments as the direct launches, so every result is bitwise equal,
on the first (recording) call, on replays, with checkpointing, with shot batches and a
ragged last group, and after a device reallocation drops the recorded graphs; the
library's count of kernel launches is the same either way."""
import numpy as np
import pytest

import fwi_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(w):
    from paper_1504_08340_gb300 import Context

    return Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho)


def _run(ctx, obs, nshots):
    J, gl, gm = ctx.adjoint_gradient(obs, 0, nshots)
    tr = ctx.forward(0, nshots)
    return J, gl.copy(), gm.copy(), tr


def _same(a, b):
    assert a[0] == b[0]
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("ckpt,batch", [(0, 1), (7, 1), (0, 2), (-1, 2)])
def test_graph_replay_is_bitwise_the_direct_path(ckpt, batch):
    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=50, f0=30.0, nrec_side=3)
    src = np.array([[6, 6, 0], [8, 7, 0], [7, 8, 0]], dtype=np.int64)
    dirs = np.array([[0.0, 0.0, 1.0], [0.3, -0.2, 0.9], [0.0, 0.5, 0.5]])
    l0, m0 = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "trial"))
    with _ctx(w) as ctx:
        ctx.set_material(l0, m0)
        ctx.set_sources(src, dirs, "ricker", w.ricker())
        ctx.set_receivers(w.receivers())
        ctx.set_checkpointing(ckpt)
        ctx.set_shot_batch(batch)
        obs = np.ascontiguousarray(np.stack([fi.synthetic_traces(w.nsteps, ctx.nrec, 30 + s) for s in range(3)]),
                                   dtype=np.float32)
        direct = _run(ctx, obs, 3)
        ctx.reset_timing()
        _run(ctx, obs, 3)
        _, launches_direct = ctx.timing(3)
        ctx.set_graphs(True)
        first = _run(ctx, obs, 3)      # records
        ctx.reset_timing()
        second = _run(ctx, obs, 3)     # replays
        _, launches_graph = ctx.timing(3)
        _same(direct, first)
        _same(direct, second)
        assert launches_graph == launches_direct
        # a reallocation (another batch width) drops the recorded graphs: the sweeps are
        # recorded again, and match the direct launches at that width (another width sums
        # the shots' FP64 gradients in another order, so it is compared with itself)
        ctx.set_shot_batch(1 if batch > 1 else 2)
        regraphed = _run(ctx, obs, 3)
        ctx.set_graphs(False)
        _same(regraphed, _run(ctx, obs, 3))
        assert regraphed[0] == direct[0] and np.array_equal(regraphed[3], direct[3])
