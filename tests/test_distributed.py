"""The shot-parallel reduction over CPU ranks (gloo): the summed misfit and gradients
equal, bitwise and on every rank, the single-process sum of the per-rank parts in
rank order; the shot ranges tile the shot list; timing takes the max over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

from paper_1504_08340_gb300.distributed import (max_over_ranks, reduce_gradient, sharded_adjoint_gradient,  # noqa: E402
                                                 shot_range)

SHAPE = (5, 7, 9)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _part(rank):
    """Seeded per-rank misfit and gradients, with magnitudes far apart so that the
    order of the sum shows in the last bits."""
    rng = np.random.default_rng(100 + rank)
    scale = 10.0 ** (3 * rank)
    gl = torch.tensor(scale * rng.standard_normal(SHAPE), dtype=torch.float64)
    gm = torch.tensor(scale * rng.standard_normal(SHAPE), dtype=torch.float64)
    return float(scale * rng.random()), gl, gm


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        J, gl, gm = _part(rank)
        Js, gls, gms = reduce_gradient(J, gl, gm)
        tmax = max_over_ranks(1.5 + rank)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), J=Js, gl=gls.numpy(), gm=gms.numpy(), tmax=tmax)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_reduce_gradient_is_the_rank_order_sum(tmp_path, world):
    import torch.multiprocessing as mp

    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    parts = [_part(r) for r in range(world)]
    J_ref, gl_ref, gm_ref = parts[0][0], parts[0][1].clone(), parts[0][2].clone()
    for J, gl, gm in parts[1:]:
        J_ref += J
        gl_ref += gl
        gm_ref += gm
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npz")
        assert float(got["J"]) == J_ref
        assert np.array_equal(got["gl"], gl_ref.numpy()) and np.array_equal(got["gm"], gm_ref.numpy())
        assert float(got["tmax"]) == 1.5 + (world - 1)


def test_reduce_without_process_group_is_identity():
    J, gl, gm = _part(0)
    Jr, glr, gmr = reduce_gradient(J, gl, gm)
    assert Jr == J and glr is gl and gmr is gm
    assert max_over_ranks(2.5) == 2.5


@pytest.mark.parametrize("nshots,world", [(16, 1), (16, 2), (16, 3), (64, 8), (5, 8), (0, 2)])
def test_shot_ranges_tile_the_shots(nshots, world):
    ranges = [shot_range(nshots, r, world) for r in range(world)]
    covered = [s for s0, n in ranges for s in range(s0, s0 + n)]
    assert covered == list(range(nshots))
    counts = [n for _, n in ranges]
    assert max(counts) - min(counts) <= 1


def test_shot_range_rejects_bad_arguments():
    for args in ((4, 2, 2), (4, -1, 2), (4, 0, 0), (-1, 0, 1)):
        with pytest.raises(ValueError):
            shot_range(*args)


class _FakeContext:
    """Stands in for the GPU context on CPU ranks: shot s contributes J = s + 1 and
    gradients scaled by 10^s, summed over the shots of a call in order."""

    def mat_shape(self):
        return SHAPE

    def adjoint_gradient(self, observed, shot0, count):
        assert observed.shape[0] == count
        J, gl, gm = 0.0, torch.zeros(SHAPE, dtype=torch.float64), torch.zeros(SHAPE, dtype=torch.float64)
        for s in range(shot0, shot0 + count):
            rng = np.random.default_rng(s)
            J += s + 1.0
            gl += torch.tensor(10.0 ** s * rng.standard_normal(SHAPE))
            gm += torch.tensor(10.0 ** s * rng.standard_normal(SHAPE))
        return J, gl, gm


def _sharded_main(rank, world, port, out_dir, nshots):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shot0, count = shot_range(nshots, rank, world)
        observed = torch.zeros((count, 3, 2, 3))  # this rank's traces
        J, gl, gm = sharded_adjoint_gradient(_FakeContext(), observed, nshots, rank, world)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), J=J, gl=gl.numpy(), gm=gm.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("nshots,world", [(5, 3), (1, 2)])
def test_sharded_gradient_over_ranks(tmp_path, nshots, world):
    """Each rank evaluates its shot range (a rank may have none) and every rank ends with
    the rank-order sum of the per-rank results."""
    import torch.multiprocessing as mp

    mp.spawn(_sharded_main, args=(world, _free_port(), str(tmp_path), nshots), nprocs=world, join=True)
    ctx = _FakeContext()
    J_ref, gl_ref, gm_ref = None, None, None
    for r in range(world):
        s0, n = shot_range(nshots, r, world)
        if n == 0:
            part = (0.0, torch.zeros(SHAPE, dtype=torch.float64), torch.zeros(SHAPE, dtype=torch.float64))
        else:
            part = ctx.adjoint_gradient(torch.zeros((n, 1)), s0, n)
        if J_ref is None:
            J_ref, gl_ref, gm_ref = part[0], part[1].clone(), part[2].clone()
        else:
            J_ref, gl_ref, gm_ref = J_ref + part[0], gl_ref + part[1], gm_ref + part[2]
    assert J_ref == sum(s + 1.0 for s in range(nshots))
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npz")
        assert float(got["J"]) == J_ref
        assert np.array_equal(got["gl"], gl_ref.numpy()) and np.array_equal(got["gm"], gm_ref.numpy())
