"""Shot-parallel gradient evaluation over ranks (one process per GPU).

Shots are independent wave problems given lambda and mu, and the misfit (7) and its
gradient are sums over the shots (Sec. 3), so the path shards by shot: each rank
evaluates a contiguous range of shots on its own GPU and the per-rank misfits and
FP64 gradients are summed once per evaluation. That sum is the only exchange.

The sum is formed in a fixed rank order, rank 0 + rank 1 + ..., so every rank holds the
same bits whatever reduction tree the backend would use. It runs as a chunked
reduce-scatter and all-gather: the flattened (J, g_lambda, g_mu) is cut into one chunk per
rank, an all-to-all hands rank r every rank's chunk r, rank r adds them in rank order,
and an all-gather returns the summed chunks to every rank. Each rank holds about three
copies of the gradient, whatever the number of ranks. The collectives run on the default
process group (or the one passed in) with tensors on the gradients' device: an NCCL group
for CUDA tensors, a gloo group for CPU ones.
"""
from __future__ import annotations


def shot_range(nshots: int, rank: int, world: int):
    """(shot0, count) of `rank`'s contiguous share of `nshots` shots; the first
    nshots % world ranks take one shot more. A rank may get no shot (count 0)."""
    if nshots < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("need nshots >= 0, world >= 1 and 0 <= rank < world")
    base, extra = divmod(nshots, world)
    shot0 = rank * base + min(rank, extra)
    return shot0, base + (1 if rank < extra else 0)


def _world(group):
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return 1
    return dist.get_world_size(group)


def reduce_gradient(J: float, g_lambda, g_mu, group=None):
    """Sum of (J, g_lambda, g_mu) over the ranks in rank order; the same bits on every
    rank. g_lambda, g_mu: FP64 tensors of equal shape on every rank. Without a process
    group (or with one rank) the inputs come back unchanged."""
    import torch
    import torch.distributed as dist

    if _world(group) == 1:
        return J, g_lambda, g_mu
    n = g_lambda.numel()
    if g_mu.numel() != n or g_lambda.dtype != torch.float64 or g_mu.dtype != torch.float64:
        raise ValueError("g_lambda and g_mu must be FP64 tensors of one size")
    world = _world(group)
    length = 1 + 2 * n
    chunk = -(-length // world)
    send = torch.zeros(world * chunk, dtype=torch.float64, device=g_lambda.device)
    send[0] = J
    send[1:1 + n] = g_lambda.reshape(-1)
    send[1 + n:length] = g_mu.reshape(-1)
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)  # recv[r chunk] = rank r's chunk of this rank
    rows = recv.view(world, chunk)
    mine = rows[0].clone()
    for r in range(1, world):
        mine += rows[r]
    parts = [torch.empty(chunk, dtype=torch.float64, device=g_lambda.device) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    total = torch.cat(parts)[:length]
    return float(total[0]), total[1:1 + n].view(g_lambda.shape), total[1 + n:].view(g_mu.shape)


def max_over_ranks(x: float, device="cpu", group=None) -> float:
    """The largest of the ranks' values of x (x itself without a process group)."""
    import torch
    import torch.distributed as dist

    if _world(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sharded_adjoint_gradient(ctx, observed, nshots: int, rank: int, world: int, group=None):
    """Misfit and gradient over shots 0 .. nshots - 1 with this rank evaluating its
    shot_range share through fwi_adjoint_gradient; observed: this rank's traces,
    [count][nsteps + 1][nrec][3] on its GPU. Returns the rank-order sums (J, g_lambda,
    g_mu) on every rank. A rank without shots contributes zeros."""
    import torch

    shot0, count = shot_range(nshots, rank, world)
    if count > 0:
        J, gl, gm = ctx.adjoint_gradient(observed, shot0, count)
    else:
        dev = observed.device if hasattr(observed, "device") else "cuda"
        J = 0.0
        gl = torch.zeros(ctx.mat_shape(), dtype=torch.float64, device=dev)
        gm = torch.zeros_like(gl)
    return reduce_gradient(J, gl, gm, group)
