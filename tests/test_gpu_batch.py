"""Shot batching: B shots advanced by one launch of each stage kernel.

Each shot is an independent wave problem on the same material (the misfit and the
gradient of Sec. 3 are sums over the shots), so batching must not change any
shot's arithmetic: traces are bitwise those of B = 1, J too (the per-shot misfits
are summed in shot order either way), and the gradients differ only by the order
of the FP64 sums over the shots. Groups that do not divide the shot count (a
ragged last group) and B larger than the shot count are covered."""
import numpy as np
import pytest

import fwi_inputs as fi
from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _workload(nsteps=50):
    return fi.build(fi.Workload("box_5x4x3", 5, 4, 3, 2, 1.0, nsteps, 30.0, 3, nshots=4, seed=5))


def _setup(w):
    from paper_1504_08340_gb300 import Context

    ctx = Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho)
    lt, mt = (_f32(a) for a in fi.medium(w, "true"))
    l0, m0 = (_f32(a) for a in fi.medium(w, "trial"))
    ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
    ctx.set_receivers(w.receivers())
    ctx.set_material(lt, mt)
    obs = torch.zeros(ctx.trace_shape(w.nshots), dtype=torch.float32, device="cuda")
    ctx.forward(0, w.nshots, out=obs)
    ctx.set_material(l0, m0)
    return ctx, obs, l0, m0


def test_batched_forward_and_misfit_are_bitwise():
    w = _workload()
    ctx, obs, _, _ = _setup(w)
    with ctx:
        ref = torch.zeros_like(obs)
        ctx.forward(0, w.nshots, out=ref)
        J1 = ctx.misfit(obs, 0, w.nshots)
        Jpart = ctx.misfit(obs[1:3], 1, 2)
        for B in (2, 3, 4, 7):
            ctx.set_shot_batch(B)
            tr = torch.full_like(obs, float("nan"))
            ctx.forward(0, w.nshots, out=tr)
            assert torch.equal(tr, ref), B
            assert ctx.misfit(obs, 0, w.nshots) == J1, B
            # a shot range that starts inside the shot list
            assert ctx.misfit(obs[1:3], 1, 2) == Jpart, B
            # host observed data go through the batch's device slots
            assert ctx.misfit(obs.cpu().numpy(), 0, w.nshots) == J1, B


@pytest.mark.parametrize("every", [0, -1, 9])
def test_batched_gradient_matches_single_shot_path(every):
    w = _workload(nsteps=61)
    ctx, obs, _, _ = _setup(w)
    with ctx:
        ctx.set_checkpointing(every)
        J1, gl1, gm1 = ctx.adjoint_gradient(obs, 0, w.nshots)
        for B in (3, 4):
            ctx.set_shot_batch(B)
            ctx.set_checkpointing(every)
            J, gl, gm = ctx.adjoint_gradient(obs, 0, w.nshots)
            assert J == J1, B
            assert rel_l2(gl.cpu().numpy(), gl1.cpu().numpy()) < 1e-12, B
            assert rel_l2(gm.cpu().numpy(), gm1.cpu().numpy()) < 1e-12, B
            ctx.set_shot_batch(1)


def test_batched_gradient_matches_oracle(oracle_mod):
    w = _workload(nsteps=40)
    ctx, obs, l0, m0 = _setup(w)
    with ctx:
        ctx.set_shot_batch(3)
        J, gl, gm = ctx.adjoint_gradient(obs, 0, w.nshots)
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
    src = [o.node_id(*s) for s in w.sources()]
    rec = [o.node_id(*r) for r in w.receivers()]
    o.set_material(l0.astype(np.float64), m0.astype(np.float64))
    ob = obs.cpu().numpy().astype(np.float64)
    dirs = w.source_dirs()
    Jo, glo, gmo = 0.0, 0.0, 0.0
    for s in range(w.nshots):  # the objective and its gradient are sums over the shots
        Js, gls, gms, _ = o.misfit_and_gradient(w.dt, w.nsteps, [src[s]], dirs[s:s + 1], rec, ob[s], "ricker",
                                                w.ricker())
        Jo, glo, gmo = Jo + Js, glo + gls, gmo + gms
    assert J == pytest.approx(Jo, rel=2e-5)
    assert rel_l2(gl.cpu().numpy().ravel(), glo.ravel()) < 1e-4
    assert rel_l2(gm.cpu().numpy().ravel(), gmo.ravel()) < 1e-4


def test_batched_step_matches_single_shot_step():
    w = _workload(nsteps=40)
    infos = []
    for B in (1, 4):
        ctx, obs, _, _ = _setup(w)
        with ctx:
            ctx.set_shot_batch(B)
            infos.append([ctx.step(obs, 0, w.nshots) for _ in range(2)])
            infos[-1].append(ctx.get_material())
    (a1, a2, (la, ma)), (b1, b2, (lb, mb)) = infos
    assert a1.J_old == b1.J_old  # same material, bitwise traces
    for x, y in ((a1, b1), (a2, b2)):
        assert x.accepted == y.accepted == 1
        assert x.J_old == pytest.approx(y.J_old, rel=1e-9)
        assert x.J_new == pytest.approx(y.J_new, rel=1e-9)
        assert x.alpha == y.alpha
    assert rel_l2(lb.ravel().astype(np.float64), la.ravel().astype(np.float64)) < 1e-6
    assert rel_l2(mb.ravel().astype(np.float64), ma.ravel().astype(np.float64)) < 1e-6


def test_shot_batch_rejects_bad_sizes():
    w = _workload(nsteps=10)
    ctx, _, _, _ = _setup(w)
    with ctx:
        for bad in (0, -1, 1025):
            with pytest.raises(Exception):
                ctx.set_shot_batch(bad)
        ctx.set_shot_batch(1024 // 256)


def test_layered_96x96x48_full_size_batched(oracle_mod):
    """The 16-shot layered 96x96x48 + 10 PML mesh (48x48 receivers) at full size, in the
    launch configuration of the shot-batch benchmark: B = 16 against B = 1 over all 16
    shots (traces bitwise, J equal, gradients to 1e-12), and one shot of the batch against
    the FP64 oracle over 4 steps (a Ricker centred at t = 0, so the first steps carry
    signal; seeded synthetic observed traces)."""
    from paper_1504_08340_gb300 import Context

    w = fi.layered_96x96x48()
    w.nsteps = 4
    wp = (w.f0, 0.0, w.amp)
    lam, mu = (_f32(a) for a in fi.medium(w, "true"))
    src, dirs, rec = w.sources(), w.source_dirs(), w.receivers()
    obs = _f32(np.stack([fi.synthetic_traces(w.nsteps, len(rec), 200 + s) for s in range(w.nshots)]))
    with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho) as ctx:
        ctx.set_material(lam, mu)
        ctx.set_sources(src, dirs, "ricker", wp)
        ctx.set_receivers(rec)
        obs_d = torch.tensor(obs, device="cuda")
        ctx.set_shot_batch(16)
        tr16 = ctx.forward(0, w.nshots)
        J16, gl16, gm16 = ctx.adjoint_gradient(obs_d, 0, w.nshots)
        gl16, gm16 = gl16.cpu().numpy(), gm16.cpu().numpy()
        ctx.set_shot_batch(1)
        tr1 = ctx.forward(0, w.nshots)
        J1, gl1, gm1 = ctx.adjoint_gradient(obs_d, 0, w.nshots)
        s = 5
        Js, gls, gms = ctx.adjoint_gradient(obs_d[s:s + 1], s, 1)
    assert np.array_equal(tr16, tr1) and J16 == J1
    assert rel_l2(gl16, gl1.cpu().numpy()) < 1e-12 and rel_l2(gm16, gm1.cpu().numpy()) < 1e-12
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
    o.set_material(lam.astype(np.float64), mu.astype(np.float64))
    sn = [o.node_id(*src[s])]
    rn = [o.node_id(*r) for r in rec]
    J_o, gl_o, gm_o, tr_o = o.misfit_and_gradient(w.dt, w.nsteps, sn, dirs[s:s + 1], rn,
                                                  obs[s].astype(np.float64), "ricker", wp)
    assert np.abs(tr_o).max() > 0
    assert rel_l2(tr16[s], tr_o) < 1e-5
    assert Js == pytest.approx(J_o, rel=2e-5)
    assert rel_l2(gls.cpu().numpy().ravel(), gl_o.ravel()) < 1e-4
    assert rel_l2(gms.cpu().numpy().ravel(), gm_o.ravel()) < 1e-4


def test_tune_shot_batch():
    """The tuner picks one of its candidates (1, 2, 4 for four shots), leaves the context
    at it with results unchanged, honours max_batch, and rejects bad arguments."""
    w = _workload(nsteps=30)
    ctx, obs, _, _ = _setup(w)
    with ctx:
        ref = ctx.forward(0, w.nshots)
        J1 = ctx.misfit(obs, 0, w.nshots)
        B = ctx.tune_shot_batch(0, w.nshots, max_batch=8, steps=5)
        assert B in (1, 2, 4)
        assert np.array_equal(ctx.forward(0, w.nshots), ref)
        assert ctx.misfit(obs, 0, w.nshots) == J1
        assert ctx.tune_shot_batch(1, 3, max_batch=1, steps=3) == 1
        good = dict(max_batch=4, steps=3, mem_fraction=0.8)
        for bad in (dict(steps=0), dict(steps=30), dict(max_batch=0), dict(mem_fraction=0.0),
                    dict(mem_fraction=1.5)):
            with pytest.raises(Exception):
                ctx.tune_shot_batch(0, w.nshots, **{**good, **bad})
        assert np.array_equal(ctx.forward(0, w.nshots), ref)


def test_sharded_gradient_matches_all_shots():
    """One rank's sharded evaluation is the whole-range call; two ranks' shares, summed
    in rank order, give the whole-range misfit and gradients up to the order of the FP64
    sums over the shots."""
    from paper_1504_08340_gb300.distributed import sharded_adjoint_gradient, shot_range

    w = _workload(nsteps=30)
    ctx, obs, _, _ = _setup(w)
    with ctx:
        J, gl, gm = ctx.adjoint_gradient(obs, 0, w.nshots)
        Js, gls, gms = sharded_adjoint_gradient(ctx, obs, w.nshots, 0, 1)
        assert Js == J and torch.equal(gls, gl) and torch.equal(gms, gm)
        parts = []
        for r in range(2):
            s0, n = shot_range(w.nshots, r, 2)
            parts.append(ctx.adjoint_gradient(obs[s0:s0 + n], s0, n))
    assert parts[0][0] + parts[1][0] == pytest.approx(J, rel=1e-12)
    assert rel_l2((parts[0][1] + parts[1][1]).cpu().numpy(), gl.cpu().numpy()) < 1e-12
    assert rel_l2((parts[0][2] + parts[1][2]).cpu().numpy(), gm.cpu().numpy()) < 1e-12


def test_tile_tuner_keeps_results_bitwise():
    """fwi_tune_tiles picks the interior kernel's planes per block and the PML warp task's
    segment width by timing; the choice changes no node's arithmetic, so traces and
    gradients are bitwise those of the default shapes."""
    from paper_1504_08340_gb300 import Context

    for w in (fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=40, f0=30.0, nrec_side=3), fi.box_8x8x4()):
        w.nsteps = 40
        l0, m0 = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "trial"))
        with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho) as ctx:
            ctx.set_material(l0, m0)
            ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
            ctx.set_receivers(w.receivers())
            obs = np.ascontiguousarray(fi.synthetic_traces(w.nsteps, ctx.nrec, 9)[None], dtype=np.float32)
            tr0 = ctx.forward()
            J0, gl0, gm0 = ctx.adjoint_gradient(obs)
            kc, seg = ctx.tune_tiles(steps=5)
            assert kc in (4, 8, 16, 32) and seg in (16, 32)
            assert np.array_equal(ctx.forward(), tr0)
            J1, gl1, gm1 = ctx.adjoint_gradient(obs)
            assert J1 == J0 and np.array_equal(gl1, gl0) and np.array_equal(gm1, gm0)
