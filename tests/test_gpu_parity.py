"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: receiver traces relative L2 <= 1e-5 and gradients <= 1e-4 (FP32
wavefields against FP64, J and gradient integrals accumulated in FP64); a
single evaluation of the right side of (6) / (15) is compared field group by
field group at <= 2e-5.
"""
import numpy as np
import pytest

import fwi_inputs as fi
from helpers import node_classes, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(w, top_pml=False, dt=None, nsteps=None, alpha0=5.0, beta0=400.0):
    from paper_1504_08340_gb300 import Context

    return Context(w.nx, w.ny, w.nz, w.npml, w.h, dt or w.dt, nsteps or w.nsteps, rho=w.rho,
                   alpha0=alpha0, beta0=beta0, top_pml=top_pml)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _as_f64_of_f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def to_gpu_layout(Y, ctx):
    """oracle [3][nnode][9] -> library [27][stride] (field 9*l + c, pitched rows)"""
    out = np.zeros((27, ctx.stride), dtype=np.float32)
    idx = ctx.state_index()
    for l in range(3):
        for c in range(9):
            out[9 * l + c, idx] = Y[l, :, c]
    return out


def from_gpu_layout(G, ctx):
    idx = ctx.state_index()
    Y = np.zeros((3, idx.size, 9))
    for l in range(3):
        for c in range(9):
            Y[l, :, c] = G[9 * l + c, idx]
    return Y


def _oracle_for(oracle_mod, w, lam, mu, top_pml=False, alpha0=5.0, beta0=400.0, threads=None):
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho, top_pml=top_pml, alpha0=alpha0,
                          beta0=beta0, threads=threads)
    o.set_material(_as_f64_of_f32(lam), _as_f64_of_f32(mu))
    return o


def _random_medium(w, seed):
    rng = np.random.default_rng(seed)
    shape = w.mat_shape
    lam = 1.6e8 * (1 + 0.2 * rng.random(shape))
    mu = 0.8e8 * (1 + 0.2 * rng.random(shape))
    return _f32(lam), _f32(mu)


MESHES = [
    dict(nx=3, ny=3, nz=2, npml=2, top=False),
    dict(nx=2, ny=3, nz=2, npml=1, top=True),
    dict(nx=2, ny=2, nz=3, npml=0, top=False),
    dict(nx=4, ny=2, nz=1, npml=3, top=False),
]


@pytest.mark.parametrize("mesh", MESHES, ids=lambda m: f"{m['nx']}x{m['ny']}x{m['nz']}+{m['npml']}{'t' if m['top'] else ''}")
@pytest.mark.parametrize("adjoint", [False, True], ids=["forward", "adjoint"])
def test_rhs_parity(oracle_mod, mesh, adjoint):
    """One evaluation of the rate of the first-order system on a random state."""
    w = fi.tiny(nx=mesh["nx"], ny=mesh["ny"], nz=mesh["nz"], npml=mesh["npml"])
    lam, mu = _random_medium(w, 4)
    o = _oracle_for(oracle_mod, w, lam, mu, top_pml=mesh["top"])
    pml, dirn = o.masks()
    Y = fi.random_state(o.nnode, pml, dirn, seed=11, scale=1.0)
    Y[:, :, 3:] *= 1e8  # stress-like scale of S
    Y = _as_f64_of_f32(Y)
    with _ctx(w, top_pml=mesh["top"]) as ctx:
        assert ctx.nnode == o.nnode and ctx.nmat == o.nmat
        ctx.set_material(lam, mu)
        if not adjoint:
            Z = Y
        else:
            D = np.ones(9)
            D[3:] = -1
            Z = np.stack([-Y[0] * D, Y[1] * D, -Y[2] * D])
        out = from_gpu_layout(ctx.rhs(to_gpu_layout(Z, ctx), adjoint=adjoint), ctx)
    ref = o.rhs(Y, adjoint=adjoint)
    if adjoint:
        D = np.ones(9)
        D[3:] = -1
        ref = np.stack([ref[0] * D, -ref[1] * D, ref[2] * D])
    _check_by_class(o, out, ref)


def _tau(S, lam, mu):
    """tau(S) = mu (S + diag S) + lam tr(S) I of symmetric tensors S[..., 6] (xx yy zz yz
    xz xy, off-diagonals as stored), with per-node lam, mu."""
    tr = S[..., 0] + S[..., 1] + S[..., 2]
    out = np.empty_like(S)
    for c in range(3):
        out[..., c] = 2.0 * mu * S[..., c] + lam * tr
    for c in range(3, 6):
        out[..., c] = mu * S[..., c]
    return out


def _node_material(o, w, lam, mu, top):
    """lambda, mu at every oracle node (natural order), the PML's taken from the nearest
    interface node of the material grid (index clamp)."""
    n = np.arange(o.nnode)
    i, j, k = n % o.nn[0], (n // o.nn[0]) % o.nn[1], n // (o.nn[0] * o.nn[1])
    lo = (w.npml, w.npml, w.npml if top else 0)
    m = lam.shape  # (k, j, i)
    kk = np.clip(k - 2 * lo[2], 0, m[0] - 1)
    jj = np.clip(j - 2 * lo[1], 0, m[1] - 1)
    ii = np.clip(i - 2 * lo[0], 0, m[2] - 1)
    return lam.astype(np.float64)[kk, jj, ii], mu.astype(np.float64)[kk, jj, ii]


@pytest.mark.parametrize("mesh", MESHES, ids=lambda m: f"{m['nx']}x{m['ny']}x{m['nz']}+{m['npml']}{'t' if m['top'] else ''}")
def test_adjoint_sweep_runs_the_forward_form_on_tau_of_T(oracle_mod, mesh):
    """The adjoint sweep advances (w, W = tau(T)) with the forward stage kernels: tau is
    linear and node-local, so applying it to the transposed system's stress rows gives the
    forward system's form (tau moves from the u rows' line points to the S rows). On a
    random state (w, T): the forward-form rate of (w, tau(T)) has the transposed rate's u
    rows and tau of its S rows, node by node."""
    w = fi.tiny(nx=mesh["nx"], ny=mesh["ny"], nz=mesh["nz"], npml=mesh["npml"])
    lam, mu = _random_medium(w, 6)
    o = _oracle_for(oracle_mod, w, lam, mu, top_pml=mesh["top"])
    pml, dirn = o.masks()
    Y = fi.random_state(o.nnode, pml, dirn, seed=17, scale=1.0)
    Y[:, :, 3:] *= 1e8
    Y = _as_f64_of_f32(Y)
    ln, mn = _node_material(o, w, lam, mu, mesh["top"])
    YW = Y.copy()
    for l in range(3):
        YW[l, :, 3:] = _tau(Y[l, :, 3:], ln, mn)
    with _ctx(w, top_pml=mesh["top"]) as ctx:
        ctx.set_material(lam, mu)
        r_adj = from_gpu_layout(ctx.rhs(to_gpu_layout(Y, ctx), adjoint=True), ctx)
        r_fwd = from_gpu_layout(ctx.rhs(to_gpu_layout(_as_f64_of_f32(YW), ctx), adjoint=False), ctx)
    ref = r_adj.copy()
    for l in range(3):
        ref[l, :, 3:] = _tau(r_adj[l, :, 3:], ln, mn)
    _check_by_class(o, r_fwd, ref)


def _check_by_class(o, out, ref, tol=2e-5):
    """Relative L2 per level, field group (u, S) and node set (interior, shell, outer-face
    PML, deep PML), so that an error confined to a small node set is not diluted by the
    others; an all-zero reference block must come out exactly zero."""
    for cls, mask in node_classes(o).items():
        if not mask.any():
            continue
        for l in range(3):
            for sl, name in ((slice(0, 3), "u"), (slice(3, 9), "S")):
                r = ref[l][mask][:, sl]
                g = out[l][mask][:, sl]
                if np.abs(r).max() == 0:
                    assert np.abs(g).max() == 0, (cls, l, name)
                    continue
                assert rel_l2(g, r) < tol, (cls, l, name, rel_l2(g, r))


def test_dims_and_pml_node_count(oracle_mod):
    w = fi.box_8x8x4()
    o = oracle_mod.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, threads=1)
    pml, _ = o.masks()
    with _ctx(w) as ctx:
        assert ctx.nn == o.nn
        assert ctx.nnode == o.nnode and ctx.nmat == o.nmat
        assert ctx.npml_nodes == int(pml.sum())
        assert ctx.nelem == o.N[0] * o.N[1] * o.N[2]
        mt = ctx.mass_tilde().ravel()
    assert np.allclose(mt, o.diag("Mtilde"), rtol=1e-14, atol=0)


def _problem(oracle_mod, w, wparams=None, threads=None):
    lt, mt = (_f32(a) for a in fi.medium(w, "true"))
    l0, m0 = (_f32(a) for a in fi.medium(w, "trial"))
    src, dirs, rec = w.sources(), w.source_dirs(), w.receivers()
    wp = wparams or w.ricker()
    o = _oracle_for(oracle_mod, w, lt, mt, threads=threads)
    sn = [o.node_id(*s) for s in src]
    rn = [o.node_id(*r) for r in rec]
    obs = o.forward(w.dt, w.nsteps, sn, dirs, "ricker", wp, rn)
    o.set_material(_as_f64_of_f32(l0), _as_f64_of_f32(m0))
    return o, (l0, m0), (src, dirs, rec, sn, rn), obs, wp


def _gpu_setup(w, l0, m0, src, dirs, rec, wp):
    ctx = _ctx(w)
    dev = torch.device("cuda:0")
    ctx.set_material(torch.tensor(l0, device=dev), torch.tensor(m0, device=dev))
    ctx.set_sources(src, dirs, "ricker", wp)
    ctx.set_receivers(rec)
    return ctx


def test_forward_traces_parity(oracle_mod):
    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=100, f0=30.0, nrec_side=3)
    o, (l0, m0), (src, dirs, rec, sn, rn), obs, wp = _problem(oracle_mod, w)
    ref = o.forward(w.dt, w.nsteps, sn, dirs, "ricker", wp, rn)
    with _gpu_setup(w, l0, m0, src, dirs, rec, wp) as ctx:
        tr = ctx.forward()[0]
        tr_dev = torch.zeros(ctx.trace_shape(1), dtype=torch.float32, device="cuda:0")
        ctx.forward(out=tr_dev)
    assert np.abs(ref).max() > 0
    assert rel_l2(tr, ref) < 1e-5
    assert np.array_equal(tr, tr_dev.cpu().numpy()[0])


def _check_gradient(oracle_mod, w, threads=None, wparams=None, tol_g=1e-4):
    o, (l0, m0), (src, dirs, rec, sn, rn), obs, wp = _problem(oracle_mod, w, wparams, threads)
    J_o, gl_o, gm_o, tr_o = o.misfit_and_gradient(w.dt, w.nsteps, sn, dirs, rn, obs, "ricker", wp)
    with _gpu_setup(w, l0, m0, src, dirs, rec, wp) as ctx:
        obs_h = _f32(obs[None])
        J, gl, gm = ctx.adjoint_gradient(obs_h)
        Jm = ctx.misfit(obs_h)
        tr = ctx.forward()[0]
        obs_d = torch.tensor(obs_h, device="cuda:0")
        J2, gl2, gm2 = ctx.adjoint_gradient(obs_d)
    assert rel_l2(tr, tr_o) < 1e-5
    assert abs(J - J_o) <= 2e-5 * J_o and abs(Jm - J) <= 1e-12 * J
    assert rel_l2(gl, gl_o) < tol_g, rel_l2(gl, gl_o)
    assert rel_l2(gm, gm_o) < tol_g, rel_l2(gm, gm_o)
    # device and host paths run the same kernels: bitwise identical
    assert J2 == J
    assert np.array_equal(gl2.cpu().numpy(), gl) and np.array_equal(gm2.cpu().numpy(), gm)


def test_gradient_parity_small(oracle_mod):
    _check_gradient(oracle_mod, fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=80, f0=30.0, nrec_side=3))


def test_gradient_parity_box_8x8x4(oracle_mod):
    """The 8x8x4 + 3 PML box with a Gaussian bump, 300 steps, 5x5 receivers."""
    _check_gradient(oracle_mod, fi.box_8x8x4())


def test_repeatable_bitwise(oracle_mod):
    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=40, f0=30.0, nrec_side=3)
    o, (l0, m0), (src, dirs, rec, sn, rn), obs, wp = _problem(oracle_mod, w)
    with _gpu_setup(w, l0, m0, src, dirs, rec, wp) as ctx:
        a = ctx.adjoint_gradient(_f32(obs[None]))
        b = ctx.adjoint_gradient(_f32(obs[None]))
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_grf_64x64x32_full_size_sampled(oracle_mod):
    """Full-size single-shot mesh (64x64x32 + 10 PML, 32x32 receivers) in the benchmark's
    launch configuration: the operator on a random state, and a short gradient run
    (a Ricker centred at t = 0 so that the first steps carry signal)."""
    w = fi.grf_64x64x32()
    lam, mu = (_f32(a) for a in fi.medium(w, "true"))
    o = _oracle_for(oracle_mod, w, lam, mu)
    pml, dirn = o.masks()
    Y = _as_f64_of_f32(fi.random_state(o.nnode, pml, dirn, seed=3, scale=1.0) * np.r_[np.ones(3), 1e8 * np.ones(6)])
    ref = o.rhs(Y)
    with _ctx(w) as ctx:
        ctx.set_material(lam, mu)
        out = from_gpu_layout(ctx.rhs(to_gpu_layout(Y, ctx)), ctx)
    _check_by_class(o, out, ref)
    del o
    w.nsteps = 4
    _check_gradient(oracle_mod, w, wparams=(w.f0, 0.0, 1e3))


def test_error_paths():
    from paper_1504_08340_gb300 import Context, FWIError

    w = fi.tiny()
    with pytest.raises(FWIError) as e:
        Context(0, 1, 1, 1, 1.0, 1e-4, 10)
    assert e.value.name == "FWI_E_INVAL"
    with _ctx(w) as ctx:
        with pytest.raises(FWIError) as e:
            ctx.forward()
        assert e.value.name == "FWI_E_STATE"
        lam, mu = (_f32(a) for a in fi.medium(w, "trial"))
        bad = lam.copy()
        bad.flat[3] = np.nan
        with pytest.raises(FWIError) as e:
            ctx.set_material(bad, mu)
        assert e.value.name == "FWI_E_NONFINITE"
        with pytest.raises(FWIError) as e:
            ctx.set_material(lam * 100, mu * 100)
        assert e.value.name == "FWI_E_UNSTABLE"
        ctx.set_material(lam, mu)
        with pytest.raises(FWIError) as e:
            ctx.set_sources([[0, 1, 1]], [[0, 0, 1]])  # on the fixed x = 0 face
        assert e.value.name == "FWI_E_INVAL"
        with pytest.raises(FWIError) as e:
            ctx.set_receivers([[5, 5, 0], [5, 5, 0]])
        assert e.value.name == "FWI_E_INVAL"
        ctx.set_sources(w.sources(), w.source_dirs(), "ricker", w.ricker())
        ctx.set_receivers(w.receivers())
        with pytest.raises(FWIError) as e:
            ctx.forward(shot0=1)
        assert e.value.name == "FWI_E_INVAL"
        # the context stays usable after these errors
        obs = np.zeros(ctx.trace_shape(1), dtype=np.float32)
        J = ctx.misfit(obs)
        assert np.isfinite(J) and J > 0


def test_multi_shot_forward_and_gradient_sum(oracle_mod):
    """Two shots in one call: traces are per shot, J and the gradients sum over shots."""
    w = fi.tiny(nx=3, ny=3, nz=2, npml=2, nsteps=40, f0=30.0, nrec_side=3)
    l0, m0 = (_f32(a) for a in fi.medium(w, "trial"))
    src = np.array([[6, 6, 0], [8, 7, 0]], dtype=np.int64)
    dirs = np.array([[0.0, 0.0, 1.0], [0.3, -0.2, 0.9]])
    rec = w.receivers()
    obs = fi.synthetic_traces(w.nsteps, len(rec), 7, 1e-9)
    with _gpu_setup(w, l0, m0, src, dirs, rec, w.ricker()) as ctx:
        both = ctx.forward(0, 2)
        one = ctx.forward(1, 1)
        assert np.array_equal(both[1], one[0])
        obs2 = _f32(np.stack([obs, 0.5 * obs]))
        J, gl, gm = ctx.adjoint_gradient(obs2, 0, 2)
        J0, gl0, gm0 = ctx.adjoint_gradient(_f32(obs2[:1]), 0, 1)
        J1, gl1, gm1 = ctx.adjoint_gradient(_f32(obs2[1:]), 1, 1)
    assert J == pytest.approx(J0 + J1, rel=1e-12)
    assert np.allclose(gl, gl0 + gl1, rtol=1e-12, atol=1e-12 * np.abs(gl).max())
    assert np.allclose(gm, gm0 + gm1, rtol=1e-12, atol=1e-12 * np.abs(gm).max())
