"""The seeded workloads against the configurations they stand for: mesh sizes, node
counts, media, shot and receiver layouts and time steps (CPU only)."""
import numpy as np
import pytest

import fwi_inputs as fi


def _velocities(w, which):
    lam, mu = fi.medium(w, which)
    vs = np.sqrt(mu / w.rho)
    vp = np.sqrt((lam + 2 * mu) / w.rho)
    return vs, vp


@pytest.mark.parametrize("make,mesh,steps,f0,nrec,nshots,nodes,mat_nodes", [
    (fi.box_8x8x4, (8, 8, 4, 3), 300, 15.0, 25, 1, 12_615, 2_601),
    (fi.grf_64x64x32, (64, 64, 32, 10), 2000, 10.0, 1024, 1, 2_427_685, 1_081_665),
    (fi.layered_96x96x48, (96, 96, 48, 10), 3000, 10.0, 2304, 16, 6_351_813, 3_613_153),
    (fi.grf_16x16x8, (16, 16, 8, 10), 2000, 10.0, 64, 1, 197_173, 18_513),
])
def test_workload_sizes(make, mesh, steps, f0, nrec, nshots, nodes, mat_nodes):
    w = make()
    assert (w.nx, w.ny, w.nz, w.npml) == mesh and w.h == 1.0 and w.rho == 2000.0
    assert w.nsteps == steps and w.f0 == f0 and w.nshots == nshots
    assert int(np.prod(w.nodes)) == nodes and int(np.prod(w.mat_shape)) == mat_nodes
    rec = w.receivers()
    assert len(rec) == nrec and len({tuple(r) for r in rec}) == nrec
    src = w.sources()
    assert len(src) == nshots and len({tuple(s) for s in src}) == nshots
    # surface points inside the interior (away from the PML and the fixed faces)
    for pts in (rec, src):
        assert np.all(pts[:, 2] == 0)
        assert np.all((pts[:, 0] >= 2 * w.npml) & (pts[:, 0] <= 2 * (w.npml + w.nx)))
        assert np.all((pts[:, 1] >= 2 * w.npml) & (pts[:, 1] <= 2 * (w.npml + w.ny)))
    # Courant number 0.5 on the h/2 node spacing at the fastest P velocity
    vp_max = max(_velocities(w, "true")[1].max(), 400.0)
    assert w.dt == pytest.approx(0.5 * 0.5 * w.h / vp_max, rel=1e-14)


def test_box_medium_has_the_ten_percent_bump():
    w = fi.box_8x8x4()
    vs0, vp0 = _velocities(w, "trial")
    assert np.all(vs0 == pytest.approx(200.0)) and np.all(vp0 == pytest.approx(400.0))
    lam, mu = fi.medium(w, "true")
    lam0, mu0 = fi.medium(w, "trial")
    r = mu / mu0 - 1
    assert np.allclose(lam / lam0 - 1, r, rtol=0, atol=1e-14)
    assert 0.09 < r.max() <= 0.10 and r.min() >= 0


def test_grf_medium_spans_twenty_percent():
    w = fi.grf_64x64x32()
    vs, vp = _velocities(w, "true")
    d = vs / 200.0 - 1
    assert np.abs(d).max() == pytest.approx(0.2, rel=1e-12)
    assert abs(d.mean()) < 1e-12
    assert np.allclose(vp / vs, 2.0, rtol=1e-12)
    # smooth: neighbouring nodes (0.5 m apart) differ far less than the field's range
    assert np.abs(np.diff(d, axis=2)).max() < 0.05
    vs0, _ = _velocities(w, "trial")
    assert np.allclose(vs0, 200.0, rtol=1e-12)


def test_layered_medium_layers_and_inclusion():
    w = fi.layered_96x96x48()
    vs, vp = _velocities(w, "true")
    assert set(np.unique(np.round(vs, 6))) == {150.0, 250.0, 400.0, 500.0}
    assert np.allclose(vp / vs, fi.vp_over_vs(0.3), rtol=1e-12)
    depth = (np.arange(2 * w.nz + 1) * 0.5 * w.h)[:, None, None] * np.ones(w.mat_shape)
    outside = vs != 500.0
    for lo, hi, v in ((0, 16, 150.0), (16, 32, 250.0), (32, 48.01, 400.0)):
        sel = outside & (depth >= lo) & (depth < hi)
        assert np.all(vs[sel] == pytest.approx(v))
    inc = np.argwhere(vs == 500.0)
    # a 16 m cube (33 nodes a side) centred at mid-plan, two thirds down
    assert len(inc) == 33 ** 3
    assert np.allclose(inc.mean(axis=0) * 0.5 * w.h, (32.0, 48.0, 48.0))
    vs0, _ = _velocities(w, "trial")
    assert np.allclose(vs0, 150.0)


def test_synthetic_traces_are_seeded():
    a = fi.synthetic_traces(20, 4, 7)
    assert a.shape == (21, 4, 3)
    assert np.array_equal(a, fi.synthetic_traces(20, 4, 7))
    assert not np.array_equal(a, fi.synthetic_traces(20, 4, 8))


def test_random_media_of_the_preconditioner_study():
    """GRF about Vs 200 / Vp 400 within the generator's bounds, seeded (same seed, same
    medium), and the time step at Courant 0.5 for the fastest medium the generator allows."""
    vmax = 0.0
    for seed in range(12):
        w = fi.media_16x16x8(seed)
        vs, vp = _velocities(w, "true")
        assert np.allclose(vp / vs, 2.0)
        assert vs.min() >= 200 * 0.8 * 0.7 - 1e-9 and vs.max() <= 200 * 1.2 * 1.3 + 1e-9
        vmax = max(vmax, vp.max())
        lam2, mu2 = fi.medium(fi.media_16x16x8(seed), "true")
        assert np.array_equal(lam2, fi.medium(w, "true")[0]) and np.array_equal(mu2, fi.medium(w, "true")[1])
        assert 0.5 * 0.5 * w.h / w.dt >= vmax
    vs0, vp0 = _velocities(fi.media_16x16x8(0), "trial")
    assert np.all(vs0 == 200.0) and np.all(vp0 == 400.0)


def test_large_workload_sizes_and_medium():
    """The large autograd workload: 160x160x80 interior + 12-element PML (3.11 M elements,
    25.2 M nodes), 64 shots on an 8x8 surface grid, 80x80 receivers, 4000 steps; a random
    field of +-20 % about Vs 200 / Vp 400 m/s with a fast (x1.4) and a slow (x0.7) sharp
    inclusion, and the Courant-0.5 step of its fastest P velocity."""
    w = fi.large_160x160x80()
    assert (w.nx, w.ny, w.nz, w.npml, w.nsteps, w.f0, w.nshots) == (160, 160, 80, 12, 4000, 10.0, 64)
    assert tuple(w.nodes) == (369, 369, 185) and int(np.prod(w.nodes)) == 25_189_785 and int(np.prod(w.mat_shape)) == 16_589_601
    assert int(np.prod(w.elements)) == 3_114_752
    src, rec = w.sources(), w.receivers()
    assert len({tuple(s) for s in src}) == 64 and len(np.unique(src[:, 0])) == 8 and len(np.unique(src[:, 1])) == 8
    assert len({tuple(r) for r in rec}) == 6400 and np.all(src[:, 2] == 0) and np.all(rec[:, 2] == 0)
    vs, vp = _velocities(w, "true")
    assert np.allclose(vp / vs, 2.0)
    # only the fast inclusion exceeds the field's +20 %, only the slow one falls below -20 %
    fast, slow = vs > 200 * 1.2 * (1 + 1e-9), vs < 200 * 0.8 * (1 - 1e-9)
    assert fast.mean() > 1e-3 and slow.mean() > 1e-3
    assert vs.max() <= 200 * 1.2 * 1.4 * (1 + 1e-9) and vs.min() >= 200 * 0.8 * 0.7 * (1 - 1e-9)
    Z, Y, X = (a.ravel() for a in np.meshgrid(*[np.arange(n) * 0.5 for n in w.mat_shape], indexing="ij"))
    assert Z[fast.ravel()].mean() < Z[slow.ravel()].mean()  # the fast one is the shallower
    assert w.dt == pytest.approx(0.5 * 0.5 * w.h / vp.max(), rel=1e-14)
    vs0, vp0 = _velocities(w, "trial")
    assert np.all(vs0 == 200.0) and np.allclose(vp0, 400.0)
