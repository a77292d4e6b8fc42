"""The interior stage kernel's plane copies: each plane of the stage input reaches the
kernel's shared-memory ring as one tensor copy (TMA) that completes on an mbarrier, and
every wait for one is bounded (fwi_set_copy_wait).

- The bounded wait: with every plane barrier expecting 16 bytes more than its copy
  delivers, no wait can complete. Each gives up after the 20 ms limit, and the sweep
  returns FWI_E_TIMEOUT instead of hanging. With the limit restored, the context gives
  the same traces as before, bit for bit. Recorded CUDA graphs are dropped by the call,
  so a replay cannot keep the old limits.
- Device buffers of fwi_rhs that do not start on a 16-byte boundary are refused on the
  host before any launch.
- The copies read zeros outside the grid: the traces on a mesh without PML, whose
  interior tile starts 4 nodes before the grid (a negative box coordinate), agree with a
  sweep that has no interior kernel at all (the persistent sweep, general formulas).
"""
import numpy as np
import pytest

import fwi_inputs as fi
from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(w, top=False):
    from paper_1504_08340_gb300 import Context

    ctx = Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho, top_pml=top)
    lam, mu = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "true"))
    ctx.set_material(lam, mu)
    p = w.npml
    kz = 2 * p if top else 0
    rec = np.array([(2 * p + 1 + i, 2 * p + 1 + j, kz) for j in range(0, 2 * w.ny - 1, 2)
                    for i in range(0, 2 * w.nx - 1, 2)])
    ctx.set_sources(rec[[0, len(rec) // 2]], np.tile([0.0, 0.0, 1.0], (2, 1)), "ricker", w.ricker())
    ctx.set_receivers(rec)
    return ctx


def test_plane_copy_wait_gives_up_with_timeout():
    from paper_1504_08340_gb300 import FWIError

    w = fi.tiny(nx=4, ny=3, nz=3, npml=2, nsteps=12, f0=30.0, nrec_side=3)
    with _ctx(w) as ctx:
        ctx.set_graphs(True)
        good = ctx.forward(0, 2)
        assert np.abs(good).max() > 0
        ctx.set_copy_wait(20.0, test_extra_bytes=16)
        with pytest.raises(FWIError) as err:
            ctx.forward(0, 2)
        assert err.value.name == "FWI_E_TIMEOUT"
        ctx.set_copy_wait(1000.0, test_extra_bytes=0)
        assert np.array_equal(ctx.forward(0, 2), good)
        ctx.set_graphs(False)
        assert np.array_equal(ctx.forward(0, 2), good)


def test_copy_wait_argument_checks():
    from paper_1504_08340_gb300 import FWIError

    w = fi.tiny(nx=2, ny=2, nz=2, npml=1, nsteps=4, f0=30.0, nrec_side=2)
    with _ctx(w) as ctx:
        for bad in [dict(wait_ms=0.0), dict(wait_ms=-1.0), dict(wait_ms=60001.0),
                    dict(wait_ms=10.0, test_extra_bytes=-1), dict(wait_ms=10.0, test_extra_bytes=65537)]:
            with pytest.raises(FWIError) as err:
                ctx.set_copy_wait(**bad)
            assert err.value.name == "FWI_E_INVAL"


def test_rhs_refuses_unaligned_device_buffers():
    from paper_1504_08340_gb300 import FWIError

    w = fi.tiny(nx=2, ny=2, nz=2, npml=1, nsteps=4, f0=30.0, nrec_side=2)
    dev = torch.device("cuda", 0)
    with _ctx(w) as ctx:
        n = ctx.state().size
        buf = torch.zeros(n + 4, dtype=torch.float32, device=dev)
        out = torch.zeros(n + 4, dtype=torch.float32, device=dev)
        for s, r in ((buf[1:n + 1], out[:n]), (buf[:n], out[2:n + 2])):
            with pytest.raises(FWIError) as err:
                ctx.rhs(s, out=r)
            assert err.value.name == "FWI_E_INVAL"
        ctx.rhs(buf[4:n + 4], out=out[:n])  # 16 bytes in: accepted


def test_boxes_read_zero_outside_the_grid():
    # no PML: the interior box starts at node 1, its first tile's copy at x = -4 (and at
    # y = -1, plane -1): the parts outside the grid must read as zero
    w = fi.tiny(nx=5, ny=3, nz=3, npml=0, nsteps=16, f0=30.0, nrec_side=3)
    with _ctx(w) as ctx:
        split = ctx.forward(0, 2)
        ctx.set_persistent(True)
        general = ctx.forward(0, 2)
    assert np.abs(split).max() > 0
    assert rel_l2(split, general) < 1e-5
