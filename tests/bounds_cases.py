"""Cases of test_gpu_bounds.py, run in a child process with the library that the
FWI_LIBRARY environment variable names (the normal or the bounds-checked build).

On meshes with a free top, a top PML, no PML and a one-element-thin interior: forward
traces of three shots in batches of two, the adjoint gradient from the stored history and
from checkpoints every 5 steps, the rates of the forward and of the adjoint system at the
final forward state, and a persistent forward sweep. Every call must return FWI_OK (the
checked build turns an out-of-range index into FWI_E_BOUNDS, which raises). The results go
to the .npz file named by the first argument."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import fwi_inputs as fi  # noqa: E402
from paper_1504_08340_gb300 import Context, fwi  # noqa: E402

MESHES = [  # nx, ny, nz, npml, top PML
    (4, 3, 2, 2, False),
    (4, 3, 2, 2, True),
    (3, 3, 2, 0, False),
    (1, 2, 1, 2, False),
]


def surface_points(nx, ny, p, kz):
    xs = sorted({2 * p + 1, 2 * p + nx, 2 * p + 2 * nx - 1})
    ys = sorted({2 * p + 1, 2 * p + ny, 2 * p + 2 * ny - 1})
    return np.array([(i, j, kz) for j in ys for i in xs])


def main(path):
    out = {"checked": np.array(int(fwi.bounds_checked()))}
    dev = torch.device("cuda", 0)
    for m, (nx, ny, nz, npml, top) in enumerate(MESHES):
        w = fi.tiny(nx=nx, ny=ny, nz=nz, npml=npml, nsteps=30, f0=30.0, nrec_side=3)
        kz = 2 * npml if top else 0  # the interior's top surface
        rec = surface_points(nx, ny, npml, kz)
        src = rec[[0, len(rec) // 2, -1]]
        dirs = np.tile([0.0, 0.0, 1.0], (3, 1))
        obs = torch.tensor(np.stack([fi.synthetic_traces(w.nsteps, len(rec), 70 + s, scale=1e-7) for s in range(3)]),
                           dtype=torch.float32, device=dev).contiguous()
        with Context(w.nx, w.ny, w.nz, w.npml, w.h, w.dt, w.nsteps, rho=w.rho, top_pml=top) as ctx:
            lt, mt = (np.ascontiguousarray(a, dtype=np.float32) for a in fi.medium(w, "true"))
            ctx.set_material(lt, mt)
            ctx.set_sources(src, dirs, "ricker", w.ricker())
            ctx.set_receivers(rec)
            ctx.set_shot_batch(2)
            out[f"m{m}_traces"] = ctx.forward(0, 3)
            state = ctx.state()
            out[f"m{m}_rate"] = ctx.rhs(state)
            out[f"m{m}_rate_adj"] = ctx.rhs(state, adjoint=True)
            for every in (0, 5):
                ctx.set_checkpointing(every)
                J, gl, gm = ctx.adjoint_gradient(obs, 0, 3)
                out[f"m{m}_J{every}"] = np.array(J)
                out[f"m{m}_gl{every}"] = gl.cpu().numpy()
                out[f"m{m}_gm{every}"] = gm.cpu().numpy()
            ctx.set_persistent(True, wait_ms=2000.0)
            out[f"m{m}_traces_persistent"] = ctx.forward(0, 3)
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
