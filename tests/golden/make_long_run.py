"""Writes tests/golden/long_run_grf_16x16x8.npz: the FP64 oracle's 2000-step single-shot
gradient evaluation on the grf_16x16x8 workload (the single-shot recipe -- Gaussian
random field medium, 10-element PML, Ricker f0 = 10 Hz, the same time step and step
count -- on a 16x16x8 interior box), used by the long-run GPU parity test.

Calls only oracle/ and the seeded input generator:
  observed = oracle forward on the true medium (stored FP32: that is what the GPU is given,
             and the oracle's misfit and gradient below use these same FP32 values),
  traces   = oracle forward on the trial medium,
  J, g_lambda, g_mu = oracle misfit (7) and adjoint gradient (C.1f)/(C.1g) at the trial
             medium against the stored observed traces.
Run from the repository root: python tests/golden/make_long_run.py  (about an hour on 8 cores).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import fwi_inputs as fi  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "long_run_grf_16x16x8.npz")


def main():
    w = fi.grf_16x16x8()
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    lt, mt = (f32(a) for a in fi.medium(w, "true"))
    l0, m0 = (f32(a) for a in fi.medium(w, "trial"))
    o = oracle.Oracle(w.nx, w.ny, w.nz, w.npml, h=w.h, rho=w.rho)
    src, dirs, rec = w.sources(), w.source_dirs(), w.receivers()
    sn = [o.node_id(*s) for s in src]
    rn = [o.node_id(*r) for r in rec]
    t = time.time()
    o.set_material(lt, mt)
    obs = o.forward(w.dt, w.nsteps, sn, dirs, "ricker", w.ricker(), rn).astype(np.float32)
    print(f"observed: {time.time() - t:.0f} s", flush=True)
    o.set_material(l0, m0)
    J, gl, gm, traces = o.misfit_and_gradient(w.dt, w.nsteps, sn, dirs, rn, obs.astype(np.float64), "ricker",
                                              w.ricker())
    print(f"gradient: {time.time() - t:.0f} s, J = {J:.6e}", flush=True)
    np.savez_compressed(OUT, observed=obs, traces=traces.astype(np.float32), J=np.float64(J),
                        g_lambda=gl.astype(np.float32), g_mu=gm.astype(np.float32),
                        nsteps=np.int64(w.nsteps), dt=np.float64(w.dt))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
