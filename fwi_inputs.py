"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle legs.

This module holds no arithmetic of the method itself: it only draws material
fields, source / receiver positions and time-step sizes for the workloads
(shapes and value ranges of the media of Sec. 4 of arXiv:1504.08340; the
paper generates all of its data synthetically, so no dataset is replaced).

Conventions: nodes are indexed (i, j, k) with i along x, j along y and k along
depth (k = 0 is the ground surface); the material grid covers the interior
nodes only, shape (2 nz + 1, 2 ny + 1, 2 nx + 1), in Pa.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

RHO = 2000.0  # kg/m^3, as in every experiment of Sec. 4


def lame_from_velocities(vs, vp, rho=RHO):
    """Eq. (29) solved for the Lame parameters: mu = rho vs^2, lambda = rho vp^2 - 2 mu."""
    mu = rho * np.asarray(vs, dtype=np.float64) ** 2
    lam = rho * np.asarray(vp, dtype=np.float64) ** 2 - 2.0 * mu
    return lam, mu


def vp_over_vs(nu):
    return math.sqrt(2.0 * (1.0 - nu) / (1.0 - 2.0 * nu))


def cfl_dt(h, vp_max, cfl=0.5):
    """Time step for a Courant number `cfl` on the LGL node spacing h/2."""
    return cfl * (0.5 * h) / vp_max


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    npml: int
    h: float
    nsteps: int
    f0: float  # Ricker peak frequency, Hz
    nrec_side: int
    nshots: int = 1
    seed: int = 0
    rho: float = RHO
    cfl: float = 0.5
    dt: float = 0.0  # filled by build()
    amp: float = 1.0e3  # N, point-load amplitude

    @property
    def mat_shape(self):
        return (2 * self.nz + 1, 2 * self.ny + 1, 2 * self.nx + 1)

    @property
    def nodes(self):
        return (2 * (self.nx + 2 * self.npml) + 1, 2 * (self.ny + 2 * self.npml) + 1,
                2 * (self.nz + self.npml) + 1)

    @property
    def elements(self):
        return (self.nx + 2 * self.npml) * (self.ny + 2 * self.npml) * (self.nz + self.npml)

    def ricker(self):
        """(f0, t0, amplitude) with t0 = 1.5 / f0, so the wavelet starts below 1e-7 of its peak."""
        return (self.f0, 1.5 / self.f0, self.amp)

    def receivers(self):
        """nrec_side x nrec_side surface receivers on evenly spaced node indices of the interior."""
        p = self.npml
        n = self.nrec_side
        xs = np.rint(np.linspace(2, 2 * self.nx - 2, n)).astype(np.int64) + 2 * p
        ys = np.rint(np.linspace(2, 2 * self.ny - 2, n)).astype(np.int64) + 2 * p
        out = [(int(i), int(j), 0) for j in ys for i in xs]
        return np.array(out, dtype=np.int64)

    def sources(self):
        """Vertical surface point loads: the centre node for one shot, else a square
        grid of shots over the interior surface."""
        p = self.npml
        if self.nshots == 1:
            return np.array([(2 * p + self.nx, 2 * p + self.ny, 0)], dtype=np.int64)
        s = int(round(math.sqrt(self.nshots)))
        assert s * s == self.nshots
        xs = np.rint(np.linspace(0, 2 * self.nx, s + 2)[1:-1]).astype(np.int64) + 2 * p
        ys = np.rint(np.linspace(0, 2 * self.ny, s + 2)[1:-1]).astype(np.int64) + 2 * p
        return np.array([(int(i), int(j), 0) for j in ys for i in xs], dtype=np.int64)

    def source_dirs(self):
        d = np.zeros((self.nshots, 3))
        d[:, 2] = 1.0
        return d


def _grid(w: Workload):
    """Physical coordinates (z, y, x) of the interior material nodes, origin at the
    top-left interior corner, depth positive downwards."""
    z = np.arange(2 * w.nz + 1) * 0.5 * w.h
    y = np.arange(2 * w.ny + 1) * 0.5 * w.h
    x = np.arange(2 * w.nx + 1) * 0.5 * w.h
    return np.meshgrid(z, y, x, indexing="ij")


def gaussian_random_field(shape, corr_len_nodes, seed, amplitude):
    """Zero-mean field with Gaussian covariance: white noise filtered in Fourier
    space, scaled so that max |field| = amplitude."""
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal(shape)
    k = np.meshgrid(*[np.fft.fftfreq(n) for n in shape], indexing="ij")
    k2 = sum(ki ** 2 for ki in k)
    filt = np.exp(-0.5 * (2 * np.pi) ** 2 * k2 * (corr_len_nodes / math.sqrt(2)) ** 2)
    f = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    f -= f.mean()
    return f * (amplitude / np.max(np.abs(f)))


def medium(w: Workload, which: str = "true"):
    """(lambda, mu) on the interior material grid for workload w.

    which = "true" gives the target medium, "trial" the starting model at which
    the gradient is evaluated (homogeneous background / top layer)."""
    shape = w.mat_shape
    if w.name.startswith("box"):
        vs = np.full(shape, 200.0)
        vp = np.full(shape, 400.0)
        lam, mu = lame_from_velocities(vs, vp, w.rho)
        if which == "true":
            rng = np.random.Generator(np.random.PCG64(w.seed))
            Z, Y, X = _grid(w)
            cz = 0.5 * w.nz * w.h
            cx = 0.5 * w.nx * w.h + rng.uniform(-0.5, 0.5) * w.h
            cy = 0.5 * w.ny * w.h + rng.uniform(-0.5, 0.5) * w.h
            bump = 0.10 * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) / (2 * 1.5 ** 2))
            lam, mu = lam * (1 + bump), mu * (1 + bump)
        return lam, mu
    if w.name.startswith("grf"):
        if which == "true":
            d = gaussian_random_field(shape, 8.0 / (0.5 * w.h), w.seed, 0.2)
        else:
            d = np.zeros(shape)
        return lame_from_velocities(200.0 * (1 + d), 400.0 * (1 + d), w.rho)
    if w.name.startswith("media"):
        if which == "true":
            return random_medium(w, w.seed)
        return lame_from_velocities(np.full(shape, 200.0), np.full(shape, 400.0), w.rho)
    if w.name.startswith("large"):
        if which == "true":
            return large_medium(w)
        return lame_from_velocities(np.full(shape, 200.0), np.full(shape, 400.0), w.rho)
    if w.name.startswith("layered"):
        r = vp_over_vs(0.3)
        Z, Y, X = _grid(w)
        depth = w.nz * w.h
        vs = np.where(Z < depth / 3, 150.0, np.where(Z < 2 * depth / 3, 250.0, 400.0))
        if which == "true":
            c = (0.5 * w.nx * w.h, 0.5 * w.ny * w.h, 2.0 * depth / 3)
            inside = (np.abs(X - c[0]) <= 8) & (np.abs(Y - c[1]) <= 8) & (np.abs(Z - c[2]) <= 8)
            vs = np.where(inside, 500.0, vs)
        else:
            vs = np.full(shape, 150.0)
        return lame_from_velocities(vs, r * vs, w.rho)
    raise ValueError(w.name)


def random_medium(w: Workload, seed: int):
    """(lambda, mu) of a seeded random medium of the learned-preconditioner study: a Gaussian
    random field (correlation length 8 m, max |delta| = 0.2 on Vs 200 and Vp 400 m/s) plus
    0-3 sharp ellipsoidal inclusions, each scaling the background Vs and Vp by 1 + c with c in
    [-0.3, 0.3] (a later inclusion overrides an earlier one where they overlap) and semi-axes of
    1.5-4 m, centred inside the interior."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = w.mat_shape
    d = gaussian_random_field(shape, 8.0 / (0.5 * w.h), int(rng.integers(1 << 30)), 0.2)
    vs0 = 200.0 * (1 + d)
    vp0 = 400.0 * (1 + d)
    vs, vp = vs0.copy(), vp0.copy()
    Z, Y, X = _grid(w)
    for _ in range(int(rng.integers(0, 4))):
        c = (rng.uniform(0.2, 0.8) * w.nx * w.h, rng.uniform(0.2, 0.8) * w.ny * w.h, rng.uniform(0.2, 0.8) * w.nz * w.h)
        r = rng.uniform(1.5, 4.0, 3)
        inside = ((X - c[0]) / r[0]) ** 2 + ((Y - c[1]) / r[1]) ** 2 + ((Z - c[2]) / r[2]) ** 2 <= 1.0
        f = 1.0 + rng.uniform(-0.3, 0.3)
        vs = np.where(inside, vs0 * f, vs)  # scales the background: overlaps do not compound
        vp = np.where(inside, vp0 * f, vp)
    return lame_from_velocities(vs, vp, w.rho)


def large_medium(w: Workload):
    """(lambda, mu) of the large inversion workload: a Gaussian random field (correlation
    length 8 m, max |delta| = 0.2 on Vs 200 and Vp 400 m/s) with two sharp ellipsoidal
    inclusions, a fast one (Vs and Vp of the background x 1.4) in the upper half and a
    slow one (x 0.7) deeper, their centres jittered by the workload's seed."""
    rng = np.random.Generator(np.random.PCG64(w.seed))
    d = gaussian_random_field(w.mat_shape, 8.0 / (0.5 * w.h), int(rng.integers(1 << 30)), 0.2)
    vs0, vp0 = 200.0 * (1 + d), 400.0 * (1 + d)
    vs, vp = vs0.copy(), vp0.copy()
    Z, Y, X = _grid(w)
    Lx, Ly, Lz = w.nx * w.h, w.ny * w.h, w.nz * w.h
    for (fx, fy, fz), radii, f in (((0.35, 0.40, 0.35), (14.0, 10.0, 8.0), 1.4),
                                   ((0.65, 0.60, 0.65), (12.0, 16.0, 9.0), 0.7)):
        c = ((fx + rng.uniform(-0.05, 0.05)) * Lx, (fy + rng.uniform(-0.05, 0.05)) * Ly,
             (fz + rng.uniform(-0.05, 0.05)) * Lz)
        inside = (((X - c[0]) / radii[0]) ** 2 + ((Y - c[1]) / radii[1]) ** 2 +
                  ((Z - c[2]) / radii[2]) ** 2) <= 1.0
        vs = np.where(inside, vs0 * f, vs)
        vp = np.where(inside, vp0 * f, vp)
    return lame_from_velocities(vs, vp, w.rho)


def vp_max(w: Workload):
    lam, mu = medium(w, "true")
    return float(np.sqrt((lam + 2 * mu) / w.rho).max())


def build(w: Workload) -> Workload:
    w.dt = cfl_dt(w.h, max(vp_max(w), 400.0), w.cfl)
    return w


# The workloads of the benchmark table (element counts: interior + PML).
def box_8x8x4():  # tiny FP64 gradient box: 8x8x4 + 3 PML, 300 steps, 5x5 receivers
    return build(Workload("box_8x8x4", 8, 8, 4, 3, 1.0, 300, 15.0, 5, seed=1))


def grf_64x64x32():  # single shot, smooth Gaussian random field, 2000 steps, 32x32 receivers
    return build(Workload("grf_64x64x32", 64, 64, 32, 10, 1.0, 2000, 10.0, 32, seed=2))


def grf_16x16x8():  # the single-shot recipe (GRF, 10-element PML, f0, dt, 2000 steps) on a 16x16x8 box
    return build(Workload("grf_16x16x8", 16, 16, 8, 10, 1.0, 2000, 10.0, 8, seed=2))


def media_16x16x8(seed=0):
    """A seeded random medium of the learned-preconditioner study: 16x16x8 + 10 PML, one
    surface shot (Ricker 20 Hz), 600 steps, 8x8 receivers; the time step covers every medium
    the generator can draw (Vp at most 400 x 1.2 x 1.3 m/s)."""
    w = Workload("media_16x16x8", 16, 16, 8, 10, 1.0, 600, 20.0, 8, seed=seed)
    w.dt = cfl_dt(w.h, 400.0 * 1.2 * 1.3, w.cfl)
    return w


def layered_96x96x48():  # 3 layers + sharp inclusion, 16 shots, 3000 steps, 48x48 receivers
    return build(Workload("layered_96x96x48", 96, 96, 48, 10, 1.0, 3000, 10.0, 48, nshots=16, seed=3))


def large_160x160x80():  # GRF + 2 sharp inclusions, 64 shots, 4000 steps, 80x80 receivers
    return build(Workload("large_160x160x80", 160, 160, 80, 12, 1.0, 4000, 10.0, 80, nshots=64, seed=4))


def tiny(nx=3, ny=3, nz=2, npml=2, nsteps=60, f0=25.0, nrec_side=3, seed=5):
    """Small boxes for the CPU pins and fast parity tests."""
    return build(Workload(f"box_{nx}x{ny}x{nz}", nx, ny, nz, npml, 1.0, nsteps, f0, nrec_side, seed=seed))


def synthetic_traces(nsteps, nrec, seed, scale=1e-9):
    """Seeded smooth traces [nsteps+1, nrec, 3], used as 'observed data' where only
    a nonzero residual is needed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.linspace(0.0, 1.0, nsteps + 1)[:, None, None]
    a = rng.standard_normal((1, nrec, 3))
    b = rng.standard_normal((1, nrec, 3))
    f = rng.uniform(1.0, 4.0, (1, nrec, 3))
    return scale * (a * np.sin(2 * np.pi * f * t) + b * np.cos(2 * np.pi * f * t) * t)


def random_state(nnode, pml_mask, dir_mask, seed, scale=1e-6):
    """Random first-order state [3, nnode, 9] that respects the Dirichlet faces and
    has history and stress only on PML nodes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Y = rng.standard_normal((3, nnode, 9)) * scale
    Y[:, dir_mask, 0:3] = 0.0
    Y[:, ~pml_mask, 3:9] = 0.0
    Y[0, ~pml_mask, 0:3] = 0.0
    return Y
