"""Reference of one iteration of Algorithm 2 (Sec. 3.2 of arXiv:1504.08340).

TEST INFRASTRUCTURE: only tests/ use it.

An iteration at material m_k = (lambda, mu) on the interior nodes:
  lines 6-8  misfit J and gradient: g_mis from the oracle's adjoint (C.1f)/(C.1g);
             the reduced gradient of (18) with R = 0 is g = Mtilde^-1 g_mis;
  line 9     L-BFGS direction (Nocedal & Wright's two-loop recursion) with m
             stored pairs; inner products in the Mtilde metric, <a, b> = a^T Mtilde b,
             for which <g, d> = g_mis . d is the exact directional derivative;
  line 10    Algorithm 1: alpha^lambda = alpha^mu = 1, halved together (rho) until
             J(m + alpha d) < J(m) + c1 alpha <g, d>;
  line 11    update (19): m_{k+1} = m_k + alpha d (stored in FP32, as the material).
With regularisation (Sec. 3.1, 3.3.1): the objective is J + R_lambda R^l + R_mu R^m with
the terms of (8) or (9) (oracle.regularization), the gradient (18) is
Mtilde^-1 (R g_reg + g_mis), and the factors follow (24) at the current material,
R_p = wp |g_mis,p| / |g_reg,p| (Euclidean norms), held fixed during the line search.
Biasing (25) of the lambda direction with weight W, Sec. 3.3.3.
Readings (the paper is silent): a pair (s, y) is kept only when <s, y> > 0;
without pairs the direction is -g scaled so that max|d| = first_step * max|m|;
trial materials with mu <= 0, lambda + 2 mu <= 0 or above the time-step limit
dt * vp_max / (h/2) <= 0.66 count as rejected trials; a biased direction that is
not a descent direction is replaced by the unbiased one; the curvature pairs use
the full (regularised) reduced gradients.
"""
from __future__ import annotations

import numpy as np


def two_loop(g, pairs, w):
    """d = -H g by the two-loop recursion in the inner product <a, b> = sum a w b.
    pairs: list of (s, y), oldest first."""
    q = g.copy()
    alphas = []
    for s, y in reversed(pairs):
        rho = 1.0 / np.sum(s * w * y)
        a = rho * np.sum(s * w * q)
        alphas.append((a, rho))
        q = q - a * y
    if pairs:
        s, y = pairs[-1]
        q = q * (np.sum(s * w * y) / np.sum(y * w * y))
    for (s, y), (a, rho) in zip(pairs, reversed(alphas)):
        b = rho * np.sum(y * w * q)
        q = q + (a - b) * s
    return -q


def dense_inverse_bfgs(pairs, w):
    """The same operator written as the BFGS inverse-Hessian recursion (dense, small n)
    in the metric W = diag(w): H0 = gamma I with gamma = <s, y>/<y, y> of the newest
    pair, then H <- (I - rho s y^T W) H (I - rho y s^T W) + rho s s^T W, rho = 1/<s, y>.
    (Euclidean BFGS in the variables W^(1/2) m, mapped back.)"""
    n = pairs[0][0].size
    W = np.diag(w)
    s, y = pairs[-1]
    H = (np.sum(s * w * y) / np.sum(y * w * y)) * np.eye(n)
    for s, y in pairs:
        rho = 1.0 / (s @ W @ y)
        U = np.eye(n) - rho * np.outer(s, y) @ W
        V = np.eye(n) - rho * np.outer(y, s) @ W
        H = U @ H @ V + rho * np.outer(s, s) @ W
    return H


def bias_direction(d, n, W):
    """(25): the lambda part d[:n] becomes |d_l| (W d_m / |d_m| + (1 - W) d_l / |d_l|)."""
    ll, mm = np.linalg.norm(d[:n]), np.linalg.norm(d[n:])
    db = d.copy()
    if ll > 0 and mm > 0:
        db[:n] = ll * (W * d[n:] / mm + (1 - W) * d[:n] / ll)
    return db


class Inversion:
    """Algorithm 2 driven by the oracle (FP64 wavefields on FP32 materials)."""

    def __init__(self, o, dt, nsteps, src_nodes, src_dirs, rec_nodes, observed, wavelet, wparams,
                 lbfgs_m=15, invert=3, c1=1e-4, rho=0.5, max_backtracks=20, first_step=0.05,
                 reg=None, reg_eps=0.0, reg_wp=0.5, bias_w=0.0):
        self.o, self.dt, self.nsteps = o, dt, nsteps
        self.src, self.dirs, self.rec, self.obs = src_nodes, src_dirs, rec_nodes, observed
        self.wavelet, self.wparams = wavelet, wparams
        self.m_keep, self.invert, self.c1, self.rho = lbfgs_m, invert, c1, rho
        self.max_bt, self.first_step = max_backtracks, first_step
        self.reg, self.reg_eps, self.reg_wp, self.bias_w = reg, reg_eps, reg_wp, bias_w
        self.w = np.concatenate([o.diag("Mtilde"), o.diag("Mtilde")])
        self.pairs = []
        self.prev = None

    def _J(self, m):
        n = m.size // 2
        self.o.set_material(m[:n], m[n:])
        tr = self.o.forward(self.dt, self.nsteps, self.src, self.dirs, self.wavelet, self.wparams, self.rec)
        return self.o.misfit(self.dt, tr, self.obs)

    def _reg_value(self, m, Rp):
        n = m.size // 2
        if self.reg is None:
            return 0.0
        return sum(Rp[p] * self.o.regularization(m[p * n:(p + 1) * n], self.reg, self.reg_eps)[0]
                   for p in range(2) if Rp[p] != 0.0)

    def admissible(self, m):
        n = m.size // 2
        lam, mu = m[:n], m[n:]
        if not (np.all(np.isfinite(m)) and np.all(mu > 0) and np.all(lam + 2 * mu > 0)):
            return False
        vp = np.sqrt((lam + 2 * mu).max() / self.o.rho)
        return self.dt * vp / (0.5 * self.o.h) <= 0.66

    def step(self, m):
        """m: FP32 material (lambda, mu) as float64 array of 2 n; returns (m_new, info)."""
        n = m.size // 2
        self.o.set_material(m[:n], m[n:])
        J0, gl, gm, _ = self.o.misfit_and_gradient(self.dt, self.nsteps, self.src, self.dirs, self.rec,
                                                   self.obs, self.wavelet, self.wparams)
        Jmis0 = J0
        Rp = [0.0, 0.0]
        if self.reg is not None:  # (18) with R_p from (24)
            gmis = [gl, gm]
            for p in range(2):
                if not self.invert & (1 << p):
                    continue
                Rf, greg = self.o.regularization(m[p * n:(p + 1) * n], self.reg, self.reg_eps)
                nr = np.linalg.norm(greg)
                Rp[p] = self.reg_wp * np.linalg.norm(gmis[p]) / nr if nr > 0 else 0.0
                gmis[p] = gmis[p] + Rp[p] * greg
                J0 += Rp[p] * Rf
            gl, gm = gmis
        mt = self.w[:n]
        g = np.concatenate([gl / mt if self.invert & 1 else 0 * gl, gm / mt if self.invert & 2 else 0 * gm])
        if self.prev is not None and self.m_keep > 0:
            s, y = m - self.prev[0], g - self.prev[1]
            if np.sum(s * self.w * y) > 0:
                self.pairs = (self.pairs + [(s, y)])[-self.m_keep:]
        for attempt in range(2):
            if self.pairs:
                d = two_loop(g, self.pairs, self.w)
            else:
                d = -g * (self.first_step * np.abs(m).max() / np.abs(g).max())
            gtd = np.sum(g * self.w * d)
            if self.bias_w > 0 and self.invert == 3 and gtd < 0:  # (25)
                db = bias_direction(d, n, self.bias_w)
                gtb = np.sum(g * self.w * db)
                if gtb < 0:
                    d, gtd = db, gtb
            if gtd < 0:
                break
            self.pairs = []
        alpha, trials = 1.0, 0
        for _ in range(self.max_bt + 1):
            mt_trial = (m + alpha * d).astype(np.float32).astype(np.float64)
            if self.admissible(mt_trial):
                trials += 1
                Jmis_t = self._J(mt_trial)
                Jt = Jmis_t + self._reg_value(mt_trial, Rp)
                if Jt < J0 + self.c1 * alpha * gtd:
                    self.prev = (m, g)
                    return mt_trial, dict(J_old=J0, J_new=Jt, alpha=alpha, gtd=gtd, trials=trials, accepted=1,
                                          R=Rp, Jmis_old=Jmis0, Jmis_new=Jmis_t)
            alpha *= self.rho
        self.pairs, self.prev = [], None
        return m, dict(J_old=J0, J_new=J0, alpha=0.0, gtd=gtd, trials=trials, accepted=0, R=Rp,
                       Jmis_old=Jmis0, Jmis_new=Jmis0)
