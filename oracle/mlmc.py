"""Control-variate coupling (Sec. 3.3) and the Monte Carlo / MLMC estimators of
Sec. 2, in float64.

* ``fine_mask``: the outcome omega_{l,m} of Sec. 2.2 is the vacancy pattern of
  sample m on level l, drawn by ``philox.vacancy_mask`` with counter
  (site, m, l, 0).  Independent levels use different level fields, so all terms
  of eq. (2.6) are independent.
* ``corner_masks``: the 2N supercell is split into four N x N corners that
  inherit its vacancies (Sec. 3.3, figure "Control variate idea"); each corner is
  then extended periodically on its own (bonds that cross a corner border are
  replaced by the corner's own periodic bonds).
* ``level_sample``: Y = Q_l(omega) - (1/4) sum_r Q_{l-1}(omega; corner r) for
  l >= 1 (0-based level index; the paper's l >= 2), and Y = Q_0(omega) on the
  first level.  The corners use the previous level's K so that
  E[Q_l^CV] = E[Q_{l-1}] holds exactly (eq. (2.5a)).
* ``mc_estimate``: eq. (2.2); ``mlmc_estimate``: eq. (2.6) with the variance of
  the unnumbered display after it (sum_l V_l / M_l).
* ``optimal_samples``: eq. (2.7).  Reading of the garbled confidence factor: the
  target variance of the estimator is (theta TOL / C_alpha)^2, the same
  squared factor eq. (2.7) carries; V_l is a scalar per level, the maximum of
  the pointwise variance over the energy grid.
* ``exhaustive_expectation``: Sec. 1 / Sec. 4.4: all 2^n vacancy outcomes of a
  small cell weighted by p^|v| (1-p)^(n-|v|).
* ``fit_rates``: the rates of the complexity models eq. (compl_model) and
  eq. (compl_model2) fitted as Sec. 4.4 does (eq. (param_est)): log-log least
  squares against N of the grid-mean sample variance of Q_l (S), of
  Y_l = Q_l - Q_l^CV (D), the grid mean of |E[Y_l]| = |E[Q_l] - E[Q_{l-1}]|
  (W: proportional to N_l^-W when N doubles) and the cost per sample (C);
  then the work exponents of eq. (Work_SLMC), eq. (Work_MLMC), eq. (Work_FS).

Pinned: telescoping with p = 0, corner tiling, CV unbiasedness (statistical),
exhaustive N = 2 expectation vs Monte Carlo, the optimality conditions of
eq. (2.7), the eq. (2.6) mean and variance on a hand-worked two-level case, and
the reported variance against the spread of independent two-level estimates
around the exact expectation (tests/test_oracle_mlmc.py).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import idos, lattice, philox


def fine_mask(prm, N: int, level: int, sample: int, seed: int) -> np.ndarray:
    return philox.vacancy_mask(seed, level, sample, 2 * N * N, prm["p"])


def corner_masks(mask: np.ndarray, N: int):
    """The four (N/2) x (N/2) corner masks, r = ri + 2 rj."""
    return [np.asarray(mask)[lattice.corner_site_map(N, r)] for r in range(4)]


def level_sample(prm, levels, level: int, sample: int, seed: int):
    """dict(Y, Q_fine, Q_coarse[4] or None, mask) for one outcome on one level.

    ``levels`` is a list of (N, K) pairs; level 0 is the coarsest."""
    N, K = levels[level]
    mask = fine_mask(prm, N, level, sample, seed)
    Qf = idos.sample_idos(N, K, mask, prm)
    if level == 0:
        return {"Y": Qf, "Q_fine": Qf, "Q_coarse": None, "mask": mask}
    Nc, Kc = levels[level - 1]
    if Nc * 2 != N:
        raise ValueError("level sizes must double")
    Qc = [idos.sample_idos(Nc, Kc, cm, prm) for cm in corner_masks(mask, N)]
    Y = Qf - 0.25 * (Qc[0] + Qc[1] + Qc[2] + Qc[3])
    return {"Y": Y, "Q_fine": Qf, "Q_coarse": Qc, "mask": mask}


def mc_estimate(samples: np.ndarray):
    """Eq. (2.2): sample mean and the variance of the mean, pointwise."""
    samples = np.asarray(samples, dtype=np.float64)
    M = samples.shape[0]
    mean = samples.mean(axis=0)
    var = samples.var(axis=0, ddof=1) / M if M > 1 else np.full_like(mean, np.inf)
    return mean, var


def mlmc_estimate(level_samples):
    """Eq. (2.6): sum over levels of the level means; Var = sum_l V_l/M_l."""
    mean = None
    var = None
    for Y in level_samples:
        m, v = mc_estimate(Y)
        mean = m if mean is None else mean + m
        var = v if var is None else var + v
    return mean, var


def optimal_samples(V, W, tol: float, theta: float = 0.5, c_alpha: float = 1.96):
    """Eq. (2.7): M_l = (C_a/(theta TOL))^2 sqrt(V_l/W_l) sum_k sqrt(W_k V_k),
    rounded up to an integer >= 1."""
    V = np.asarray(V, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    s = np.sum(np.sqrt(W * V))
    M = (c_alpha / (theta * tol)) ** 2 * np.sqrt(V / W) * s
    return np.maximum(1, np.ceil(M)).astype(np.int64), M


def fit_rates(N, Y_levels, Q_levels, cost=None):
    """Rates W, S, D, C from per-level sample arrays (Y_levels[l], Q_levels[l]:
    (M_l, n_E); level 0 is the coarsest) and an optional cost per sample per
    level.  Norm: the arithmetic mean over the energy grid."""
    N = np.asarray(N, dtype=np.float64)

    def slope(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        ok = (x > 0) & (y > 0)
        if ok.sum() < 2:
            return float("nan")
        return float(np.polyfit(np.log(x[ok]), np.log(y[ok]), 1)[0])

    xs, vq, xd, vy, xw, bias = [], [], [], [], [], []
    for l in range(len(N)):
        Y = np.asarray(Y_levels[l], dtype=np.float64)
        Q = np.asarray(Q_levels[l], dtype=np.float64)
        if Y.shape[0] >= 2:
            xs.append(N[l])
            vq.append(np.mean(Q.var(axis=0, ddof=1)))
            if l > 0:
                xd.append(N[l])
                vy.append(np.mean(Y.var(axis=0, ddof=1)))
        if Y.shape[0] >= 1 and l > 0:
            xw.append(N[l])
            bias.append(np.mean(np.abs(Y.mean(axis=0))))
    S = -slope(xs, vq)
    D = -slope(xd, vy)
    W = -slope(xw, bias)
    C = slope(N, cost) if cost is not None else float("nan")
    return {"W": W, "S": S, "D": D, "C": C, "work_mc": 2 + (C - S) / W, "work_mlmc": 2 + (C - D) / W,
            "work_fs": 2 * C / S, "theta_mc": 1 / (1 + (C - S) / W)}


def exhaustive_expectation(prm, N: int, K: int):
    """E[Q_N] over all 2^(2N^2) vacancy outcomes (only for tiny cells)."""
    n = 2 * N * N
    p = prm["p"]
    acc = None
    for bits in itertools.product((0, 1), repeat=n):
        v = np.array(bits, dtype=np.uint8)
        nv = int(v.sum())
        w = (p ** nv) * ((1.0 - p) ** (n - nv))
        Q = idos.sample_idos(N, K, v, prm)
        acc = w * Q if acc is None else acc + w * Q
    return acc
