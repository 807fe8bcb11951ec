"""Pins of the oracle's control-variate coupling (Sec. 3.3) and estimators
(Sec. 2): telescoping, exhaustive enumeration (Sec. 1, Sec. 4.4), the CV
unbiasedness condition eq. (2.5a), and the optimality of eq. (2.7)."""
import numpy as np
import pytest

from oracle import idos, lattice, mlmc
from synthetic import GRAPHENE


def prm(**kw):
    d = dict(GRAPHENE)
    d.update(p=0.05, e_min=-9.0, e_max=9.0, n_E=201, delta=0.1, smoothing="gauss")
    d.update(kw)
    return d


def test_telescoping_pristine():
    """With p = 0 every corner equals the pristine coarse cell, so
    Y_0 + Y_1 + Y_2 = Q(N_2, K_2) exactly; a sign error or a wrong coarse K
    breaks this."""
    P = prm(p=0.0)
    levels = [(1, 6), (2, 3), (4, 2)]
    Ys = [mlmc.level_sample(P, levels, l, 0, 1)["Y"] for l in range(3)]
    Q2 = idos.sample_idos(4, 2, np.zeros(32, np.uint8), P)
    assert np.allclose(Ys[0] + Ys[1] + Ys[2], Q2, atol=1e-13)
    # and the level-1 difference is the pure k-grid refinement effect
    Q1 = idos.sample_idos(1, 6, np.zeros(2, np.uint8), P)
    assert np.allclose(Ys[0], Q1, atol=1e-15)


def test_exhaustive_n2_matches_monte_carlo():
    """E[Q] over all 2^8 outcomes of the N = 2 cell vs the Monte Carlo mean of
    400 seeded samples (eq. (2.2)): every energy within 5 standard errors."""
    P = prm(p=0.2, n_E=61, e_min=-9, e_max=9)
    ex = mlmc.exhaustive_expectation(P, 2, 2)
    Ys = np.array([mlmc.level_sample(P, [(2, 2)], 0, m, 99)["Y"] for m in range(400)])
    mean, var = mlmc.mc_estimate(Ys)
    z = np.abs(mean - ex) / np.sqrt(np.maximum(var, 1e-30))
    assert np.max(z[var > 1e-20]) < 5.0
    # saturation of the expectation: E[n_act]/|F| = (1 - p) 2 N^2 / |F|
    assert ex[-1] == pytest.approx(0.8 * 8 / lattice.supercell_area(2, P["a"]), rel=1e-12)


def test_cv_unbiased():
    """Eq. (2.5a): the mean of the coarse control variate on level 1 equals the
    mean of independent level-0 samples (4 standard errors of the difference)."""
    P = prm(p=0.2, n_E=41)
    levels = [(2, 2), (4, 2)]
    M = 150
    cv = []
    q0 = []
    for m in range(M):
        s = mlmc.level_sample(P, levels, 1, m, 5)
        cv.append(0.25 * sum(s["Q_coarse"]))
        q0.append(mlmc.level_sample(P, levels, 0, m, 5)["Y"])
    a, va = mlmc.mc_estimate(cv)
    b, vb = mlmc.mc_estimate(q0)
    z = np.abs(a - b) / np.sqrt(va + vb + 1e-30)
    assert np.max(z[(va + vb) > 1e-20]) < 4.5


def test_cv_exact_at_saturation():
    """At energies above the whole spectrum Q = n_act/|F| and the four corners
    partition the sites, so Y = 0 there for every outcome."""
    P = prm(p=0.3, n_E=21)
    s = mlmc.level_sample(P, [(2, 2), (4, 2)], 1, 3, 8)
    assert abs(s["Y"][-1]) < 1e-13


def test_optimal_samples_is_optimal():
    """Eq. (2.7) minimises sum_l M_l W_l subject to
    sum_l V_l/M_l = (theta TOL / C_a)^2: check the constraint and the Lagrange
    condition M_l^2 W_l / V_l = const on the unrounded values."""
    V = np.array([2e-4, 1e-5, 1e-6, 1e-7])
    W = np.array([6e6, 1.2e8, 3.3e9, 5.8e10])
    tol, th, ca = 1e-3, 0.5, 1.96
    Mi, M = mlmc.optimal_samples(V, W, tol, th, ca)
    assert np.sum(V / M) == pytest.approx((th * tol / ca) ** 2, rel=1e-12)
    lag = M ** 2 * W / V
    assert np.allclose(lag, lag[0], rtol=1e-12)
    assert np.all(Mi >= M) and np.all(Mi - M < 1)
    # any other allocation meeting the constraint costs at least as much
    rng = np.random.default_rng(0)
    for _ in range(20):
        Malt = M * np.exp(rng.normal(scale=0.3, size=4))
        Malt *= np.sum(V / Malt) / (th * tol / ca) ** 2
        assert np.sum(Malt * W) >= np.sum(M * W) * (1 - 1e-12)


def test_mlmc_combine_hand_computed():
    """Eq. (2.6) and the variance display after it, worked by hand: level A
    holds Y = 1, 3 (mean 2, unbiased sample variance 2, M = 2), level B holds
    Y = 0, 2, 4 (mean 2, sample variance 4, M = 3).  The estimate is 2 + 2 = 4
    and its variance V_A/M_A + V_B/M_B = 2/2 + 4/3 = 7/3.  A biased (ddof 0)
    sample variance gives 1/2 + 8/9, a missing 1/M_l gives 6, a doubled one
    1/2 + 4/9: all differ from 7/3."""
    A = np.array([[1.0], [3.0]])
    B = np.array([[0.0], [2.0], [4.0]])
    mean, var = mlmc.mlmc_estimate([A, B])
    assert mean[0] == pytest.approx(4.0, abs=1e-15)
    assert var[0] == pytest.approx(7.0 / 3.0, rel=1e-15)
    m1, v1 = mlmc.mc_estimate(A)
    assert m1[0] == pytest.approx(2.0, abs=1e-15) and v1[0] == pytest.approx(1.0, rel=1e-15)
    # one sample: the variance of the mean is unknown, not zero
    m0, v0 = mlmc.mc_estimate(np.array([[5.0]]))
    assert m0[0] == 5.0 and np.isinf(v0[0])


def test_mlmc_variance_matches_spread_of_estimates():
    """Statistical pin of the eq. (2.6) variance against the exact expectation.
    Levels (N, K) = (1, 4), (2, 2) at p = 0.2: the estimate is unbiased for
    E[Q(N = 2, K = 2)], known exactly from all 2^8 outcomes (Sec. 1).  Over R
    independent estimates (disjoint sample indices) two unbiased estimators of
    the estimator's variance must agree: the mean of the reported
    sum_l V_l/M_l, and the mean squared deviation of the estimates from the
    exact expectation.  For R = 250 their ratio has a relative standard error
    of about 0.1 (seeds 21, 22, 23 give 0.98, 1.07, 0.98); the bound
    [0.7, 1.45] rejects a missing or doubled 1/M_l (a factor of 3 to 64) and a
    dropped level term (with M = 64 and 3 samples each level carries between
    0.4 and 0.6 of the variance here, which the test also checks)."""
    P = prm(p=0.2, n_E=31)
    levels = [(1, 4), (2, 2)]
    ex = mlmc.exhaustive_expectation(P, 2, 2)
    R, M0, M1 = 250, 64, 3
    dev2 = np.zeros(P["n_E"])
    rep = np.zeros(P["n_E"])
    share0 = np.zeros(P["n_E"])
    for r in range(R):
        Y0 = np.array([mlmc.level_sample(P, levels, 0, r * M0 + m, 21)["Y"] for m in range(M0)])
        Y1 = np.array([mlmc.level_sample(P, levels, 1, r * M1 + m, 21)["Y"] for m in range(M1)])
        mean, var = mlmc.mlmc_estimate([Y0, Y1])
        dev2 += (mean - ex) ** 2
        rep += var
        share0 += mlmc.mc_estimate(Y0)[1]
    live = rep > 1e-3 * rep.max()
    ratio = dev2[live].sum() / rep[live].sum()
    assert 0.7 < ratio < 1.45, ratio
    frac0 = share0[live].sum() / rep[live].sum()
    assert 0.4 < frac0 < 0.75, frac0
