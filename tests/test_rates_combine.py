"""Host arithmetic of the estimator behind the C ABI (no device needed): the
eq. (2.6) combine (idos_combine_level_stats) against the oracle's pinned
mlmc_estimate, and the rate fit of Sec. 2.1-2.2 / Sec. 4.4 (idos_fit_rates and
oracle.mlmc.fit_rates) on synthetic level samples whose grid-mean variances,
level means and costs follow exact power laws in N."""
import numpy as np
import pytest

from oracle import mlmc

N_LEVELS = [4, 8, 16, 32]
TRUE = {"W": 1.5, "S": 2.0, "D": 3.0, "C": 4.0}


@pytest.fixture(scope="module")
def pkg():
    from paper_1611_09784_gb300 import build
    build.build()
    import paper_1611_09784_gb300 as p
    p.load_library()
    return p


def power_law_samples(n_E=17, reps=2):
    """Per-level samples (Y, Q) with exactly
    mean_j Var(Q_l) = 3 N^-S, mean_j Var(Y_l) = 7 N^-D (l >= 1),
    mean_j |E[Y_l]| = 5 N^-W (l >= 1), built from pairs x = mu +- d per grid
    point (unbiased variance 2 d^2) scaled by a fixed profile over the grid."""
    prof = 0.5 + np.linspace(0.0, 1.0, n_E)          # positive profile, mean 1
    prof /= prof.mean()
    sgn = np.where(np.arange(n_E) % 3 == 0, -1.0, 1.0)
    Ys, Qs = [], []
    for l, N in enumerate(N_LEVELS):
        vq = 3.0 * N ** -TRUE["S"] * prof
        Q = np.stack([1.0 + np.sqrt(vq / 2), 1.0 - np.sqrt(vq / 2)] * (reps // 2))
        if l == 0:
            Y = Q.copy()
        else:
            vy = 7.0 * N ** -TRUE["D"] * prof
            b = 5.0 * N ** -TRUE["W"] * prof * sgn
            Y = np.stack([b + np.sqrt(vy / 2), b - np.sqrt(vy / 2)] * (reps // 2))
        Ys.append(Y)
        Qs.append(Q)
    cost = 2.0 * np.asarray(N_LEVELS, dtype=np.float64) ** TRUE["C"]
    return Ys, Qs, cost


def moments_of(Ys, Qs):
    return np.stack([np.stack([Y.sum(0), (Y ** 2).sum(0), Q.sum(0), (Q ** 2).sum(0)]) for Y, Q in zip(Ys, Qs)])


def test_oracle_fit_recovers_power_laws():
    Ys, Qs, cost = power_law_samples()
    r = mlmc.fit_rates(N_LEVELS, Ys, Qs, cost)
    for k, v in TRUE.items():
        assert r[k] == pytest.approx(v, abs=1e-9), k


def test_paper_rates_give_paper_work_exponents():
    """Sec. 4.4 prints W = 1.5, S = 2, D = 3, C = 4 and the exponents
    TOL^-10/3 (standard MC, eq. (Work_SLMC)) and TOL^-8/3 (MLMC,
    eq. (Work_MLMC)); eq. (Work_FS) gives 2C/S = 4."""
    Ys, Qs, cost = power_law_samples()
    r = mlmc.fit_rates(N_LEVELS, Ys, Qs, cost)
    assert r["work_mc"] == pytest.approx(10.0 / 3.0, abs=1e-9)
    assert r["work_mlmc"] == pytest.approx(8.0 / 3.0, abs=1e-9)
    assert r["work_fs"] == pytest.approx(4.0, abs=1e-9)
    assert r["theta_mc"] == pytest.approx(1.0 / (1.0 + 2.0 / 1.5), abs=1e-12)


def test_library_fit_matches_power_laws_and_oracle(pkg):
    Ys, Qs, cost = power_law_samples(reps=4)
    M = [Y.shape[0] for Y in Ys]
    r = pkg.fit_rates(N_LEVELS, M, moments_of(Ys, Qs), cost)
    ro = mlmc.fit_rates(N_LEVELS, Ys, Qs, cost)
    for k, v in TRUE.items():
        assert r[k] == pytest.approx(v, abs=1e-9), k
        assert r[k] == pytest.approx(ro[k], abs=1e-9), k
    assert (r["n_S"], r["n_D"], r["n_W"], r["n_C"]) == (4, 3, 3, 4)
    assert r["S_se"] == pytest.approx(0.0, abs=1e-7)   # exact power law: no residual
    for k in ("work_mc", "work_mlmc", "work_fs", "theta_mc"):
        assert r[k] == pytest.approx(ro[k], abs=1e-9), k


def test_library_fit_skips_levels_without_samples(pkg):
    Ys, Qs, cost = power_law_samples()
    mo = moments_of(Ys, Qs)
    M = [2, 0, 2, 2]
    mo[1] = 0.0
    r = pkg.fit_rates(N_LEVELS, M, mo, None)
    assert (r["n_S"], r["n_D"], r["n_W"], r["n_C"]) == (3, 2, 2, 0)
    assert r["S"] == pytest.approx(TRUE["S"], abs=1e-9)
    assert r["D"] == pytest.approx(TRUE["D"], abs=1e-9)
    assert np.isnan(r["C"])


def test_library_combine_matches_oracle(pkg):
    rng = np.random.default_rng(11)
    levels = [rng.normal(1.0, 0.5, size=(40, 9)), rng.normal(0.1, 0.05, size=(10, 9)),
              rng.normal(0.01, 0.02, size=(3, 9))]
    counts = np.array([Y.shape[0] for Y in levels])
    sums = np.stack([np.stack([Y.sum(0), (Y ** 2).sum(0)]) for Y in levels])
    mean, var = pkg.combine_level_stats(counts, sums)
    mref, vref = mlmc.mlmc_estimate(levels)
    assert np.allclose(mean, mref, rtol=0, atol=1e-14)
    assert np.allclose(var, vref, rtol=1e-10, atol=0)
    # the hand-worked case of the oracle pin: estimate 4, variance 7/3
    m2, v2 = pkg.combine_level_stats([2, 3], np.array([[[4.0], [10.0]], [[6.0], [20.0]]]))
    assert m2[0] == pytest.approx(4.0, abs=1e-15) and v2[0] == pytest.approx(7.0 / 3.0, rel=1e-14)
    # a level with no samples is left out
    m3, v3 = pkg.combine_level_stats([2, 0], np.array([[[4.0], [10.0]], [[0.0], [0.0]]]))
    assert m3[0] == pytest.approx(2.0) and v3[0] == pytest.approx(1.0)


def test_library_combine_rejects_bad_counts(pkg):
    for counts in ([1, 3], [0, 0], [-2, 3]):
        with pytest.raises(pkg.IdosError) as ei:
            pkg.combine_level_stats(counts, np.zeros((2, 2, 4)))
        assert ei.value.status == -1
