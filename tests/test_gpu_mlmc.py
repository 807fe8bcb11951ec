"""The adaptive MLMC estimator (idos_mlmc_estimate, eq. (2.6)-(2.7)) against
the oracle: the same estimator recomputed by the oracle on the same samples,
a one-level estimate against the exact expectation over every vacancy
outcome of a 2 x 2 cell, and sample counts that depend on the seed alone."""
import numpy as np
import pytest

from oracle import mlmc as omlmc

from gpu_common import IDOS_TOL, cfg_and_prm

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_1611_09784_gb300")


@pytest.mark.parametrize("persistent", [1, 0])
def test_estimate_equals_oracle_on_the_same_samples(persistent):
    """Level l uses samples 0 .. M_l - 1 of the seed: the oracle's level
    differences over those samples give the same mean (eq. (2.6)) within the
    per-sample IDoS tolerance, and the same level variances."""
    levels = [(2, 4), (4, 3), (8, 2)]
    w, cfg, prm = cfg_and_prm(precision="fp32", p=0.1)
    cfg = dict(cfg, levels=levels, persistent=persistent)
    seed = 4242
    with pkg.create_model(cfg) as m:
        est = m.mlmc_estimate(8e-3, theta=0.5, c_alpha=1.96, pilot_samples=8, max_rounds=3, seed=seed)
    M = [int(x) for x in est["M"]]
    assert all(x >= 2 for x in M) and est["rounds"] >= 1
    assert est["h2d_bytes"] > 0 and est["d2h_bytes"] > 0
    mean = np.zeros_like(est["mean"])
    var = np.zeros_like(est["var"])
    for l, Ml in enumerate(M):
        Y = np.array([omlmc.level_sample(prm, levels, l, s, seed)["Y"] for s in range(Ml)])
        mean += Y.mean(0)
        var += Y.var(0, ddof=1) / Ml
        # per-sample differences below IDOS_TOL move a variance by at most
        # about 2 IDOS_TOL max|Y - mean| + IDOS_TOL^2
        assert abs(est["V"][l] - Y.var(0, ddof=1).max()) <= 4 * IDOS_TOL * np.abs(Y).max() + 2 * IDOS_TOL ** 2
    assert np.max(np.abs(est["mean"] - mean)) < len(levels) * IDOS_TOL
    assert np.max(np.abs(np.sqrt(est["var"]) - np.sqrt(var))) < len(levels) * IDOS_TOL


def test_one_level_estimate_matches_exhaustive_expectation():
    """Plain MC on a 2 x 2 cell (eq. (2.6) with one level): within four
    standard errors of E[Q] summed over all 2^8 vacancy outcomes."""
    w, cfg, prm = cfg_and_prm(precision="fp32", p=0.3)
    K = 3
    cfg = dict(cfg, levels=[(2, K)])
    prm = dict(prm, p=0.3)
    exact = omlmc.exhaustive_expectation(prm, 2, K)
    with pkg.create_model(cfg) as m:
        est = m.mlmc_estimate(2e-3, theta=0.5, c_alpha=1.96, pilot_samples=64, max_rounds=3, seed=77)
    se = np.sqrt(est["var"])
    assert int(est["M"][0]) >= 64
    assert np.all(np.abs(est["mean"] - exact) <= 4.0 * se + IDOS_TOL)


def test_bench_levels_estimate_at_tol_matches_oracle():
    """The benchmark's estimate: graphene levels N = 4, 8, 16, 32 at TOL = 1e-3
    (pilot 32, three rounds, float32 with one float64 pass, tensor-core
    update).  (1) The oracle recomputes eq. (2.6) on the very samples the
    library drew: means agree within the per-sample tolerance times the
    levels.  (2) An independent oracle plain Monte Carlo estimate at N = 32
    (eq. (2.2), samples of another key) agrees with it within four combined
    standard errors (both estimate E[Q_32])."""
    import oracle_pool
    w, cfg, prm = cfg_and_prm(precision="fp32", refine=1)
    cfg = dict(cfg, tc_products=6)
    seed = 515
    with pkg.create_model(cfg) as m:
        est = m.mlmc_estimate(w["tol"], theta=w["theta"], c_alpha=w["c_alpha"], pilot_samples=32, max_rounds=3,
                              seed=seed)
    M = [int(x) for x in est["M"]]
    levels = [tuple(x) for x in w["levels"]]
    jobs = [(prm, levels, l, s, seed) for l in reversed(range(len(M))) for s in range(M[l])]
    n_mc = 48
    jobs += [(prm, [levels[-1]], 0, s, seed + 1) for s in range(n_mc)]
    with oracle_pool.pool() as p:
        res = p.map(oracle_pool.level_y, jobs, chunksize=4)
    per = [[] for _ in M]
    mc = []
    for i, (l, s, Y) in enumerate(res):
        (mc if i >= len(jobs) - n_mc else per[l]).append(Y)
    mean = sum(np.mean(np.array(y), axis=0) for y in per)
    assert np.max(np.abs(est["mean"] - mean)) < len(M) * IDOS_TOL
    mc_mean, mc_var = omlmc.mc_estimate(np.array(mc))
    z = np.abs(est["mean"] - mc_mean) / np.sqrt(est["var"] + mc_var + 1e-30)
    assert np.max(z) < 4.0, float(np.max(z))


def test_sample_counts_depend_on_seed_only():
    """Three levels: the finest level's pilot runs beside the other levels'
    pilots and provisional rounds of eq. (2.7); with profiling on the same
    calls run one after the other.  With the flop-model W_l, the same seed
    gives the same samples per level whatever the timing (two unprofiled
    calls) and with profiling on, hence the same eq. (2.6) mean up to the
    summation order of the level sums."""
    levels = [(2, 4), (4, 3), (8, 2)]
    w, cfg, prm = cfg_and_prm(precision="fp32", p=0.1)
    cfg = dict(cfg, levels=levels)
    kw = dict(theta=0.5, c_alpha=1.96, pilot_samples=8, max_rounds=3, seed=2024)
    with pkg.create_model(cfg) as m:
        a = m.mlmc_estimate(8e-3, **kw)
        b = m.mlmc_estimate(8e-3, **kw)
        m.set_profiling(1)
        c = m.mlmc_estimate(8e-3, **kw)
        m.set_profiling(0)
    for e in (b, c):
        assert list(e["M"]) == list(a["M"])
        assert e["rounds"] == a["rounds"]
        np.testing.assert_allclose(e["mean"], a["mean"], rtol=0, atol=1e-12)
        np.testing.assert_allclose(e["var"], a["var"], rtol=1e-9, atol=1e-15)
    # every level below the finest took at least the pilot
    assert all(int(x) >= 8 for x in a["M"][:-1]) and int(a["M"][-1]) >= 4
