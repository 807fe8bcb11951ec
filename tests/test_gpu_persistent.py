"""The persistent launch over every level's shared-memory matrices (fine and
corner cells of all levels in one size-sorted work list) against the
per-level launches and against the oracle."""
import numpy as np
import pytest

from oracle import mlmc as omlmc

from gpu_common import IDOS_TOL, cfg_and_prm

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_1611_09784_gb300")


def _stats(cfg, counts, seed, firsts):
    with pkg.create_model(cfg) as m:
        m.sample_levels(counts, seed, firsts)
        return [m.get_level_stats(l)[:3] for l in range(len(counts))]


@pytest.mark.parametrize("p", [0.05, 0.6, 0.0, 1.0])
@pytest.mark.parametrize("counts", [[37, 5, 3, 1], [4, 0, 2, 0], [0, 3, 0, 0]])
def test_persistent_bit_identical_to_per_level_launches(p, counts):
    """Same kernels per matrix, same reduction orders: identical sums, also
    with ragged cells (p = 0.6), empty cells (p = 1), pristine cells and
    levels without samples."""
    w, cfg, prm = cfg_and_prm(precision="fp32", p=p)
    firsts = [1000, 2000, 3000, 4000]
    a = _stats(dict(cfg, persistent=1, sm_split=0), counts, w["seed"], firsts)
    b = _stats(dict(cfg, persistent=0, sm_split=0), counts, w["seed"], firsts)
    c = _stats(dict(cfg, persistent=1), counts, w["seed"], firsts)   # on the SM partition
    for x, y, z in zip(a, b, c):
        assert x[0] == y[0] == z[0]
        assert np.array_equal(x[1], y[1]) and np.array_equal(x[2], y[2])
        assert np.array_equal(x[1], z[1]) and np.array_equal(x[2], z[2])
    if p == 1.0:   # every site removed: Q = 0 on both levels of each pair
        for x in a:
            assert np.all(x[1] == 0.0)


def test_persistent_level_sums_match_oracle():
    """Level sums of Y and Y^2 from one persistent-mode call against the
    oracle's per-sample level differences (levels 0..2: n = 32 and 128 on the
    persistent launch, n = 512 on the two-stage path)."""
    w, cfg, prm = cfg_and_prm(precision="fp32")
    counts, firsts = [3, 2, 1, 0], [500, 501, 502, 0]
    got = _stats(dict(cfg, persistent=1), counts, w["seed"], firsts)
    for l, n in enumerate(counts):
        if n == 0:
            assert got[l][0] == 0
            continue
        Y = np.array([omlmc.level_sample(prm, w["levels"], l, firsts[l] + s, w["seed"])["Y"] for s in range(n)])
        M, s1, s2 = got[l]
        assert M == n
        assert np.max(np.abs(s1 - Y.sum(0))) < n * IDOS_TOL
        bound = n * IDOS_TOL * (2.0 * np.max(np.abs(Y)) + IDOS_TOL)
        assert np.max(np.abs(s2 - (Y ** 2).sum(0))) < bound


def test_persistent_field_validated():
    w, cfg, prm = cfg_and_prm(precision="fp32")
    with pytest.raises(Exception):
        pkg.create_model(dict(cfg, persistent=2))


@pytest.mark.parametrize("levels", [[(4, 6), (8, 3)], [(4, 6)], [(2, 4), (4, 3), (8, 2)]])
def test_persistent_other_level_sets(levels):
    """Two levels (the finest level's own small sets on the persistent launch,
    partition on), one level, and three small levels (up to 5 segments)."""
    w, cfg, prm = cfg_and_prm(precision="fp32")
    cfg = dict(cfg, levels=levels)
    counts = [7, 3, 2][:len(levels)]
    firsts = [300, 301, 302][:len(levels)]
    a = _stats(dict(cfg, persistent=1), counts, w["seed"], firsts)
    b = _stats(dict(cfg, persistent=0, sm_split=0), counts, w["seed"], firsts)
    for x, y in zip(a, b):
        assert x[0] == y[0]
        assert np.array_equal(x[1], y[1]) and np.array_equal(x[2], y[2])
