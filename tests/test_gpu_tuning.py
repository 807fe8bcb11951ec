"""Installed configurations (idos_set_tuning) and the timeline trace: every
configuration the autotuner can pick gives the same level statistics as the
defaults (the same kernels per matrix; only the W kernel's and the update's
float rounding differ), and timeline mode traces every launch."""
import numpy as np
import pytest

from gpu_common import IDOS_TOL, cfg_and_prm

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_1611_09784_gb300")

COUNTS = [40, 4, 2, 1]
BASE = dict(sm_split=0, small_max_n=-1, persistent=1, graph=1, w_tile=1, chase_pair=1, placement=0,
            panel_cluster=0, her2k_lower=1, persist_reserve=0)


def _stats(m, tuning, seed=31):
    m.reset_level_stats(-1)
    if tuning is not None:
        m.set_tuning(tuning)
    for k in range(2):
        m.sample_levels(COUNTS, seed, [k * c for c in COUNTS])
    return [m.get_level_stats(l) for l in range(4)]


@pytest.mark.parametrize("change", [dict(sm_split=24, placement=2), dict(sm_split=32, placement=1),
                                    dict(w_tile=2), dict(her2k_lower=0), dict(persist_reserve=16),
                                    dict(graph=0, persistent=0), dict(panel_cluster=2, chase_pair=0)])
def test_installed_configuration_matches_defaults(change):
    w, cfg, prm = cfg_and_prm(precision="fp32")
    with pkg.create_model(cfg) as m:
        ref = _stats(m, dict(BASE))
        got = _stats(m, dict(BASE, **change))
    for (M0, s0, q0, _), (M1, s1, q1, _) in zip(ref, got):
        assert M0 == M1
        # sums over M_l samples of per-sample values within 1e-5 each
        assert np.max(np.abs(np.asarray(s1) - np.asarray(s0))) <= M0 * 2 * IDOS_TOL


def test_set_tuning_rejects_out_of_range():
    w, cfg, prm = cfg_and_prm(precision="fp32")
    with pkg.create_model(cfg) as m:
        with pytest.raises(pkg.IdosError):
            m.set_tuning(dict(BASE, w_tile=3))
        with pytest.raises(pkg.IdosError):
            m.set_tuning(dict(BASE, placement=-1))


def test_timeline_trace_covers_every_launch():
    w, cfg, prm = cfg_and_prm(precision="fp32")
    with pkg.create_model(cfg) as m:
        m.set_tuning(dict(BASE, sm_split=24, placement=2))
        m.sample_levels(COUNTS, 5, [0] * 4)
        m.set_profiling(2)
        m.sample_levels(COUNTS, 5, list(COUNTS))
        m.set_profiling(False)
        tr = m.get_trace()
        prof = m.get_profile()
    assert tr, "empty trace"
    kernels = {e["kernel"] for e in tr}
    assert {"k_small_tridiag", "k_bisect", "k_idos", "k_ts_chase"} <= kernels
    assert all(e["t1_ms"] >= e["t0_ms"] >= -1e-3 for e in tr)
    # the trace's launches are the profile's launches
    assert sum(e["launches"] for e in tr) == sum(n for _, n in prof.values())
    assert len({e["lane"] for e in tr}) >= 2   # the levels kept their own streams
