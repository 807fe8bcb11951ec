"""idos_sample_levels replayed as a captured CUDA graph: the same results as
direct launches, call after call with new seeds and sample indices (read by
the replayed mask kernels from a device buffer), recaptured when the sample
counts change."""
import numpy as np
import pytest

from gpu_common import cfg_and_prm

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_1611_09784_gb300")

CALLS = [([6, 3, 2, 1], 11, [0, 0, 0, 0]),
         ([6, 3, 2, 1], 12, [6, 3, 2, 1]),
         ([6, 3, 2, 1], 12, [100, 50, 20, 9]),
         ([9, 0, 1, 0], 13, [7, 0, 4, 0]),      # new counts: a new capture
         ([9, 0, 1, 0], 14, [70, 0, 40, 0])]


def _run(cfg):
    out = []
    with pkg.create_model(cfg) as m:
        for counts, seed, firsts in CALLS:
            m.sample_levels(counts, seed, firsts)
            out.append([m.get_level_stats(l)[:3] for l in range(4)])
        info = m.graph_info()
    return out, info


@pytest.mark.parametrize("sm_split", [-1, 0])
@pytest.mark.parametrize("persistent", [1, 0])
def test_graph_replay_matches_direct_launches(sm_split, persistent):
    w, cfg, prm = cfg_and_prm(precision="fp32")
    cfg = dict(cfg, sm_split=sm_split, persistent=persistent)
    got, info = _run(dict(cfg, graph=1))
    ref, info0 = _run(dict(cfg, graph=0))
    replays, captures, why = info
    assert why == "", why
    # a call whose workspace must first grow runs directly (then the next
    # one captures); a repeated key replays without a new capture
    assert captures >= 2 and replays >= captures + 1
    assert info0[:2] == (0, 0)
    for a, b in zip(got, ref):
        for x, y in zip(a, b):
            assert x[0] == y[0]
            assert np.array_equal(x[1], y[1]) and np.array_equal(x[2], y[2])


def test_graph_replay_fp64_model():
    """The float64 path (per-level launches, two-stage solves at n = 512 and
    2048) replays too."""
    w, cfg, prm = cfg_and_prm(precision="fp64")
    got, info = _run(dict(cfg, graph=1))
    ref, _ = _run(dict(cfg, graph=0))
    assert info[2] == "" and info[0] >= 2
    for a, b in zip(got, ref):
        for x, y in zip(a, b):
            assert np.array_equal(x[1], y[1]) and np.array_equal(x[2], y[2])


def test_graph_replay_tmdc_model():
    """The TMDC-shaped model (two-stage path at every size, per-level launches)
    replays with the same sums as direct launches."""
    from synthetic import model_params, workload
    w = workload("tmdc_sweep")
    cfg = dict(w["model"])
    cfg.update(p=w["p"], levels=[(4, 2), (8, 1)], e_min=w["e_min"], e_max=w["e_max"], n_E=w["n_E"],
               delta=w["delta"], smoothing=w["smoothing"], precision="fp32", refine64_iters=1)
    calls = [([3, 1], 5, [0, 0]), ([3, 1], 6, [3, 1]), ([3, 1], 6, [10, 20])]
    out = {}
    for graph in (1, 0):
        with pkg.create_model(dict(cfg, graph=graph)) as m:
            res = []
            for counts, seed, firsts in calls:
                m.sample_levels(counts, seed, firsts)
                res.append([m.get_level_stats(l)[:3] for l in range(2)])
            out[graph] = (res, m.graph_info())
    assert out[1][1][2] == "" and out[1][1][0] >= 1
    for a, b in zip(out[1][0], out[0][0]):
        for x, y in zip(a, b):
            assert np.array_equal(x[1], y[1]) and np.array_equal(x[2], y[2])
