"""The request loop (idos_server_*): a request's level sums are the same
alone, in a mix of concurrent requests of other levels and sizes, and through
the model's own idos_sample_level; requests overlap on the device within the
HBM budget, and a budget smaller than any request serialises them."""
import numpy as np
import pytest

from gpu_common import cfg_and_prm

pytestmark = pytest.mark.gpu

MIX = [(0, 300), (2, 3), (1, 40), (3, 1), (0, 7), (1, 5), (2, 1), (0, 64), (3, 1), (1, 17)]


def _server(**kw):
    import paper_1611_09784_gb300 as pkg
    w, cfg, prm = cfg_and_prm(precision="fp32")
    return w, cfg, pkg.Server(cfg, **kw)


def test_same_alone_in_the_mix_and_through_the_model():
    import paper_1611_09784_gb300 as pkg
    w, cfg, srv = _server(n_workers=4)
    seed = w["seed"]
    probes = [(1, 12, 100), (3, 1, 7), (0, 200, 5000)]
    alone = {}
    for lv, n, first in probes:
        s1, s2, lat, dev = srv.wait(srv.submit(lv, n, seed, first))
        assert lat > 0 and dev > 0
        alone[(lv, n, first)] = (s1, s2)
    tickets = {}
    for i, (lv, n) in enumerate(MIX):
        tickets[("mix", i)] = srv.submit(lv, n, seed, 10_000 + 1000 * i)
        if i % 3 == 0:
            p = probes[(i // 3) % len(probes)]
            tickets[p + (i,)] = srv.submit(p[0], p[1], seed, p[2])
    for key, t in tickets.items():
        s1, s2, lat, dev = srv.wait(t)
        if key[0] != "mix":
            a1, a2 = alone[key[:3]]
            assert np.array_equal(s1, a1) and np.array_equal(s2, a2), key
    srv.close()
    m = pkg.create_model(dict(cfg, sm_split=0))
    for lv, n, first in probes:
        m.reset_level_stats(-1)
        m.sample_level(lv, n, seed, first)
        M, s1, s2, _ = m.get_level_stats(lv)
        assert M == n
        assert np.array_equal(s1, alone[(lv, n, first)][0]) and np.array_equal(s2, alone[(lv, n, first)][1])
    m.close()


def test_requests_overlap_within_the_budget():
    w, cfg, srv = _server(n_workers=4, hbm_budget_bytes=0)
    t = [srv.submit(lv, n, w["seed"], 50_000 + 100 * i) for i, (lv, n) in enumerate(MIX)]
    for x in t:
        srv.wait(x)
    info = srv.info()
    assert info["completed"] == len(MIX) and info["queued"] == 0 and info["in_flight_bytes"] == 0
    peak_overlapped = info["peak_bytes"]
    srv.close()
    # a one-byte budget admits one request at a time: the peak is the largest single footprint
    w, cfg, one = _server(n_workers=4, hbm_budget_bytes=1)
    t = [one.submit(lv, n, w["seed"], 50_000 + 100 * i) for i, (lv, n) in enumerate(MIX)]
    for x in t:
        one.wait(x)
    peak_single = one.info()["peak_bytes"]
    one.close()
    assert peak_overlapped > peak_single


def test_invalid_requests_are_rejected():
    import paper_1611_09784_gb300 as pkg
    w, cfg, srv = _server(n_workers=2)
    with pytest.raises(pkg.IdosError):
        srv.submit(9, 1, w["seed"], 0)
    with pytest.raises(pkg.IdosError):
        srv.submit(0, 0, w["seed"], 0)
    with pytest.raises(pkg.IdosError):
        srv.wait(123456)
    srv.close()
