"""Replica path on CPU: two gloo ranks with disjoint sample ranges merge their
level accumulators and reproduce the single-process MLMC estimate.  The level
samples come from the oracle (no GPU); what is tested is the replica logic
(the exchange, and the library's host-arithmetic eq. (2.6) combine of the
merged sums)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

LEVELS = [(2, 2), (4, 2)]
COUNTS = [6, 4]


def _prm():
    from synthetic import GRAPHENE
    d = dict(GRAPHENE)
    d.update(p=0.2, e_min=-9.0, e_max=9.0, n_E=31, delta=0.3, smoothing="gauss")
    return d


def _level_sums(level, samples, seed=17):
    from oracle import mlmc
    prm = _prm()
    Y = np.array([mlmc.level_sample(prm, LEVELS, level, m, seed)["Y"] for m in samples])
    return len(samples), Y.sum(0), (Y ** 2).sum(0)


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    from paper_1611_09784_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    counts = np.zeros(len(LEVELS), dtype=np.int64)
    sums = np.zeros((len(LEVELS), 2, 31))
    for l, c in enumerate(COUNTS):
        mine = [m for m in range(c) if m % world == rank]   # disjoint sample indices
        M, s1, s2 = _level_sums(l, mine)
        counts[l], sums[l, 0], sums[l, 1] = M, s1, s2
    mc, ms = replicas.merge(counts, sums)
    mean, var = replicas.combine(mc, ms)
    q.put((rank, mc.tolist(), mean.tolist(), var.tolist()))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_1611_09784_gb300 import build
    build.build()


def test_two_gloo_ranks_reproduce_single_process():
    from oracle import mlmc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # single process over all samples
    prm = _prm()
    per_level = [np.array([mlmc.level_sample(prm, LEVELS, l, m, 17)["Y"] for m in range(c)])
                 for l, c in enumerate(COUNTS)]
    mean_ref, var_ref = mlmc.mlmc_estimate(per_level)
    for rank, counts, mean, var in res:
        assert counts == COUNTS
        assert np.allclose(mean, mean_ref, rtol=0, atol=1e-13)
        assert np.allclose(var, var_ref, rtol=1e-9, atol=1e-18)


def test_combine_rejects_single_sample_levels():
    from paper_1611_09784_gb300 import IdosError, replicas
    with pytest.raises(IdosError):
        replicas.combine([1, 3], np.zeros((2, 2, 4)))
