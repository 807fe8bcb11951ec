"""The benchmark's algorithmic work model for the bidiagonal small kernels
(bench.py gk_flops, n_act_of with sublattices): hand-computed counts and a
direct count of kept sites."""
import numpy as np

import bench


def test_gk_flops_hand_counts():
    # p = q = 16: 16 sum_{k=0}^{15} ((k + 1) k + k^2) = 16 (2 * 1240 + 120)
    assert bench.gk_flops([[16, 16]]) == 41600.0
    # p = 1: the left reflector touches no later column, there is no right one
    assert bench.gk_flops([[1, 5]]) == 0.0
    assert bench.gk_flops([[0, 7]]) == 0.0
    # p = 2, q = 3: j = 0 only, 16 ((3 - 0)(2 - 1) + (3 - 1)(2 - 1)) = 80, either order
    assert bench.gk_flops([[2, 3]]) == 80.0
    assert bench.gk_flops([[3, 2], [2, 3]]) == 160.0


def test_n_act_of_sublattice_counts():
    rng = np.random.default_rng(7)
    N = 4
    masks = (rng.random((6, 2 * N * N)) < 0.2).astype(np.uint8)
    fine, corners = bench.n_act_of(masks, N, sublattice=True)
    total, _ = bench.n_act_of(masks, N)
    for s in range(6):
        keep = 1 - masks[s]
        # site m = 2 (i + N j) + sublattice
        assert fine[s, 0] == keep[0::2].sum() and fine[s, 1] == keep[1::2].sum()
        assert fine[s].sum() == total[s]
    assert corners.shape == (6, 4, 2)
    assert np.array_equal(corners.sum(axis=(1, 2)), fine.sum(axis=1))
