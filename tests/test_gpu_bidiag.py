"""Graphene's matrices up to n = 128 in the bidiagonal form (eigenvalues eps
+- the singular values of the block between the sublattices, |n_A - n_B| more
at eps): its degenerate cases against the oracle's dense eigenvalues of H(k)
and its IDoS, on both float32 kernels (half-warp for n <= 32, 64-thread CTA
above) and the float64 half-warp kernel."""
import numpy as np
import pytest

from oracle import idos as oidos

from gpu_common import EIG_TOL, IDOS_TOL, cfg_and_prm, sorted_active

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_1611_09784_gb300")


def crafted_masks(N, rng):
    """mask[m] = 1 removes site m = 2 (i + N j) + sublattice."""
    n = 2 * N * N
    out = {"pristine": np.zeros(n, np.uint8)}
    no_a = np.zeros(n, np.uint8)
    no_a[0::2] = 1                       # p = 0: every kept site isolated at eps
    out["no A sites"] = no_a
    no_b = np.zeros(n, np.uint8)
    no_b[1::2] = 1
    out["no B sites"] = no_b
    few_a = np.zeros(n, np.uint8)
    few_a[2 * rng.permutation(N * N)[: max(1, (3 * N * N) // 4)]] = 1   # n_B - n_A zero modes
    out["3/4 of A removed"] = few_a
    out["half removed"] = (rng.random(n) < 0.5).astype(np.uint8)
    pair = np.ones(n, np.uint8)
    pair[0] = 0                          # one A site and its same-cell B neighbour
    pair[1] = 0
    out["one bond"] = pair
    return out


CASES = [("fp32", N) for N in (1, 2, 4, 5, 8)] + [("fp64", N) for N in (1, 2, 4)]


@pytest.mark.parametrize("eps", [0.0, 0.37])
@pytest.mark.parametrize("precision,N", CASES)
def test_bidiagonal_degenerate_cells(precision, N, eps):
    w, cfg, prm = cfg_and_prm(precision=precision, refine=1)
    cfg.update(eps_onsite=eps, tc_products=6)
    prm["eps_onsite"] = eps
    K = 2
    rng = np.random.default_rng(100 + N)
    with pkg.create_model(cfg) as m:
        for name, mk in crafted_masks(N, rng).items():
            Q, E = m.eval_idos(N, K, mask=mk, want_eigs=True)
            Eo = oidos.band_energies(N, K, mk, prm)
            for kk, (g, r) in enumerate(zip(sorted_active(E), Eo)):
                assert g.shape == r.shape, (name, kk)
                if g.size:
                    assert np.max(np.abs(g - r)) < EIG_TOL, (name, kk, float(np.max(np.abs(g - r))))
            assert np.max(np.abs(Q - oidos.sample_idos(N, K, mk, prm))) < IDOS_TOL, name
