"""Pins of the TMDC-shaped oracle (oracle/tmdc.py) against what the mathematics
fixes: Hermiticity, the band folding of a pristine supercell onto the primitive
cell, the trace identity, the bipartite nearest-neighbour limit (particle-hole
symmetry, sublattice zero modes), removal equals sentinel, hop counts, and IDoS
saturation."""
import numpy as np
import pytest

from oracle import idos, lattice, tmdc
from synthetic import TMDC


def _prm(**over):
    d = dict(TMDC)
    d.update(p=0.05, e_min=-40.0, e_max=40.0, n_E=41, delta=0.05, smoothing="gauss")
    d.update(over)
    return d


def _rand_k(a, seed):
    rng = np.random.default_rng(seed)
    b = lattice.reciprocal_vectors(a)
    return rng.uniform(-1, 1) * b[0] + rng.uniform(-1, 1) * b[1]


def test_parameter_layout_and_range():
    eps, T1, T2M, T2X = tmdc.params(TMDC["model_seed"])
    assert eps.shape == (11,) and T1.shape == (3, 5, 6) and T2M.shape == (3, 5, 5) and T2X.shape == (3, 6, 6)
    allp = np.concatenate([eps, T1.ravel(), T2M.ravel(), T2X.ravel()])
    assert allp.size == 284 and np.all(allp >= -2.0) and np.all(allp < 2.0)
    assert len(np.unique(allp)) == 284


@pytest.mark.parametrize("N", [1, 2, 3])
def test_hermitian_with_vacancies(N):
    prm = _prm()
    mask = np.zeros(N * N, dtype=np.uint8)
    mask[::2] = 1
    H = tmdc.hamiltonian(N, _rand_k(prm["a"], N), mask, prm)
    assert np.allclose(H, H.conj().T, atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_hop_counts(N):
    nn, mm, xx = tmdc.hops(N, TMDC["a"])
    assert len(nn) == 3 * N * N            # three pairs per metal atom
    assert len(mm) == 6 * N * N and len(xx) == 6 * N * N   # six second neighbours each
    for lst in (mm, xx):
        for d in range(3):
            assert sum(1 for h in lst if h[2] == d and h[3] > 0) == N * N


@pytest.mark.parametrize("N", [2, 3])
def test_trace_is_sum_of_active_onsite_energies(N):
    prm = _prm()
    eps = tmdc.params(prm["model_seed"])[0]
    mask = np.zeros(N * N, dtype=np.uint8)
    mask[1] = 1
    H = tmdc.hamiltonian(N, _rand_k(prm["a"], 7), mask, prm)
    n_pairs = N * N - int(mask.sum())
    expect = N * N * eps[:5].sum() + n_pairs * eps[5:].sum() + 6 * int(mask.sum()) * prm["sentinel"]
    assert abs(np.trace(H).real - expect) < 1e-9 and abs(np.trace(H).imag) < 1e-12


@pytest.mark.parametrize("N", [2, 3])
def test_band_folding_onto_primitive_cell(N):
    prm = _prm()
    a = prm["a"]
    b = lattice.reciprocal_vectors(a)
    k = _rand_k(a, 11 + N)
    E_sc = np.linalg.eigvalsh(tmdc.hamiltonian(N, k, np.zeros(N * N, dtype=np.uint8), prm))
    E_pc = []
    for g1 in range(N):
        for g2 in range(N):
            kk = k + (g1 * b[0] + g2 * b[1]) / N
            E_pc.append(np.linalg.eigvalsh(tmdc.hamiltonian(1, kk, np.zeros(1, dtype=np.uint8), prm)))
    assert np.allclose(np.sort(E_sc), np.sort(np.concatenate(E_pc)), atol=1e-10)


def _nn_only(prm):
    eps, T1, T2M, T2X = tmdc.params(prm["model_seed"])
    return dict(prm, tmdc_params=(np.zeros(11), T1, np.zeros_like(T2M), np.zeros_like(T2X)))


@pytest.mark.parametrize("N,vac", [(2, [0]), (3, [1, 4])])
def test_nearest_neighbour_limit_is_bipartite(N, vac):
    prm = _nn_only(_prm())
    mask = np.zeros(N * N, dtype=np.uint8)
    mask[vac] = 1
    n_vac = 6 * len(vac)
    E = idos.eigenvalues(tmdc.hamiltonian(N, _rand_k(prm["a"], 3), mask, prm), n_vac)
    assert np.allclose(np.sort(E), np.sort(-E), atol=1e-10)        # particle-hole symmetric
    n_metal, n_pair = 5 * N * N, 6 * (N * N - len(vac))
    assert int(np.sum(np.abs(E) < 1e-9)) >= abs(n_pair - n_metal)  # rank of the off-diagonal block


def test_removal_equals_sentinel():
    prm = _prm()
    N = 2
    mask = np.array([0, 1, 0, 1], dtype=np.uint8)
    k = _rand_k(prm["a"], 5)
    H = tmdc.hamiltonian(N, k, mask, prm)
    keep = tmdc.orbital_mask(mask) == 0
    Hc = H[np.ix_(keep, keep)]
    assert np.allclose(idos.eigenvalues(H, 12), np.linalg.eigvalsh(Hc), atol=1e-10)


def test_idos_saturates_at_active_orbitals():
    prm = _prm()
    N, K = 2, 2
    mask = np.array([1, 0, 0, 0], dtype=np.uint8)
    E = tmdc.band_energies(N, K, mask, prm)
    assert E.max() < prm["e_max"] - 10 * prm["delta"] and E.min() > prm["e_min"] + 10 * prm["delta"]
    Q = tmdc.sample_idos(N, K, mask, prm)
    n_act = 11 * N * N - 6
    assert abs(Q[-1] - n_act / lattice.supercell_area(N, prm["a"])) < 1e-12
    assert abs(Q[0]) < 1e-12


def test_corner_tiling_identity():
    # a pristine N x N supercell on a K grid is the 2 x 2 tiling of its
    # (N/2) x (N/2) corners on a 2K grid (for even K both Monkhorst-Pack grids
    # fold onto the same primitive momenta): same spectrum multiset, same IDoS
    prm = _prm(e_min=-12.0, e_max=12.0, n_E=25, delta=0.3)
    N, K = 2, 2
    fine = np.zeros(N * N, dtype=np.uint8)
    corners = tmdc.corner_masks(fine, N)
    assert len(corners) == 4 and all(c.shape == (1,) for c in corners)
    qf = tmdc.sample_idos(N, K, fine, prm)
    qc = tmdc.sample_idos(N // 2, 2 * K, corners[0], prm)
    assert np.allclose(qf, qc, atol=1e-12)


def test_corner_masks_partition_the_cells():
    rng = np.random.default_rng(2)
    N = 6
    mask = (rng.random(N * N) < 0.5).astype(np.uint8)
    c = tmdc.corner_masks(mask, N)
    assert sum(int(x.sum()) for x in c) == int(mask.sum())
    m = mask.reshape(N, N)
    assert c[1][0] == m[0, 3] and c[2][0] == m[3, 0] and c[3][-1] == m[5, 5]
