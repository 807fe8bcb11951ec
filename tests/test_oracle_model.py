"""Pins of the oracle's H(k) assembly, eigenvalues and smoothed IDoS.

Each test checks the oracle against a fact the paper's model fixes
independently of the code (closed-form bands, band folding, bipartite
symmetry, state counts, normal-distribution tables, a 2x2 tiling identity).
"""
import math

import numpy as np
import pytest

from oracle import hamiltonian, idos, jacobi, lattice, mlmc, philox
from synthetic import GRAPHENE
from synthetic import matrices as synth

A = GRAPHENE["a"]
T = GRAPHENE["t"]


def prm(**kw):
    d = dict(GRAPHENE)
    d.update(p=0.05, e_min=-9.0, e_max=9.0, n_E=201, delta=0.1, smoothing="gauss")
    d.update(kw)
    return d


def closed_form(k):
    """Pristine graphene bands +-|t||1 + e^{ik.a1} + e^{ik.a2}| (eps_2p = 0):
    the 2x2 H_AB of Sec. 3.1 summed over the three neighbour directions."""
    av = lattice.primitive_vectors(A)
    f = 1 + np.exp(1j * (k @ av[0])) + np.exp(1j * (k @ av[1]))
    return np.array([-abs(T) * abs(f), abs(T) * abs(f)])


def random_k(rng, N):
    bv = lattice.reciprocal_vectors(A) / N
    u = rng.uniform(-0.5, 0.5, size=2)
    return u[0] * bv[0] + u[1] * bv[1]


def test_n1_closed_form_bands():
    rng = np.random.default_rng(1)
    for _ in range(20):
        k = random_k(rng, 1)
        H = hamiltonian.hamiltonian(1, k, np.zeros(2, np.uint8), T, 0.0, A, 1e3)
        assert np.allclose(np.linalg.eigvalsh(H), np.sort(closed_form(k)), atol=1e-12)
    # Dirac point K = (2 b1 + b2)/3 is a zero of both bands
    bv = lattice.reciprocal_vectors(A)
    H = hamiltonian.hamiltonian(1, (2 * bv[0] + bv[1]) / 3, np.zeros(2, np.uint8), T, 0.0, A, 1e3)
    assert np.allclose(np.linalg.eigvalsh(H), 0.0, atol=1e-12)
    # Gamma point: +-3|t|
    H = hamiltonian.hamiltonian(1, np.zeros(2), np.zeros(2, np.uint8), T, 0.0, A, 1e3)
    assert np.allclose(np.linalg.eigvalsh(H), [-3 * abs(T), 3 * abs(T)], atol=1e-12)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_band_folding(N):
    """N x N pristine supercell at k = union of primitive bands at k + G,
    G = (g1 b1 + g2 b2)/N (Sec. 4.2: the supercell BZ is the primitive one
    shrunk by 1/N)."""
    rng = np.random.default_rng(N)
    bv = lattice.reciprocal_vectors(A)
    for _ in range(3):
        k = random_k(rng, N)
        H = hamiltonian.hamiltonian(N, k, np.zeros(2 * N * N, np.uint8), T, 0.0, A, 1e3)
        got = np.linalg.eigvalsh(H)
        want = np.sort(np.concatenate([closed_form(k + (g1 * bv[0] + g2 * bv[1]) / N)
                                       for g1 in range(N) for g2 in range(N)]))
        assert np.allclose(got, want, atol=1e-11)


def test_pristine_idos_folding_equals_primitive():
    """For even N and K the N x N supercell on a K x K grid samples exactly the
    primitive bands on an NK x NK grid, so the IDoS per area is identical."""
    P = prm(p=0.0)
    q_super = idos.sample_idos(4, 2, np.zeros(32, np.uint8), P)
    q_prim = idos.sample_idos(1, 8, np.zeros(2, np.uint8), P)
    assert np.allclose(q_super, q_prim, atol=1e-13)
    # saturation of the pristine sheet: 2 states per primitive cell
    assert q_prim[-1] == pytest.approx(2.0 / lattice.cell_area(A), abs=1e-12)
    assert q_prim[-1] == pytest.approx(0.381618, abs=1e-6)


def test_smoothing_normal_table():
    """g(x) = P(Z > x) for Z ~ N(0,1); values from standard normal tables."""
    g = idos.smooth_gauss
    assert g(0.0) == pytest.approx(0.5, abs=1e-16)
    assert g(1.0) == pytest.approx(0.15865525393145707, abs=1e-14)
    assert g(2.0) == pytest.approx(0.022750131948179209, abs=1e-15)
    assert g(-1.959963984540054) == pytest.approx(0.975, abs=1e-13)
    assert g(3.0) == pytest.approx(0.0013498980316301, abs=1e-15)
    x = np.linspace(-5, 5, 101)
    assert np.allclose(g(x) + g(-x), 1.0, atol=1e-15)


def test_poly_smoothing_meets_eq_4_2():
    from scipy.integrate import quad
    g = lambda x: float(idos.smooth_poly(x))
    assert g(-1.0) == 1.0 and g(1.0) == 0.0 and g(-3.0) == 1.0 and g(2.0) == 0.0
    for q in (0, 1):
        val = quad(lambda x: x ** q * ((1.0 if x < 0 else 0.0) - g(x)), -1, 0)[0] + \
            quad(lambda x: x ** q * (0.0 - g(x)), 0, 1)[0]
        assert abs(val) < 1e-12


def test_energy_grid():
    e = idos.energy_grid(-9.0, 9.0, 201)
    assert e[0] == -9.0 and e[200] == 9.0 and e[100] == 0.0
    assert np.allclose(np.diff(e), 0.09, atol=1e-14)


def _random_mask(N, seed, p):
    return philox.vacancy_mask(seed, 0, 0, 2 * N * N, p)


@pytest.mark.parametrize("N,seed", [(2, 3), (3, 11), (4, 5)])
def test_particle_hole_saturation_zero_modes(N, seed):
    """Bipartite hopping, eps_2p = 0: the spectrum is symmetric at every k, so
    Q(e) + Q(-e) = n_act/|F| on the symmetric grid; Q(e_max) = n_act/|F|; and at
    least |n_A - n_B| eigenvalues vanish (rank of the A-B block)."""
    P = prm(p=0.3)
    mask = _random_mask(N, seed, 0.3)
    n_act = int((mask == 0).sum())
    area = lattice.supercell_area(N, A)
    Q = idos.sample_idos(N, 2, mask, P)
    assert np.allclose(Q + Q[::-1], n_act / area, atol=1e-12)
    assert Q[-1] == pytest.approx(n_act / area, abs=1e-12)
    nA = int(((mask == 0) & (np.arange(2 * N * N) % 2 == 0)).sum())
    nB = n_act - nA
    E = idos.band_energies(N, 2, mask, P)
    for row in E:
        assert np.sum(np.abs(row) < 1e-8) >= abs(nA - nB)
        assert np.allclose(np.sort(row), np.sort(-row), atol=1e-10)


def test_single_vacancy_n1():
    """N = 1 with site B removed leaves one isolated A orbital at eps_2p."""
    P = prm(p=0.5)
    mask = np.array([0, 1], np.uint8)
    E = idos.band_energies(1, 3, mask, P)
    assert np.allclose(E, 0.0, atol=1e-12)
    Q = idos.sample_idos(1, 3, mask, P)
    en = idos.energy_grid(-9, 9, 201)
    assert np.allclose(Q, idos.smooth_gauss(-en / 0.1) / lattice.cell_area(A), atol=1e-14)


def test_sentinel_equals_removal():
    """Eigenvalues kept from the sentinel matrix equal those of the matrix with
    the vacancy rows and columns deleted (Sec. 3.2)."""
    N = 3
    mask = _random_mask(N, 9, 0.25)
    keep = np.nonzero(mask == 0)[0]
    k = lattice.kpoints(N, 3, A)[4]
    H = hamiltonian.hamiltonian(N, k, mask, T, 0.0, A, 1e3)
    Hc = hamiltonian.hamiltonian(N, k, np.zeros_like(mask), T, 0.0, A, 1e3)[np.ix_(keep, keep)]
    assert np.allclose(idos.eigenvalues(H, int(mask.sum())), np.linalg.eigvalsh(Hc), atol=1e-11)


@pytest.mark.parametrize("N", [2, 4])
def test_jacobi_crosscheck(N):
    mask = _random_mask(N, 17, 0.2)
    k = lattice.kpoints(N, 2, A)[1]
    H = hamiltonian.hamiltonian(N, k, mask, T, 0.0, A, 1e3)
    assert np.allclose(jacobi.jacobi_eigvalsh(H), np.linalg.eigvalsh(H), atol=1e-10)
    R = synth.hermitian(12, 4)
    assert np.allclose(jacobi.jacobi_eigvalsh(R), np.linalg.eigvalsh(R), atol=1e-12)


@pytest.mark.parametrize("Nf,K", [(4, 2), (8, 2)])
def test_corner_tiling_identity(Nf, K):
    """A fine mask made of one corner pattern repeated 2x2 is a 2x2 supercell of
    that corner: its IDoS on a K x K grid equals the corner's on a 2K x 2K grid
    (K even).  This pins the corner slicing and the supercell assembly with
    vacancies (Sec. 3.3)."""
    h = Nf // 2
    P = prm(p=0.2)
    c = _random_mask(h, 23 + Nf, 0.2)
    fine = np.zeros(2 * Nf * Nf, np.uint8)
    for r in range(4):
        fine[lattice.corner_site_map(Nf, r)] = c
    for cm in mlmc.corner_masks(fine, Nf):
        assert np.array_equal(cm, c)
    qf = idos.sample_idos(Nf, K, fine, P)
    qc = idos.sample_idos(h, 2 * K, c, P)
    assert np.allclose(qf, qc, atol=1e-12)


# ---- overlap s != 0 (eq. (3.2c)-(3.2d)) and the DoS -----------------------
S_OV = 0.129
T_PAPER = -3.033


def test_overlap_n1_closed_form():
    """With S_AB = s f, H_AB = t f (f = sum of the three bond phases), the 2x2
    generalized problem has E = (eps + t|f|)/(1 + s|f|) and (eps - t|f|)/(1 - s|f|)."""
    rng = np.random.default_rng(4)
    av = lattice.primitive_vectors(A)
    for _ in range(10):
        k = random_k(rng, 1)
        mask = np.zeros(2, np.uint8)
        H = hamiltonian.hamiltonian(1, k, mask, T_PAPER, 0.0, A, 1e3)
        S = hamiltonian.overlap(1, k, mask, S_OV, A)
        f = abs(1 + np.exp(1j * (k @ av[0])) + np.exp(1j * (k @ av[1])))
        ref = np.sort([T_PAPER * f / (1 + S_OV * f), -T_PAPER * f / (1 - S_OV * f)])
        assert np.allclose(idos.generalized_eigenvalues(H, S, 0), ref, atol=1e-12)


def test_overlap_zero_is_the_standard_problem():
    rng = np.random.default_rng(5)
    N = 3
    mask = (rng.random(2 * N * N) < 0.2).astype(np.uint8)
    p0 = prm(s=0.0)
    p1 = prm(s=1e-14)
    assert np.allclose(idos.band_energies(N, 2, mask, p0), idos.band_energies(N, 2, mask, p1), atol=1e-11)


def test_overlap_generalized_eigenpairs_solve_the_pencil():
    rng = np.random.default_rng(6)
    N = 2
    mask = np.array([0, 1, 0, 0, 0, 0, 1, 0], dtype=np.uint8)
    k = random_k(rng, N)
    H = hamiltonian.hamiltonian(N, k, mask, T_PAPER, 0.0, A, 1e3)
    S = hamiltonian.overlap(N, k, mask, S_OV, A)
    assert np.allclose(S, S.conj().T) and np.min(np.linalg.eigvalsh(S)) > 1 - 3 * S_OV - 1e-12
    for E in idos.generalized_eigenvalues(H, S, 2):
        sv = np.linalg.svd(H - E * S, compute_uv=False)
        assert sv[-1] < 1e-9 * np.max(sv)


def test_dos_differentiation_is_exact_on_quadratics():
    e = idos.energy_grid(-3.0, 5.0, 33)
    Q = 0.7 * e ** 2 - 1.3 * e + 2.0
    D = idos.dos_from_idos(Q, -3.0, 5.0)
    assert np.allclose(D[1:-1], 1.4 * e[1:-1] - 1.3, atol=1e-12)
    h = e[1] - e[0]
    assert np.isclose(D[0], (Q[1] - Q[0]) / h) and np.isclose(D[-1], (Q[-1] - Q[-2]) / h)
