"""Pins of the honeycomb geometry (Sec. 3.1) and the k-grid (Sec. 4.2)."""
import math

import numpy as np
import pytest

from oracle import hamiltonian, lattice

A = 2.46


def test_reciprocal_duality():
    av = lattice.primitive_vectors(A)
    bv = lattice.reciprocal_vectors(A)
    assert np.allclose(av @ bv.T, 2 * math.pi * np.eye(2), atol=1e-13)


def test_cell_area_value():
    # sqrt(3)/2 a^2 = 5.24084 A^2 for a = 2.46 A
    assert lattice.cell_area(A) == pytest.approx(math.sqrt(3) / 2 * A * A, rel=1e-14)
    assert lattice.cell_area(A) == pytest.approx(5.24084, abs=5e-6)
    assert lattice.supercell_area(32, A) == pytest.approx(5366.62, abs=0.01)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 8])
def test_three_neighbours_each(N):
    ms, ns, rs = hamiltonian.bonds(N, A)
    n = 2 * N * N
    assert len(ms) == 3 * n
    counts = np.bincount(ms, minlength=n)
    assert np.all(counts == 3)
    assert np.allclose(np.linalg.norm(rs, axis=1), A / math.sqrt(3), atol=1e-12)
    # bipartite: every bond joins sublattice A (even index) to B (odd index)
    assert np.all((ms % 2) != (ns % 2))


@pytest.mark.parametrize("N,K", [(1, 1), (4, 6), (8, 3), (16, 2), (3, 5)])
def test_kgrid_reduced_coordinates(N, K):
    ks = lattice.kpoints(N, K, A)
    av = lattice.primitive_vectors(A)
    red = N * (ks @ av.T) / (2 * math.pi)      # reduced coordinates on b_j/N
    frac = np.array([(2 * i - K - 1) / (2 * K) for i in range(1, K + 1)])
    for q in range(K * K):
        i1, i2 = q % K, q // K
        assert red[q, 0] == pytest.approx(frac[i1], abs=1e-13)
        assert red[q, 1] == pytest.approx(frac[i2], abs=1e-13)
    assert np.allclose(ks.mean(axis=0), 0.0, atol=1e-13)


@pytest.mark.parametrize("N", [2, 4, 8])
def test_corners_partition_sites(N):
    maps = [lattice.corner_site_map(N, r) for r in range(4)]
    allsites = np.sort(np.concatenate(maps))
    assert np.array_equal(allsites, np.arange(2 * N * N))
    pos = lattice.site_positions(N, A)
    h = N // 2
    av = lattice.primitive_vectors(A)
    for r, mp in enumerate(maps):
        ri, rj = r % 2, r // 2
        # the corner's own positions, shifted by its origin, are the (N/2)-cell positions
        local = lattice.site_positions(h, A) + ri * h * av[0] + rj * h * av[1]
        assert np.allclose(pos[mp], local, atol=1e-12)
