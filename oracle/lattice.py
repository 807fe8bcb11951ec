"""Honeycomb geometry of Sec. 3.1 and the supercell / Brillouin-zone sampling of
Sec. 4.2, in plain float64.

Readings (the paper names the lattice but fixes no coordinates):
* primitive vectors a1 = a(1, 0), a2 = a(1/2, sqrt(3)/2);
* basis tau_A = 0, tau_B = (a1 + a2)/3 (nearest-neighbour distance a/sqrt(3));
* supercell site index m = 2(i + N j) + s for cell (i, j) in [0, N)^2 and
  sublattice s in {A = 0, B = 1}; position i a1 + j a2 + tau_s;
* reciprocal vectors b_j with a_i . b_j = 2 pi delta_ij; the N x N supercell has
  reciprocal vectors b_j / N;
* Brillouin-zone points: a K x K Monkhorst-Pack grid on the supercell cell,
  k = sum_j (2 i_j - K - 1)/(2K) b_j / N, i_j = 1..K, ordered i_1 fastest.  The
  paper's rhombus-corner grid (Sec. 4.2) is replaced by this uniform grid; the
  BZ integral of eq. (4.1) becomes the mean over the K^2 points (Sec. 4.3,
  nearest-point band approximation).

Pinned in tests/test_oracle_lattice.py: a_i . b_j = 2 pi delta_ij, neighbour
distances, reduced coordinates of the grid, cell area = |a1 x a2|.
"""
from __future__ import annotations

import math

import numpy as np


def primitive_vectors(a: float) -> np.ndarray:
    """Rows a1, a2 (Angstrom)."""
    return np.array([[a, 0.0], [0.5 * a, 0.5 * math.sqrt(3.0) * a]], dtype=np.float64)


def basis(a: float) -> np.ndarray:
    """Rows tau_A, tau_B."""
    av = primitive_vectors(a)
    return np.array([[0.0, 0.0], (av[0] + av[1]) / 3.0], dtype=np.float64)


def reciprocal_vectors(a: float) -> np.ndarray:
    """Rows b1, b2 with a_i . b_j = 2 pi delta_ij."""
    av = primitive_vectors(a)
    return 2.0 * math.pi * np.linalg.inv(av).T


def cell_area(a: float) -> float:
    """|F| of the primitive cell: |a1 x a2|."""
    av = primitive_vectors(a)
    return abs(av[0, 0] * av[1, 1] - av[0, 1] * av[1, 0])


def supercell_area(N: int, a: float) -> float:
    """|F| of the N x N supercell."""
    return N * N * cell_area(a)


def site_index(i: int, j: int, s: int, N: int) -> int:
    return 2 * (i + N * j) + s


def site_positions(N: int, a: float) -> np.ndarray:
    """float64[2N^2, 2] positions of the supercell sites, in site-index order."""
    av = primitive_vectors(a)
    tau = basis(a)
    pos = np.zeros((2 * N * N, 2), dtype=np.float64)
    for j in range(N):
        for i in range(N):
            for s in range(2):
                pos[site_index(i, j, s, N)] = i * av[0] + j * av[1] + tau[s]
    return pos


def mp_fractions(K: int) -> np.ndarray:
    """(2i - K - 1)/(2K), i = 1..K."""
    return np.array([(2 * i - K - 1) / (2.0 * K) for i in range(1, K + 1)], dtype=np.float64)


def kpoints(N: int, K: int, a: float) -> np.ndarray:
    """float64[K*K, 2] Monkhorst-Pack points of the N x N supercell, index
    i1 + K*i2 (i1 fastest)."""
    bv = reciprocal_vectors(a) / N
    u = mp_fractions(K)
    ks = np.zeros((K * K, 2), dtype=np.float64)
    for i2 in range(K):
        for i1 in range(K):
            ks[i1 + K * i2] = u[i1] * bv[0] + u[i2] * bv[1]
    return ks


def corner_site_map(N: int, r: int) -> np.ndarray:
    """int[2(N/2)^2]: fine-cell site index of every site of corner r of Sec. 3.3.

    Corner r = ri + 2 rj covers cells i in [ri N/2, (ri+1) N/2), j likewise; its
    own site index is m' = 2(i' + (N/2) j') + s with i' = i - ri N/2."""
    if N % 2:
        raise ValueError("corner partition needs even N")
    h = N // 2
    ri, rj = r % 2, r // 2
    out = np.zeros(2 * h * h, dtype=np.int64)
    for jl in range(h):
        for il in range(h):
            for s in range(2):
                out[site_index(il, jl, s, h)] = site_index(il + ri * h, jl + rj * h, s, N)
    return out
