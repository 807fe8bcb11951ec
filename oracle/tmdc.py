"""TMDC-shaped 11-orbital tight-binding model on an N x N supercell (the MoS2
example of Sec. 3.1 and the chalcogen-pair vacancies of Sec. 3.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper takes the 11-band MoS2 model and its parameters from another work
whose table is not available here.  This model keeps the structure the paper
describes and draws the parameters from the seeded generator:

* the honeycomb lattice a1 = a(1, 0), a2 = a(1/2, sqrt3/2); a metal atom with 5 d
  orbitals (q = 0..4) on the A site tau_M = 0 and a chalcogen pair with 6 p
  orbitals (q = 5..10; two atoms stacked perpendicular to the plane, one
  projected position) on the B site tau_X = (a1 + a2)/3;
* 11 on-site energies eps[q];
* nearest-neighbour metal -> pair blocks T1[b] (5 x 6) for the three bonds
  R_0 = tau_X, R_1 = tau_X - a1, R_2 = tau_X - a2 (the pair -> metal hop is the
  conjugate transpose);
* second-neighbour metal-metal blocks T2M[d] (5 x 5) and pair-pair blocks
  T2X[d] (6 x 6) along delta_0 = a1, delta_1 = a2, delta_2 = a2 - a1; the hop
  along -delta_d is T[d]^T (the blocks are real, so H is Hermitian).

    H_{(c,q),(c',q')}(k) = sum over hops (c,q) -> (c',q') of block entry * exp(i k . R),

R the true vector from the first atom to the second (atomic gauge, eq. (3.2b)).
Orbital index o = 11 c + q, cell c = i + N j.  A removed pair (mask[c] = 1)
takes out orbitals 11c+5 .. 11c+10: the oracle zeroes their rows and columns and
puts the sentinel on the diagonal, as for graphene.

Parameters: uniform_params(model_seed, 284, lo, hi) in the order eps[11],
T1[3][5][6], T2M[3][5][5], T2X[3][6][6] (row-major).

Hops are found by brute force: every pair of atoms and every periodic image of
the supercell within one supercell vector, classified by distance (a/sqrt3 for
the nearest neighbours, a for the second) and by matching the displacement to
R_b or +-delta_d.

Pinned by (tests/test_oracle_tmdc.py): Hermiticity, band folding of the pristine
supercell onto the primitive cell, the trace identity Tr H = sum of on-site
energies of the active orbitals, sublattice zero modes and particle-hole symmetry of
the nearest-neighbour-only limit, removal equals sentinel.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from . import idos, lattice, philox

N_ORB = 11
N_M = 5
N_X = 6
N_PARAMS = 11 + 3 * 5 * 6 + 3 * 5 * 5 + 3 * 6 * 6   # 284


def params(model_seed: int, lo: float = -2.0, hi: float = 2.0):
    """(eps[11], T1[3,5,6], T2M[3,5,5], T2X[3,6,6]) drawn from the generator."""
    p = philox.uniform_params(model_seed, N_PARAMS, lo, hi)
    eps = p[0:11].copy()
    T1 = p[11:101].reshape(3, 5, 6).copy()
    T2M = p[101:176].reshape(3, 5, 5).copy()
    T2X = p[176:284].reshape(3, 6, 6).copy()
    return eps, T1, T2M, T2X


def atom_positions(N: int, a: float):
    """(metal positions [N^2, 2], pair positions [N^2, 2]) of cells c = i + N j."""
    av = lattice.primitive_vectors(a)
    tau_x = (av[0] + av[1]) / 3.0
    M = np.array([i * av[0] + j * av[1] for j in range(N) for i in range(N)], dtype=np.float64)
    return M, M + tau_x[None, :]


@functools.lru_cache(maxsize=16)
def hops(N: int, a: float):
    """Lists of hops found by distance and direction:
    nn: (cell_M, cell_X, b, R) metal -> pair nearest neighbours;
    mm, xx: (cell, cell', d, sign, R) second neighbours (sign +1 along +delta_d)."""
    av = lattice.primitive_vectors(a)
    tau_x = (av[0] + av[1]) / 3.0
    Rb = [tau_x, tau_x - av[0], tau_x - av[1]]
    deltas = [av[0], av[1], av[1] - av[0]]
    M, X = atom_positions(N, a)
    shifts = np.array([u * N * av[0] + v * N * av[1] for u in (-1, 0, 1) for v in (-1, 0, 1)])
    tol = 1e-6 * a
    nn = []
    for cm in range(N * N):
        d = X[None, :, :] + shifts[:, None, :] - M[cm][None, None, :]
        dist = np.sqrt((d ** 2).sum(axis=2))
        for img, cx in zip(*np.nonzero(np.abs(dist - a / math.sqrt(3.0)) < tol)):
            R = d[img, cx]
            b = [k for k in range(3) if np.linalg.norm(R - Rb[k]) < tol]
            assert len(b) == 1
            nn.append((cm, int(cx), b[0], R))
    second = []
    for P in (M, X):
        lst = []
        for c in range(N * N):
            d = P[None, :, :] + shifts[:, None, :] - P[c][None, None, :]
            dist = np.sqrt((d ** 2).sum(axis=2))
            for img, c2 in zip(*np.nonzero(np.abs(dist - a) < tol)):
                R = d[img, c2]
                hit = [(k, s) for k in range(3) for s in (1, -1) if np.linalg.norm(R - s * deltas[k]) < tol]
                assert len(hit) == 1
                lst.append((c, int(c2), hit[0][0], hit[0][1], R))
        second.append(lst)
    return nn, second[0], second[1]


def hamiltonian(N: int, k, mask, prm) -> np.ndarray:
    """complex128[11 N^2, 11 N^2] H(k); mask[c] = 1 removes cell c's pair."""
    if "tmdc_params" in prm:   # explicit (eps, T1, T2M, T2X), e.g. special cases in the pins
        eps, T1, T2M, T2X = prm["tmdc_params"]
    else:
        eps, T1, T2M, T2X = params(prm["model_seed"], prm.get("param_lo", -2.0), prm.get("param_hi", 2.0))
    a = prm["a"]
    n = N_ORB * N * N
    kv = np.asarray(k, dtype=np.float64)
    H = np.zeros((n, n), dtype=np.complex128)
    nn, mm, xx = hops(N, a)
    for cm, cx, b, R in nn:
        ph = np.exp(1j * float(R @ kv))
        rows = N_ORB * cm + np.arange(N_M)
        cols = N_ORB * cx + N_M + np.arange(N_X)
        H[np.ix_(rows, cols)] += T1[b] * ph
        H[np.ix_(cols, rows)] += T1[b].T * np.conj(ph)
    for lst, T, off, size in ((mm, T2M, 0, N_M), (xx, T2X, N_M, N_X)):
        for c, c2, dd, sign, R in lst:
            ph = np.exp(1j * float(R @ kv))
            rows = N_ORB * c + off + np.arange(size)
            cols = N_ORB * c2 + off + np.arange(size)
            H[np.ix_(rows, cols)] += (T[dd] if sign > 0 else T[dd].T) * ph
    for c in range(N * N):
        H[N_ORB * c + np.arange(N_ORB), N_ORB * c + np.arange(N_ORB)] += eps
    mask = np.asarray(mask)
    for c in range(N * N):
        if mask[c]:
            for q in range(N_M, N_ORB):
                o = N_ORB * c + q
                H[o, :] = 0.0
                H[:, o] = 0.0
                H[o, o] = prm["sentinel"]
    return H


def orbital_mask(mask) -> np.ndarray:
    """u8[11 N^2]: 1 for every orbital a removed pair takes out."""
    mask = np.asarray(mask, dtype=np.uint8)
    out = np.zeros(N_ORB * mask.shape[0], dtype=np.uint8)
    for c, m in enumerate(mask):
        if m:
            out[N_ORB * c + N_M:N_ORB * c + N_ORB] = 1
    return out


def band_energies(N: int, K: int, mask, prm) -> np.ndarray:
    """float64[K^2, n_act]: E_n(k) on the grid (kept orbitals only)."""
    mask = np.asarray(mask, dtype=np.uint8)
    n_vac = N_X * int(mask.sum())
    out = []
    for k in lattice.kpoints(N, K, prm["a"]):
        out.append(idos.eigenvalues(hamiltonian(N, k, mask, prm), n_vac))
    return np.array(out)


def sample_idos(N: int, K: int, mask, prm) -> np.ndarray:
    """Per-sample IDoS Q(eps_j) of the N x N supercell with the given pair mask."""
    E = band_energies(N, K, mask, prm)
    en = idos.energy_grid(prm["e_min"], prm["e_max"], prm["n_E"])
    return idos.idos_from_bands(E, lattice.supercell_area(N, prm["a"]), en, prm["delta"],
                                prm.get("smoothing", "gauss"))


def pair_mask(prm, N: int, level: int, sample: int, seed: int) -> np.ndarray:
    """u8[N^2]: the chalcogen pairs of sample `sample` on `level` that are removed
    (the vacancy generator with site index = cell index, Sec. 3.2)."""
    return philox.vacancy_mask(seed, level, sample, N * N, prm["p"])


def corner_masks(mask, N: int):
    """The four (N/2) x (N/2) corner pair masks of a fine pair mask (Sec. 3.3:
    corner r = ri + 2 rj takes cells i in [ri N/2, (ri+1) N/2), j in
    [rj N/2, (rj+1) N/2); local cell i' + (N/2) j')."""
    h = N // 2
    m = np.asarray(mask, dtype=np.uint8).reshape(N, N)   # [j][i]
    return [m[rj * h:(rj + 1) * h, ri * h:(ri + 1) * h].reshape(-1).copy() for rj in range(2) for ri in range(2)]

