"""Bloch Hamiltonian of the nearest-neighbour graphene model, eq. (3.2a)-(3.2b),
on an N x N supercell with vacancies (Sec. 3.2).

    H_mm(k) = eps_2p,     H_mn(k) = sum over bonds m->n of t exp(i k . R_mn),

R_mn the true vector from atom m to atom n (atomic gauge, as eq. (3.2b) states).
Bonds are found by brute force: every pair of sites and every periodic image of
the supercell within one supercell vector, kept when the distance equals the
nearest-neighbour distance a/sqrt(3).  For N = 1 the three bonds join the same
pair of sites and their phases add, which is how the paper's 2x2 H_AB of Sec.
3.1 arises.  The overlap S(k) of eq. (3.2c)-(3.2d) is the identity (s = 0).

A vacancy (Sec. 3.2) removes the site's rows and columns.  The oracle keeps the
matrix size fixed, zeroes those rows and columns and puts a large sentinel on
the diagonal; ``idos`` then drops exactly the sentinel eigenvalues, which
equals removal because the sentinel block is decoupled.

Pinned by: closed-form pristine bands (N = 1), band folding (N > 1),
particle-hole symmetry and zero-mode counts with vacancies, and the 2x2 tiling
identity of the control-variate corners (tests/test_oracle_model.py).
"""
from __future__ import annotations

import functools
import math

import numpy as np

from . import lattice


@functools.lru_cache(maxsize=32)
def bonds(N: int, a: float):
    """(m, n, R) arrays of all directed nearest-neighbour bonds of the supercell
    (both directions), found by distance over the 9 nearest supercell images."""
    pos = lattice.site_positions(N, a)
    av = lattice.primitive_vectors(a)
    nn = a / math.sqrt(3.0)
    shifts = np.array([u * N * av[0] + v * N * av[1] for u in (-1, 0, 1) for v in (-1, 0, 1)])
    ms, ns, rs = [], [], []
    for m in range(pos.shape[0]):
        d = pos[None, :, :] + shifts[:, None, :] - pos[m][None, None, :]   # (9, n, 2)
        dist = np.sqrt((d ** 2).sum(axis=2))
        img, n = np.nonzero(np.abs(dist - nn) < 1e-6 * a)
        for q, nidx in zip(img, n):
            ms.append(m)
            ns.append(int(nidx))
            rs.append(d[q, nidx])
    return np.array(ms), np.array(ns), np.array(rs)


def hamiltonian(N: int, k, mask, t: float, eps_onsite: float, a: float,
                sentinel: float) -> np.ndarray:
    """complex128[2N^2, 2N^2] H(k) with vacancies (mask[m] = 1 removes site m)."""
    n = 2 * N * N
    ms, ns, rs = bonds(N, a)
    H = np.zeros((n, n), dtype=np.complex128)
    kv = np.asarray(k, dtype=np.float64)
    # np.add.at accumulates repeated (m, n) pairs: for N = 1 the three bonds
    # A->B land on the same entry and their phases add.
    np.add.at(H, (ms, ns), t * np.exp(1j * (rs @ kv)))
    H[np.arange(n), np.arange(n)] += eps_onsite
    mask = np.asarray(mask)
    for m in range(n):
        if mask[m]:
            H[m, :] = 0.0
            H[:, m] = 0.0
            H[m, m] = sentinel
    return H


def overlap(N: int, k, mask, s: float, a: float) -> np.ndarray:
    """complex128[2N^2, 2N^2] S(k) of eq. (3.2c)-(3.2d): 1 on the diagonal,
    s exp(i k . R_mn) on every nearest-neighbour bond (found by the same
    brute-force search as H); a removed site keeps only its diagonal 1, so
    its generalized eigenvalue is H's sentinel."""
    n = 2 * N * N
    ms, ns, rs = bonds(N, a)
    S = np.zeros((n, n), dtype=np.complex128)
    np.add.at(S, (ms, ns), s * np.exp(1j * (rs @ np.asarray(k, dtype=np.float64))))
    mask = np.asarray(mask)
    for m in range(n):
        if mask[m]:
            S[m, :] = 0.0
            S[:, m] = 0.0
    S[np.arange(n), np.arange(n)] += 1.0
    return S

