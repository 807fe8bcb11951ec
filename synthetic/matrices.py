"""Seeded random Hermitian and real symmetric tridiagonal matrices for
eigensolver parity tests (numpy's PCG64 generator, float64)."""
from __future__ import annotations

import numpy as np


def hermitian(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """complex128[n, n] Hermitian matrix with entries of size ~scale."""
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return (scale / np.sqrt(2.0 * n)) * (X + X.conj().T)


def tridiagonal(n: int, seed: int):
    """(d[n], e[n-1]) of a random real symmetric tridiagonal matrix."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=n), rng.normal(size=max(n - 1, 0))
