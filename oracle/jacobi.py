"""Cyclic Jacobi eigenvalue iteration for a complex Hermitian matrix, plain
Python/NumPy, used only to cross-check LAPACK's eigvalsh on small matrices
(n <= 32) so that the oracle's eigenvalues rest on two unrelated algorithms.

Each rotation zeroes one off-diagonal pair (p, q): with the phase of A_pq
removed the 2x2 block is real symmetric and the classical Jacobi angle
tan(2 theta) = 2|A_pq| / (A_qq - A_pp) annihilates it (Golub & Van Loan,
Sec. 8.5).  Sweeps repeat until the off-diagonal Frobenius norm is below
tol * ||A||_F.
"""
from __future__ import annotations

import math

import numpy as np


def jacobi_eigvalsh(A, tol: float = 1e-14, max_sweeps: int = 60) -> np.ndarray:
    A = np.array(A, dtype=np.complex128)
    n = A.shape[0]
    scale = np.linalg.norm(A)
    if scale == 0.0:
        return np.zeros(n)
    for _ in range(max_sweeps):
        off = math.sqrt(max(0.0, np.linalg.norm(A) ** 2 - float(np.sum(np.abs(np.diag(A)) ** 2))))
        if off <= tol * scale:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                r = abs(apq)
                if r <= 1e-300:
                    continue
                ph = apq / r                          # A_pq = r * ph
                app, aqq = A[p, p].real, A[q, q].real
                theta = 0.5 * math.atan2(2.0 * r, aqq - app)
                c, s = math.cos(theta), math.sin(theta)
                # unitary G acting on columns p, q: [c, s*ph; -s*conj(ph), c]
                G = np.eye(n, dtype=np.complex128)
                G[p, p] = c
                G[q, q] = c
                G[p, q] = s * ph
                G[q, p] = -s * np.conj(ph)
                A = G.conj().T @ A @ G
                A[p, q] = 0.0
                A[q, p] = 0.0
    return np.sort(np.real(np.diag(A)))
