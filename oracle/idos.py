"""Smoothed integrated density of states per unit area of one sampled supercell,
eq. (4.1) with the approximations of Sec. 4.3:

    Q(eps_j) = 1/(|F| K^2) * sum_{k in grid} sum_{n active} g((E_n(k) - eps_j)/delta)

* |F| = N^2 |a1 x a2| is the supercell area (eq. (4.1) normalises by the area of
  the fundamental cell of the periodic problem, here the supercell);
* the BZ average of eq. (4.1) is the mean over the K x K grid (Sec. 4.3: E_n(k)
  replaced by its value at the nearest grid point);
* the indicator is smoothed as in eq. (4.2).  Reading: g(x) = erfc(x/sqrt 2)/2,
  the upper tail of the standard normal (delta is its standard deviation); it
  satisfies the q = 0 moment condition by symmetry but is not compactly
  supported.  ``smooth_poly`` is the paper-conforming alternative:
  g(x) = 1/2 - 9x/8 + 5x^3/8 on [-1, 1] (1 below, 0 above) meets g(-1) = 1,
  g(1) = 0 and both moment conditions of eq. (4.2);
* energies eps_j = e_min + j (e_max - e_min)/(n_E - 1), j = 0..n_E-1 (Sec. 4.3,
  uniform grid);
* eigenvalues come from LAPACK (numpy.linalg.eigvalsh) on the full matrix with
  sentinels; eigenvalues above E_cut are the vacancies' and are dropped, with
  a check that exactly n_vac of them are.

Pinned: g against normal-distribution table values, saturation at n_act/|F|,
particle-hole identity Q(e) + Q(-e) = n_act/|F|, band folding, closed form.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh
from scipy.special import erfc

from . import hamiltonian, lattice

E_CUT = 500.0   # eigenvalues above this are vacancy sentinels (sentinel = 1e3 eV)


def energy_grid(e_min: float, e_max: float, n_E: int) -> np.ndarray:
    return np.array([e_min + j * (e_max - e_min) / (n_E - 1) for j in range(n_E)], dtype=np.float64)


def smooth_gauss(x):
    return 0.5 * erfc(np.asarray(x, dtype=np.float64) / np.sqrt(2.0))


def smooth_poly(x):
    x = np.asarray(x, dtype=np.float64)
    mid = 0.5 - 1.125 * x + 0.625 * x ** 3
    return np.where(x <= -1.0, 1.0, np.where(x >= 1.0, 0.0, mid))


SMOOTHERS = {"gauss": smooth_gauss, "poly": smooth_poly}


def eigenvalues(H: np.ndarray, n_vac: int) -> np.ndarray:
    """Ascending eigenvalues of the active block: all eigenvalues of H below
    E_CUT; asserts that exactly n_vac sentinel eigenvalues were dropped."""
    E = np.linalg.eigvalsh(H)
    keep = E < E_CUT
    if int((~keep).sum()) != n_vac:
        raise AssertionError("sentinel eigenvalue count differs from vacancy count")
    return E[keep]


def generalized_eigenvalues(H: np.ndarray, S: np.ndarray, n_vac: int) -> np.ndarray:
    """Ascending eigenvalues E of H u = E S u (eq. (3.1), S Hermitian positive
    definite) below E_CUT, by LAPACK's generalized Hermitian solver; asserts
    that exactly n_vac sentinel eigenvalues were dropped."""
    E = eigh(H, S, eigvals_only=True)
    keep = E < E_CUT
    if int((~keep).sum()) != n_vac:
        raise AssertionError("sentinel eigenvalue count differs from vacancy count")
    return np.sort(E[keep])


def band_energies(N: int, K: int, mask, prm) -> np.ndarray:
    """float64[K^2, n_act]: E_n(k) for every grid point (graphene model); with
    a nonzero overlap prm["s"] the generalized problem H u = E S u of
    eq. (3.1)-(3.2d)."""
    mask = np.asarray(mask, dtype=np.uint8)
    n_vac = int(mask.sum())
    ks = lattice.kpoints(N, K, prm["a"])
    s = float(prm.get("s", 0.0))
    out = []
    for k in ks:
        H = hamiltonian.hamiltonian(N, k, mask, prm["t"], prm["eps_onsite"], prm["a"], prm["sentinel"])
        if s != 0.0:
            out.append(generalized_eigenvalues(H, hamiltonian.overlap(N, k, mask, s, prm["a"]), n_vac))
        else:
            out.append(eigenvalues(H, n_vac))
    return np.array(out)


def idos_from_bands(E: np.ndarray, area: float, energies: np.ndarray, delta: float,
                    smoothing: str = "gauss") -> np.ndarray:
    """float64[n_E] from band energies E[K^2, n_act] (eq. (4.1)-(4.2))."""
    g = SMOOTHERS[smoothing]
    nk = E.shape[0]
    Q = np.zeros(energies.shape[0], dtype=np.float64)
    for j, eps in enumerate(energies):
        Q[j] = g((E.ravel() - eps) / delta).sum()
    return Q / (area * nk)


def sample_idos(N: int, K: int, mask, prm) -> np.ndarray:
    """Per-sample IDoS Q(eps_j) of the N x N supercell with the given mask."""
    E = band_energies(N, K, mask, prm)
    en = energy_grid(prm["e_min"], prm["e_max"], prm["n_E"])
    return idos_from_bands(E, lattice.supercell_area(N, prm["a"]), en, prm["delta"],
                           prm.get("smoothing", "gauss"))


def dos_from_idos(Q, e_min: float, e_max: float) -> np.ndarray:
    """Density of states from an IDoS on the uniform grid by numerical
    differentiation (Sec. 4.3): central differences (Q_{j+1} - Q_{j-1})/(2h)
    inside, one-sided differences at the two ends; h = (e_max - e_min)/(n_E - 1)."""
    Q = np.asarray(Q, dtype=np.float64)
    n = Q.shape[-1]
    h = (e_max - e_min) / (n - 1)
    D = np.empty_like(Q)
    D[..., 1:-1] = (Q[..., 2:] - Q[..., :-2]) / (2.0 * h)
    D[..., 0] = (Q[..., 1] - Q[..., 0]) / h
    D[..., -1] = (Q[..., -1] - Q[..., -2]) / h
    return D

