"""The fact the GPU path's bidiagonal form rests on, checked on the oracle's own
H(k) (eq. (3.2a)-(3.2b)): nearest-neighbour hopping only joins the two
sublattices, and a vacancy removes a site without changing that, so with the
kept sites ordered (A, B) the Hamiltonian is eps I + [[0, T], [T^H, 0]] and
its spectrum is eps +- the singular values of T together with |n_A - n_B|
eigenvalues at eps."""
import numpy as np
import pytest

from oracle import hamiltonian, lattice
from synthetic import GRAPHENE


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("eps", [0.0, 0.37])
def test_spectrum_is_eps_plus_minus_singular_values(N, eps):
    rng = np.random.default_rng(10 * N + int(eps > 0))
    t, a = GRAPHENE["t"], GRAPHENE["a"]
    n = 2 * N * N
    for trial in range(6):
        mask = (rng.random(n) < rng.choice([0.0, 0.1, 0.3, 0.6])).astype(np.uint8)
        keep = np.flatnonzero(mask == 0)
        if keep.size == 0:
            continue
        k = lattice.kpoints(N, 2, a)[trial % 4]
        H = hamiltonian.hamiltonian(N, k, mask, t, eps, a, 1e3)[np.ix_(keep, keep)]
        A = keep[keep % 2 == 0]           # site m = 2 (i + N j) + sublattice
        B = keep[keep % 2 == 1]
        ia = np.searchsorted(keep, A)
        ib = np.searchsorted(keep, B)
        # no bond inside a sublattice
        assert np.allclose(H[np.ix_(ia, ia)], eps * np.eye(ia.size))
        assert np.allclose(H[np.ix_(ib, ib)], eps * np.eye(ib.size))
        T = H[np.ix_(ia, ib)]
        sv = np.linalg.svd(T, compute_uv=False) if T.size else np.zeros(0)
        zero_modes = abs(ia.size - ib.size)
        expect = np.sort(np.concatenate([eps + sv, eps - sv, np.full(zero_modes, eps)]))
        got = np.linalg.eigvalsh(H)
        assert got.shape == expect.shape
        assert np.max(np.abs(got - expect)) < 1e-10
