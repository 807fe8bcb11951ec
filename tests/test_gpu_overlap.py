"""Graphene with the paper's overlap (t = -3.033 eV, s = 0.129, eq. (3.2a)-(3.2d)):
the GPU path's generalized eigenvalues and IDoS against the oracle's LAPACK
generalized Hermitian solver (scipy.linalg.eigh(H, S)), with vacancies, and a
level sample with the control-variate coupling."""
import numpy as np
import pytest

from oracle import idos as oidos
from oracle import mlmc as omlmc
from oracle import philox as ophilox
from synthetic import GRAPHENE

pytestmark = pytest.mark.gpu

EIG_TOL = 1e-4
IDOS_TOL = 1e-5


def _cfg(levels, precision):
    prm = dict(GRAPHENE, t=-3.033, s=0.129, p=0.1, e_min=-9.0, e_max=12.0, n_E=211, delta=0.1, smoothing="gauss")
    cfg = dict(prm, levels=levels, precision=precision, refine64_iters=2)
    return cfg, prm


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,K", [(1, 4), (2, 3), (4, 2), (8, 1)])
def test_generalized_eigenvalues_and_idos(N, K, precision):
    import paper_1611_09784_gb300 as pkg
    cfg, prm = _cfg([(N, K)], precision)
    m = pkg.create_model(cfg)
    for sample in range(2):
        mask = ophilox.vacancy_mask(11, 0, sample, 2 * N * N, prm["p"])
        Q, E = m.eval_idos(N, K, mask=mask, want_eigs=True)
        E_ref = oidos.band_energies(N, K, mask, prm)
        for k in range(K * K):
            got = E[k][~np.isnan(E[k])]
            # still ascending after the map (equal eigenvalues, e.g. a pair of
            # zero modes, may come out in either order within rounding)
            assert np.all(np.diff(got) >= -1e-9)
            assert np.max(np.abs(got - E_ref[k])) < EIG_TOL
        assert np.max(np.abs(Q - oidos.sample_idos(N, K, mask, prm))) < IDOS_TOL
    m.close()


def test_level_sample_with_overlap():
    import paper_1611_09784_gb300 as pkg
    levels = [(4, 2), (8, 1)]
    cfg, prm = _cfg(levels, "fp64")
    m = pkg.create_model(cfg)
    Y, Qf, Qc = m.sample_level_detail(1, 2, 21, 4)
    for s in range(2):
        ref = omlmc.level_sample(prm, levels, 1, 4 + s, 21)
        assert np.max(np.abs(Y[s] - ref["Y"])) < 2 * IDOS_TOL
    m.close()
