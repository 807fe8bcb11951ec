"""GPU parity of the TMDC-shaped 11-orbital model (chalcogen-pair vacancies)
against the oracle (oracle/tmdc.py), through the C ABI: pair masks bit-exact,
H(k) entries, per-sample eigenvalues and IDoS, the MLMC level coupling, and
one full-size sample (N = 16, n = 2816)."""
import numpy as np
import pytest

from oracle import lattice
from oracle import tmdc as otmdc
from synthetic import model_params, workload

pytestmark = pytest.mark.gpu

EIG_TOL = 1e-4
IDOS_TOL = 1e-5


def _cfg(levels, precision="fp64", **over):
    w = workload("tmdc_sweep")
    w.update(over)
    prm = model_params(w)
    cfg = dict(w["model"])
    cfg.update(p=w["p"], levels=levels, e_min=w["e_min"], e_max=w["e_max"], n_E=w["n_E"], delta=w["delta"],
               smoothing=w["smoothing"], precision=precision, refine64_iters=2)
    return w, cfg, prm


def test_pair_masks_bit_exact():
    import paper_1611_09784_gb300 as pkg
    w, cfg, prm = _cfg([(4, 2), (8, 1)], p=0.3)
    m = pkg.create_model(cfg)
    for level, N in ((0, 4), (1, 8)):
        got = m.vacancy_masks(N, level, w["seed"], 5, 6)
        for s in range(6):
            assert np.array_equal(got[s], otmdc.pair_mask(prm, N, level, 5 + s, w["seed"]))
    m.close()


@pytest.mark.parametrize("N", [1, 2, 3])
def test_hamiltonian_entries(N):
    import paper_1611_09784_gb300 as pkg
    w, cfg, prm = _cfg([(N, 2)])
    m = pkg.create_model(cfg)
    rng = np.random.default_rng(N)
    mask = (rng.random(N * N) < 0.4).astype(np.uint8)
    ks = lattice.kpoints(N, 2, prm["a"])
    for ki in range(4):
        H = m.hamiltonian(N, 2, ki, mask)
        ref = otmdc.hamiltonian(N, ks[ki], mask, prm)
        assert np.max(np.abs(H - ref)) < 1e-12
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,K", [(1, 3), (2, 2), (4, 2)])
def test_sample_idos_and_eigenvalues(N, K, precision):
    import paper_1611_09784_gb300 as pkg
    w, cfg, prm = _cfg([(N, K)], precision=precision)
    m = pkg.create_model(cfg)
    for sample in range(2):
        mask = otmdc.pair_mask(prm, N, 0, sample, w["seed"])
        Q, E = m.eval_idos(N, K, mask=None, seed=w["seed"], level=0, sample=sample, want_eigs=True)
        E_ref = otmdc.band_energies(N, K, mask, prm)
        for kk in range(K * K):
            got = np.sort(E[kk][~np.isnan(E[kk])])
            assert got.shape == E_ref[kk].shape
            assert np.max(np.abs(got - E_ref[kk])) < EIG_TOL
        Q_ref = otmdc.sample_idos(N, K, mask, prm)
        err = np.max(np.abs(Q - Q_ref))
        print(f"tmdc N={N} K={K} {precision} sample {sample}: max|dQ| = {err:.3e}, "
              f"max|dE| = {max(np.max(np.abs(np.sort(E[k][~np.isnan(E[k])]) - E_ref[k])) for k in range(K * K)):.3e}")
        assert err < IDOS_TOL
    m.close()


def test_level_coupling_matches_oracle():
    import paper_1611_09784_gb300 as pkg
    levels = [(4, 2), (8, 1)]
    w, cfg, prm = _cfg(levels)
    m = pkg.create_model(cfg)
    Y, Qf, Qc = m.sample_level_detail(1, 2, w["seed"], 3)
    for s in range(2):
        fine = otmdc.pair_mask(prm, 8, 1, 3 + s, w["seed"])
        qf = otmdc.sample_idos(8, 1, fine, prm)
        qc = [otmdc.sample_idos(4, 2, c, prm) for c in otmdc.corner_masks(fine, 8)]
        assert np.max(np.abs(Qf[s] - qf)) < IDOS_TOL
        for r in range(4):
            assert np.max(np.abs(Qc[s][r] - qc[r])) < IDOS_TOL
        assert np.max(np.abs(Y[s] - (qf - 0.25 * sum(qc)))) < 2 * IDOS_TOL
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_sample_n2816(precision):
    import paper_1611_09784_gb300 as pkg
    w, cfg, prm = _cfg([(16, 1)], precision=precision)
    m = pkg.create_model(cfg)
    mask = otmdc.pair_mask(prm, 16, 0, 0, w["seed"])
    Q, E = m.eval_idos(16, 1, mask=None, seed=w["seed"], level=0, sample=0, want_eigs=True)
    E_ref = otmdc.band_energies(16, 1, mask, prm)
    got = np.sort(E[0][~np.isnan(E[0])])
    assert got.shape == E_ref[0].shape
    assert np.max(np.abs(got - E_ref[0])) < EIG_TOL
    assert np.max(np.abs(Q - otmdc.sample_idos(16, 1, mask, prm))) < IDOS_TOL
    m.close()
