"""Workload definitions (sizes, parameters, seeds) for the synthetic inputs.

graphene_plain_mc   plain Monte Carlo, graphene N = 4 (n = 32), p = 0.05,
                    6x6 Monkhorst-Pack grid, 1000 samples, 201 energies on
                    [-9, 9] eV, delta = 0.1 eV, float64 throughout.
graphene_mlmc       four MLMC levels N = 4, 8, 16, 32 (n = 32 ... 2048), k-grid
                    sides 6, 3, 2, 1 (K_side^2 N^2 close to 576 from above),
                    p = 0.05, TOL = 1e-3 states/A^2, float32 reduction with
                    float64 refinement / statistics.
tmdc_sweep          11-orbital TMDC-shaped model, N = 4, 8, 12, 16
                    (n = 176 ... 2816), 4x4 grid, chalcogen-pair vacancies with
                    p = 0.05, 401 energies on [-6, 6] eV, delta = 0.05 eV.
graphene_stress     graphene N = 64 (n = 8192), p = 0.02, 2x2 grid, 128 samples.
"""
from __future__ import annotations

import copy

BASE_SEED = 161109784

GRAPHENE = {"kind": "graphene", "t": -2.7, "eps_onsite": 0.0, "a": 2.46, "sentinel": 1.0e3}
TMDC = {"kind": "tmdc", "t": 0.0, "eps_onsite": 0.0, "a": 3.19, "sentinel": 1.0e3,
        "model_seed": 20150921, "param_lo": -2.0, "param_hi": 2.0}

WORKLOADS = {
    "graphene_plain_mc": {
        "model": GRAPHENE, "p": 0.05, "levels": [(4, 6)], "samples": [1000],
        "e_min": -9.0, "e_max": 9.0, "n_E": 201, "delta": 0.1,
        "smoothing": "gauss", "precision": "fp64", "seed": BASE_SEED,
    },
    "graphene_mlmc": {
        "model": GRAPHENE, "p": 0.05, "levels": [(4, 6), (8, 3), (16, 2), (32, 1)],
        "tol": 1.0e-3, "theta": 0.5, "c_alpha": 1.96,
        "e_min": -9.0, "e_max": 9.0, "n_E": 201, "delta": 0.1,
        "smoothing": "gauss", "precision": "fp32", "seed": BASE_SEED,
    },
    "tmdc_sweep": {
        "model": TMDC, "p": 0.05, "sizes": [4, 8, 12, 16], "K": 4, "samples_per_size": 32,
        "e_min": -6.0, "e_max": 6.0, "n_E": 401, "delta": 0.05,
        "smoothing": "gauss", "precision": "fp32", "seed": BASE_SEED,
    },
    "graphene_stress": {
        "model": GRAPHENE, "p": 0.02, "levels": [(64, 2)], "samples": [128],
        "e_min": -9.0, "e_max": 9.0, "n_E": 201, "delta": 0.1,
        "smoothing": "gauss", "precision": "fp32", "seed": BASE_SEED,
    },
}


def workload(name: str) -> dict:
    return copy.deepcopy(WORKLOADS[name])


def model_params(w: dict) -> dict:
    """Flat parameter dict (model constants + energy grid + p) of a workload."""
    prm = dict(w["model"])
    for key in ("p", "e_min", "e_max", "n_E", "delta", "smoothing"):
        prm[key] = w[key]
    return prm
