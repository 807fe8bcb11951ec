"""Shared helpers of the GPU parity tests (model configs from the synthetic
workloads, the oracle's parameter dicts)."""
import numpy as np

from synthetic import GRAPHENE, model_params, workload

# Tolerances: vacancy masks bit-exact; eigenvalues 1e-4 eV; per-sample IDoS
# 1e-5 states/A^2 (absolute).
EIG_TOL = 1e-4
IDOS_TOL = 1e-5


def cfg_and_prm(name="graphene_mlmc", precision="fp32", refine=2, **over):
    w = workload(name)
    w.update(over)
    prm = model_params(w)
    cfg = dict(w["model"])
    cfg.update(p=w["p"], levels=w["levels"], e_min=w["e_min"], e_max=w["e_max"], n_E=w["n_E"],
               delta=w["delta"], smoothing=w["smoothing"], precision=precision, refine64_iters=refine)
    return w, cfg, prm


def graphene_prm(**over):
    d = dict(GRAPHENE)
    d.update(p=0.05, e_min=-9.0, e_max=9.0, n_E=201, delta=0.1, smoothing="gauss")
    d.update(over)
    return d


def sorted_active(E):
    """Rows of GPU eigenvalues with the NaN padding removed."""
    return [np.sort(row[~np.isnan(row)]) for row in E]
