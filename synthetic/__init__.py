"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

This package holds workload parameters (model constants, supercell sizes,
k-grid sides, energy grids, vacancy probabilities, seeds and sample ranges)
and seeded random Hermitian / tridiagonal matrices for eigensolver parity.  It
contains none of the method's arithmetic: vacancy patterns and model
parameters are drawn inside each implementation by the counter-based
generator, from the seeds given here.
"""
from .workloads import (BASE_SEED, GRAPHENE, TMDC, WORKLOADS, workload, model_params)  # noqa: F401
