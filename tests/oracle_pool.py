"""A spawn-started process pool running oracle level samples with one BLAS
thread per process (the GPU tests' way to run many oracle samples; spawn, so
that no worker is forked from a process holding a CUDA context)."""
import os

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")


def level_y(args):
    from oracle import mlmc
    prm, levels, level, sample, seed = args
    return level, sample, mlmc.level_sample(prm, levels, level, sample, seed)["Y"]


def pool():
    import multiprocessing as mp
    # the workers inherit the environment at spawn: one BLAS thread each
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return mp.get_context("spawn").Pool(max(1, n))
