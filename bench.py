"""Benchmark: MLMC estimate of the expected IDoS of graphene with vacancies
(levels N = 4, 8, 16, 32; TOL = 1e-3 states/A^2) on GB300.

One step = one pass of the whole path over the workload's fixed per-level
sample allocation M_l (tests/golden/mlmc_allocation_graphene.json, written by
an oracle-only script from eq. (2.7)): vacancy masks, corner slicing, H(k)
assembly, Householder reduction, Sturm bisection, smoothed IDoS, level
differences and float64 statistics on the device, then the eq. (2.6) combine
on the host.  Metric: eigen-solves per second (higher is better).

Also reported: `e2e` (the adaptive public call idos_mlmc_estimate(TOL) with
host outputs, wall clock, aggregated over 16 seeds), time-to-TOL of MLMC vs plain MC at the finest level
on the same GPU, per-kernel CUDA-event times, the roofline of the dominant
kernel, the oracle timed on the host cores (`cpu_baseline`), and SM clocks
sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU: replicas only (weak scaling), each rank draws disjoint samples.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALLOC_FILE = os.path.join(ROOT, "tests", "golden", "mlmc_allocation_graphene.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
WORKLOAD = "graphene_mlmc"
METRIC = "eigsolves/s (MLMC IDoS estimate, TOL=1e-3)"
UNIT = "eigsolves/s"
REFINE64 = 1
TC_PRODUCTS = 6   # split-bf16 products of the tensor-core trailing update
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20
E2E_CALLS = 16    # seeded adaptive estimates behind the e2e value (at least --steps)


# ------------------------------------------------------------------ helpers --
def load_alloc():
    with open(ALLOC_FILE) as f:
        return json.load(f)


def eigsolves_per_sample(levels, level):
    N, K = levels[level]
    n = K * K
    if level > 0:
        n += 4 * levels[level - 1][1] ** 2
    return n


def workload_config(alloc, w, precision=None):
    return {"workload": WORKLOAD, "model": "graphene pz NN tight-binding, t=-2.7 eV, a=2.46 A",
            "p": w["p"], "levels_N_K": w["levels"], "samples_per_level": alloc["M"], "tol": w["tol"],
            "n_E": w["n_E"], "delta": w["delta"],
            "precision": precision or f"fp32 reduction + {REFINE64} fp64 Newton/Sturm pass, fp64 sums",
            "l2": "flushed (256 MiB write) between timed steps", "parallelism": "replicas"}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash(name):
    path = os.path.join(ROOT, "paper_1611_09784_gb300", "csrc", name)
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic(kernel, algorithmic_per_launch):
    """DRAM bytes per launch of `kernel`: the committed ncu capture's DRAM bytes
    per algorithmic unit (flop or byte) times this run's algorithmic units per
    launch; None when there is no capture or the kernel's source file changed
    since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            for ln in f:
                if ln.startswith("#") or not ln.strip():
                    continue
                k, src, h, ratio = ln.split()[:4]
                if k == kernel and kernel_source_hash(src) == h:
                    return float(ratio) * algorithmic_per_launch
    except Exception:
        pass
    return None


# --------------------------------------------------------- algorithmic work --
def n_act_of(masks, N, sublattice=False):
    """Kept-site counts of the fine cells and of their 4 corners (site index
    m = 2(i + N j) + s, corner r = ri + 2 rj); with `sublattice`, the counts
    per sublattice s (last axis of 2)."""
    import numpy as np
    S = masks.shape[0]
    keep = 1 - masks.reshape(S, N, N, 2)
    fine = keep.reshape(S, -1, 2).sum(1) if sublattice else keep.reshape(S, -1).sum(1)
    h = N // 2
    corners = []
    for r in range(4):
        ri, rj = r % 2, r // 2
        blk = keep[:, rj * h:(rj + 1) * h, ri * h:(ri + 1) * h, :]
        corners.append(blk.reshape(S, -1, 2).sum(1) if sublattice else blk.reshape(S, -1).sum(1))
    return fine, np.stack(corners, 1)


def gk_flops(nAB):
    """Real flops of the Golub-Kahan bidiagonalisation of graphene's q x p
    sublattice block (p = min(n_A, n_B), q = max) as the kernels do it:
    per left reflector j the dot and the update over rows j .. q-1 of columns
    j+1 .. p-1, per right reflector the row products and the update over rows
    j+1 .. q-1 of the same columns, 8 flops per complex multiply-add."""
    import numpy as np
    nAB = np.asarray(nAB).reshape(-1, 2)
    total = 0.0
    pairs, counts = np.unique(np.sort(nAB, axis=1), axis=0, return_counts=True)
    for (p, q), c in zip(pairs, counts):
        j = np.arange(int(p), dtype=np.float64)
        total += c * float(np.sum(16.0 * ((q - j) * (p - 1 - j) + (q - 1 - j) * (p - 1 - j))))
    return total


# Kernel families of the library's profiler and what bounds each one:
# "alu" (float32 FMA issue), "alu64" (float64 FMA issue), "tensor" (bf16 MMA),
# "hbm" (DRAM bytes).  W runs on the FP32 pipe unless the autotuner picked the
# tensor-core W (w_tile 2).
FAMILIES = {"k_small_tridiag": "alu", "k_ts_panel": "alu", "k_ts_w": "tensor", "k_ts_z": "hbm", "k_ts_her2k": "tensor",
            "k_ts_chase": "alu", "k_bisect": "alu64", "k_idos": "hbm"}


def algorithmic_work(m, levels, M, seed, firsts, refine=REFINE64, n_E=201, bw=16):
    """Exact algorithmic work of one step from the samples' kept-site counts,
    per kernel family (flops, or bytes for the HBM-bound families):
    - k_small_tridiag: graphene n <= 128: the Golub-Kahan bidiagonalisation
      of the sublattice block (gk_flops); otherwise the Householder
      tridiagonal reduction, 16/3 n^3 real flops per matrix;
    - per stage-1 panel of bw columns with m rows below it (float32 complex,
      8 bytes per entry): panel QR 8 m bw^2 flops, W = A22 (Y T) 8 m^2 bw
      flops, Z = W - 1/2 Y (T^H M) 4 bw m x 8 bytes (W and Y twice read, Z
      written once), the rank-2bw update 16 m^2 bw flops;
    - k_ts_chase: per sweep step the right and left reflector applications to
      the bw x bw bulge block (2 x 8 bw^2) and the two-sided update of the
      bw x bw diagonal block (3 x 8 bw^2);
    - k_bisect: the float64 refinement passes, 4 flops per row of the
      characteristic-polynomial recurrence, refine x n^2 rows per matrix;
    - k_idos: the eigenvalues read (8 bytes each) and Q written (8 n_E bytes
      per cell)."""
    import numpy as np
    work = {k: 0.0 for k in FAMILIES}

    def add(n_ab, K2, big, n_sites):
        n_arr = n_ab.sum(-1)
        n = n_arr.astype(np.float64)
        work["k_bisect"] += K2 * float(np.sum(4.0 * refine * n ** 2))
        work["k_idos"] += float(np.sum(8.0 * K2 * n + 8.0 * n_E))
        if not big:
            if n_sites <= 128:
                work["k_small_tridiag"] += K2 * gk_flops(n_ab)
            else:
                work["k_small_tridiag"] += K2 * float(np.sum(16.0 / 3.0 * n ** 3))
            return
        for nn in n_arr:
            nn = int(nn)
            for k in range(0, nn - bw, bw):
                mm = nn - k - bw
                work["k_ts_panel"] += K2 * 8.0 * mm * bw * bw
                work["k_ts_w"] += K2 * 8.0 * bw * mm * mm
                work["k_ts_z"] += K2 * 4.0 * bw * mm * 8.0
                work["k_ts_her2k"] += K2 * 16.0 * bw * mm * mm
            steps = sum((nn - 2 - i) // bw + 1 for i in range(0, nn - 2))
            work["k_ts_chase"] += K2 * 40.0 * bw * bw * steps
    for l, (N, K) in enumerate(levels):
        if not M[l]:
            continue
        masks = m.vacancy_masks(N, l, seed, firsts[l], M[l])
        fine, corners = n_act_of(masks, N, sublattice=True)
        add(fine, K * K, 2 * N * N > 160, 2 * N * N)
        if l > 0:
            Kc = levels[l - 1][1]
            add(corners.reshape(-1, 2), Kc * Kc, 2 * (N // 2) ** 2 > 160, 2 * (N // 2) ** 2)
    return work


AGGREGATE_SCOPES = ("k_lg_band (stage 1, all)",)


def roofline(prof, work, steps, pk, pk_kind, fma, tc_products=6, w_tile=1):
    """Roofline objects of the kernel families; the first is the single kernel
    family (not an aggregate scope) with the largest event time.  fma: the
    FMA peaks measured in this run (TFLOP/s, float32 and float64); w_tile: the
    W kernel the run used (2 = tensor cores, six products whatever
    tc_products)."""
    singles = sorted(((k, v) for k, v in prof.items() if k not in AGGREGATE_SCOPES), key=lambda kv: -kv[1][0])
    out = []
    for name, (ms, launches) in singles:
        bound = FAMILIES.get(name)
        if bound is None or not launches or not ms:
            continue
        if bound == "tensor" and (not tc_products or (name == "k_ts_w" and w_tile != 2)):
            bound = "alu"
        per_launch_s = ms * 1e-3 / launches
        units_per_launch = work[name] * steps / launches
        executed = units_per_launch
        if bound == "tensor":
            # the trailing update and W run on the tensor cores: split-bf16 MMA
            # flops per algorithmic flop (tc_products for the update, six for
            # W), against the measured bf16 GEMM rate (sustained: the kernels
            # are timed inside a long replay)
            nprod = 6 if name == "k_ts_w" else tc_products
            executed = units_per_launch * nprod
            achieved, unit = executed / per_launch_s / 1e12, "TFLOP/s"
            peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))
            src = f"{pk_kind} bf16 GEMM, sustained; achieved counts the {nprod} split-bf16 products per algorithmic flop"
        elif bound == "hbm":
            achieved, unit = units_per_launch / per_launch_s / 1e9, "GB/s"
            peak = pk.get("hbm_gbs", 6800.0)
            src = f"{pk_kind} HBM copy bandwidth"
        elif bound == "alu64":
            achieved, unit = units_per_launch / per_launch_s / 1e12, "TFLOP/s"
            peak = fma["fp64_tflops"]
            src = "measured in this run: float64 FMA microbenchmark (idos_measure_fma_peak)"
        else:
            achieved, unit = units_per_launch / per_launch_s / 1e12, "TFLOP/s"
            peak = fma["fp32_tflops"]
            src = "measured in this run: float32 FMA microbenchmark (idos_measure_fma_peak)"
        out.append({"kernel": name, "bound": "alu" if bound == "alu64" else bound,
                    "pipe": {"alu": "fp32", "alu64": "fp64", "tensor": "bf16 mma", "hbm": "dram"}[bound],
                    "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                    # (the committed capture is of the FP32-pipe W)
                    "traffic": None if (name == "k_ts_w" and bound == "tensor") else ncu_traffic(name, units_per_launch),
                    "algorithmic_per_launch": units_per_launch, "executed_per_launch": executed,
                    "launches": launches, "avg_launch_ms": per_launch_s * 1e3, "peak_source": src})
    dominant = singles[0][0] if singles else None
    first = next((r for r in out if r["kernel"] == dominant), out[0] if out else None)
    if first is not None:
        first = dict(first, dominant_by_event_time=dominant)
    return first, out


def measure_fma_peaks(pkg, stream, clock_gpu=0):
    """FMA issue rates of this GPU (float32, float64) with the SM clock
    sampled meanwhile; each launch runs for a few hundred milliseconds."""
    clocks = ClockSampler(clock_gpu)
    clocks.start()
    f32, ms32 = pkg.measure_fma_peak("fp32", 1 << 21, stream)
    f64, ms64 = pkg.measure_fma_peak("fp64", 1 << 15, stream)
    clk = clocks.stop()
    out = {"fp32_tflops": f32 / 1e12, "fp64_tflops": f64 / 1e12, "fp32_ms": ms32, "fp64_ms": ms64,
           "kernel": "k_fma_peak: 8 CTAs x 256 threads per SM, 8 independent FMA chains per thread",
           "clocks": clk}
    if clk:
        out["fp32_tflops_per_ghz"] = out["fp32_tflops"] / (clk["sm_mhz"] / 1e3)
    return out


# ------------------------------------------------------------- oracle (CPU) --
def _oracle_job(args):
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle import mlmc as omlmc
    from synthetic import model_params, workload
    level, sample, seed = args
    w = workload(WORKLOAD)
    prm = model_params(w)
    t0 = time.perf_counter()
    omlmc.level_sample(prm, w["levels"], level, sample, seed)
    return level, time.perf_counter() - t0


def _oracle_check_job(args):
    """The oracle's level sample (Y, Q_fine, Q_coarse) and, when asked, the
    fine cell's band energies, for the GPU-vs-oracle check of the bench line."""
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    from oracle import idos as oidos
    from oracle import mlmc as omlmc
    from synthetic import model_params, workload
    level, sample, seed, want_bands = args
    w = workload(WORKLOAD)
    prm = model_params(w)
    r = omlmc.level_sample(prm, w["levels"], level, sample, seed)
    out = {"level": level, "sample": sample, "Y": r["Y"], "Q_fine": r["Q_fine"], "Q_coarse": r["Q_coarse"]}
    if want_bands:
        N, K = w["levels"][level]
        out["E"] = oidos.band_energies(N, K, r["mask"], prm)
    return out


def oracle_pool():
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return mp.get_context("spawn").Pool(cores), cores


def oracle_sample_counts(alloc, frac=1.0 / 16):
    return [max(1, int(math.ceil(Ml * frac))) for Ml in alloc["M"]]


def oracle_measure(pool, cores, alloc, levels, frac=1.0 / 16, first=50_000_000, seed=161109784):
    """Time the oracle (float64, LAPACK eigvalsh) on a bounded, workload-shaped
    sample: ceil(M_l / 16) level samples of every level (at least one), run on
    all host cores (one process per core, BLAS single-threaded).  value =
    eigen-solves of the sample / its wall time; nothing is extrapolated."""
    counts = oracle_sample_counts(alloc, frac)
    jobs = [(l, first + s, seed) for l in range(len(counts)) for s in range(counts[l])]
    jobs.sort(key=lambda j: -j[0])
    t0 = time.perf_counter()
    res = pool.map(_oracle_job, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    per = [[] for _ in counts]
    for l, t in res:
        per[l].append(t)
    mean = [sum(x) / len(x) for x in per]
    eig = sum(c * eigsolves_per_sample(levels, l) for l, c in enumerate(counts))
    return {"value": eig / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{counts} level samples of levels 0..3 (1/16 of the allocation {alloc['M']}, at least one "
                       f"per level; {eig} eigen-solves) on {cores} host processes, 1 BLAS thread each, "
                       f"{wall:.1f} s wall; value = those eigen-solves / that wall time (measured, not extrapolated)"),
            "wall_s": wall, "eigsolves": eig, "per_level_mean_core_s": [round(x, 4) for x in mean]}


def gpu_oracle_check(model, levels, seed, counts=(4, 2, 2, 1), first=90_000_000):
    """GPU side of the oracle check at the bench's settings: per level the
    level samples (Y, Q_fine, Q_coarse) and the first sample's fine-cell
    eigenvalues (NaN-padded rows)."""
    out = []
    for l, c in enumerate(counts):
        Y, Qf, Qc = model.sample_level_detail(l, c, seed, first)
        N, K = levels[l]
        _, E = model.eval_idos(N, K, seed=seed, level=l, sample=first, want_eigs=True)
        out.append({"Y": Y, "Q_fine": Qf, "Q_coarse": Qc, "E": E})
    return out


def oracle_check_jobs(seed, counts=(4, 2, 2, 1), first=90_000_000):
    return [(l, first + s, seed, s == 0) for l in range(len(counts)) for s in range(counts[l])]


def compare_oracle_check(gpu, oracle_res, counts=(4, 2, 2, 1), first=90_000_000):
    """Max absolute differences GPU - oracle per level: Y, Q_fine, Q_coarse
    (states/A^2) and eigenvalues (eV, the first sample's fine cell, as sorted
    multisets per grid point)."""
    import numpy as np
    by = {(r["level"], r["sample"]): r for r in oracle_res}
    per_level = []
    for l, c in enumerate(counts):
        g = gpu[l]
        dY = dQ = dC = 0.0
        for s in range(c):
            r = by[(l, first + s)]
            dY = max(dY, float(np.max(np.abs(g["Y"][s] - r["Y"]))))
            dQ = max(dQ, float(np.max(np.abs(g["Q_fine"][s] - r["Q_fine"]))))
            if l > 0:
                dC = max(dC, float(np.max(np.abs(g["Q_coarse"][s] - np.stack(r["Q_coarse"])))))
        Eo = by[(l, first)]["E"]
        dE = 0.0
        for row, ref in zip(g["E"], Eo):
            act = np.sort(row[~np.isnan(row)])
            if act.shape != ref.shape:
                dE = float("inf")
                break
            dE = max(dE, float(np.max(np.abs(act - ref))) if ref.size else 0.0)
        per_level.append({"level": l, "samples": c, "max_abs_dY": dY, "max_abs_dQ_fine": dQ,
                          "max_abs_dQ_coarse": dC, "max_abs_dE_eV": dE})
    worst_q = max(max(p["max_abs_dY"], p["max_abs_dQ_fine"], p["max_abs_dQ_coarse"]) for p in per_level)
    worst_e = max(p["max_abs_dE_eV"] for p in per_level)
    return {"per_level": per_level, "max_abs_dQ": worst_q, "max_abs_dE_eV": worst_e,
            "tolerance": {"Q": 1e-5, "E_eV": 1e-4}, "pass": bool(worst_q < 1e-5 and worst_e < 1e-4),
            "what": ("GPU (bench settings: float32 reduction, tensor-core update with 6 split-bf16 products, "
                     f"{REFINE64} float64 pass) against the float64 oracle on the same seeded samples "
                     f"{first}.. of every level, computed outside the timed region")}


def level_cost_model(levels, l):
    """Flop-model work of one level-l sample: sum of n^3 over its eigen-solves
    (fine cell at K_l^2 points, the four corners at K_{l-1}^2 points)."""
    N, K = levels[l]
    c = K * K * float(2 * N * N) ** 3
    if l > 0:
        Nc, Kc = levels[l - 1]
        c += 4 * Kc * Kc * float(2 * Nc * Nc) ** 3
    return c


# ------------------------------------------------ other workloads (extras) --
def tmdc_sweep(pkg, torch, stream, samples=(32, 32, 32, 8)):
    """TMDC-shaped 11-orbital model, N = 4, 8, 12, 16 (n = 176 .. 2816), 4 x 4
    grid, float32 reduction + one float64 refinement pass: eigen-solves/s of
    one sample_level call per size (CUDA events on the model stream)."""
    from synthetic import workload
    w = workload("tmdc_sweep")
    out = []
    for N, S in zip(w["sizes"], samples):
        cfg = dict(w["model"], p=w["p"], levels=[(N, w["K"])], e_min=w["e_min"], e_max=w["e_max"], n_E=w["n_E"],
                   delta=w["delta"], smoothing=w["smoothing"], precision="fp32", refine64_iters=REFINE64,
                   tc_products=TC_PRODUCTS)
        m = pkg.create_model(cfg, stream=stream.cuda_stream)
        m.sample_level(0, 1, w["seed"] + 1, 0)          # warm-up (workspace, first launches)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        m.sample_level(0, S, w["seed"], 0)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out.append({"N": N, "n": 11 * N * N, "K": w["K"], "samples": S, "ms": round(ms, 2),
                    "eigsolves_per_s": S * w["K"] ** 2 / (ms * 1e-3)})
        m.close()
    return out


def stress(pkg, torch, stream, samples=2, fp64_check=True):
    """Graphene N = 64 (n = 8192), p = 0.02, 2 x 2 grid: `samples` samples
    (4 solves each) on the float32 path with the tensor-core trailing update
    (CUDA events), the tensor-core update's achieved MMA rate from a profiled
    replay of the same call, and the eigenvalue difference to the float64 GPU
    path on one grid point of sample 0 (K = 1 model, same mask)."""
    import numpy as np
    from synthetic import workload
    w = workload("graphene_stress")
    base = dict(w["model"], p=w["p"], e_min=w["e_min"], e_max=w["e_max"], n_E=w["n_E"], delta=w["delta"],
                smoothing=w["smoothing"], refine64_iters=REFINE64, tc_products=TC_PRODUCTS)
    m = pkg.create_model(dict(base, levels=w["levels"], precision="fp32"), stream=stream.cuda_stream)
    m.sample_level(0, 1, w["seed"] + 1, 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    m.sample_level(0, samples, w["seed"], 0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    m.reset_profile()
    m.set_profiling(True)
    m.sample_level(0, 1, w["seed"], 0)
    m.set_profiling(False)
    prof = m.get_profile()
    m.close()
    out = {"N": 64, "n": 8192, "K": 2, "samples": samples, "of_samples": 128, "ms": round(ms, 1),
           "eigsolves_per_s": samples * 4 / (ms * 1e-3),
           "precision": f"fp32 reduction, tensor-core trailing update ({TC_PRODUCTS} split-bf16 products), "
                        f"{REFINE64} fp64 pass",
           "kernels_ms_per_sample": {k: round(v[0], 2) for k, v in prof.items()}}
    # executed MMA flops of the trailing update of one n = 8192 matrix (x 4
    # grid points): tc_products x 16 bw m^2 per panel
    n, bw = 8192, 16
    flops = 4 * TC_PRODUCTS * sum(16.0 * bw * (n - k - bw) ** 2 for k in range(0, n - bw, bw))
    if "k_ts_her2k" in prof and prof["k_ts_her2k"][0] > 0:
        out["tensor_core_update_tflops"] = flops / (prof["k_ts_her2k"][0] * 1e-3) / 1e12
    if fp64_check:
        # eigenvalues of one grid point on both paths (K = 1: the zone centre
        # of the Monkhorst-Pack grid), same mask
        w1 = dict(base, levels=[(64, 1)])
        m32 = pkg.create_model(dict(w1, precision="fp32"), stream=stream.cuda_stream)
        _, E32 = m32.eval_idos(64, 1, seed=w["seed"], level=0, sample=0, want_eigs=True)
        m32.close()
        m64 = pkg.create_model(dict(w1, precision="fp64", refine64_iters=2), stream=stream.cuda_stream)
        t0 = time.perf_counter()
        _, E64 = m64.eval_idos(64, 1, seed=w["seed"], level=0, sample=0, want_eigs=True)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        m64.close()
        a32 = np.sort(E32[0][~np.isnan(E32[0])])
        a64 = np.sort(E64[0][~np.isnan(E64[0])])
        out["fp32_vs_fp64_gpu"] = {"max_abs_dE_eV": float(np.max(np.abs(a32 - a64))), "n_act": int(a32.size),
                                   "fp64_seconds_one_solve": t64, "what": "one n = 8192 matrix (sample 0, K = 1)"}
    return out


def fp64_paths(pkg, torch, stream, cfg, levels, M, seed):
    """The float64 GPU path (the paper's own precision): config 1, plain Monte
    Carlo, graphene N = 4, 6 x 6 grid, 1000 samples (36 000 eigen-solves), and
    one step of the MLMC allocation on the float64 path; CUDA events on the
    model stream."""
    from synthetic import workload
    out = {}
    w1 = workload("graphene_plain_mc")
    c1 = dict(w1["model"], p=w1["p"], levels=w1["levels"], e_min=w1["e_min"], e_max=w1["e_max"], n_E=w1["n_E"],
              delta=w1["delta"], smoothing=w1["smoothing"], precision="fp64", refine64_iters=2)
    m = pkg.create_model(c1, stream=stream.cuda_stream)
    m.sample_level(0, 8, w1["seed"] + 1, 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    m.sample_level(0, w1["samples"][0], w1["seed"], 0)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    m.close()
    N, K = w1["levels"][0]
    solves = w1["samples"][0] * K * K
    out["config1_plain_mc_fp64"] = {"N": N, "K": K, "samples": w1["samples"][0], "eigsolves": solves, "ms": round(ms, 2),
                                    "eigsolves_per_s": solves / (ms * 1e-3)}
    m = pkg.create_model(dict(cfg, precision="fp64", refine64_iters=2, sm_split=-1, graph=-1), stream=stream.cuda_stream)
    m.sample_levels([1] * len(M), seed + 3, [10 ** 9] * len(M))
    torch.cuda.synchronize()
    e0.record(stream)
    m.sample_levels(M, seed + 3, [0] * len(M))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    m.close()
    eig = sum(Ml * eigsolves_per_sample(levels, l) for l, Ml in enumerate(M))
    out["config2_mlmc_fp64_step"] = {"samples_per_level": M, "ms": round(ms, 1), "eigsolves_per_s": eig / (ms * 1e-3),
                                     "precision": "fp64 reduction, bisection and 2 fp64 passes"}
    return out


def serving_trace(rng, rate, n_req, bmax, probs):
    import numpy as np
    gaps = rng.exponential(1.0 / rate, n_req)
    lv = rng.choice(len(probs), size=n_req, p=probs)
    nb = [int(round(math.exp(rng.uniform(0.0, math.log(bmax[l]))))) for l in lv]
    return np.cumsum(gaps), lv, nb


def serve_trace(pkg, cfg, arrive, lv, nb, seed, workers):
    """Replays one arrival trace through the request loop; latency =
    submission to completion (library clock)."""
    import numpy as np
    srv = pkg.Server(dict(cfg, sm_split=0), n_workers=workers)
    for l in sorted(set(int(x) for x in lv)):            # warm-up: workspaces, first launches
        srv.wait(srv.submit(l, 1, seed + 5, 0))
    t0 = time.perf_counter()
    tickets = []
    for i in range(len(lv)):
        dt = t0 + arrive[i] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append(srv.submit(int(lv[i]), nb[i], seed, 1_000_000 + 10_000 * i))
    lat = [srv.wait(t)[2] for t in tickets]
    elapsed = time.perf_counter() - t0
    srv.close()
    return {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "wall_s": elapsed}, elapsed


def serving(pkg, cfg, levels, seed, rates=(10.0, 30.0, 100.0, 300.0, 1000.0, 2000.0), trace_seed=7):
    """The request loop under Poisson arrivals of level requests like the ones
    the adaptive driver emits, for both models: graphene levels N = 4 ... 32
    (probability 0.4, 0.3, 0.2, 0.1; batch log-uniform in [1, 512, 512, 32, 4]
    samples) and the TMDC-shaped model at N = 4, 8, 16 (n = 176, 704, 2816;
    0.5, 0.35, 0.15; batch up to 64, 8, 1).  Every trace is served by 4 worker
    streams (concurrent) and by 1 (one request at a time).  Requests per trace:
    about 2 s of arrivals, 20 to 120.  Throughput = eigen-solves / (last
    completion - first arrival)."""
    import numpy as np
    from synthetic import workload
    rng = np.random.default_rng(trace_seed)
    wt = workload("tmdc_sweep")
    tm_levels = [(4, wt["K"]), (8, wt["K"]), (16, wt["K"])]
    tm_cfg = dict(wt["model"], p=wt["p"], levels=tm_levels, e_min=wt["e_min"], e_max=wt["e_max"], n_E=wt["n_E"],
                  delta=wt["delta"], smoothing=wt["smoothing"], precision="fp32", refine64_iters=REFINE64,
                  tc_products=TC_PRODUCTS)
    models = {"graphene": (cfg, levels, [512, 512, 32, 4], [0.4, 0.3, 0.2, 0.1]),
              "tmdc": (tm_cfg, tm_levels, [64, 8, 1], [0.5, 0.35, 0.15])}
    out = []
    for name, (mcfg, mlev, bmax, probs) in models.items():
        for rate in rates:
            n_req = int(min(120, max(20, 2 * rate)))
            arrive, lv, nb = serving_trace(rng, rate, n_req, bmax, probs)
            eig = sum(n * eigsolves_per_sample(mlev, int(l)) for l, n in zip(lv, nb))
            row = {"model": name, "rate_per_s": rate, "requests": n_req, "eigsolves": int(eig)}
            for workers in (4, 1):
                r, elapsed = serve_trace(pkg, mcfg, arrive, lv, nb, seed, workers)
                r["eigsolves_per_s"] = eig / elapsed
                row["concurrent_4" if workers == 4 else "one_at_a_time"] = r
            out.append(row)
    return out


# ------------------------------------------------------------------- GPU arm --
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pool = cores = None
    if rank == 0 and world == 1 and not args.skip_extras:
        pool, cores = oracle_pool()     # spawn pool before the first GPU call
    if world > 1:
        dist.init_process_group("nccl", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1611_09784_gb300 as pkg
    from synthetic import workload

    w = workload(WORKLOAD)
    alloc = load_alloc()
    levels = [tuple(x) for x in w["levels"]]
    M = list(alloc["M"])
    if args.levels is not None:
        keep = {int(x) for x in args.levels.split(",")}
        M = [Ml if l in keep else 0 for l, Ml in enumerate(M)]
    stream = torch.cuda.Stream(device=dev)
    cfg = dict(w["model"], p=w["p"], levels=levels, e_min=w["e_min"], e_max=w["e_max"], n_E=w["n_E"],
               delta=w["delta"], smoothing=w["smoothing"], precision="fp32", refine64_iters=REFINE64,
               tc_products=TC_PRODUCTS, sm_split=args.sm_split, graph=args.graph)
    model = pkg.create_model(cfg, stream=stream.cuda_stream)
    seed = w["seed"] + 1000 * rank
    eig_step = sum(Ml * eigsolves_per_sample(levels, l) for l, Ml in enumerate(M))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # the project's autotuner picks the SM partition and the small/two-stage
    # cutoff for this allocation (timed on sample indices outside the run's)
    tuning = model.autotune(M, reps=1) if args.sm_split < 0 else {"fixed_sm_split": args.sm_split}

    def step(idx):
        # every level of the allocation at once (concurrent level streams)
        model.sample_levels(M, seed, [idx * Ml for Ml in M])

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    model.reset_level_stats(-1)
    clocks = ClockSampler(local) if not args.no_clocks else None
    barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    evs = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(args.warmup + k)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    g_replays, g_captures, g_note = model.graph_info()
    graph_line = {"replays": g_replays, "captures": g_captures, "note": g_note,
                  "what": "idos_sample_levels captured once as a CUDA graph (all level streams), replayed per step"}
    # combine (eq. (2.6), idos_combine_level_stats) from the device
    # accumulators, summed over replicas
    from paper_1611_09784_gb300 import replicas
    counts, sums = replicas.model_stats(model)
    level_span_ms = [round(model.get_level_stats(l)[3] * 1e3 / args.steps, 3) for l in range(len(M))]
    # the four accumulator rows and their sample counts, read together (the
    # profiled replay below adds to the accumulators)
    mom = [model.get_level_moments(l) for l in range(len(M))]
    moments = np.stack([x[1] for x in mom])
    mom_counts = [x[0] for x in mom]
    if world > 1:
        counts, sums = replicas.merge(counts, sums, device=dev)
    mean, var = replicas.combine(counts, sums)
    # Per-kernel CUDA-event times: the timed steps run the levels on
    # concurrent streams, where one kernel's event span includes time spent
    # waiting for SMs held by kernels of other levels.  So the kernels are
    # timed on the same work (the timed steps' samples, the same launches)
    # replayed with profiling on, which issues them in order on one stream,
    # events on that stream around every launch.
    model.reset_profile()
    model.set_profiling(True)
    for k in range(args.steps):
        model.sample_levels(M, seed, [(args.warmup + k) * Ml for Ml in M])
    torch.cuda.synchronize()
    model.set_profiling(False)
    prof = model.get_profile()
    t_max = torch.tensor([total_ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    total_ms_max = float(t_max.item())
    value = world * args.steps * eig_step / (total_ms_max * 1e-3)

    # algorithmic work of the timed steps (exact kept-site counts)
    firsts_steps = [[(args.warmup + k) * Ml for Ml in M] for k in range(args.steps)]
    work = {}
    for firsts in firsts_steps:
        wk = algorithmic_work(model, levels, M, seed, firsts, n_E=w["n_E"])
        for k2 in wk:
            work[k2] = work.get(k2, 0.0) + wk[k2] / args.steps
    pk, pk_kind = peaks()
    fma = measure_fma_peaks(pkg, stream.cuda_stream, local)
    w_tile = tuning.get("w_tile", 1) if isinstance(tuning, dict) else 1
    roof, roofs = roofline(prof, work, args.steps, pk, pk_kind, fma, tc_products=TC_PRODUCTS, w_tile=w_tile)

    # rates W, S, D, C (Sec. 2.1-2.2, fitted as Sec. 4.4 does) from the timed
    # steps' level accumulators; cost per sample: each level alone on the
    # model stream (CUDA events), and the flop model sum n^3
    rates = None
    if all(M):
        Ns = [N for N, _ in levels]
        cnt = mom_counts
        cost_s = []
        for l in range(len(M)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            model.sample_level(l, M[l], seed + 7, 1 << 41)
            b.record(stream)
            torch.cuda.synchronize()
            cost_s.append(a.elapsed_time(b) * 1e-3 / M[l])
        flop = [level_cost_model(levels, l) for l in range(len(M))]
        rates = {"measured_gpu_cost": pkg.fit_rates(Ns, cnt, moments, cost_s),
                 "flop_model_cost": pkg.fit_rates(Ns, cnt, moments, flop),
                 "C_last_two_levels_gpu": math.log(cost_s[-1] / cost_s[-2]) / math.log(Ns[-1] / Ns[-2]),
                 "gpu_seconds_per_sample": cost_s, "samples_per_level": cnt,
                 "norm": "arithmetic mean over the energy grid",
                 "paper_printed": {"W": 1.5, "S": 2, "D": 3, "C": 4, "work_mc": 10 / 3, "work_mlmc": 8 / 3}}

    if args.skip_extras:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
                              "partial": "timed steps only (--skip-extras)", "samples_per_level": M,
                              "level_span_ms_per_step": level_span_ms,
                              "kernels_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in prof.items()},
                              "roofline": roof, "rooflines": roofs, "fma_peaks": fma, "rates": rates,
                              "clocks": clk, "graph": graph_line, "autotune": tuning}),
                  flush=True)
        model.close()
        if pool is not None:
            pool.close()
        return

    # ---- e2e: the public adaptive call, host outputs, wall clock ----
    # One model, set up once with the configuration the autotuner chose for
    # this allocation (as a user would keep it); one untimed call sizes its
    # workspaces; then each timed call is a whole estimate from zeroed level
    # statistics on fresh sample indices.  The samples an estimate needs vary
    # with its seed (about one seed in five needs a fifth finest sample, one
    # more n = 2048 chain), so the value is the aggregate over E2E_CALLS
    # seeds: all their eigen-solves over all their wall time.
    e2e_n, e2e_s, h2d, d2h, est = [], [], 0, 0, None
    model2 = pkg.create_model(cfg, stream=stream.cuda_stream)
    if isinstance(tuning, dict) and "best_ms" in tuning:
        model2.set_tuning(tuning)
    model2.mlmc_estimate(w["tol"], theta=w["theta"], c_alpha=w["c_alpha"], pilot_samples=32, max_rounds=3,
                         seed=seed + 16)
    e2e_M = []
    for k in range(max(args.steps, E2E_CALLS)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        est = model2.mlmc_estimate(w["tol"], theta=w["theta"], c_alpha=w["c_alpha"], pilot_samples=32,
                                   max_rounds=3, seed=seed + 17 + k)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e_n.append(sum(int(est["M"][l]) * eigsolves_per_sample(levels, l) for l in range(len(levels))))
        e2e_s.append(dt)
        e2e_M.append([int(x) for x in est["M"]])
        h2d, d2h = max(h2d, est["h2d_bytes"]), max(d2h, est["d2h_bytes"])
    model2.close()
    e2e_value = world * sum(e2e_n) / sum(e2e_s)
    e2e_mean_s = sum(e2e_s) / len(e2e_s)

    # ---- time-to-TOL: plain MC at the finest level on the same GPU ----
    Nf, Kf = levels[-1]
    mc_cfg = dict(cfg, levels=[(Nf, Kf)])
    mc = pkg.create_model(mc_cfg, stream=stream.cuda_stream)
    pilot = 32
    mc.sample_level(0, pilot, seed + 99, 0)
    Mp, s1, s2, _ = mc.get_level_stats(0)
    mu = s1 / Mp
    v_mc = float(np.max(np.maximum(s2 - Mp * mu * mu, 0) / (Mp - 1)))
    m_mc = int(math.ceil((w["c_alpha"] / (w["theta"] * w["tol"])) ** 2 * v_mc))
    # warm (workspaces sized by an untimed call of the same size), as the MLMC call above
    mc.sample_level(0, m_mc, seed + 98, pilot)
    mc.reset_level_stats(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mc.sample_level(0, m_mc, seed + 99, pilot)
    torch.cuda.synchronize()
    mc_s = time.perf_counter() - t0
    mc.close()

    sweep = tmdc_sweep(pkg, torch, stream)
    stress_line = stress(pkg, torch, stream)
    serve = serving(pkg, cfg, levels, seed)
    fp64 = fp64_paths(pkg, torch, stream, cfg, levels, M, seed)

    # GPU against the oracle at the bench's settings, outside the timed region
    chk = None
    if pool is not None and not args.no_oracle_check:
        chk_async = pool.map_async(_oracle_check_job, oracle_check_jobs(seed), chunksize=1)
        gpu_chk = gpu_oracle_check(model, levels, seed)
        chk = compare_oracle_check(gpu_chk, chk_async.get())

    cpu = None
    if pool is not None:
        if not args.no_cpu_baseline:
            cpu = oracle_measure(pool, cores, alloc, levels)
        pool.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (reduction, bisection) + f64 (refine, sums)",
            "data": "synthetic (seeded Philox vacancy masks)",
            "config": workload_config(alloc, w),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "call": "idos_mlmc_estimate(TOL=1e-3) adaptive, host outputs, wall clock",
                    "calls": len(e2e_s), "value_is": "all calls' eigen-solves / all calls' wall time",
                    "seconds_per_call": e2e_mean_s, "seconds_per_call_median": statistics.median(e2e_s),
                    "seconds_per_call_p90": float(np.percentile(e2e_s, 90)),
                    "samples_per_level_median": [int(x) for x in np.median(np.array(e2e_M), axis=0)],
                    "samples_per_level_max": [int(x) for x in np.max(np.array(e2e_M), axis=0)]},
            "time_to_tol": {"mlmc_adaptive_s": e2e_mean_s, "mlmc_adaptive_s_median": statistics.median(e2e_s),
                            "mlmc_fixed_alloc_s": total_ms_max / args.steps * 1e-3,
                            "plain_mc_s": mc_s, "plain_mc_samples": m_mc, "plain_mc_level": [Nf, Kf],
                            "speedup_mlmc_vs_mc": mc_s / e2e_mean_s},
            "gpu_launches": int(sum(v[1] for v in prof.values()) // args.steps),
            "kernels_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in sorted(prof.items(), key=lambda x: -x[1][0])},
            "level_span_ms_per_step": level_span_ms,
            "kernels_timing": "CUDA events per launch, the timed steps' launches replayed in order on one stream (unprofiled timed steps run the levels concurrently)",
            "roofline": roof,
            "rooflines": roofs,
            "clocks": clk,
            "cpu_baseline": cpu,
            "autotune": tuning,
            "graph": graph_line,
            "serving": serve,
            "tmdc_sweep": sweep,
            "stress": stress_line,
            "fp64_path": fp64,
            "estimate_check": {"Q_at_e_max": float(mean[-1]), "max_std": float(np.sqrt(np.max(var)))},
            "oracle_check": chk,
            "rates": rates,
            "fma_peaks": fma,
        }
        print(json.dumps(line), flush=True)
    model.close()
    if world > 1:
        dist.destroy_process_group()


# -------------------------------------------------------------- reference arm --
def run_reference(args):
    """The oracle as it stands (float64, LAPACK eigvalsh) on the host cores:
    each step is one bounded, workload-shaped sample (oracle_measure), timed
    for real; value and ms_per_step are medians over the timed steps."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synthetic import workload
    w = workload(WORKLOAD)
    alloc = load_alloc()
    levels = [tuple(x) for x in w["levels"]]
    pool, cores = oracle_pool()
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        r = oracle_measure(pool, cores, alloc, levels, first=60_000_000 + 10_000 * i)
        if i >= args.warmup:
            vals.append(r["value"])
            secs.append(r["wall_s"])
    pool.close()
    value = statistics.median(vals)
    cfg = workload_config(alloc, w, precision="fp64 throughout (the oracle: numpy / LAPACK eigvalsh, float64 sums)")
    cfg["step"] = "one bounded sample of the allocation per step: " + r["sample"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Philox vacancy masks)", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": r["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------- profiling helpers --
# ncu kernel names -> the library profiler's kernel families
NCU_FAMILY = [("k_small_persistent", "k_small_tridiag"), ("k_small_tridiag", "k_small_tridiag"),
              ("k_ts_panel", "k_ts_panel"), ("k_ts_wm", "k_ts_z"), ("k_ts_zc", "k_ts_z"), ("k_ts_w", "k_ts_w"),
              ("k_tc_w", "k_ts_w"), ("k_tc_operands", "k_ts_her2k"), ("k_tc_her2k", "k_ts_her2k"), ("k_ts_her2k", "k_ts_her2k"),
              ("k_ts_to_band", "k_ts_chase"), ("k_ts_chase", "k_ts_chase"), ("k_bisect", "k_bisect"),
              ("k_idos", "k_idos"), ("k_level", "k_level_stats"), ("k_fine_masks", "k_masks"),
              ("k_corner_masks", "k_masks"), ("k_cell_maps", "k_masks"), ("k_lg_assemble", "k_lg_assemble")]
FAMILY_SOURCE = {"k_small_tridiag": "k_small.cu", "k_ts_panel": "k_large.cu", "k_ts_w": "k_large.cu",
                 "k_ts_z": "k_large.cu", "k_ts_her2k": "k_tc.cu", "k_ts_chase": "k_chase.cu",
                 "k_bisect": "k_bisect.cu", "k_idos": "k_idos.cu"}


def ncu_family(name):
    # the first identifier of the library's kernel naming (k_...), whatever
    # return type, namespaces or template arguments ncu prints around it
    m = re.search(r"\b(k_[A-Za-z0-9_]+)", name)
    base = m.group(1) if m else ""
    for prefix, fam in NCU_FAMILY:
        if base.startswith(prefix):
            return fam
    return None


def run_profile_step(args):
    """One step of the workload for an ncu capture: direct launches on shared
    SMs, no autotuner, no warm-up, no clock sampler; the allocation scaled by
    --scale (at least one sample per level).  Writes the step's algorithmic
    work per kernel family to --work-json."""
    import numpy as np
    import torch
    import paper_1611_09784_gb300 as pkg
    from synthetic import workload
    w = workload(WORKLOAD)
    levels = [tuple(x) for x in w["levels"]]
    M = [max(1, int(round(Ml * args.scale))) for Ml in load_alloc()["M"]]
    if args.levels is not None:
        keep = {int(x) for x in args.levels.split(",")}
        M = [Ml if l in keep else 0 for l, Ml in enumerate(M)]
    cfg = dict(w["model"], p=w["p"], levels=levels, e_min=w["e_min"], e_max=w["e_max"], n_E=w["n_E"],
               delta=w["delta"], smoothing=w["smoothing"], precision="fp32", refine64_iters=REFINE64,
               tc_products=TC_PRODUCTS, sm_split=0, graph=0)
    torch.cuda.set_device(0)
    m = pkg.create_model(cfg)
    seed = w["seed"]
    firsts = [0] * len(M)
    m.sample_levels(M, seed, firsts)
    torch.cuda.synchronize()
    work = algorithmic_work(m, levels, M, seed, firsts, n_E=w["n_E"])
    m.close()
    if args.work_json:
        with open(args.work_json, "w") as f:
            json.dump({"samples_per_level": M, "work": work}, f)
    print(json.dumps({"profile_step": True, "samples_per_level": M}), flush=True)


def traffic_table(csv_path, work_json):
    """From an ncu CSV of one profile step (--metrics dram__bytes_read.sum,
    dram__bytes_write.sum, gpu__time_duration.sum) and that step's work file:
    per kernel family the launches, device time, share and DRAM bytes per
    algorithmic unit, and the profiles/traffic.txt lines."""
    import csv
    with open(work_json) as f:
        wk = json.load(f)["work"]
    rows = {}
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for rec in csv.DictReader(lines):
        fam = ncu_family(rec.get("Kernel Name", ""))
        if fam is None:
            continue
        r = rows.setdefault(fam, {"launch_ids": set(), "ns": 0.0, "dram": 0.0})
        r["launch_ids"].add(rec["ID"])
        val = float(rec["Metric Value"].replace(",", "")) if rec.get("Metric Value") else 0.0
        unit = rec.get("Metric Unit", "")
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1, "usecond": 1e3,
                 "msecond": 1e6}.get(unit, 1)
        if rec["Metric Name"] == "gpu__time_duration.sum":
            r["ns"] += val * scale
        elif rec["Metric Name"].startswith("dram__bytes"):
            r["dram"] += val * scale
    total = sum(r["ns"] for r in rows.values()) or 1.0
    out = []
    for fam, r in sorted(rows.items(), key=lambda kv: -kv[1]["ns"]):
        ratio = r["dram"] / wk[fam] if wk.get(fam) else None
        out.append({"family": fam, "launches": len(r["launch_ids"]), "ms": r["ns"] / 1e6, "share": r["ns"] / total,
                    "dram_bytes": r["dram"], "algorithmic": wk.get(fam), "dram_per_unit": ratio})
    print(json.dumps(out, indent=1))
    for o in out:
        if o["dram_per_unit"] is not None and o["family"] in FAMILY_SOURCE:
            src = FAMILY_SOURCE[o["family"]]
            print(f"{o['family']} {src} {kernel_source_hash(src)} {o['dram_per_unit']:.4e}")


def run_case(args):
    """Single-kernel cases for ncu captures: her2k:N:B (the tensor-core
    trailing update of B random n = N panels, twice) and eigvalsh:N:B (B random
    Hermitian matrices through the float32 path at the bench settings, twice)."""
    import numpy as np
    import paper_1611_09784_gb300 as pkg
    from synthetic import matrices as synth
    kind, N, B = args.case.split(":")
    N, B = int(N), int(B)
    rng = np.random.default_rng(5)
    t0 = time.perf_counter()
    if kind == "her2k":
        A = np.stack([synth.hermitian(N, 10 + b, scale=3.0) for b in range(B)])
        Y = rng.standard_normal((B, 16, N)) + 1j * rng.standard_normal((B, 16, N))
        Z = rng.standard_normal((B, 16, N)) + 1j * rng.standard_normal((B, 16, N))
        for _ in range(2):
            pkg.her2k(A, Y, Z, tc_products=TC_PRODUCTS)
    elif kind == "eigvalsh":
        H = np.stack([synth.hermitian(N, 20 + b, scale=3.0) for b in range(B)])
        for _ in range(2):
            pkg.eigvalsh(H, precision="fp32", refine64_iters=REFINE64, tc_products=TC_PRODUCTS)
    else:
        raise SystemExit(f"unknown case {kind}")
    print(json.dumps({"case": args.case, "wall_s": time.perf_counter() - t0}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--levels", default=None,
                    help="comma list of level indices to run (profiling a part of the workload)")
    ap.add_argument("--sm-split", type=int, default=-1,
                    help="SMs reserved for the finest level (0: shared SMs, -1: library default)")
    ap.add_argument("--graph", type=int, default=-1, choices=[-1, 0, 1],
                    help="graph replay of idos_sample_levels (-1: library default / autotuner; 0 for ncu runs, "
                         "which cannot follow a stream capture)")
    ap.add_argument("--no-clocks", action="store_true",
                    help="do not sample nvidia-smi clocks (profiler runs)")
    ap.add_argument("--skip-extras", action="store_true",
                    help="only the timed steps: no e2e / plain-MC / CPU-baseline measurements")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the GPU-vs-oracle check at the bench settings")
    ap.add_argument("--profile-step", action="store_true",
                    help="profiling: run exactly one step (direct launches, shared SMs, no autotuner, no warm-up)")
    ap.add_argument("--scale", type=float, default=1.0, help="profiling: scale of the allocation in --profile-step")
    ap.add_argument("--work-json", default=None, help="profiling: where --profile-step writes the step's work")
    ap.add_argument("--traffic-table", nargs=2, metavar=("NCU_CSV", "WORK_JSON"), default=None,
                    help="summarise an ncu capture of --profile-step (no GPU needed)")
    ap.add_argument("--case", default=None, help="profiling: her2k:N:B or eigvalsh:N:B")
    args = ap.parse_args()
    if args.traffic_table:
        traffic_table(*args.traffic_table)
        return
    if args.case:
        run_case(args)
        return
    if args.profile_step:
        run_profile_step(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
