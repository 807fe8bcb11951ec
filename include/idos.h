/*
 * idos.h - C ABI of the GB300 MLMC integrated-density-of-states library
 * (libidos.so).
 *
 * The library computes, for honeycomb tight-binding sheets with random
 * vacancies, the smoothed integrated density of states (IDoS) per unit area
 * of eq. (4.1)-(4.2) of Plechac & von Schwerin, "Multi-level Monte Carlo
 * acceleration of computations on multi-layer materials with random
 * defects", sample by sample, and the multilevel Monte Carlo estimator of
 * its expectation, eq. (2.6), with the control variates of Sec. 3.3.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an idos_status code: 0 = IDOS_OK, negative on
 *    error.  No C++ exception crosses the ABI.  idos_status_string() gives a
 *    static message; idos_last_error() gives the last detailed message of the
 *    calling thread.
 *  - All pointers named *_out / out and all input arrays are HOST pointers
 *    owned by the caller, unless a parameter says otherwise.  The model owns
 *    all device memory it allocates; nothing returned aliases it.
 *  - A model runs every kernel on the CUDA stream given at creation (a
 *    cudaStream_t passed as void*; NULL = the legacy default stream).  Calls
 *    that return host results synchronise that stream before returning.
 *  - A model must not be used from two threads at once.
 *  - Level index 0 is the paper's level l = 1 (the coarsest supercell).
 *  - Units: eV, Angstrom; IDoS in states per Angstrom^2 (no spin factor).
 *  - Site index inside an N x N supercell: m = 2(i + N j) + s, cell (i, j),
 *    sublattice s (A = 0, B = 1); lattice a1 = a(1,0), a2 = a(1/2, sqrt3/2),
 *    tau_B = (a1 + a2)/3.  k-points: K x K Monkhorst-Pack grid on the
 *    supercell reciprocal cell, index i1 + K i2.
 */
#ifndef IDOS_H
#define IDOS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IDOS_MAX_LEVELS 8

enum idos_status {
  IDOS_OK = 0,
  IDOS_ERR_INVALID_ARG = -1,   /* bad pointer, size, level, or descriptor field */
  IDOS_ERR_OUT_OF_MEMORY = -2, /* device or pinned allocation failed           */
  IDOS_ERR_CUDA = -3,          /* a CUDA runtime call or kernel launch failed   */
  IDOS_ERR_TIMEOUT = -4,       /* a bounded device-side wait gave up            */
  IDOS_ERR_NOT_CONVERGED = -5, /* an iteration hit its limit, or a reduced matrix came out non-finite */
  IDOS_ERR_UNSUPPORTED = -6,   /* valid request the library does not implement  */
  IDOS_ERR_NO_DEVICE = -7      /* no CUDA device of compute capability 10.3     */
};

/* Model kinds (Sec. 3.1).  Sizes below use V = vacancy sites and n = orbitals
 * of an N x N supercell:
 * IDOS_GRAPHENE: nearest-neighbour pz model, eq. (3.2a)-(3.2b): V = n = 2 N^2
 *   (site m = 2(i + N j) + s, one orbital each; a vacancy removes the site).
 * IDOS_TMDC: the TMDC-shaped 11-orbital model (the MoS2 example of Sec. 3.1
 *   with the pair vacancies of Sec. 3.2): metal with 5 d orbitals on the A
 *   site, chalcogen pair with 6 p orbitals on the B site; V = N^2 (site = the
 *   pair of cell c = i + N j), n = 11 N^2 (orbital 11 c + q, q < 5 metal);
 *   a vacancy removes the pair's 6 orbitals.  Real parameters drawn from
 *   model_seed (Philox4x64-10, counter (i, 0, 0, 0), key (model_seed, 2),
 *   value -2 + 4 (w0 >> 11) 2^-53 eV): 11 on-site energies, metal -> pair
 *   blocks (5 x 6) for the bonds tau_B, tau_B - a1, tau_B - a2, second-neighbour
 *   metal (5 x 5) and pair (6 x 6) blocks along a1, a2, a2 - a1 (transposed
 *   for the reverse hop); t, eps_onsite are unused.  N <= 24. */
enum idos_kind { IDOS_GRAPHENE = 0, IDOS_TMDC = 1 };

/* Arithmetic of the per-k eigen-solve.
 * IDOS_FP64: Householder reduction and smoothing in float64; eigenvalues by a
 *   float32 Sturm bracket then safeguarded float64 Newton on the float64
 *   tridiagonal's characteristic polynomial, to float64 resolution.
 * IDOS_FP32_REFINE64: reduction and Sturm bisection in float32, then
 *   refine64_iters float64 passes (Sturm count + Newton step each) on the
 *   float32 tridiagonal; the smoothing argument and every sum are float64,
 *   erfc is evaluated in float32.  Graphene matrices up to n = 128 are
 *   reduced in the bidiagonal form of the block between the two sublattices
 *   (H(k) = eps I + [[0, T], [T^H, 0]]): the tridiagonal handed to the
 *   bisection has diagonal eps and off-diagonals the bidiagonal's entries,
 *   with exactly the eigenvalues eps +- sigma_i(T) and |n_A - n_B| at eps. */
enum idos_precision { IDOS_FP64 = 0, IDOS_FP32_REFINE64 = 1 };

/* Smoothed step g of eq. (4.2).
 * IDOS_SMOOTH_GAUSS: g(x) = erfc(x / sqrt 2) / 2 (delta = standard deviation).
 * IDOS_SMOOTH_POLY:  g(x) = 1/2 - 9x/8 + 5x^3/8 on [-1, 1], 1 below, 0 above
 *                    (compact, both moment conditions of eq. (4.2)). */
enum idos_smoothing { IDOS_SMOOTH_GAUSS = 0, IDOS_SMOOTH_POLY = 1 };

/* Model description (Sec. 3.1-3.3, Sec. 4.2-4.3).  Plain data, copied by
 * idos_create_model. */
typedef struct idos_model_desc {
  int32_t kind;        /* idos_kind                                         */
  int32_t precision;   /* idos_precision                                    */
  int32_t smoothing;   /* idos_smoothing                                    */
  int32_t n_levels;    /* 1 .. IDOS_MAX_LEVELS                              */
  int32_t N[IDOS_MAX_LEVELS];     /* supercell side per level; N[l] = 2 N[l-1]
                                     when n_levels > 1 (Sec. 2.2, 3.3)       */
  int32_t Kside[IDOS_MAX_LEVELS]; /* Monkhorst-Pack side per level (>= 1)    */
  double t;            /* nearest-neighbour hopping, eq. (3.2b) (eV)        */
  double eps_onsite;   /* on-site energy eps_2p, eq. (3.2a) (eV)            */
  double a;            /* lattice constant (Angstrom)                       */
  double p;            /* vacancy probability, Sec. 3.2, in [0, 1]          */
  double sentinel;     /* diagonal of a removed site in idos_hamiltonian()  */
  double e_min, e_max; /* energy grid eps_j = e_min + j (e_max-e_min)/(n_E-1) */
  double delta;        /* smoothing width, eq. (4.2) (> 0)                  */
  int32_t n_E;         /* number of energies, 2 .. 1024                     */
  int32_t refine64_iters; /* float64 Newton/Sturm passes (FP32_REFINE64)  */
  uint64_t model_seed; /* parameter seed of the TMDC-shaped model           */
  int64_t workspace_bytes; /* device workspace cap; 0 = library default      */
  int32_t tc_products; /* IDOS_FP32_REFINE64, n > 160: trailing rank-2BW update
                          of the two-stage reduction on the FP32 pipe (0) or on
                          the tensor cores with 3 or 6 split-bfloat16 products
                          (6: float32-class sums, 3: ~5x their error)        */
  int32_t sm_split;    /* idos_sample_levels: SMs reserved (green context)
                          for the finest level, the other levels share the
                          rest, in calls where the other levels' work (flop
                          model, sum of n^3) is at least half the finest
                          level's; 0 = all levels always share all SMs,
                          -1 = library default (48).  Rounded up to the
                          device's partition granularity (8 SMs on sm_103).
                          Results do not depend on it.                       */
  double overlap_s;    /* graphene: nearest-neighbour overlap s of eq. (3.2c)-
                          (3.2d), |s| < 1/3; 0 = the standard problem.  With
                          S = I + s B and H = eps_onsite I + t B (B the bond-
                          phase matrix on the kept sites) the generalized
                          eigenvalues of eq. (3.1) are E = (eps_onsite + l) /
                          (1 + (s/t) l), l the eigenvalues of t B.           */
  int32_t persistent;  /* idos_sample_levels, graphene, IDOS_FP32_REFINE64:
                          1 = the shared-memory reductions (n <= 160) of
                          every level, fine and corner cells, in one
                          persistent launch over a size-sorted work list
                          (larger matrices first, one per CTA; n <= 32 one
                          per warp, taken by whichever warp is free); 0 = one
                          launch per cell set on its level's stream; -1 =
                          library default (1).  Results are bit-identical.  */
  int32_t graph;       /* idos_sample_levels: 1 = a call that repeats the
                          previous call's sample counts and settings is
                          captured as a CUDA graph (all level streams) and
                          later such calls replay it, the seed and first
                          sample indices read by the mask kernels from a
                          device buffer (a first call with new counts runs
                          directly); 0 = direct launches; -1 = library
                          default (1).  Results are bit-identical.           */
} idos_model_desc;

typedef struct idos_model idos_model;

/* Create a model on the current CUDA device: the tight-binding model of
 * Sec. 3.1 (graphene, eq. (3.2a)-(3.2d), or the TMDC-shaped model), its
 * vacancy law (Sec. 3.2), the MLMC level hierarchy N_l = 2 N_{l-1} with the
 * control variates of Sec. 3.3, and the Brillouin-zone grid and smoothed IDoS
 * of Sec. 4.2-4.3.  Validates d (IDOS_ERR_INVALID_ARG before any device call),
 * allocates the level accumulators and a workspace.  *out receives the handle
 * (NULL on error).  cuda_stream: cudaStream_t as void*, or NULL. */
int idos_create_model(const idos_model_desc* d, void* cuda_stream, idos_model** out);

/* Free every device buffer of the model created by idos_create_model (the
 * model of Sec. 3.1-3.3 and the grids of Sec. 4.2-4.3); synchronises its
 * stream first.  NULL ok. */
void idos_destroy_model(idos_model* m);

/* The SM partition idos_sample_levels uses: *sms_finest SMs for the finest
 * level and *sms_rest for the others, or 0 and 0 when all levels share all
 * SMs (sm_split = 0, one level, or no green-context support in the driver;
 * *why then holds the reason, a static string, "" when none). */
int idos_get_partition(const idos_model* m, int* sms_finest, int* sms_rest, const char** why);

/* Graph replay of idos_sample_levels: how many calls replayed a graph and
 * how many captures were made; *why: "" while graph mode is on, else the
 * reason it was given up (a static string valid until the next call on m). */
int idos_get_graph_info(const idos_model* m, int64_t* replays, int64_t* captures, const char** why);

/* Static text for a status code. */
const char* idos_status_string(int status);

/* Detailed message of the last error on the calling thread ("" if none). */
const char* idos_last_error(void);

/* Draw n_samples outcomes of level `level` (sample indices first_sample ..
 * first_sample + n_samples - 1, generator key `seed`), compute for each
 *   Y = Q_l(omega) - (1/4) sum_r Q_{l-1}(omega; corner r)   (level >= 1)
 *   Y = Q_0(omega)                                         (level == 0)
 * (eq. (2.6) and the control variate of Sec. 3.3; corners use level l-1's
 * Kside) and add sum Y, sum Y^2 (float64, fixed summation order) and the
 * sample count to the model's level accumulators.
 * per_sample_Y: NULL, or host float64[n_samples * n_E] receiving every Y.
 * Errors: INVALID_ARG (level out of range, n_samples < 0), CUDA, OUT_OF_MEMORY. */
int idos_sample_level(idos_model* m, int level, int64_t n_samples, uint64_t seed,
                      int64_t first_sample, double* per_sample_Y);

/* Same as idos_sample_level, but also returns the per-sample fine IDoS
 * Q_l (host float64[n_samples * n_E], may be NULL) and the four corner IDoS
 * (host float64[n_samples * 4 * n_E], corner r = ri + 2 rj, may be NULL;
 * ignored on level 0).  Parity entry point. */
int idos_sample_level_detail(idos_model* m, int level, int64_t n_samples, uint64_t seed,
                             int64_t first_sample, double* per_sample_Y,
                             double* Q_fine, double* Q_coarse);

/* All levels at once: n_samples[l] outcomes of every level l (0 skips a
 * level), sample indices first_sample[l] ... (or, when first_sample is NULL,
 * continuing after the samples the level already holds), generator key seed.
 * Same results as one idos_sample_level call per level; the levels run
 * concurrently on streams of their own (each with its own workspace), after
 * the work already queued on the model's stream, so that the latency-bound
 * phases of the largest matrices overlap the other levels' work.  Returns
 * when every level is done. */
int idos_sample_levels(idos_model* m, const int64_t* n_samples, uint64_t seed, const int64_t* first_sample);

/* Read the accumulators of one level: *M samples, sum[n_E], sumsq[n_E]
 * (host, may be NULL), *seconds of GPU time spent on the level (may be NULL). */
int idos_get_level_stats(const idos_model* m, int level, int64_t* M, double* sum,
                         double* sumsq, double* seconds);

/* All four float64 accumulators of one level: moments host float64[4 * n_E],
 * rows sum Y, sum Y^2 (the level term of eq. (2.6), as idos_get_level_stats),
 * sum Q_l, sum Q_l^2 (the fine IDoS Q_l of the same outcomes alone, whose
 * variance decay is the rate S of eq. (Q_variance)); *M samples, *seconds
 * GPU time (both may be NULL). */
int idos_get_level_moments(const idos_model* m, int level, int64_t* M, double* moments, double* seconds);

/* Eq. (2.6) and the variance display after it, from level accumulators (host
 * arithmetic, no device needed): mean[j] = sum_l S1_l[j] / M_l and
 * var[j] = sum_l V_l[j] / M_l with V_l[j] = (S2_l[j] - M_l mean_l[j]^2) /
 * (M_l - 1) the unbiased sample variance.  M: int64[n_levels]; a level with
 * M_l = 0 is left out.  sums: float64[n_levels * 2 * n_E], per level the rows
 * S1 = sum Y, S2 = sum Y^2.  mean, var: host float64[n_E].  INVALID_ARG for a
 * level with M_l = 1 or M_l < 0, no level with samples, or bad sizes. */
int idos_combine_level_stats(int n_levels, const int64_t* M, const double* sums, int n_E, double* mean,
                             double* var);

/* Rates of the complexity models of Sec. 2.1-2.2 (eq. (compl_model):
 * Q - E[Q_N] ~ N^-W, Var(Q_N) ~ N^-S, cost per sample ~ N^C; eq.
 * (compl_model2): Var(Q_l - Q_l^CV) ~ N^-D), fitted as Sec. 4.4 does
 * (eq. (param_est)), and the asymptotic work exponents they imply. */
typedef struct idos_rates {
  double W, S, D, C;              /* fitted exponents (NaN with < 2 usable levels)      */
  double W_se, S_se, D_se, C_se;  /* standard errors of the slopes (0 with 2 points)   */
  int32_t n_W, n_S, n_D, n_C;     /* levels each fit used                              */
  double work_mc;    /* eq. (Work_SLMC): Work_MC ~ TOL^-(2 + (C - S)/W)                 */
  double work_mlmc;  /* eq. (Work_MLMC): Work_MLMC ~ TOL^-(2 + (C - D)/W) (for D < C)   */
  double work_fs;    /* eq. (Work_FS): one sample on a large cell, TOL^-(2 C / S)      */
  double theta_mc;   /* the MC bias/statistics split 1 / (1 + (C - S)/W) of Sec. 2.1   */
} idos_rates;

/* Fit the rates from level accumulators (host arithmetic, no device needed).
 * N: int32[n_levels] supercell sides (doubling); M: int64[n_levels]; moments:
 * float64[n_levels * 4 * n_E] as idos_get_level_moments returns them; cost:
 * float64[n_levels] work per sample (seconds or a flop model), or NULL (C is
 * then NaN); a level with cost <= 0 is left out of C.  Norm: the arithmetic
 * mean over the energy grid, as the paper's convergence plots use.  Each rate
 * is minus (C: plus) the least-squares slope of log(value) against log N_l:
 * S from the grid-mean sample variance of Q_l over levels with M_l >= 2; D
 * from that of Y_l over levels l >= 1 (0-based) with M_l >= 2; W from the
 * grid mean of |sum Y_l / M_l| over levels l >= 1 with M_l >= 1 (E[Y_l] =
 * E[Q_l] - E[Q_{l-1}] is proportional to N_l^-W when N doubles); C from cost.
 * INVALID_ARG for bad sizes or pointers. */
int idos_fit_rates(int n_levels, const int32_t* N, const int64_t* M, const double* moments, const double* cost,
                   int n_E, idos_rates* out);

/* Zero the accumulators of one level, or of all levels when level == -1. */
int idos_reset_level_stats(idos_model* m, int level);

/* IDoS Q(eps_j) of eq. (4.1)-(4.2) for ONE supercell configuration: side N,
 * Kside x Kside grid.  mask: host u8[V] (1 = vacancy site removed; V as in
 * idos_kind), or NULL to draw it from (seed, level, sample) exactly as
 * idos_sample_level does.  idos_out: host float64[n_E].  eigs_out: NULL or
 * host float64[Kside^2 * n]: per k the ascending eigenvalues of the active
 * block (equal eigenvalues may come out in either order within their
 * rounding), then NaN padding to n. */
int idos_eval_idos(idos_model* m, int N, int Kside, const uint8_t* mask, uint64_t seed,
                   int level, int64_t sample, double* idos_out, double* eigs_out);

/* Options of the adaptive estimator. */
typedef struct idos_mlmc_opts {
  double tol;            /* TOL of Sec. 2 (states / Angstrom^2)                  */
  double theta;          /* statistical share of TOL (0 < theta < 1)             */
  double c_alpha;        /* confidence quantile (1.96)                           */
  int64_t pilot_samples; /* pilot samples on level 0 (>= 2); with three or more
                            levels also on every level below the finest; the
                            finest (every level l > 0 with fewer levels) takes
                            max(4, ceil(pilot_samples sqrt(W_0/W_l))), W = flop model */
  int32_t work_model;    /* 0: W_l from the flop model sum n^3; 1: measured time */
  int32_t max_rounds;    /* eq. (2.7) rounds after the pilots (>= 1); with three or
                            more levels also the most provisional rounds of the
                            levels below the finest beside its pilot          */
  uint64_t seed;         /* generator key                                        */
} idos_mlmc_opts;

/* Result of the adaptive estimator; every array is caller-owned host memory. */
typedef struct idos_estimate {
  double* mean;    /* float64[n_E]: eq. (2.6)                               */
  double* var;     /* float64[n_E]: sum_l V_l(eps)/M_l                       */
  int64_t* M;      /* int64[n_levels]: samples used per level               */
  double* V;       /* float64[n_levels]: max over eps of the level variance  */
  double* W;       /* float64[n_levels]: work per sample used in eq. (2.7)   */
  double seconds;  /* wall time of the call                                  */
  int32_t rounds;  /* eq. (2.7) rounds with every level's pilot in           */
  int64_t h2d_bytes; /* bytes copied host -> device during the call          */
  int64_t d2h_bytes; /* bytes copied device -> host during the call          */
} idos_estimate;

/* Adaptive MLMC (Sec. 2.2): pilot round (see pilot_samples), V_l and
 * W_l, M_l from eq. (2.7) with target variance (theta tol / c_alpha)^2, extra
 * samples, combine by eq. (2.6).  With three or more levels the finest
 * level's pilot is issued first, on its own SM partition, and the other
 * levels run beside it: their pilots, then up to max_rounds provisional
 * rounds sized by eq. (2.7) with the finest level's term estimated from the
 * variance decay of the two levels below it (half of it counted); once the
 * finest pilot is in, the rounds top up every level to eq. (2.7) with all
 * pilots.  With profiling on the same calls run one after the other: with
 * work_model 0 the sample counts depend on the seed and the options only,
 * neither on timing nor on profiling.  Starts from zeroed accumulators.  Sample indices
 * continue from 0 on every level. */
int idos_mlmc_estimate(idos_model* m, const idos_mlmc_opts* o, idos_estimate* out);

/* ---- kernel timing (tracing) ----
 * With profiling enabled every kernel launch of the model is bracketed by a
 * pair of CUDA events on the model's stream; the pairs are resolved when the
 * call that launched them synchronises, and accumulated per kernel family.
 * The events add a few microseconds per launch. */

/* enable = 1 turns timing on: idos_sample_levels then issues every level's
 * launches in order on one stream, without the SM partition or a graph, so
 * that each event pair spans its own kernel alone.  enable = 2 (timeline):
 * the levels keep their streams and partition but run without a graph
 * (launches issued directly, levels in the library's issue order, so a
 * level's first kernel can start only once the host has issued it), each
 * pair's span includes any time its kernel waited for SMs, and
 * idos_sample_levels also keeps a trace of its launches (idos_get_trace).
 * 0 turns timing off.  Does not clear the totals. */
int idos_set_profiling(idos_model* m, int enable);

/* Number of kernel families (valid kid values are 0 .. count-1). */
int idos_profile_count(void);

/* Totals of kernel family kid since the last reset: *name (static string,
 * may be NULL), *ms summed event time, *launches. */
int idos_get_profile(const idos_model* m, int kid, const char** name, double* ms, int64_t* launches);

/* Zero the totals (and the trace). */
int idos_reset_profile(idos_model* m);

/* One timed scope of the last idos_sample_levels call made in timeline mode. */
typedef struct idos_trace_entry {
  int32_t kid;        /* kernel family (idos_get_profile's kid)                */
  int32_t lane;       /* stream, numbered in order of first use within the call */
  int32_t launches;   /* kernel launches inside the scope (0: aggregating scope) */
  int32_t reserved;
  double t0_ms;       /* start and end, ms after the call was issued (the     */
  double t1_ms;       /* origin stream's event before the levels fork off)    */
} idos_trace_entry;

/* Copies up to `capacity` entries of that trace (host array, caller-owned)
 * and sets *count to the trace's length (which may exceed capacity). */
int idos_get_trace(const idos_model* m, int64_t capacity, idos_trace_entry* out, int64_t* count);

/* ---- parity / diagnostic entry points (same kernels as the hot path) ---- */

/* Vacancy masks of samples first_sample .. first_sample + n_samples - 1 of
 * `level` for an N x N cell: host u8[n_samples * V] (1 = removed),
 * computed on the device by the hot path's generator (Philox4x64-10, key
 * (seed, 1), counter (site, sample, level, 0), vacant iff word0 < p 2^64). */
int idos_vacancy_masks(idos_model* m, int N, int level, uint64_t seed, int64_t first_sample,
                       int64_t n_samples, uint8_t* out);

/* H(k) of the model for one configuration (mask: host u8[V]) and one grid
 * point, as the assembly kernel builds it, written as a full n x n complex128
 * matrix (row-major, interleaved re/im: host float64[2 n^2]) with removed
 * orbitals' rows and columns zero and m->sentinel on their diagonal.
 * N <= 32 (graphene), <= 12 (TMDC-shaped). */
int idos_hamiltonian(idos_model* m, int N, int Kside, int k_index, const uint8_t* mask,
                     double* out);

/* All eigenvalues of `batch` dense Hermitian n x n matrices (host complex128,
 * row-major, interleaved re/im, float64[batch * 2 n^2]) through the hot
 * path's Householder reduction and Sturm bisection in `precision`
 * (tc_products as in idos_model_desc); eigs_out: host float64[batch * n],
 * ascending per matrix.  cuda_stream as above. */
int idos_eigvalsh(int precision, int refine64_iters, int tc_products, int n, int64_t batch,
                  const double* H, double* eigs_out, void* cuda_stream);

/* The real symmetric tridiagonal (d, e^2) that the hot path's Householder
 * reduction (Sec. 4.2's dense eigensolver; shared-memory path or two-stage
 * path by size, tc_products as in idos_model_desc) makes of `batch` dense
 * Hermitian n x n matrices (H as in idos_eigvalsh): d_out, e2_out: host
 * float64[batch * n]; e2_out[b n + i] = |e_i|^2 couples rows i and i + 1
 * (the last entry of every matrix is 0).  Its eigenvalues are those of H.
 * Parity entry point (checks the reduction apart from the bisection). */
int idos_tridiagonalize(int precision, int tc_products, int n, int64_t batch, const double* H, double* d_out,
                        double* e2_out, void* cuda_stream);

/* The trailing update of one stage-1 panel of the two-stage reduction
 * (compact-WY form of the two-sided Householder update, Sec. 4.2's dense
 * eigensolver): A_out = A - (Y Z^H + Z Y^H) for `batch` complex n x n
 * matrices, computed in float32 storage by the kernel the large path runs:
 * tc_products = 0 on the FP32 pipe, 3 or 6 on the tensor cores with that many
 * split-bfloat16 products (see idos_model_desc).  A: host complex128
 * float64[batch * 2 n^2] row-major; Y, Z: host complex128 float64[batch * 2 *
 * 16 n], column c of matrix b at Y[b][c][0..n) (the 16 = band half-width
 * columns of one panel); A_out: host float64[batch * 2 n^2].  Inputs are
 * rounded to float32.  Allocates and frees its own device buffers; blocking. */
int idos_her2k(int tc_products, int n, int64_t batch, const double* A, const double* Y, const double* Z,
               double* A_out);

/* The product W = A22 V of one stage-1 panel (the first factor of the
 * compact-WY two-sided update, Sec. 4.2's dense eigensolver in two-stage
 * form): A22 = rows and columns k + 16 .. n-1 of A (m = n - k - 16, k a
 * multiple of 16 with 0 <= k < n - 16), V = columns 0..m-1 of YT.  mode =
 * the kernel the large path runs: 2 = tensor cores (six split-bfloat16
 * products, n even), 1 = FP32 pipe with 128-row register tiles (n even), 0 =
 * FP32 pipe with 64-row tiles; the partial sums of the kernel's K splits are
 * added in split order on the host.  A: host complex128 float64[batch * 2 n^2]
 * row-major; YT: host float64[batch * 2 * 16 n], column c of matrix b at
 * YT[b][c][0..n); W_out: host float64[batch * 2 * 16 n] in the same layout,
 * entries m..n-1 of each column zero.  Inputs are rounded to float32.
 * Allocates and frees its own device buffers; blocking. */
int idos_stage1_w(int mode, int n, int64_t batch, int k, const double* A, const double* YT, double* W_out);

/* Density of states from an IDoS on the uniform energy grid (host float64
 * Q[n_E], n_E >= 2) by numerical differentiation, as the paper suggests for
 * the expected IDoS: central differences (Q[j+1] - Q[j-1]) / (2h) inside,
 * one-sided differences at the ends, h = (e_max - e_min) / (n_E - 1); dos:
 * host float64[n_E].  Host arithmetic only (no device needed). */
int idos_dos_from_idos(const double* Q, int n_E, double e_min, double e_max, double* dos);

/* FMA throughput of the current device, the denominator of the ALU
 * rooflines (the paper has no counterpart; it times one CPU core): a grid of
 * 8 CTAs x 256 threads per SM, each thread running 8 independent dependent
 * FMA chains for `iters` iterations, timed with CUDA events on cuda_stream
 * after one untimed launch.  precision: IDOS_FP32_REFINE64 (float32 FMA) or
 * IDOS_FP64 (float64 FMA).  *flops_per_s: 2 flops per FMA; *ms (nullable):
 * the timed launch.  Blocking.  INVALID_ARG for iters outside 1 .. 2^30. */
int idos_measure_fma_peak(int precision, int64_t iters, void* cuda_stream, double* flops_per_s, double* ms);

/* ---- autotuning ----
 * Times idos_sample_levels(n_samples) on this model for every candidate
 * configuration and installs the fastest: the SMs reserved for the finest
 * level (sm_split: 0, 24, 32, 40, 48, 56, 64 where the device allows) and the
 * largest n the shared-memory kernel takes before the two-stage path (64, or
 * whatever fits: 160 float32 / 112 float64) and, with the latter, the
 * persistent launch on or off (graphene, IDOS_FP32_REFINE64; on with graph
 * replay in each of the three placements below; off without graph replay),
 * then the winner's split +- 4 SMs where the partition alignment gives a size
 * not yet timed, then the winner with graph replay switched (unless
 * the model gave graphs up), then the two-stage kernel shapes (the W tile,
 * one or two warps per sweep in clustered band chases, and 1, 2 or 4 CTAs
 * in the panel QR cluster).  Each candidate
 * runs twice untimed (a direct
 * call, then the graph capture) and `reps` times timed (best kept), on
 * sample indices from 2^40 on;
 * the level statistics are restored afterwards.  Results do not depend on the
 * choice beyond float rounding of the path choice; out: the choice and every
 * candidate's best step time. */
#define IDOS_TUNE_MAX 56
typedef struct idos_tuning {
  int32_t sm_split;      /* chosen SMs reserved for the finest level (0 = shared; the partition's
                            actual size) */
  int32_t small_max_n;   /* chosen limit of the shared-memory kernel (-1 = what fits) */
  double best_ms;        /* step time of the chosen configuration */
  int32_t n_tried;
  int32_t tried_split[IDOS_TUNE_MAX];
  int32_t tried_small[IDOS_TUNE_MAX];
  double tried_ms[IDOS_TUNE_MAX];
  int32_t persistent;    /* chosen persistent setting (idos_model_desc.persistent) */
  int32_t tried_persistent[IDOS_TUNE_MAX];
  int32_t graph;         /* chosen graph setting (idos_model_desc.graph) */
  int32_t tried_graph[IDOS_TUNE_MAX];
  int32_t w_tile;        /* stage-1 W kernel: 1 = 128-row register tiles (default), 0 = 64-row
                            tiles, 2 = tensor cores (with tc_products > 0) */
  int32_t chase_pair;    /* clustered band chases: 1 = two warps per sweep, 0 = one */
  int32_t tried_w_tile[IDOS_TUNE_MAX];
  int32_t tried_chase_pair[IDOS_TUNE_MAX];
  int32_t placement;     /* persistent route on the partition: 0 = every level on its own
                            partition; 1 = a level below the finest whose fine cells take the
                            two-stage path runs on the finest level's SMs; 2 = the finest
                            level's corner cells run on the other levels' SMs */
  int32_t tried_placement[IDOS_TUNE_MAX];
  int32_t panel_cluster; /* CTAs of the stage-1 panel QR cluster (0 = the default rule) */
  int32_t tried_panel_cluster[IDOS_TUNE_MAX];
  int32_t her2k_lower;   /* tensor-core trailing update: 1 = lower-triangle tiles with mirrored
                            blocks (default), 0 = the full tile grid */
  int32_t tried_her2k_lower[IDOS_TUNE_MAX];
  int32_t persist_reserve; /* SMs of its partition the persistent small-matrix launch leaves free
                              for the two-stage chains beside it (0 = none) */
  int32_t tried_persist_reserve[IDOS_TUNE_MAX];
} idos_tuning;
int idos_autotune(idos_model* m, const int64_t* n_samples, int reps, idos_tuning* out);

/* Installs the configuration fields of `t` (sm_split, small_max_n,
 * persistent, graph, w_tile, chase_pair, placement, panel_cluster,
 * her2k_lower, persist_reserve; the timing
 * and tried_* fields are ignored), e.g. a choice an earlier idos_autotune
 * returned, without timing anything.  sm_split 0 shares all SMs; a split the
 * driver cannot make leaves every level on all SMs (idos_autotune's rule).
 * Results do not depend on the configuration beyond float rounding of the
 * path choice (small_max_n, w_tile).  Invalid values: IDOS_ERR_INVALID_ARG,
 * nothing changed. */
int idos_set_tuning(idos_model* m, const idos_tuning* t);

/* ---- serving ----
 * A request loop over the level sampler (a scheduler thread inside the
 * library).  Requests arrive from any host thread; they are admitted in
 * arrival order onto n_workers device streams, each with its own workspace,
 * while the summed workspace of the requests in flight (their HBM footprint)
 * stays within hbm_budget_bytes (0 = 8 GiB; a request larger than the budget
 * still runs when nothing else is in flight), so requests of different levels
 * and sizes overlap on the device.  A request's result is the float64 sum of
 * Y and of Y^2 (the level terms of eq. (2.6), Y as in idos_sample_level) over
 * its samples first_sample .. first_sample + n_samples - 1 of `level`; its
 * launch shapes depend only on the request, so the result is the same whether
 * it runs alone or among others.  The model described by d is created inside
 * the server (its sm_split is ignored). */
typedef struct idos_server idos_server;
int idos_server_create(const idos_model_desc* d, int n_workers, int64_t hbm_budget_bytes, idos_server** out);

/* Queue one request; *ticket identifies it.  Does not block. */
int idos_server_submit(idos_server* s, int level, int64_t n_samples, uint64_t seed, int64_t first_sample,
                       int64_t* ticket);

/* Block until the request is done; sum, sumsq: host float64[n_E] (nullable);
 * latency_s: seconds from submission to completion; device_ms: CUDA-event
 * time of its work.  Returns the request's status; the ticket is then freed. */
int idos_server_wait(idos_server* s, int64_t ticket, double* sum, double* sumsq, double* latency_s,
                     double* device_ms);

/* Counters: requests completed, queued, bytes of the workspace in flight now
 * and at peak (all nullable). */
int idos_server_info(const idos_server* s, int64_t* completed, int64_t* queued, int64_t* in_flight_bytes,
                     int64_t* peak_bytes);

/* Finish the queued requests, stop the loop, free everything.  NULL ok. */
void idos_server_destroy(idos_server* s);

/* ---- allocation-free evaluation ----
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc: code that owns all device memory through its
 * own pool and forbids outside allocations, code that must not trigger the
 * implicit device-wide synchronisation of cudaMalloc / cudaFree in a
 * latency-critical loop, or code that cannot create a model (model creation
 * allocates its accumulators and workspace).
 *
 * Computes exactly what idos_eval_idos computes for one configuration (same
 * kernels, same results), without a model and without allocating: its
 * scratch (kept-site maps, tridiagonals, eigenvalues when eigs_dev_out is
 * NULL) lives in one file-scope static device array of 1 MiB that every GPU
 * which loads libidos.so holds until the process exits.
 *  - d: model description (only the single-configuration fields are used:
 *    kind (graphene only), precision, smoothing, t, eps_onsite, a, p, e_min,
 *    e_max, delta, n_E, refine64_iters, overlap_s (|s| < 1/3, nonzero t)).
 *  - N, Kside: supercell side and k-grid side.  Only matrices of the
 *    shared-memory path are accepted (2N^2 <= 160 in float32, <= 112 in
 *    float64), and the scratch must fit 1 MiB (about 2 K^2 2N^2 (2 s + 8)
 *    bytes, s = 4 or 8); larger requests return IDOS_ERR_INVALID_ARG with the
 *    byte count in idos_last_error().
 *  - mask_dev: DEVICE u8[2N^2] (1 = removed), or NULL to draw the mask from
 *    (seed, level, sample) as idos_sample_level does.
 *  - idos_dev_out: DEVICE float64[n_E]; eigs_dev_out: NULL or DEVICE
 *    float64[Kside^2 * 2N^2] (layout as in idos_eval_idos).  Caller-owned.
 *  - cuda_stream: cudaStream_t as void* (NULL = legacy default stream).  The
 *    call enqueues its kernels and returns without synchronising.
 * Set-up: every call whose stream is not being captured looks up the static
 * array's device address (cudaGetSymbolAddress, no allocation), so the
 * address stays valid across a cudaDeviceReset; a call on a capturing stream
 * reuses the address of the last uncaptured call on that device, so make the
 * first call on a device before any stream capture.  The first call on a
 * device may also load the library's kernel modules (CUDA loads modules
 * lazily by default), which takes device memory once: make it outside the
 * region that must not allocate, as a warm-up.  After that no call allocates.
 * All calls share the array and every call overwrites all of the scratch it
 * reads, so nothing needs clearing between calls (a call after a larger one
 * sees none of its contents); calls whose kernels overlap on the GPU (other
 * streams, other host threads) race on the array and must be serialised by
 * the caller. */
int idos_eval_idos_noalloc(const idos_model_desc* d, int N, int Kside, const uint8_t* mask_dev,
                           uint64_t seed, int level, int64_t sample, double* idos_dev_out,
                           double* eigs_dev_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* IDOS_H */
