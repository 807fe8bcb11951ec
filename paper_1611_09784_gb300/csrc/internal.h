// internal.h - host-side declarations shared by the libidos translation units:
// the model object behind the C ABI, the device workspace arena and the
// kernel launchers of each stage of the path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/idos.h"
#include "common.cuh"
#include "profiler.h"

namespace idos {

// Bump allocator over one device buffer.  reset() at the start of every API
// call; grow() reallocates (after a stream sync) when a call needs more.
// Returned by Arena::reserve when the arena would have to grow while its
// stream is being captured into a graph (never leaves the library).
constexpr int kErrGrowDuringCapture = -1000;

struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  size_t peak = 0;
  uint64_t gen = 0;   // bumped on every (re)allocation: graphs hold pointers into it
  int reserve(size_t bytes, cudaStream_t s);   // ensure capacity >= bytes
  void reset() { used = 0; }
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    size_t need = off + count * sizeof(T);
    if (need > cap) return nullptr;
    used = need;
    if (used > peak) peak = used;
    return reinterpret_cast<T*>(base + off);
  }
  void release();
};

// Vacancy sites and orbitals per unit cell of each model kind: graphene has
// two sites with one orbital each; the TMDC-shaped model one removable
// chalcogen pair and 11 orbitals (5 metal + 6 pair).
inline int vac_per_cell(int kind) { return kind == IDOS_TMDC ? 1 : 2; }
inline int orb_per_cell(int kind) { return kind == IDOS_TMDC ? 11 : 2; }

// One set of supercell configurations of equal side N ("cells"): vacancy
// masks and the compaction maps from orbital index to active row.
struct CellSet {
  int kind = IDOS_GRAPHENE;
  int N = 0;
  int n_sites = 0;   // orbitals per cell: orb_per_cell(kind) N^2
  int n_vac = 0;     // vacancy sites per cell: vac_per_cell(kind) N^2
  int64_t count = 0;
  uint8_t* vmask = nullptr; // [count][n_vac], 1 = removed (the same buffer as mask for graphene)
  uint8_t* mask = nullptr;  // [count][n_sites], 1 = orbital removed
  int* n_act = nullptr;     // [count]
  int* act = nullptr;       // [count][n_sites] active orbitals, ascending
  int* inv = nullptr;       // [count][n_sites] orbital -> active row, or -1
};

// Inputs of one batched eigen-solve: every cell of a CellSet at every point
// of a Kside x Kside grid (matrix index = cell * K^2 + k), or `count`
// explicit Hermitian matrices (H != nullptr, Kside = 1, n_act = n_max).
int check_device(int& sm_count);   // IDOS_ERR_NO_DEVICE unless the current device is sm_103

struct SolveArgs {
  const CellSet* cells = nullptr;
  int Kside = 1;
  int n_max = 0;            // matrix dimension capacity = orbitals per cell
  int64_t n_mat = 0;
  double t = 0, eps = 0;    // graphene: hopping and on-site energy
  int kind = IDOS_GRAPHENE;
  const double* tmdc_p = nullptr;   // TMDC-shaped model: device parameter table
  const double2* H = nullptr;
  void* d = nullptr;        // T[n_mat][n_max] diagonal of the tridiagonal
  void* e2 = nullptr;       // T[n_mat][n_max] squared off-diagonal (e2[i] couples i, i+1)
  cudaStream_t stream = 0;
  Arena* ws = nullptr;
  // Device status word, zero on entry, set nonzero by a kernel whose bounded
  // dependency wait ran out.  With it the caller checks after its own
  // synchronisation; without it the large path checks (and synchronises).
  int* err = nullptr;
  // float32 large path: 0 = trailing update on the FP32 pipe, 3 or 6 =
  // tensor cores with that many split-bfloat16 products
  int tc_np = 0;
  // SMs the launches of this call run on (0 = the whole device; launch
  // shapes do not depend on it) and the largest thread-block cluster they may
  // form (SM partitions guarantee 8; the band chase computes the same values
  // for every cluster size, the panel QR never exceeds 8)
  int sm_avail = 0;
  int max_cluster = 16;
  // kernel shapes of the two-stage path (set by the autotuner): the float32
  // W = A22 (Y T) with 128-row register tiles (1), 64-row tiles (0) or on the
  // tensor cores (2, with the tensor-core trailing update; else as 1);
  // clustered band chases with two warps per sweep (1) or one (0)
  int w_tile = 1;
  int chase_pair = 1;
  // CTAs of the stage-1 panel QR cluster (0: the smallest power of two whose
  // shared memory holds the panel, grown while the batch leaves SMs idle)
  int panel_cluster = 0;
  // tensor-core trailing update on lower-triangle tiles with mirrored blocks
  // (1) or on the full tile grid (0)
  int her2k_lower = 1;
};

// Two green contexts splitting the device's SMs (partition.cu): ctx[0] has
// sms[0] SMs (reserved for one stream's work), ctx[1] the rest.
struct SmPartition {
  void* ctx[2] = {nullptr, nullptr};
  int sms[2] = {0, 0};
  bool shared = false;   // owned by the process-wide cache (never destroyed by a model)
};
int partition_create(int big_sms, SmPartition& p);
int partition_rounded(int big_sms);   // the SM count a request of big_sms rounds up to
int partition_stream(const SmPartition& p, int which, int priority, cudaStream_t* out);
void partition_destroy(SmPartition& p);

struct Model {
  idos_model_desc d{};
  cudaStream_t stream = 0;
  // one stream, workspace and event pair per level for idos_sample_levels
  cudaStream_t lstream[IDOS_MAX_LEVELS] = {};   // shared SMs, priorities by cost
  cudaStream_t pstream[IDOS_MAX_LEVELS] = {};   // the same on the SM partition (null without one)
  // second stream per level for the corners' solve beside the fine one
  cudaStream_t lstream2[IDOS_MAX_LEVELS] = {}, pstream2[IDOS_MAX_LEVELS] = {};
  // streams of the levels below the finest on the finest level's partition:
  // with placement 1 a level whose fine cells take the two-stage path runs
  // there (its latency-bound chain beside the finest level's) instead of
  // waiting for the persistent launch to free the other partition's SMs
  cudaStream_t pstreamF[IDOS_MAX_LEVELS] = {};
  // placement of work on the partition: 0 = levels on their own partitions;
  // 1 = the levels above (pstreamF); 2 = the finest level's corner solve
  // (many medium matrices, throughput work) on the other partition, leaving
  // the finest partition to the latency-bound chain of the large matrices.
  // 0 by default; the autotuner may pick another.
  int placement = 0;
  cudaEvent_t lfork2[IDOS_MAX_LEVELS] = {}, ljoin2[IDOS_MAX_LEVELS] = {};
  cudaStream_t stream2 = nullptr;                // the same for calls on the model's stream
  cudaEvent_t fork2 = nullptr, join2 = nullptr;
  Arena lws[IDOS_MAX_LEVELS];
  cudaEvent_t lev0[IDOS_MAX_LEVELS] = {}, lev1[IDOS_MAX_LEVELS] = {};
  cudaEvent_t fork = nullptr;
  // persistent launch over the levels' shared-memory matrices: per-level
  // "inputs ready" events, the launch's completion, its work counters (three
  // per level: a launch uses those of the lowest level it serves)
  cudaEvent_t lprep[IDOS_MAX_LEVELS] = {};
  cudaEvent_t small_done = nullptr;
  unsigned long long* small_ctr = nullptr;
  // graph replay of idos_sample_levels: per-call values (seed, first sample
  // of every level) read by the mask kernels from dyn_dev; the executable
  // graph of the last key (sample counts, route, partition, arena
  // generations) and how often it was captured / replayed
  int graph = 1;
  cudaStream_t gstream = nullptr;   // origin stream of idos_sample_levels (non-blocking)
  cudaEvent_t fork0 = nullptr;      // caller's stream -> origin stream
  uint64_t* dyn_dev = nullptr;
  uint64_t* dyn_host = nullptr;   // pinned
  cudaEvent_t ljoin[IDOS_MAX_LEVELS] = {};
  cudaGraphExec_t gexec = nullptr;
  std::vector<int64_t> gkey;
  std::vector<int64_t> glast;     // key of the previous call (a repeat is captured)
  int64_t graph_replays = 0, graph_captures = 0;
  std::string graph_note;         // why graph mode was given up ("" while it works)
  uint64_t part_gen = 0;          // bumped by every partition rebuild
  SmPartition part;               // SM split of idos_sample_levels (ctx null: shared SMs)
  std::string part_note;          // why there is no split (empty when there is one or none was asked)
  int lsms[IDOS_MAX_LEVELS] = {};  // SMs of each level stream's partition (0: whole device)
  int sm_split_now = 0;           // SMs reserved for the finest level now (0: no partition)
  int small_max_n = -1;           // largest n on the shared-memory kernel (-1: whatever fits)
  int persistent = 1;             // one persistent launch for the levels' shared-memory matrices
  int w_tile = 1, chase_pair = 1;  // two-stage kernel shapes (SolveArgs)
  int panel_cluster = 0;           // stage-1 panel QR cluster size (SolveArgs)
  int her2k_lower = 1;             // trailing update on lower-triangle tiles (SolveArgs)
  int persist_reserve = 0;         // SMs of its partition the persistent launch leaves free
  double* acc = nullptr;          // device [n_levels][kAccRows][n_E]: sum Y, Y^2, Q_fine, Q_fine^2
  double* tmdc_p = nullptr;       // device parameter table of the TMDC-shaped model (null for graphene)
  int* err = nullptr;             // device [IDOS_MAX_LEVELS + 1] status words: level streams, then the model stream
  int64_t M[IDOS_MAX_LEVELS] = {};
  double seconds[IDOS_MAX_LEVELS] = {};
  Arena ws;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int sm_count = 0;
  Profiler prof;
};

// ---- stage launchers (return idos_status) ----
// dyn (optional, device): [0] seed, read in place of `seed`; [1 + level]
// first sample, to which `first_sample` is added as an offset.
int launch_fine_masks(uint8_t* out, int n_sites, int64_t count, uint64_t seed, int level,
                      int64_t first_sample, double p, cudaStream_t s, const uint64_t* dyn = nullptr);
int launch_corner_masks(const uint8_t* fine, int N, int per_cell, int64_t count, uint8_t* out, cudaStream_t s);
// TMDC-shaped model: orbital masks [count][11 N^2] from pair masks [count][N^2]
int launch_orbital_masks(const uint8_t* pairs, int N, int64_t count, uint8_t* out, cudaStream_t s);
int launch_cell_maps(CellSet& c, cudaStream_t s);
int launch_assemble_dense(const SolveArgs& a, int k_index, double2* out, double sentinel);
// The TMDC-shaped model's parameter table (kTmdcParams doubles, host) drawn
// from model_seed: value i = lo + (hi - lo) u_i, u_i = (w0 >> 11) 2^-53 with w0
// word 0 of Philox4x64-10(counter (i, 0, 0, 0), key (model_seed, 2)).
void tmdc_draw_params(uint64_t model_seed, double lo, double hi, double* out);

// Householder reduction to real symmetric tridiagonal (d, e^2).
bool small_path_fits(int precision, int n_max);
int solve_small(int precision, const SolveArgs& a);

// One segment of the persistent shared-memory launch: every matrix (cell x
// k-point) of one graphene cell set, reduced to float32 (d, e^2).
constexpr int kMaxSmallSegs = 8;
struct SmallSeg {
  const int* n_act = nullptr;
  const int* act = nullptr;
  const int* inv = nullptr;
  int N = 0, Kside = 0, n_max = 0;
  int64_t n_mat = 0;
  float* d = nullptr;
  float* e2 = nullptr;
};
// Largest n_max the persistent launch takes (float32).
constexpr int kPersistMaxN = 160;
// Reduces the matrices of all segments (n_max <= kPersistMaxN each) by
// persistent launches of at most `ctas` - `reserve` CTAs (ctas 0: one per SM
// of the device), each CTA filling one SM, so that `reserve` SMs stay free
// for other streams' kernels: matrices with n_max > 32 are CTA work items,
// handed out largest first; the n_max <= 32 ones are warp work items taken
// one at a time by any warp that is free.  counters: device [3] uint64
// scratch, zeroed here on the stream.
int solve_small_persistent(const SmallSeg* segs, int n_segs, double t, double eps, unsigned long long* counters,
                           int ctas, int reserve, cudaStream_t s);
int solve_large(int precision, const SolveArgs& a);
// Workspace the large-matrix path needs to hold n_mat matrices in one batch.
size_t large_path_bytes(int precision, int n_max, int64_t n_mat);

// Sturm-count bisection: eigs[mat][n_max] ascending, NaN beyond n_act.
// err (nullable, device): status word; bit 2 is set when a matrix's (d, e^2)
// holds a non-finite entry (the reduction broke down).  sym != 0: every
// spectrum is symmetric about `center`; only indices >= n/2 are bisected and
// the rest mirrored.
int launch_bisect(int precision, int refine64_iters, const void* d, const void* e2,
                  const int* n_act_cell, int K2, int n_max, int64_t n_mat, double* eigs,
                  cudaStream_t s, int* err = nullptr, int sym = 0, double center = 0.0);

// Overlap s != 0 (graphene): eigenvalues l of t B -> generalized eigenvalues
// (eps + l) / (1 + sigma l), sigma = s / t, kept ascending.
int launch_overlap_map(double* eigs, const int* n_act_cell, int K2, int n_max, int64_t n_mat, double eps,
                       double sigma, cudaStream_t s);

// Smoothed IDoS per cell (eq. (4.1)-(4.2)): Q[cell][n_E].
struct EnergyGrid { double e_min, e_max, delta; int n_E; int smoothing; int fp32_erfc; };
int launch_idos(const double* eigs, const int* n_act_cell, int K2, int n_max, int64_t n_cells,
                double area, const EnergyGrid& g, double* Q, cudaStream_t s);

// Rows of a level accumulator (float64 [kAccRows][n_E]): sum Y, sum Y^2 (the
// level term of eq. (2.6)), sum Q_fine, sum Q_fine^2 (the fine IDoS alone,
// whose variance decay is the rate S of Sec. 2.1).
constexpr int kAccRows = 4;

// Level difference and float64 statistics: Y = Qf - (1/4) sum_r Qc[r] (or Qf),
// acc[0][j] += sum_s Y, acc[1][j] += sum_s Y^2, acc[2][j] += sum_s Qf,
// acc[3][j] += sum_s Qf^2, optional Y export.
int launch_level_stats(const double* Qf, const double* Qc, int64_t S, int n_E, double* Y,
                       double* acc, Arena& ws, cudaStream_t s);

double cell_area(double a);   // |a1 x a2| = sqrt(3)/2 a^2

// Level sampling for other drivers (api.cu): n_samples of `level` on stream st
// with workspace ws, float64 sums added to acc [kAccRows][n_E] (device, zeroed
// by the caller), err (device status word) zeroed first; ev0 / ev1 recorded
// around the work; returns without waiting.
int level_run_async(Model* M, int level, int64_t n_samples, uint64_t seed, int64_t first, cudaStream_t st,
                    Arena& ws, cudaEvent_t ev0, cudaEvent_t ev1, int* err, double* acc);
// Device workspace such a call reserves (its HBM footprint).
size_t level_footprint(const Model* M, int level, int64_t n_samples);
// Reads a status word after the work that sets it completed.
int read_status_word(const int* err);
// The idos_status of a status word already on the host (0 = IDOS_OK).
int status_of_word(int h);

}  // namespace idos

// The opaque handle of the C ABI is the model object itself.
struct idos_model : public idos::Model {};
