// large.cuh - definitions shared by the two stages of the large-matrix
// reduction (k_large.cu: dense -> band; k_chase.cu: band -> tridiagonal).
#pragma once

#include <cuda.h>

#include "internal.h"

namespace idos {
namespace lg {

constexpr int BW = 16;          // band half-width
constexpr int ND = 2 * BW + 1;  // stored diagonals during the chase

template <typename T> __device__ __forceinline__ T tiny_rest();
template <> __device__ __forceinline__ float tiny_rest<float>() { return 1e-30f; }
template <> __device__ __forceinline__ double tiny_rest<double>() { return 1e-290; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ c2<T> shfl_c(c2<T> v, int src) {
  return mk<T>(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

struct Batch {
  int n_max;
  int B;
  int K2;
  int64_t mat0;
  const int* n_act_cell;   // may be null (all n_max)
};

__device__ __forceinline__ int batch_n(const Batch& b, int m) {
  return b.n_act_cell ? b.n_act_cell[(b.mat0 + m) / b.K2] : b.n_max;
}

// Launch plan of the band chase for matrices of capacity n_max: the dataflow
// kernel on a cluster of csz CTAs (warps per CTA, log2 of the band columns
// per CTA, dynamic shared memory), or csz = 0 for the barrier-per-time-step
// kernel (bands too large for 16 CTAs).
struct ChasePlan {
  int csz = 0, cwarps = 0, ccwl = 0;
  int pair = 0;   // clustered chase with two warps per sweep (k_ts_chase_pair)
  size_t csmem = 0;
  int threads = 0, slots = 0, band_in_smem = 0;
  size_t smem = 0;
};

// Picks the plan for `batch` matrices per launch on `sms` SMs with clusters of
// at most max_cluster CTAs and sets the kernels' shared-memory attributes.
template <typename T>
int chase_plan(int n_max, int64_t batch, int sms, int max_cluster, ChasePlan& p, bool allow_pair = true);

// Copies the band of the dense matrices A (the stage-1 output) into Bd and
// reduces it: d = diagonal, e2 = squared subdiagonal of each tridiagonal.
// err: device status word, set when a dataflow wait gives up.
template <typename T>
int chase_run(const ChasePlan& p, const Batch& bt, const c2<T>* A, c2<T>* Bd, T* d, T* e2, int* err, cudaStream_t s);

// Tensor-core trailing update (k_tc.cu), float32 storage: per batch, the
// split-bfloat16 operand buffers (Aop [B][n_max][64 np], Bop [B][2 n_max][64 np])
// and their TMA descriptors.
struct TcPlan {
  CUtensorMap mapA, mapB, mapC;
  CUtensorMap mapB2, mapCm;   // the lower-triangle update: B boxes of 256 rows, 16-row reduce-add boxes
  CUtensorMap mapWB;          // W's operand B' (in Bop's memory)
  int kw = 0;                 // its row length (bfloat16)
  int lower = 1;              // 1: lower-triangle tiles with mirrored blocks, 0: the full tile grid
  int np = 6;
  int n_max = 0;
  void* Aop = nullptr;
  void* Bop = nullptr;
};

// Device bytes of the operand buffers per matrix of capacity n_max.
size_t tc_operand_bytes(int n_max, int np);

// Encodes the TMA descriptors of the operand buffers and of the dense batch A
// ([batch][n_max][n_max] complex float32, n_max even) for `batch` matrices and
// sets the kernel's shared-memory attribute.  np = 3 or 6 split products.
int tc_plan(TcPlan& p, int n_max, int64_t batch, int np, void* Aop, void* Bop, void* A);

// A22 -= Y Z^H + Z Y^H for every matrix of the batch at panel offset k (the
// trailing block starts at row and column k + BW; k = -BW updates the whole
// matrix).  Y, Z: [B][BW][n_max] complex float32; A is the plan's batch.
int tc_her2k(const TcPlan& p, const Batch& bt, int k, const c2<float>* Y, const c2<float>* Z, int* err, cudaStream_t s);

// W = A22 (Y T) on the tensor cores (six split-bfloat16 products) for every
// matrix of the plan's batch at panel offset k >= 0: partial sums over nsplit
// ranges of A22's columns into Wp[b][split][BW][n_max] (complex float32),
// each range's slice written in full.  YT: [B][BW][n_max].
int tc_w(const TcPlan& p, const Batch& bt, int k, const c2<float>* YT, c2<float>* Wp, int nsplit, int* err,
         cudaStream_t s);

}  // namespace lg
}  // namespace idos
