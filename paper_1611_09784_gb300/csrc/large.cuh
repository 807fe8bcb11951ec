// large.cuh - definitions shared by the two stages of the large-matrix
// reduction (k_large.cu: dense -> band; k_chase.cu: band -> tridiagonal).
#pragma once

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
  size_t csmem = 0;
  int threads = 0, slots = 0, band_in_smem = 0;
  size_t smem = 0;
};

// Picks the plan for `batch` matrices per launch on `sms` SMs and sets the
// kernels' shared-memory attributes.
template <typename T>
int chase_plan(int n_max, int64_t batch, int sms, ChasePlan& p);

// Copies the band of the dense matrices A (the stage-1 output) into Bd and
// reduces it: d = diagonal, e2 = squared subdiagonal of each tridiagonal.
// err: device status word, set when a dataflow wait gives up.
template <typename T>
int chase_run(const ChasePlan& p, const Batch& bt, const c2<T>* A, c2<T>* Bd, T* d, T* e2, int* err, cudaStream_t s);

}  // namespace lg
}  // namespace idos
