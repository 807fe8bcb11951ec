// k_peak.cu - FMA issue-rate microbenchmark: the denominators of the ALU
// rooflines (float32 and float64 FMA throughput of this device at the clocks
// it runs at), measured with the same CUDA-event timing as the kernels they
// are compared with.
//
// Every thread runs kChains independent dependent-FMA chains a <- a b + c, so
// each SM sub-partition has enough independent FMAs in flight to cover the
// pipe latency; the grid is a whole number of CTAs per SM.  The sum of the
// chains is stored only when the runtime argument `store` is nonzero, so the
// compiler keeps the arithmetic; the host always passes 0 (and no buffer), so
// the kernel touches no memory.
#include <cuda_runtime.h>

#include "internal.h"

namespace idos {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

// Chain i uses its own multiplier b + i db (runtime values), so no two chains
// can be merged.
template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int iters, T b, T db, T c, int store, T* __restrict__ out) {
  T a[kChains], bi[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    a[i] = T(threadIdx.x + i) * T(1e-3);
    bi[i] = b + T(i) * db;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], bi[i], c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (store) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace idos

using namespace idos;

extern "C" int idos_measure_fma_peak(int precision, int64_t iters, void* cuda_stream, double* flops_per_s,
                                     double* ms_out) {
  if (!flops_per_s || (precision != IDOS_FP64 && precision != IDOS_FP32_REFINE64) || iters < 1 ||
      iters > (int64_t)1 << 30) {
    set_error("null output, precision not IDOS_FP64 / IDOS_FP32_REFINE64, or iters outside 1 .. 2^30");
    return IDOS_ERR_INVALID_ARG;
  }
  int sms = 0;
  IDOS_TRY(check_device(sms));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  // 8 CTAs of 256 threads per SM: 64 warps, 16 per sub-partition
  const unsigned grid = (unsigned)sms * 8;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  IDOS_CUDA_TRY(cudaEventCreate(&e0));
  cudaError_t err = cudaEventCreate(&e1);
  float ms = 0.f;
  if (err == cudaSuccess) {
    // warm-up launch (clocks up, module loaded), then the timed one
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {
      if (rep == 1) err = cudaEventRecord(e0, s);
      if (err != cudaSuccess) break;
      if (precision == IDOS_FP64)
        k_fma_peak<double><<<grid, kPeakThreads, 0, s>>>((int)(rep ? iters : iters / 8 + 1), 0.9999999, 1e-9, 1e-7, 0, nullptr);
      else
        k_fma_peak<float><<<grid, kPeakThreads, 0, s>>>((int)(rep ? iters : iters / 8 + 1), 0.9999f, 1e-6f, 1e-4f, 0, nullptr);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    set_error(std::string("fma peak: ") + cudaGetErrorString(err));
    return IDOS_ERR_CUDA;
  }
  const double flops = 2.0 * kChains * (double)iters * grid * kPeakThreads;
  *flops_per_s = flops / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return IDOS_OK;
}
