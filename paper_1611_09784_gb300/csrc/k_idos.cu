// k_idos.cu - smoothed IDoS per supercell (eq. (4.1)-(4.2), Sec. 4.3) and
// the MLMC level difference with its float64 statistics (eq. (2.6) and the
// variance display after it).
//
// Q(eps_j) = 1/(|F| K^2) sum_k sum_n g((E_n(k) - eps_j)/delta).  Per grid
// point the eigenvalues are ascending, so for every energy the terms with
// (E - eps_j)/delta < -c contribute exactly 1 and those above +c exactly 0
// (to below float64 resolution for c = 8.5 with the Gaussian; exactly for
// the compact polynomial with c = 1): a binary search gives the count below
// the window and only the window's terms are evaluated.  All sums float64.
#include <cfloat>

#include "internal.h"

namespace idos {

namespace {

constexpr int IDOS_THREADS = 256;

__device__ __forceinline__ double smooth_g(double x, int smoothing, int fp32_erfc) {
  if (smoothing == IDOS_SMOOTH_POLY) {
    if (x <= -1.0) return 1.0;
    if (x >= 1.0) return 0.0;
    return 0.5 - 1.125 * x + 0.625 * x * x * x;
  }
  if (fp32_erfc) return 0.5 * (double)erfcf((float)(x * 0.70710678118654752440));
  return 0.5 * erfc(x * 0.70710678118654752440);
}

// One CTA per cell; threads stride over energies.
__global__ void __launch_bounds__(IDOS_THREADS)
k_idos(const double* __restrict__ eigs, const int* __restrict__ n_act_cell, int K2, int n_max,
       double inv_norm, double e_min, double span, double delta, int n_E, int smoothing, int fp32_erfc,
       double* __restrict__ Q) {
  extern __shared__ double sE[];
  const int64_t cell = blockIdx.x;
  const int n = n_act_cell ? n_act_cell[cell] : n_max;
  const double c = (smoothing == IDOS_SMOOTH_POLY) ? 1.0 : 8.5;
  const double inv_delta = 1.0 / delta;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};   // up to 4 energies per thread (n_E <= 1024)
  for (int k = 0; k < K2; ++k) {
    const double* E = eigs + (cell * K2 + k) * (int64_t)n_max;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) sE[i] = E[i];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = threadIdx.x + q * IDOS_THREADS;
      if (j >= n_E) break;
      const double eps = e_min + ((double)j * span) / (double)(n_E - 1);   // eps_j as defined
      const double lo = eps - c * delta, hi = eps + c * delta;
      // first index with E >= lo
      int a = 0, b = n;
      while (a < b) {
        const int m = (a + b) >> 1;
        if (sE[m] < lo) a = m + 1; else b = m;
      }
      double s = (double)a;
      for (int i = a; i < n && sE[i] < hi; ++i) s += smooth_g((sE[i] - eps) * inv_delta, smoothing, fp32_erfc);
      acc[q] += s;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = threadIdx.x + q * IDOS_THREADS;
    if (j < n_E) Q[cell * n_E + j] = acc[q] * inv_norm;
  }
}

constexpr int STAT_CHUNK = 64;

// partial[chunk][0|1][j] over STAT_CHUNK samples, fixed order.
__global__ void k_level_partial(const double* __restrict__ Qf, const double* __restrict__ Qc, int64_t S,
                                int n_E, double* __restrict__ Y, double* __restrict__ partial) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t chunk = blockIdx.y;
  if (j >= n_E) return;
  double s1 = 0.0, s2 = 0.0;
  const int64_t s0 = chunk * STAT_CHUNK, s_end = min(S, s0 + STAT_CHUNK);
  for (int64_t smp = s0; smp < s_end; ++smp) {
    double y = Qf[smp * n_E + j];
    if (Qc) {
      const double* q = Qc + smp * 4 * (int64_t)n_E + j;
      y -= 0.25 * (q[0] + q[n_E] + q[2 * n_E] + q[3 * n_E]);
    }
    if (Y) Y[smp * n_E + j] = y;
    s1 += y;
    s2 += y * y;
  }
  partial[(chunk * 2 + 0) * n_E + j] = s1;
  partial[(chunk * 2 + 1) * n_E + j] = s2;
}

__global__ void k_level_final(const double* __restrict__ partial, int64_t n_chunks, int n_E,
                              double* __restrict__ acc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_E) return;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t c = 0; c < n_chunks; ++c) {
    s1 += partial[(c * 2 + 0) * n_E + j];
    s2 += partial[(c * 2 + 1) * n_E + j];
  }
  acc[j] += s1;
  acc[n_E + j] += s2;
}

}  // namespace

int launch_idos(const double* eigs, const int* n_act_cell, int K2, int n_max, int64_t n_cells,
                double area, const EnergyGrid& g, double* Q, cudaStream_t s) {
  if (n_cells == 0) return IDOS_OK;
  if (g.n_E > 4 * IDOS_THREADS) {
    set_error("n_E above 1024 is not supported by the IDoS kernel");
    return IDOS_ERR_UNSUPPORTED;
  }
  const double span = g.e_max - g.e_min;
  const double inv_norm = 1.0 / (area * K2);
  const size_t smem = sizeof(double) * (size_t)n_max;
  IDOS_CUDA_TRY(cudaFuncSetAttribute(k_idos, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope ps(KID_IDOS, s);
  k_idos<<<(unsigned)n_cells, IDOS_THREADS, smem, s>>>(eigs, n_act_cell, K2, n_max, inv_norm, g.e_min, span,
                                                       g.delta, g.n_E, g.smoothing, g.fp32_erfc, Q);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

int launch_level_stats(const double* Qf, const double* Qc, int64_t S, int n_E, double* Y, double* acc,
                       Arena& ws, cudaStream_t s) {
  if (S == 0) return IDOS_OK;
  const int64_t n_chunks = (S + STAT_CHUNK - 1) / STAT_CHUNK;
  double* partial = ws.take<double>((size_t)n_chunks * 2 * n_E);
  if (!partial) {
    set_error("workspace too small for level statistics");
    return IDOS_ERR_OUT_OF_MEMORY;
  }
  const dim3 grid((n_E + 127) / 128, (unsigned)n_chunks);
  ProfScope ps(KID_LEVEL_STATS, s);
  k_level_partial<<<grid, 128, 0, s>>>(Qf, Qc, S, n_E, Y, partial);
  IDOS_CHECK_LAUNCH();
  k_level_final<<<(n_E + 127) / 128, 128, 0, s>>>(partial, n_chunks, n_E, acc);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

}  // namespace idos
