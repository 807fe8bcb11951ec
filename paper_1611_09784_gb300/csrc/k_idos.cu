// k_idos.cu - smoothed IDoS per supercell (eq. (4.1)-(4.2), Sec. 4.3) and
// the MLMC level difference with its float64 statistics (eq. (2.6) and the
// variance display after it).
//
// Q(eps_j) = 1/(|F| K^2) sum_k sum_n g((E_n(k) - eps_j)/delta).  Only the
// terms inside a window of smoothing widths around eps_j are evaluated; the
// eigenvalues below it count 1 each (see k_idos).
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "internal.h"

namespace idos {

namespace {

constexpr int IDOS_THREADS = 256;

// One CTA per cell; threads stride over energies.  Per grid point the
// eigenvalues (ascending) are mapped to grid coordinates u = (E - e_min)/h
// (float64), split into the bucket ju = floor(u) and the fraction f = u - ju;
// then for energy j, x_j(E) = (E - eps_j)/delta = ((ju - j) + f) h/delta.
// Eigenvalues with ju < j - W have x < -c (their term is 1 to below the
// working precision), those with ju > j + W have x > c (term 0), so the sum
// is a count (a binary search on the non-decreasing ju) plus the terms of
// the 2W + 1 buckets around j.  F32: the window terms and their sum are
// float32 (erfcf), the count and the sums over k are float64.
template <bool F32>
__global__ void __launch_bounds__(IDOS_THREADS)
k_idos(const double* __restrict__ eigs, const int* __restrict__ n_act_cell, int K2, int n_max, double inv_norm,
       double e_min, double inv_h, double h_over_delta, int W, int n_E, int smoothing, double* __restrict__ Q) {
  using R = typename std::conditional<F32, float, double>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* sju = reinterpret_cast<int*>(smem_raw);
  R* sf = reinterpret_cast<R*>(smem_raw + (((size_t)n_max * sizeof(int) + 15) & ~size_t(15)));
  const int64_t cell = blockIdx.x;
  const int n = n_act_cell ? n_act_cell[cell] : n_max;
  const R r = (R)h_over_delta;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};   // up to 4 energies per thread (n_E <= 1024)
  for (int k = 0; k < K2; ++k) {
    const double* E = eigs + (cell * K2 + k) * (int64_t)n_max;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double u = (E[i] - e_min) * inv_h;
      const double fl = floor(u);
      sju[i] = (int)fl;
      sf[i] = (R)(u - fl);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = threadIdx.x + q * IDOS_THREADS;
      if (j >= n_E) break;
      // lo: first index with ju >= j - W;  hi: first index with ju > j + W
      int lo = 0, hi = n;
      {
        int a = 0, b = n;
        while (a < b) { const int m = (a + b) >> 1; if (sju[m] < j - W) a = m + 1; else b = m; }
        lo = a;
        b = n;
        while (a < b) { const int m = (a + b) >> 1; if (sju[m] <= j + W) a = m + 1; else b = m; }
        hi = a;
      }
      R sum = R(0);
      for (int i = lo; i < hi; ++i) {
        const R x = ((R)(sju[i] - j) + sf[i]) * r;
        R g;
        if (smoothing == IDOS_SMOOTH_POLY) {
          g = x <= R(-1) ? R(1) : (x >= R(1) ? R(0) : R(0.5) - R(1.125) * x + R(0.625) * x * x * x);
        } else if constexpr (F32) {
          g = 0.5f * erfcf(x * 0.70710678118654752440f);
        } else {
          g = 0.5 * erfc(x * 0.70710678118654752440);
        }
        sum += g;
      }
      acc[q] += (double)lo + (double)sum;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = threadIdx.x + q * IDOS_THREADS;
    if (j < n_E) Q[cell * n_E + j] = acc[q] * inv_norm;
  }
}

constexpr int STAT_CHUNK = 64;

// partial[chunk][r][j] over STAT_CHUNK samples in a fixed order, rows r of
// the level accumulator: sum Y, sum Y^2, sum Q_fine, sum Q_fine^2.
__global__ void k_level_partial(const double* __restrict__ Qf, const double* __restrict__ Qc, int64_t S,
                                int n_E, double* __restrict__ Y, double* __restrict__ partial) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t chunk = blockIdx.y;
  if (j >= n_E) return;
  double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
  const int64_t s0 = chunk * STAT_CHUNK, s_end = min(S, s0 + STAT_CHUNK);
  for (int64_t smp = s0; smp < s_end; ++smp) {
    const double qf = Qf[smp * n_E + j];
    double y = qf;
    if (Qc) {
      const double* q = Qc + smp * 4 * (int64_t)n_E + j;
      y -= 0.25 * (q[0] + q[n_E] + q[2 * n_E] + q[3 * n_E]);
    }
    if (Y) Y[smp * n_E + j] = y;
    s1 += y;
    s2 += y * y;
    s3 += qf;
    s4 += qf * qf;
  }
  double* pc = partial + chunk * kAccRows * n_E + j;
  pc[0] = s1;
  pc[n_E] = s2;
  pc[2 * n_E] = s3;
  pc[3 * n_E] = s4;
}

__global__ void k_level_final(const double* __restrict__ partial, int64_t n_chunks, int n_E,
                              double* __restrict__ acc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_E) return;
  double s[kAccRows] = {};
  for (int64_t c = 0; c < n_chunks; ++c)
#pragma unroll
    for (int r = 0; r < kAccRows; ++r) s[r] += partial[(c * kAccRows + r) * n_E + j];
#pragma unroll
  for (int r = 0; r < kAccRows; ++r) acc[r * n_E + j] += s[r];
}

}  // namespace

int launch_idos(const double* eigs, const int* n_act_cell, int K2, int n_max, int64_t n_cells,
                double area, const EnergyGrid& g, double* Q, cudaStream_t s) {
  if (n_cells == 0) return IDOS_OK;
  if (g.n_E > 4 * IDOS_THREADS) {
    set_error("n_E above 1024 is not supported by the IDoS kernel");
    return IDOS_ERR_UNSUPPORTED;
  }
  const double h = (g.e_max - g.e_min) / (g.n_E - 1);
  const double inv_norm = 1.0 / (area * K2);
  // half-width of the window in smoothing widths: the Gaussian tail beyond
  // 8.5 (float64) / 6.5 (float32) standard deviations is below the working
  // precision; the compact polynomial vanishes beyond 1
  const double c = g.smoothing == IDOS_SMOOTH_POLY ? 1.0 : (g.fp32_erfc ? 6.5 : 8.5);
  const int W = (int)std::ceil(c * g.delta / h) + 1;
  const size_t smem = (((size_t)n_max * sizeof(int) + 15) & ~size_t(15)) + sizeof(double) * (size_t)n_max;
  ProfScope ps(KID_IDOS, s);
  if (g.fp32_erfc) {
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_idos<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_idos<true><<<(unsigned)n_cells, IDOS_THREADS, smem, s>>>(eigs, n_act_cell, K2, n_max, inv_norm, g.e_min,
                                                               1.0 / h, h / g.delta, W, g.n_E, g.smoothing, Q);
  } else {
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_idos<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_idos<false><<<(unsigned)n_cells, IDOS_THREADS, smem, s>>>(eigs, n_act_cell, K2, n_max, inv_norm, g.e_min,
                                                                1.0 / h, h / g.delta, W, g.n_E, g.smoothing, Q);
  }
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

int launch_level_stats(const double* Qf, const double* Qc, int64_t S, int n_E, double* Y, double* acc,
                       Arena& ws, cudaStream_t s) {
  if (S == 0) return IDOS_OK;
  const int64_t n_chunks = (S + STAT_CHUNK - 1) / STAT_CHUNK;
  double* partial = ws.take<double>((size_t)n_chunks * kAccRows * n_E);
  if (!partial) {
    set_error("workspace too small for level statistics");
    return IDOS_ERR_OUT_OF_MEMORY;
  }
  const dim3 grid((n_E + 127) / 128, (unsigned)n_chunks);
  ProfScope ps(KID_LEVEL_STATS, s, 2);
  k_level_partial<<<grid, 128, 0, s>>>(Qf, Qc, S, n_E, Y, partial);
  IDOS_CHECK_LAUNCH();
  k_level_final<<<(n_E + 127) / 128, 128, 0, s>>>(partial, n_chunks, n_E, acc);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

}  // namespace idos
