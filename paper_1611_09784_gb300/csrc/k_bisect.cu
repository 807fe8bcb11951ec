// k_bisect.cu - eigenvalues of the real symmetric tridiagonal (d, e^2) by
// Sturm-count bisection (E_n(k), the n-th smallest eigenvalue, Sec. 4.3).
//
// count(x) = number of eigenvalues below x = number of negative pivots of
// the LDL^T factorisation of T - x I:
//   q_0 = d_0 - x,  q_i = (d_i - x) - e_{i-1}^2 / q_{i-1},
// with a pivot of magnitude below pivmin replaced by -pivmin (a perturbation
// of x by at most pivmin).  Eigenvalue k (0-based) is the smallest x with
// count(x) >= k + 1; each thread bisects one index inside the Gershgorin
// interval, all threads of a group reading the same (d, e^2) from shared
// memory (broadcast).  IDOS_FP32_REFINE64 bisects in float32 to convergence
// and then continues `refine` steps in float64 on the same tridiagonal.
#include <cfloat>

#include "internal.h"

namespace idos {

namespace {

template <typename T, typename S>
__device__ __forceinline__ int sturm_count(const S* __restrict__ d, const S* __restrict__ e2, int n,
                                           T x, T pivmin) {
  T q = T(d[0]) - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int cnt = q < T(0);
  for (int i = 1; i < n; ++i) {
    T r;
    if constexpr (sizeof(T) == 4) r = __fdividef(T(e2[i - 1]), q);
    else r = T(e2[i - 1]) / q;
    q = (T(d[i]) - x) - r;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < T(0);
  }
  return cnt;
}

template <typename T>
__device__ __forceinline__ T ulp_of(T x) {
  if constexpr (sizeof(T) == 4) return fabsf(x) * FLT_EPSILON + FLT_MIN;
  else return fabs(x) * DBL_EPSILON + DBL_MIN;
}

// Bisect [lo, hi] for eigenvalue index k: count(lo) <= k < count(hi).
template <typename T, typename S>
__device__ __forceinline__ void bisect_index(const S* d, const S* e2, int n, int k, T pivmin, T& lo,
                                             T& hi, int max_iter) {
  for (int it = 0; it < max_iter; ++it) {
    const T mid = T(0.5) * (lo + hi);
    if (!(mid > lo && mid < hi)) break;                     // no representable midpoint left
    if (hi - lo <= T(2) * ulp_of<T>(fabs(lo) > fabs(hi) ? lo : hi)) break;
    if (sturm_count<T, S>(d, e2, n, mid, pivmin) >= k + 1) hi = mid;
    else lo = mid;
  }
}

// One group of G threads per matrix, MPB groups per CTA.  S = storage type of
// (d, e^2); float64 bisection when S is double, float32 + refine otherwise.
template <typename S, int G, int MPB>
__global__ void __launch_bounds__(G* MPB)
k_bisect(const S* __restrict__ d_in, const S* __restrict__ e2_in, const int* __restrict__ n_act_cell,
         int K2, int n_max, int64_t n_mat, int refine, double* __restrict__ eigs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int gid = threadIdx.x / G, tid = threadIdx.x % G;
  const int64_t mat = (int64_t)blockIdx.x * MPB + gid;
  if (mat >= n_mat) return;
  S* d = reinterpret_cast<S*>(smem_raw) + (size_t)gid * 2 * n_max;
  S* e2 = d + n_max;
  __shared__ double red_lo[MPB][G / 32], red_hi[MPB][G / 32], red_e[MPB][G / 32];
  const int n = n_act_cell ? n_act_cell[mat / K2] : n_max;
  double* out = eigs + mat * n_max;
  for (int i = tid; i < n_max; i += G) {
    if (i >= n) out[i] = __longlong_as_double(0x7ff8000000000000ll);   // NaN padding
  }
  if (n <= 0) return;
  // Gershgorin bounds and the largest e^2, in double for safety
  double glo = 1e300, ghi = -1e300, emax = 0.0;
  for (int i = tid; i < n; i += G) {
    const S di = d_in[mat * n_max + i];
    const S ei = (i < n - 1) ? e2_in[mat * n_max + i] : S(0);
    d[i] = di;
    e2[i] = ei;
    const double el = (i > 0) ? sqrt((double)e2_in[mat * n_max + i - 1]) : 0.0;
    const double er = sqrt((double)ei);
    glo = fmin(glo, (double)di - el - er);
    ghi = fmax(ghi, (double)di + el + er);
    emax = fmax(emax, (double)ei);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
  if constexpr (G > 32) {
    const int w = tid >> 5;
    if ((tid & 31) == 0) { red_lo[gid][w] = glo; red_hi[gid][w] = ghi; red_e[gid][w] = emax; }
    group_sync<G, MPB>(gid);
    for (int q = 0; q < G / 32; ++q) {
      glo = fmin(glo, red_lo[gid][q]);
      ghi = fmax(ghi, red_hi[gid][q]);
      emax = fmax(emax, red_e[gid][q]);
    }
  }
  group_sync<G, MPB>(gid);
  const double span = fmax(ghi - glo, 1e-30);
  glo -= 1e-6 * span + 1e-12;   // float rounding of the reduced bounds
  ghi += 1e-6 * span + 1e-12;
  for (int k = tid; k < n; k += G) {
    if constexpr (sizeof(S) == 8) {
      const double piv = 1e-290 * fmax(1.0, emax);
      double lo = glo, hi = ghi;
      bisect_index<double, S>(d, e2, n, k, piv, lo, hi, 200);
      out[k] = 0.5 * (lo + hi);
    } else {
      const float piv = 1e-30f * fmaxf(1.0f, (float)emax);
      float lo = (float)glo, hi = (float)ghi;
      bisect_index<float, S>(d, e2, n, k, piv, lo, hi, 100);
      double dlo = lo, dhi = hi;
      const double piv64 = 1e-290 * fmax(1.0, emax);
      for (int it = 0; it < refine; ++it) {
        const double mid = 0.5 * (dlo + dhi);
        if (sturm_count<double, S>(d, e2, n, mid, piv64) >= k + 1) dhi = mid;
        else dlo = mid;
      }
      out[k] = 0.5 * (dlo + dhi);
    }
  }
}

template <typename S, int G, int MPB>
int run_bisect(const void* d, const void* e2, const int* n_act_cell, int K2, int n_max, int64_t n_mat,
               int refine, double* eigs, cudaStream_t s) {
  const size_t smem = sizeof(S) * 2 * (size_t)n_max * MPB;
  auto kern = k_bisect<S, G, MPB>;
  IDOS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t blocks = (n_mat + MPB - 1) / MPB;
  ProfScope ps(KID_BISECT, s);
  kern<<<(unsigned)blocks, G * MPB, smem, s>>>(reinterpret_cast<const S*>(d), reinterpret_cast<const S*>(e2),
                                               n_act_cell, K2, n_max, n_mat, refine, eigs);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

template <typename S>
int bisect_t(int refine, const void* d, const void* e2, const int* n_act_cell, int K2, int n_max,
             int64_t n_mat, double* eigs, cudaStream_t s) {
  if (n_max <= 32) return run_bisect<S, 32, 8>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s);
  if (n_max <= 64) return run_bisect<S, 64, 4>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s);
  if (n_max <= 128) return run_bisect<S, 128, 2>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s);
  if (n_max <= 256) return run_bisect<S, 256, 1>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s);
  if (n_max <= 512) return run_bisect<S, 512, 1>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s);
  return run_bisect<S, 1024, 1>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s);
}

}  // namespace

int launch_bisect(int precision, int refine64_iters, const void* d, const void* e2,
                  const int* n_act_cell, int K2, int n_max, int64_t n_mat, double* eigs,
                  cudaStream_t s) {
  if (n_mat == 0) return IDOS_OK;
  if (precision == IDOS_FP64)
    return bisect_t<double>(0, d, e2, n_act_cell, K2, n_max, n_mat, eigs, s);
  return bisect_t<float>(refine64_iters, d, e2, n_act_cell, K2, n_max, n_mat, eigs, s);
}

}  // namespace idos
