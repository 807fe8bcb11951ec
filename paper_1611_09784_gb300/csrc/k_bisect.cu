// k_bisect.cu - eigenvalues of the real symmetric tridiagonal (d, e^2) by
// Sturm-count bisection (E_n(k), the n-th smallest eigenvalue, Sec. 4.3).
//
// count(x) = number of eigenvalues below x = number of negative pivots of
// the LDL^T factorisation of T - x I:
//   q_0 = d_0 - x,  q_i = (d_i - x) - e_{i-1}^2 / q_{i-1},
// with a pivot of magnitude below pivmin replaced by -pivmin (a perturbation
// of x by at most pivmin).  Eigenvalue k (0-based) is the smallest x with
// count(x) >= k + 1; each thread bisects one index inside the Gershgorin
// interval in float32, all threads of a group reading the same (d, e^2)
// from shared memory (broadcast).
//
// The float64 stage works on the characteristic polynomials of the leading
// blocks, p_0 = 1, p_1 = d_0 - x, p_{i+1} = (d_i - x) p_i - e_{i-1}^2 p_{i-1}
// (a pivot is p_{i+1}/p_i, so the count is the number of sign changes), and
// their x-derivatives, rescaled by exact powers of two: no division.  One
// pass gives the count at x and the Newton step -p_n/p_n', used inside the
// current bracket (safeguarded Newton: bisect when the step leaves it).
// Every matrix is first scaled by an exact power of two so that its
// Gershgorin interval lies within [-1, 1] (results scaled back exactly).
//   IDOS_FP32_REFINE64: float32 bisection to 2 ulp or 2 eps |T|, whichever is
//     wider, then refine64_iters passes starting at the bracket midpoint, with
//     count and p_n in float64 and p_n' in float32;
//   IDOS_FP64: float32 bisection on the rounded tridiagonal gives a bracket,
//     checked and widened in float64, then safeguarded Newton, all in float64,
//     to float64 resolution.
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

// Sign, zero and exponent tests on the bit pattern (integer pipe); the
// float64 pipe is kept for the recurrence itself.
__device__ __forceinline__ bool dneg(double v) { return __double2hiint(v) < 0; }
__device__ __forceinline__ bool dzero(double v) { return (__double_as_longlong(v) << 1) == 0; }
__device__ __forceinline__ int dexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

// One float64 pass over (d, e^2) held in float64: count of eigenvalues below
// x and the Newton step -p_n(x)/p_n'(x) of the characteristic polynomial.
// Five float64 operations per row: t = d_i - x, p' = t p - b p_prev and
// q' = t q - (b q_prev + p) as two fused pairs (four with CD: every d_i equal
// to d_0 bit for bit, t formed once with the same value).
template <bool CD>
__device__ __forceinline__ int sturm_newton64(const double* __restrict__ d, const double* __restrict__ e2, int n,
                                              double x, double& step) {
  const double t0 = d[0] - x;
  double p0 = 1.0, p1 = t0;                     // p_{i-1}, p_i
  double q0 = 0.0, q1 = -1.0;                   // derivatives
  if (dzero(p1)) p1 = -0x1p-1000;              // exact zero pivot counts as negative
  int cnt = dneg(p1);
  for (int i = 1; i < n; ++i) {
    const double t = CD ? t0 : d[i] - x, b = e2[i - 1];
    double p2 = fma(t, p1, -(b * p0));
    const double q2 = fma(t, q1, -fma(b, q0, p1));
    if (dzero(p2)) p2 = -copysign(fmax(fabs(p1) * 0x1p-52, 0x1p-1000), p1);   // zero pivot -> negative
    cnt += dneg(p2) != dneg(p1);
    p0 = p1; p1 = p2; q0 = q1; q1 = q2;
    if ((i & 15) == 0) {
      // keep the sequence in range: exact scaling by 2^-e, e the largest
      // binary exponent (biased exponent fields compared as integers)
      const int eb = max(max(dexp(p0), dexp(p1)), max(dexp(q0), dexp(q1)));
      if ((eb > 1023 + 400 && eb < 2047) || (eb > 0 && eb < 1023 - 400)) {
        const double sc = __hiloint2double((2046 - eb) << 20, 0);   // 2^(1023 - eb)
        p0 *= sc; p1 *= sc; q0 *= sc; q1 *= sc;
      }
    }
  }
  step = (q1 != 0.0) ? -p1 / q1 : 0.0;
  return cnt;
}

__device__ __forceinline__ int fexp(float v) { return (__float_as_int(v) >> 23) & 0xff; }

// The float32 path keeps its rows interleaved: de[i] = (d_i, e^2_{i-1}) in
// float32 and dde[i] the same pair in float64, so a row is one 8-byte
// (16-byte) shared-memory load.  sturm_count_pairs is sturm_count on de.
// sturm_newton_mixed_pairs is the float64 pass above with the derivative
// carried in float32: the count and p_n(x) (the residual, where the
// cancellation is) stay float64 - three float64 operations per row - while p'
// only sets the Newton step length, for which float32 accuracy is ample (a
// relative error r in p' leaves an error r times the step; a wild value is
// caught by the bracket safeguard).  The float32 recurrence runs on a float32
// copy of p (from de, the same normalised tridiagonal rounded to float32), so
// no per-row float64 -> float32 conversion is needed.  With |T| <= 1 (the
// caller normalises) a value grows by at most 3x per row, so an exponent
// check every 8 rows that rescales all values by 2^-e once the largest binary
// exponent e leaves [-60, 60] keeps the float32 values far from overflow.
__device__ __forceinline__ int sturm_count_pairs(const float2* __restrict__ de, int n, float x, float pivmin) {
  float q = de[0].x - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = q < 0.f;
  for (int i = 1; i < n; ++i) {
    const float2 r = de[i];
    q = (r.x - x) - __fdividef(r.y, q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.f;
  }
  return cnt;
}

// CD: every diagonal entry equals the first (bit for bit), so d_i - x is the
// same in every row and is formed once: two float64 operations per row
// instead of three, with exactly the values of the general recurrence.
template <bool CD>
__device__ __forceinline__ int sturm_newton_mixed_pairs(const double2* __restrict__ dde, const float2* __restrict__ de,
                                                        int n, double x, double& step) {
  const float x32 = (float)x;
  const double t0 = dde[0].x - x;
  const float t0f = de[0].x - x32;
  double p0 = 1.0, p1 = t0;
  float r0 = 1.0f, r1 = t0f;
  float q0 = 0.0f, q1 = -1.0f;
  if (dzero(p1)) p1 = -0x1p-1000;
  int cnt = dneg(p1);
  bool lost = false;
  for (int i = 1; i < n; ++i) {
    const double2 rd = dde[i];
    const float2 rf = de[i];
    const double t = CD ? t0 : rd.x - x;
    double p2 = fma(t, p1, -(rd.y * p0));
    const float t32 = CD ? t0f : rf.x - x32, b32 = rf.y;
    const float r2 = fmaf(t32, r1, -(b32 * r0));
    const float q2 = fmaf(t32, q1, -fmaf(b32, q0, r1));
    if (dzero(p2)) p2 = dneg(p1) ? 0x1p-1000 : -0x1p-1000;
    cnt += dneg(p2) != dneg(p1);
    p0 = p1; p1 = p2; r0 = r1; r1 = r2; q0 = q1; q1 = q2;
    if ((i & 7) == 0) {
      const int ep = max(dexp(p0), dexp(p1));
      const int eq = max(fexp(q0), fexp(q1));
      const int e = max(ep > 0 ? ep - 1023 : -2000, eq > 0 ? eq - 127 : -2000);
      if (e > 60 || (e < -60 && e > -2000)) {
        const int ed = min(max(e, -1000), 1000), ef = min(max(e, -126), 126);
        const double sd = __hiloint2double((1023 - ed) << 20, 0);
        const float sf = __int_as_float((127 - ef) << 23);
        p0 *= sd; p1 *= sd;
        r0 *= sf; r1 *= sf; q0 *= sf; q1 *= sf;
        lost |= ed != ef;
      }
    }
  }
  step = (!lost && q1 != 0.0f) ? -p1 * (double)(1.0f / q1) : 0.0;
  return cnt;
}

// Safeguarded Newton for eigenvalue k inside [lo, hi] (count(lo) <= k < count(hi)).
// Pass(x, step) returns count(x) and sets the Newton step.
template <typename Pass>
__device__ __forceinline__ double newton_polish(Pass pass, int k, double lo, double hi, int passes) {
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < passes; ++it) {
    double step;
    const int c = pass(x, step);
    if (c >= k + 1) hi = x; else lo = x;
    const double xn = x + step;
    const bool inside = xn > lo && xn < hi;
    const double nx = inside ? xn : 0.5 * (lo + hi);
    if (nx == x || hi - lo <= 4.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 1e-300) { x = nx; break; }
    if (inside && fabs(step) <= 2.0 * DBL_EPSILON * fabs(x)) { x = nx; break; }
    x = nx;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T ulp_of(T x) {
  if constexpr (sizeof(T) == 4) return fabsf(x) * FLT_EPSILON + FLT_MIN;
  else return fabs(x) * DBL_EPSILON + DBL_MIN;
}

// Bisect [lo, hi] for eigenvalue index k: count(lo) <= k < count(hi).  The
// bracket stops shrinking at 2 ulp of the eigenvalue or at atol, whichever is
// larger: the float32 count itself is only backward stable to a perturbation
// of order ulp * |T| of the matrix, so narrowing a bracket around an
// eigenvalue near zero (a zero mode) below that scale buys no accuracy, and it
// would hold the whole warp for up to ~100 iterations instead of ~24.
template <typename T, typename S>
__device__ __forceinline__ void bisect_index(const S* d, const S* e2, int n, int k, T pivmin, T& lo,
                                             T& hi, int max_iter, T atol) {
  for (int it = 0; it < max_iter; ++it) {
    const T mid = T(0.5) * (lo + hi);
    if (!(mid > lo && mid < hi)) break;                     // no representable midpoint left
    if (hi - lo <= fmax(T(2) * ulp_of<T>(fabs(lo) > fabs(hi) ? lo : hi), atol)) break;
    if (sturm_count<T, S>(d, e2, n, mid, pivmin) >= k + 1) hi = mid;
    else lo = mid;
  }
}

__device__ __forceinline__ void bisect_index_pairs(const float2* de, int n, int k, float pivmin, float& lo, float& hi,
                                                   int max_iter, float atol) {
  for (int it = 0; it < max_iter; ++it) {
    const float mid = 0.5f * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (hi - lo <= fmaxf(2.0f * ulp_of<float>(fabsf(lo) > fabsf(hi) ? lo : hi), atol)) break;
    if (sturm_count_pairs(de, n, mid, pivmin) >= k + 1) hi = mid;
    else lo = mid;
  }
}

// Byte offset of the float64 pair copies in the float32 layout (16-byte aligned).
__host__ __device__ __forceinline__ size_t bisect_pair_offset(int n_max, int mpb) {
  return (sizeof(float) * 2 * (size_t)(n_max + 1) * mpb + 15) & ~size_t(15);
}

// One group of G threads per (matrix, chunk of `chunk` eigenvalue indices),
// MPB groups per CTA; every group holds its matrix's whole (d, e^2) in shared
// memory.  S = storage type of (d, e^2).
// sym != 0: the spectrum is symmetric about `center` (a bipartite hopping
// matrix plus center I: chiral symmetry), so only the indices k >= n / 2 are
// bisected and lambda_{n-1-k} = 2 center - lambda_k is written beside them.
template <typename S, int G, int MPB>
__global__ void __launch_bounds__(G* MPB)
k_bisect(const S* __restrict__ d_in, const S* __restrict__ e2_in, const int* __restrict__ n_act_cell,
         int K2, int n_max, int64_t n_mat, int chunk, int refine, double* __restrict__ eigs, int* __restrict__ err,
         int sym, double center) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int gid = threadIdx.x / G, tid = threadIdx.x % G;
  const int n_chunks = (n_max + chunk - 1) / chunk;
  const int64_t gidx = (int64_t)blockIdx.x * MPB + gid;
  const int64_t mat = gidx / n_chunks;
  const int c_lo = (int)(gidx - mat * n_chunks) * chunk;
  const int c_hi = min(n_max, c_lo + chunk);
  if (mat >= n_mat) return;
  // float64 storage: d[n_max], e2[n_max] per group.  float32 storage: the
  // same bytes hold de[n_max] = (d_i, e^2_{i-1}) pairs, then (16-byte
  // aligned) their float64 copies dde[n_max].
  // per-group arrays padded by one element: two half-warp groups reading
  // the same row index then hit different banks
  const int gs = n_max + 1;
  S* d = reinterpret_cast<S*>(smem_raw) + (size_t)gid * 2 * gs;
  S* e2 = d + n_max;
  float2* de = reinterpret_cast<float2*>(smem_raw) + (size_t)gid * gs;
  double2* dde = reinterpret_cast<double2*>(smem_raw + bisect_pair_offset(n_max, MPB)) + (size_t)gid * gs;
  double* dd = reinterpret_cast<double*>(d);   // float64 path: the same arrays
  double* ee = dd + n_max;
  constexpr int NW = G >= 32 ? G / 32 : 1;
  __shared__ double red_lo[MPB][NW], red_hi[MPB][NW], red_e[MPB][NW];
  __shared__ int red_cd[MPB][NW];
  // the lanes of this group (half-warp groups shuffle within their half)
  const unsigned gmask = G >= 32 ? 0xffffffffu : (0xFFFFu << (16 * (gid & 1)));
  __shared__ int ms_cnt[MPB][G];
  const int n = n_act_cell ? n_act_cell[mat / K2] : n_max;
  double* out = eigs + mat * n_max;
  for (int i = c_lo + tid; i < c_hi; i += G) {
    if (i >= n) out[i] = __longlong_as_double(0x7ff8000000000000ll);   // NaN padding
  }
  const int h0 = sym ? n / 2 : 0;   // first bisected index
  if (n <= 0 || c_lo >= n || c_hi <= h0) return;
  // Gershgorin bounds and the largest e^2 in the storage precision (widened
  // below by far more than their rounding)
  S glo_s = S(1e30), ghi_s = S(-1e30), emax_s = S(0);
  const S d_first = d_in[mat * n_max];
  bool cdiag = true;   // every diagonal entry equal to the first, bit for bit
  for (int i = tid; i < n; i += G) {
    const S di = d_in[mat * n_max + i];
    if constexpr (sizeof(S) == 4) cdiag = cdiag && __float_as_int(di) == __float_as_int(d_first);
    else cdiag = cdiag && __double_as_longlong(di) == __double_as_longlong(d_first);
    const S ei = (i < n - 1) ? e2_in[mat * n_max + i] : S(0);
    // a non-finite entry means the reduction broke down: report it (status
    // bit 2) rather than return eigenvalues of a corrupted matrix
    if (err && !(isfinite(di) && isfinite(ei))) atomicOr(err, 2);
    if constexpr (sizeof(S) == 4) {
      float* def = reinterpret_cast<float*>(de);
      def[2 * i] = di;
      if (i + 1 < n) def[2 * (i + 1) + 1] = ei;
      if (i == 0) def[1] = 0.0f;
    } else {
      d[i] = di;
      e2[i] = ei;
    }
    const S el = (i > 0) ? sqrt(e2_in[mat * n_max + i - 1]) : S(0);
    const S er = sqrt(ei);
    glo_s = fmin(glo_s, di - el - er);
    ghi_s = fmax(ghi_s, di + el + er);
    emax_s = fmax(emax_s, ei);
  }
#pragma unroll
  for (int o = G >= 32 ? 16 : G / 2; o > 0; o >>= 1) {
    glo_s = fmin(glo_s, __shfl_xor_sync(gmask, glo_s, o));
    ghi_s = fmax(ghi_s, __shfl_xor_sync(gmask, ghi_s, o));
    emax_s = fmax(emax_s, __shfl_xor_sync(gmask, emax_s, o));
  }
  cdiag = __all_sync(gmask, cdiag);
  double glo = (double)glo_s, ghi = (double)ghi_s, emax = (double)emax_s;
  if constexpr (G > 32) {
    const int w = tid >> 5;
    if ((tid & 31) == 0) { red_lo[gid][w] = glo; red_hi[gid][w] = ghi; red_e[gid][w] = emax; red_cd[gid][w] = cdiag; }
    group_sync<G, MPB>(gid);
    for (int q = 0; q < G / 32; ++q) {
      glo = fmin(glo, red_lo[gid][q]);
      ghi = fmax(ghi, red_hi[gid][q]);
      emax = fmax(emax, red_e[gid][q]);
      cdiag = cdiag && red_cd[gid][q] != 0;
    }
  }
  // Normalise by an exact power of two, sc = 2^-e with max(|glo|, |ghi|) =
  // m 2^e, m in [0.5, 1): every pass below works on T' = sc T (eigenvalues
  // sc lambda, counts unchanged), so the float32 values of the mixed pass
  // stay in range whatever the scale of the input; results are scaled back
  // exactly.
  int ex = 0;
  const double tn = fmax(fabs(glo), fabs(ghi));
  if (tn > 0.0 && tn < 1e300) frexp(tn, &ex);
  ex = sizeof(S) == 4 ? min(max(ex, -60), 60) : min(max(ex, -900), 900);
  const double sc = ldexp(1.0, -ex), isc = ldexp(1.0, ex);
  group_sync<G, MPB>(gid);
  const S sc_s = (S)sc;   // 2^-ex, |ex| <= 900: exact in float64; float32 uses |ex| <= 60
  for (int i = tid; i < n; i += G) {
    if constexpr (sizeof(S) == 4) {
      float2 r = de[i];
      r.x = r.x * sc_s;
      r.y = r.y * sc_s * sc_s;
      de[i] = r;
      dde[i] = make_double2((double)r.x, (double)r.y);
    } else {
      d[i] = d[i] * sc_s;
      e2[i] = e2[i] * sc_s * sc_s;
    }
  }
  group_sync<G, MPB>(gid);
  glo *= sc;
  ghi *= sc;
  emax *= sc * sc;
  const double span = fmax(ghi - glo, 1e-30);
  glo -= 1e-6 * span + 1e-12;   // float rounding of the reduced bounds
  ghi += 1e-6 * span + 1e-12;
  const float piv32 = 1e-30f * fmaxf(1.0f, (float)emax);
  const float atol32 = 2.0f * FLT_EPSILON * (float)fmax(fabs(glo), fabs(ghi));
  // Multisection start: thread t counts the eigenvalues below the interior
  // point x_t = glo + (t + 1) (ghi - glo) / (G + 1) of the Gershgorin
  // interval; eigenvalue k then starts from the two neighbouring points whose
  // counts bracket it (a binary search that keeps count(lo) <= k < count(hi)
  // for whatever counts it reads), saving about log2(G + 1) - 1 bisection
  // steps per eigenvalue for one count per thread.
  // (float32 points from one float64 step: no float64 division per point)
  const float ms_lo = (float)glo, ms_step = (float)((ghi - glo) / (double)(G + 1));
  const auto x_ms = [&](int t) { return fmaf((float)(t + 1), ms_step, ms_lo); };
  {
    int c;
    if constexpr (sizeof(S) == 4) c = sturm_count_pairs(de, n, x_ms(tid), piv32);
    else c = sturm_count<float, S>(d, e2, n, x_ms(tid), piv32);
    ms_cnt[gid][tid] = c;
  }
  group_sync<G, MPB>(gid);
  const auto ms_bracket = [&](int k, float& lo, float& hi) {
    int L = -1, H = G;   // x_{-1} = glo (count 0), x_G = ghi (count n)
    while (H - L > 1) {
      const int mid = (L + H) >> 1;
      if (ms_cnt[gid][mid] >= k + 1) H = mid;
      else L = mid;
    }
    lo = L < 0 ? (float)glo : x_ms(L);
    hi = H >= G ? (float)ghi : x_ms(H);
  };
  for (int k = max(c_lo, h0) + tid; k < min(n, c_hi); k += G) {
    double lam;
    if constexpr (sizeof(S) == 8) {
      // float32 bracket on the rounded tridiagonal (float64 data read and
      // rounded on the fly), widened, checked in float64, then polished
      float lo32, hi32;
      ms_bracket(k, lo32, hi32);
      bisect_index<float, S>(d, e2, n, k, piv32, lo32, hi32, 100, atol32);
      const double w = 64.0 * (double)FLT_EPSILON * fmax(fabs(glo), fabs(ghi)) + 1e-12;
      double lo = fmax(glo, (double)lo32 - w), hi = fmin(ghi, (double)hi32 + w);
      double st;
      const auto pass = [&](double x, double& step) {
        return cdiag ? sturm_newton64<true>(dd, ee, n, x, step) : sturm_newton64<false>(dd, ee, n, x, step);
      };
      if (pass(lo, st) > k) lo = glo;      // bracket lost: fall back
      if (pass(hi, st) < k + 1) hi = ghi;
      lam = isc * newton_polish(pass, k, lo, hi, 60);
    } else {
      float lo, hi;
      ms_bracket(k, lo, hi);
      bisect_index_pairs(de, n, k, piv32, lo, hi, 100, atol32);
      if (refine <= 0) {
        lam = isc * 0.5 * ((double)lo + (double)hi);
      } else if (cdiag) {
        const auto pass = [&](double x, double& step) { return sturm_newton_mixed_pairs<true>(dde, de, n, x, step); };
        lam = isc * newton_polish(pass, k, (double)lo, (double)hi, refine);
      } else {
        const auto pass = [&](double x, double& step) { return sturm_newton_mixed_pairs<false>(dde, de, n, x, step); };
        lam = isc * newton_polish(pass, k, (double)lo, (double)hi, refine);
      }
    }
    // an upper-half eigenvalue of a symmetric spectrum is >= center; a
    // rounding-level value below it (a zero mode) is raised to it, so that
    // the mirrored sequence stays ascending across the middle
    if (sym) lam = fmax(lam, center);
    out[k] = lam;
    if (sym && n - 1 - k != k) out[n - 1 - k] = 2.0 * center - lam;
  }
}

template <typename S, int G, int MPB>
int run_bisect(const void* d, const void* e2, const int* n_act_cell, int K2, int n_max, int64_t n_mat,
               int refine, double* eigs, cudaStream_t s, int chunk, int* err, int sym, double center) {
  const size_t smem = sizeof(S) == 4 ? bisect_pair_offset(n_max, MPB) + sizeof(double) * 2 * (size_t)(n_max + 1) * MPB
                                     : sizeof(S) * 2 * (size_t)(n_max + 1) * MPB;
  auto kern = k_bisect<S, G, MPB>;
  IDOS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t groups = n_mat * ((n_max + chunk - 1) / chunk);
  const int64_t blocks = (groups + MPB - 1) / MPB;
  ProfScope ps(KID_BISECT, s);
  kern<<<(unsigned)blocks, G * MPB, smem, s>>>(reinterpret_cast<const S*>(d), reinterpret_cast<const S*>(e2),
                                               n_act_cell, K2, n_max, n_mat, chunk, refine, eigs, err, sym, center);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

template <typename S>
int bisect_t(int refine, const void* d, const void* e2, const int* n_act_cell, int K2, int n_max,
             int64_t n_mat, double* eigs, cudaStream_t s, int* err, int sym, double center) {
  if (sym) {
    // half the indices per matrix: groups of half the size
    if (n_max <= 32)
      return run_bisect<S, 16, 16>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s, n_max, err, 1, center);
    if (n_max <= 64)
      return run_bisect<S, 32, 8>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s, n_max, err, 1, center);
    if (n_max <= 128)
      return run_bisect<S, 64, 4>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s, n_max, err, 1, center);
    if (n_max <= 256)
      return run_bisect<S, 128, 2>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s, n_max, err, 1, center);
    // chunks of 128 indices; the chunks below n / 2 return at once
    return run_bisect<S, 128, 1>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s, 128, err, 1, center);
  }
  if (n_max <= 32) return run_bisect<S, 32, 8>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s, n_max, err, 0, 0.0);
  if (n_max <= 64) return run_bisect<S, 64, 4>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s, n_max, err, 0, 0.0);
  if (n_max <= 128) return run_bisect<S, 128, 2>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s, n_max, err, 0, 0.0);
  // larger matrices: 128 eigenvalue indices per CTA, so one matrix spreads over n/128 SMs
  return run_bisect<S, 128, 1>(d, e2, n_act_cell, K2, n_max, n_mat, refine, eigs, s, 128, err, 0, 0.0);
}

}  // namespace

// Generalized eigenvalues of the graphene pencil (H, S) = (eps I + t B,
// I + s B): E = (eps + l) / (1 + sigma l), sigma = s / t, l the eigenvalues of
// t B (ascending on entry).  The map is monotone, increasing when
// 1 - sigma eps > 0 and decreasing otherwise; thread i maps the pair (i,
// n-1-i) and writes it back ascending either way.
__global__ void k_overlap_map(double* __restrict__ eigs, const int* __restrict__ n_act_cell, int K2, int n_max,
                              int64_t n_mat, double eps, double sigma) {
  const int64_t mat = blockIdx.x;
  if (mat >= n_mat) return;
  const int n = n_act_cell ? n_act_cell[mat / K2] : n_max;
  double* e = eigs + mat * n_max;
  const bool rev = 1.0 - sigma * eps < 0.0;
  for (int i = threadIdx.x; i < (n + 1) / 2; i += blockDim.x) {
    const int jj = n - 1 - i;
    const double a = e[i], b = e[jj];
    const double fa = (eps + a) / (1.0 + sigma * a), fb = (eps + b) / (1.0 + sigma * b);
    if (rev) {
      e[i] = fb;
      e[jj] = fa;
    } else {
      e[i] = fa;
      e[jj] = fb;
    }
  }
}

int launch_overlap_map(double* eigs, const int* n_act_cell, int K2, int n_max, int64_t n_mat, double eps,
                       double sigma, cudaStream_t s) {
  if (n_mat == 0) return IDOS_OK;
  k_overlap_map<<<(unsigned)n_mat, 128, 0, s>>>(eigs, n_act_cell, K2, n_max, n_mat, eps, sigma);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

int launch_bisect(int precision, int refine64_iters, const void* d, const void* e2,
                  const int* n_act_cell, int K2, int n_max, int64_t n_mat, double* eigs,
                  cudaStream_t s, int* err, int sym, double center) {
  if (n_mat == 0) return IDOS_OK;
  if (precision == IDOS_FP64)
    return bisect_t<double>(0, d, e2, n_act_cell, K2, n_max, n_mat, eigs, s, err, sym, center);
  return bisect_t<float>(refine64_iters, d, e2, n_act_cell, K2, n_max, n_mat, eigs, s, err, sym, center);
}

}  // namespace idos
