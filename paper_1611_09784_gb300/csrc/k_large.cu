// k_large.cu - blocked Householder tridiagonalisation of large Hermitian
// matrices held in global memory (L2 / HBM), batched, in ONE persistent
// cooperative kernel per batch.
//
// Same reflectors as k_small.cu (real tau, |e_j| = ||x||), organised in
// panels of NB columns (the LATRD arrangement): inside a panel the trailing
// matrix keeps its panel-start value and every column is corrected on the fly
// by the panel's earlier (v, w) pairs,  A_cur = A_start - V W^H - W V^H,  so the
// matrix-vector product of each column is a GEMV with the panel-start matrix
// plus thin corrections; after the panel, A -= V W^H + W V^H (rank 2NB).
//
// All CTAs of the grid walk the columns in lockstep; one column is two
// phases separated by grid barriers:
//   R   rows (256-row tiles): finish column j-1 (p = tau (y - V s1 - W s2),
//       w = p - K v with K = tau^2/2 (Re v^H y - 2 Re s2^H s1), all from
//       partials) and start column j: corrected column -> x (kept in V[i]),
//       d_j, partial ||x||^2, partial W^H x, V^H x
//   G   GEMV tiles (256 rows x 64 columns): partial y = A22 v and v^H y
// and every panel ends with the rank-2NB update (two more barriers).
// Reductions go through per-tile partials (double-buffered by column parity)
// that every consumer re-sums in a fixed order, so results are deterministic.
// Data written by other CTAs is read with L1-bypassing loads.
//
// Grid barrier: sense-reversal on a global counter; every wait is bounded
// (~2 s); on timeout the kernel sets an error flag, all CTAs leave, and the
// host returns IDOS_ERR_TIMEOUT.
#include "graphene.cuh"
#include "internal.h"

namespace idos {

namespace {

constexpr int NB = 32;    // panel width
constexpr int PT = 256;   // threads per CTA = rows per tile
constexpr int CS = 64;    // GEMV column slice
constexpr int HT = 32;    // her2k tile side

template <typename T> __device__ __forceinline__ T tiny_rest();
template <> __device__ __forceinline__ float tiny_rest<float>() { return 1e-30f; }
template <> __device__ __forceinline__ double tiny_rest<double>() { return 1e-290; }

template <typename T> __device__ __forceinline__ c2<T> ldcg(const c2<T>* p);
template <> __device__ __forceinline__ float2 ldcg<float>(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ldcg<double>(const double2* p) { return __ldcg(p); }

template <typename T>
struct PState {
  int n_max, B, K2, ntile, nslice;
  int64_t mat0;
  const int* n_act_cell;    // may be null (all n_max)
  c2<T>* A;                 // [B][n_max][n_max]
  c2<T>* V;                 // [B][NB][n_max]
  c2<T>* W;                 // [B][NB][n_max]
  c2<T>* part;              // [B][nslice][n_max] GEMV partials
  T* prest;                 // [2][B][ntile]
  T* gvy;                   // [2][B][ntile][nslice] partials of Re(v^H A22 v)
  c2<T>* ps;                // [2][B][ntile][2 NB]
  c2<T>* alpha;             // [2][B]
  T* d_out;                 // [B][n_max]
  T* e2_out;                // [B][n_max]
  unsigned int* bar;        // [0] count, [1] generation
  int* err;
};

template <typename T>
__device__ __forceinline__ int mat_n(const PState<T>& s, int b) {
  return s.n_act_cell ? s.n_act_cell[(s.mat0 + b) / s.K2] : s.n_max;
}

// Bounded sense-reversal grid barrier.  Returns false when the grid must stop.
__device__ __forceinline__ bool grid_sync(unsigned int* bar, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = bar + 1;
    const unsigned int gen = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (*(volatile int*)err) break;
        if (++spins > (1ll << 24)) {   // ~2 s with the back-off below
          atomicExch(err, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = *(volatile int*)err == 0;
  }
  __syncthreads();
  return s_ok;
}

// sigma^2, alpha, tau and v_{j+1} of column j from the partials.
template <typename T>
struct Reflector {
  T rest, sigma2, tau;
  c2<T> alpha, v1;
  int tr;
};

template <typename T>
__device__ __forceinline__ Reflector<T> reflector(const PState<T>& s, int b, int par) {
  Reflector<T> R;
  T rest = T(0);
  const T* pr = s.prest + ((size_t)par * s.B + b) * s.ntile;
  for (int t = 0; t < s.ntile; ++t) rest += __ldcg(pr + t);
  R.rest = rest;
  R.alpha = ldcg<T>(s.alpha + (size_t)par * s.B + b);
  const T aa2 = cabs2<T>(R.alpha);
  R.sigma2 = aa2 + rest;
  R.tr = rest > tiny_rest<T>();
  R.tau = T(0);
  R.v1 = mk<T>(T(0), T(0));
  if (R.tr) {
    const T sigma = sqrt(R.sigma2), aa = sqrt(aa2);
    const c2<T> ph = aa > T(0) ? cscale<T>(R.alpha, T(1) / aa) : mk<T>(T(1), T(0));
    R.tau = T(1) / (sigma * (sigma + aa));
    R.v1 = cadd<T>(R.alpha, cscale<T>(ph, sigma));
  }
  return R;
}

// Fixed-order block sum of one value per thread (PT threads).
template <typename T>
__device__ __forceinline__ T block_reduce(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = T(0);
#pragma unroll
  for (int w = 0; w < PT / 32; ++w) s += red[w];
  return s;
}

// Everything every row unit needs about column j once its GEMV is done:
// the reflector, s1 = W^H v, s2 = V^H v (q < i), K, and p at row j + 1.
template <typename T>
struct ColumnInfo {
  Reflector<T> R;
  T K;
  c2<T> s1[NB], s2[NB];
  c2<T> p1;     // p_{j+1}
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reflector of column j computed by one warp (lanes load the tile partials).
template <typename T>
__device__ __forceinline__ Reflector<T> reflector_warp(const PState<T>& s, int b, int par) {
  const int lane = threadIdx.x & 31;
  T rest = T(0);
  const T* pr = s.prest + ((size_t)par * s.B + b) * s.ntile;
  for (int t = lane; t < s.ntile; t += 32) rest += __ldcg(pr + t);
  rest = warp_sum<T>(rest);
  Reflector<T> R;
  R.rest = rest;
  R.alpha = ldcg<T>(s.alpha + (size_t)par * s.B + b);
  const T aa2 = cabs2<T>(R.alpha);
  R.sigma2 = aa2 + rest;
  R.tr = rest > tiny_rest<T>();
  R.tau = T(0);
  R.v1 = mk<T>(T(0), T(0));
  if (R.tr) {
    const T sigma = sqrt(R.sigma2), aa = sqrt(aa2);
    const c2<T> ph = aa > T(0) ? cscale<T>(R.alpha, T(1) / aa) : mk<T>(T(1), T(0));
    R.tau = T(1) / (sigma * (sigma + aa));
    R.v1 = cadd<T>(R.alpha, cscale<T>(ph, sigma));
  }
  return R;
}

template <typename T>
__device__ void column_info(const PState<T>& s, int b, int j, int i, ColumnInfo<T>& ci, T* red) {
  using C = c2<T>;
  const int nm = s.n_max, par = j & 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const C* Vb = s.V + (size_t)b * NB * nm;
  const C* Wb = s.W + (size_t)b * NB * nm;
  const int n_b = mat_n(s, b);
  if (warp == 0) {
    const Reflector<T> R = reflector_warp<T>(s, b, par);
    if (lane == 0) ci.R = R;
  }
  __syncthreads();
  const C v1 = ci.R.v1;
  // s1_q (warp 1..) and s2_q: one thread per (q, which), tile partials in order
  if (threadIdx.x < 2 * i) {
    const int q = threadIdx.x % i, which = threadIdx.x / i;   // 0: s1 (W), 1: s2 (V)
    C acc = mk<T>(T(0), T(0));
    const C* pp = s.ps + ((size_t)par * s.B + b) * s.ntile * (2 * NB);
    for (int tt = 0; tt < s.ntile; ++tt) acc = cadd<T>(acc, ldcg<T>(pp + (size_t)tt * 2 * NB + which * NB + q));
    acc = cadd<T>(acc, cjmul<T>(ldcg<T>((which == 0 ? Wb : Vb) + (size_t)q * nm + j + 1), v1));
    if (which == 0) ci.s1[q] = acc; else ci.s2[q] = acc;
  }
  // Re(v^H A22 v) from the GEMV partials of the (tile, slice) units that ran
  const int ng = s.ntile * s.nslice;
  T vy = T(0);
  for (int x = threadIdx.x; x < ng; x += PT) {
    const int tt = x / s.nslice, sl = x % s.nslice;
    const bool ran = (tt + 1) * PT > j + 1 && tt * PT < n_b && (sl + 1) * CS > j + 1 && sl * CS < n_b;
    if (ran) vy += __ldcg(s.gvy + ((size_t)par * s.B + b) * ng + x);
  }
  vy = block_reduce<T>(vy, red);   // has __syncthreads: s1/s2 visible afterwards
  if (warp == 0) {
    // cross term and p at row j + 1, lanes over q and over slices
    T cross = T(0);
    C y = mk<T>(T(0), T(0));
    for (int q = lane; q < i; q += 32) {
      cross += ci.s2[q].x * ci.s1[q].x + ci.s2[q].y * ci.s1[q].y;   // Re(conj(s2) s1)
      y = csub<T>(y, cmul<T>(ldcg<T>(Vb + (size_t)q * nm + j + 1), ci.s1[q]));
      y = csub<T>(y, cmul<T>(ldcg<T>(Wb + (size_t)q * nm + j + 1), ci.s2[q]));
    }
    for (int sl = (j + 1) / CS + lane; sl < s.nslice && sl * CS < n_b; sl += 32)
      y = cadd<T>(y, ldcg<T>(s.part + ((size_t)b * s.nslice + sl) * nm + j + 1));
    cross = warp_sum<T>(cross);
    y.x = warp_sum<T>(y.x);
    y.y = warp_sum<T>(y.y);
    if (lane == 0) {
      const T tau = ci.R.tau;
      ci.K = T(0.5) * tau * tau * (vy - T(2) * cross);
      ci.p1 = cscale<T>(y, tau);
    }
  }
  __syncthreads();
}

// R3 of column j on the tile's rows r > j: p = tau (y - V s1 - W s2),
// w = p - K v, stored as W[i][r]; the owner of row j+1 also stores v_{j+1},
// e_j^2.  No transform: v = w = 0.
template <typename T>
__device__ void phase_r3(const PState<T>& s, int b, int t, int j, int i, const ColumnInfo<T>& ci) {
  using C = c2<T>;
  const int n = mat_n(s, b);
  const int nm = s.n_max;
  C* Vi = s.V + ((size_t)b * NB + i) * nm;
  C* Wi = s.W + ((size_t)b * NB + i) * nm;
  const int r = t * PT + threadIdx.x;
  if (t == (j + 1) / PT && threadIdx.x == 0) {
    Vi[j + 1] = ci.R.v1;
    s.e2_out[(size_t)b * nm + j] = ci.R.sigma2;
  }
  if (r <= j || r >= n) return;
  if (!ci.R.tr) {
    if (r > j + 1) Vi[r] = mk<T>(T(0), T(0));
    Wi[r] = mk<T>(T(0), T(0));
    return;
  }
  const C* Vb = s.V + (size_t)b * NB * nm;
  const C* Wb = s.W + (size_t)b * NB * nm;
  C y = mk<T>(T(0), T(0));
  const int sl0 = (j + 1) / CS;
  const int sl1 = min(s.nslice, (n + CS - 1) / CS);
#pragma unroll 8
  for (int sl = sl0; sl < sl1; ++sl) y = cadd<T>(y, ldcg<T>(s.part + ((size_t)b * s.nslice + sl) * nm + r));
  for (int q0 = 0; q0 < i; q0 += 4) {
    C vq[4], wq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (q0 + u < i) {
        vq[u] = ldcg<T>(Vb + (size_t)(q0 + u) * nm + r);
        wq[u] = ldcg<T>(Wb + (size_t)(q0 + u) * nm + r);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (q0 + u < i) {
        y = csub<T>(y, cmul<T>(vq[u], ci.s1[q0 + u]));
        y = csub<T>(y, cmul<T>(wq[u], ci.s2[q0 + u]));
      }
    }
  }
  const C p = cscale<T>(y, ci.R.tau);
  const C v = (r == j + 1) ? ci.R.v1 : ldcg<T>(Vi + r);
  Wi[r] = csub<T>(p, cscale<T>(v, ci.K));
}

// R1 for column j (panel index i): corrected column j -> x (kept in V[i]),
// d_j, alpha, partial ||x||^2 and W^H x, V^H x over rows >= j + 2.  For
// i > 0, v and w of column j-1 at row j are v_prev_j, w_prev_j, computed by
// every unit (their owner stores them concurrently).
template <typename T>
__device__ void phase_r1(const PState<T>& s, int b, int t, int j, int i, c2<T> w_prev_j, c2<T> v_prev_j,
                         T* red) {
  using C = c2<T>;
  __shared__ C sWj[NB], sVj[NB];
  __shared__ C sa[PT];
  const int n = mat_n(s, b);
  const int nm = s.n_max;
  C* Vb = s.V + (size_t)b * NB * nm;
  const C* Wb = s.W + (size_t)b * NB * nm;
  if (threadIdx.x < i) {
    const int q = threadIdx.x;
    sVj[q] = (q < i - 1) ? ldcg<T>(Vb + (size_t)q * nm + j) : v_prev_j;
    sWj[q] = (q < i - 1) ? ldcg<T>(Wb + (size_t)q * nm + j) : w_prev_j;
  }
  __syncthreads();
  const int r = t * PT + threadIdx.x;
  const int par = j & 1;
  C a = mk<T>(T(0), T(0));
  T rest = T(0);
  if (r >= j && r < n) {
    a = conjg<T>(ldcg<T>(s.A + ((size_t)b * nm + j) * nm + r));   // A[r][j] = conj(A[j][r])
    for (int q0 = 0; q0 < i; q0 += 4) {
      C vq[4], wq[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (q0 + u < i) {
          vq[u] = (r == j) ? sVj[q0 + u] : ldcg<T>(Vb + (size_t)(q0 + u) * nm + r);
          wq[u] = (r == j) ? sWj[q0 + u] : ldcg<T>(Wb + (size_t)(q0 + u) * nm + r);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (q0 + u < i) {
          a = csub<T>(a, cmulc<T>(vq[u], sWj[q0 + u]));
          a = csub<T>(a, cmulc<T>(wq[u], sVj[q0 + u]));
        }
      }
    }
    if (r == j) s.d_out[(size_t)b * nm + j] = a.x;
    else if (r == j + 1) s.alpha[(size_t)par * s.B + b] = a;
    else rest = cabs2<T>(a);
    if (r > j) Vb[(size_t)i * nm + r] = a;
  }
  sa[threadIdx.x] = (r >= j + 2 && r < n) ? a : mk<T>(T(0), T(0));
  rest = block_reduce<T>(rest, red);
  if (threadIdx.x == 0) s.prest[((size_t)par * s.B + b) * s.ntile + t] = rest;
  // tile partials of W_q^H x and V_q^H x over rows >= j + 2 (warp per q)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  C* ps = s.ps + (((size_t)par * s.B + b) * s.ntile + t) * (2 * NB);
  for (int q = warp; q < i; q += PT / 32) {
    C a1 = mk<T>(T(0), T(0)), a2 = mk<T>(T(0), T(0));
#pragma unroll
    for (int x = lane; x < PT; x += 32) {
      const int rr = t * PT + x;
      if (rr < j + 2 || rr >= n) continue;
      const C xa = sa[x];
      a1 = cadd<T>(a1, cjmul<T>(ldcg<T>(Wb + (size_t)q * nm + rr), xa));
      a2 = cadd<T>(a2, cjmul<T>(ldcg<T>(Vb + (size_t)q * nm + rr), xa));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a1.x += __shfl_xor_sync(0xffffffffu, a1.x, o);
      a1.y += __shfl_xor_sync(0xffffffffu, a1.y, o);
      a2.x += __shfl_xor_sync(0xffffffffu, a2.x, o);
      a2.y += __shfl_xor_sync(0xffffffffu, a2.y, o);
    }
    if (lane == 0) {
      ps[q] = a1;
      ps[NB + q] = a2;
    }
  }
  __syncthreads();
}

// G: partial y over one (row tile, column slice): part[b][sl][r] = sum_c conj(A[c][r]) v_c,
// and the tile-slice partial of v^H y.
template <typename T>
__device__ void phase_gemv(const PState<T>& s, int b, int t, int sl, int j, int i, T* red) {
  using C = c2<T>;
  __shared__ C sv[CS];
  __shared__ int s_tr;
  __shared__ C s_v1;
  const int n = mat_n(s, b);
  if (j >= n - 1) return;
  const int c0 = max(j + 1, sl * CS), c1 = min(n, (sl + 1) * CS);
  if (c0 >= c1 || t * PT >= n || (t + 1) * PT <= j + 1) return;
  const int nm = s.n_max;
  if (threadIdx.x < 32) {
    const Reflector<T> R = reflector_warp<T>(s, b, j & 1);
    if (threadIdx.x == 0) {
      s_tr = R.tr;
      s_v1 = R.v1;
    }
  }
  __syncthreads();
  const int tr = s_tr;
  const C* Vi = s.V + ((size_t)b * NB + i) * nm;
  if (tr) {
    for (int c = c0 + threadIdx.x; c < c1; c += PT) sv[c - c0] = (c == j + 1) ? s_v1 : ldcg<T>(Vi + c);
  }
  __syncthreads();
  const int r = t * PT + threadIdx.x;
  T vy = T(0);
  if (tr && r > j && r < n) {
    const C* Ab = s.A + (size_t)b * nm * nm + r;
    C acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = mk<T>(T(0), T(0));
    int c = c0;
    for (; c + 8 <= c1; c += 8) {
      C av[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) av[u] = ldcg<T>(Ab + (size_t)(c + u) * nm);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u & 3] = cadd<T>(acc[u & 3], cjmul<T>(av[u], sv[c + u - c0]));
    }
    for (; c < c1; ++c) acc[0] = cadd<T>(acc[0], cjmul<T>(ldcg<T>(Ab + (size_t)c * nm), sv[c - c0]));
    const C y = cadd<T>(cadd<T>(acc[0], acc[1]), cadd<T>(acc[2], acc[3]));
    s.part[((size_t)b * s.nslice + sl) * nm + r] = y;
    const C v = (r == j + 1) ? s_v1 : ldcg<T>(Vi + r);
    vy = v.x * y.x + v.y * y.y;   // Re(conj(v_r) y_r)
  }
  vy = block_reduce<T>(vy, red);
  if (threadIdx.x == 0)
    s.gvy[((size_t)(j & 1) * s.B + b) * s.ntile * s.nslice + (size_t)t * s.nslice + sl] = vy;
  __syncthreads();
}

// Panel update A[r][c] -= sum_q V[q][r] conj(W[q][c]) + W[q][r] conj(V[q][c]), r, c >= jn.
template <typename T>
__device__ void phase_her2k(const PState<T>& s, int b, int tr_, int tc, int jn, c2<T>* sm) {
  using C = c2<T>;
  const int n = mat_n(s, b);
  const int r0 = jn + tr_ * HT, c0 = jn + tc * HT;
  if (r0 >= n || c0 >= n) return;
  const int nm = s.n_max;
  C* sVr = sm;
  C* sWr = sVr + NB * (HT + 1);
  C* sVc = sWr + NB * (HT + 1);
  C* sWc = sVc + NB * (HT + 1);
  const C* Vb = s.V + (size_t)b * NB * nm;
  const C* Wb = s.W + (size_t)b * NB * nm;
  for (int idx = threadIdx.x; idx < NB * HT; idx += PT) {
    const int q = idx / HT, x = idx % HT;
    const int r = r0 + x, c = c0 + x;
    sVr[q * (HT + 1) + x] = r < n ? ldcg<T>(Vb + (size_t)q * nm + r) : mk<T>(T(0), T(0));
    sWr[q * (HT + 1) + x] = r < n ? ldcg<T>(Wb + (size_t)q * nm + r) : mk<T>(T(0), T(0));
    sVc[q * (HT + 1) + x] = c < n ? ldcg<T>(Vb + (size_t)q * nm + c) : mk<T>(T(0), T(0));
    sWc[q * (HT + 1) + x] = c < n ? ldcg<T>(Wb + (size_t)q * nm + c) : mk<T>(T(0), T(0));
  }
  __syncthreads();
  const int cx = threadIdx.x % HT, ry = threadIdx.x / HT;   // 8 row groups
  C* Ab = s.A + (size_t)b * nm * nm;
#pragma unroll
  for (int k = 0; k < HT / 8; ++k) {
    const int rl = ry + 8 * k;
    C acc = mk<T>(T(0), T(0));
#pragma unroll 8
    for (int q = 0; q < NB; ++q) {
      acc = cadd<T>(acc, cmulc<T>(sVr[q * (HT + 1) + rl], sWc[q * (HT + 1) + cx]));
      acc = cadd<T>(acc, cmulc<T>(sWr[q * (HT + 1) + rl], sVc[q * (HT + 1) + cx]));
    }
    const int r = r0 + rl, c = c0 + cx;
    if (r < n && c < n) {
      C* e = Ab + (size_t)r * nm + c;
      *e = csub<T>(ldcg<T>(e), acc);
    }
  }
  __syncthreads();
}

// One column step j of every matrix, in order:
//   [R3 of column j-1 + R1 of column j]  barrier  [GEMV of column j]  barrier
// with the panel's rank-2NB update (and its two barriers) when j starts a panel.
template <typename T>
__global__ void __launch_bounds__(PT, 3)
k_lg_persist(PState<T> s) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c2<T>* sm = reinterpret_cast<c2<T>*>(smem_raw);
  __shared__ ColumnInfo<T> ci;
  __shared__ T red[PT / 32];
  const int nrow_units = s.B * s.ntile;
  const int ngemv_units = nrow_units * s.nslice;
  for (int j = 0; j < s.n_max; ++j) {
    const int j0 = j - j % NB, i = j - j0;
    const bool panel_start = (i == 0);
    if (panel_start && j > 0) {
      // finish the previous panel's last column (R3), then the rank-2NB update
      for (int u = blockIdx.x; u < nrow_units; u += gridDim.x) {
        const int b = u / s.ntile, t = u % s.ntile;
        if (j - 1 >= mat_n(s, b) - 1) continue;
        column_info<T>(s, b, j - 1, NB - 1, ci, red);
        phase_r3<T>(s, b, t, j - 1, NB - 1, ci);
        __syncthreads();
      }
      if (!grid_sync(s.bar, s.err)) return;
      const int nt = (s.n_max - j + HT - 1) / HT;
      const int units = s.B * nt * nt;
      for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int b = u / (nt * nt), rem = u % (nt * nt);
        phase_her2k<T>(s, b, rem / nt, rem % nt, j, sm);
      }
      if (!grid_sync(s.bar, s.err)) return;
    }
    // R3 of column j-1 (inside the panel) fused with R1 of column j
    for (int u = blockIdx.x; u < nrow_units; u += gridDim.x) {
      const int b = u / s.ntile, t = u % s.ntile;
      const int n = mat_n(s, b);
      if (j >= n) continue;
      c2<T> w_prev = mk<T>(T(0), T(0)), v_prev = mk<T>(T(0), T(0));
      if (!panel_start) {
        column_info<T>(s, b, j - 1, i - 1, ci, red);   // j - 1 < n - 1 here
        phase_r3<T>(s, b, t, j - 1, i - 1, ci);
        if (ci.R.tr) {
          v_prev = ci.R.v1;
          w_prev = csub<T>(ci.p1, cscale<T>(ci.R.v1, ci.K));
        }
        __syncthreads();
      }
      phase_r1<T>(s, b, t, j, i, w_prev, v_prev, red);
    }
    if (!grid_sync(s.bar, s.err)) return;
    for (int u = blockIdx.x; u < ngemv_units; u += gridDim.x) {
      const int b = u / (s.ntile * s.nslice), rem = u % (s.ntile * s.nslice);
      phase_gemv<T>(s, b, rem / s.nslice, rem % s.nslice, j, i, red);
    }
    if (!grid_sync(s.bar, s.err)) return;
  }
}

// Assembly of H(k) into global memory (rows of kept sites only; the buffer is
// zeroed beforehand).  One thread per (matrix, row).
template <typename T>
__global__ void k_lg_assemble(int64_t n_mat_batch, int64_t mat0, int n_max, int K2,
                              const int* __restrict__ n_act_cell, const int* __restrict__ act,
                              const int* __restrict__ inv, int N, int K, double t_hop, double eps,
                              const double2* __restrict__ Hin, c2<T>* __restrict__ A) {
  using C = c2<T>;
  const int64_t total = n_mat_batch * (int64_t)n_max;
  const int n_sites = 2 * N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t mat = idx / n_max;
    const int a = (int)(idx - mat * n_max);
    C* Am = A + mat * (int64_t)n_max * n_max;
    if (Hin) {
      const double2* src = Hin + mat * (int64_t)n_max * n_max + (int64_t)a * n_max;
      for (int c = 0; c < n_max; ++c) Am[(int64_t)a * n_max + c] = mk<T>((T)src[c].x, (T)src[c].y);
      continue;
    }
    const int64_t gmat = mat0 + mat;
    const int64_t cell = gmat / K2;
    const int kidx = (int)(gmat - cell * K2);
    if (a >= n_act_cell[cell]) continue;
    int nb[3];
    bool fromB;
    graphene_neighbours(N, act[cell * n_sites + a], nb, fromB);
    C* row = Am + (int64_t)a * n_max;
    for (int b = 0; b < 3; ++b) {
      const int col = inv[cell * n_sites + nb[b]];
      if (col < 0) continue;
      const double2 p = graphene_phase(N, K, kidx, b);
      const double im = fromB ? -p.y : p.y;
      row[col] = cadd<T>(row[col], mk<T>((T)(t_hop * p.x), (T)(t_hop * im)));
    }
    row[a].x += (T)eps;
  }
}

template <typename T>
size_t per_matrix_bytes(int nm) {
  using C = c2<T>;
  const int ntile = (nm + PT - 1) / PT, nslice = (nm + CS - 1) / CS;
  return sizeof(C) * ((size_t)nm * nm + 2 * (size_t)NB * nm + (size_t)nslice * nm) +
         2 * (sizeof(T) * ntile * (1 + nslice) + sizeof(C) * ntile * 2 * NB + sizeof(C)) + 512;
}

template <typename T>
int solve_large_t(const SolveArgs& a) {
  using C = c2<T>;
  const int nm = a.n_max;
  const int ntile = (nm + PT - 1) / PT;
  const int nslice = (nm + CS - 1) / CS;
  const CellSet* cells = a.cells;
  const int K2 = a.Kside * a.Kside;
  const size_t smem = sizeof(C) * 4 * NB * (HT + 1);   // her2k tiles
  auto kern = k_lg_persist<T>;
  IDOS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  IDOS_CUDA_TRY(cudaGetDevice(&dev));
  IDOS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  IDOS_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  IDOS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PT, smem));
  if (!coop || per_sm < 1) {
    set_error("cooperative launch of the large-matrix kernel is not possible on this device");
    return IDOS_ERR_UNSUPPORTED;
  }
  const int grid = sms * std::min(per_sm, 4);
  // per-matrix bytes: A + V + W + P + GEMV partials (+ small partials)
  const size_t per_mat = per_matrix_bytes<T>(nm);
  const size_t room = a.ws->cap > a.ws->used ? a.ws->cap - a.ws->used : 0;
  int64_t batch = std::max<int64_t>(1, (int64_t)((room > 65536 ? room - 65536 : 0) / per_mat));
  batch = std::min<int64_t>(batch, a.n_mat);
  const size_t mark = a.ws->used;
  PState<T> s{};
  s.n_max = nm;
  s.K2 = K2;
  s.ntile = ntile;
  s.nslice = nslice;
  s.n_act_cell = cells ? cells->n_act : nullptr;
  s.A = a.ws->take<C>((size_t)batch * nm * nm);
  s.V = a.ws->take<C>((size_t)batch * NB * nm);
  s.W = a.ws->take<C>((size_t)batch * NB * nm);
  s.part = a.ws->take<C>((size_t)batch * nslice * nm);
  s.prest = a.ws->take<T>((size_t)2 * batch * ntile);
  s.gvy = a.ws->take<T>((size_t)2 * batch * ntile * nslice);
  s.ps = a.ws->take<C>((size_t)2 * batch * ntile * 2 * NB);
  s.alpha = a.ws->take<C>((size_t)2 * batch);
  s.bar = a.ws->take<unsigned int>(2);
  s.err = a.ws->take<int>(1);
  if (!s.A || !s.V || !s.W || !s.part || !s.prest || !s.gvy || !s.ps || !s.alpha || !s.bar || !s.err) {
    set_error("large-matrix workspace does not fit");
    return IDOS_ERR_OUT_OF_MEMORY;
  }
  for (int64_t m0 = 0; m0 < a.n_mat; m0 += batch) {
    const int64_t nb_mat = std::min<int64_t>(batch, a.n_mat - m0);
    s.B = (int)nb_mat;
    s.mat0 = m0;
    s.d_out = reinterpret_cast<T*>(a.d) + m0 * nm;
    s.e2_out = reinterpret_cast<T*>(a.e2) + m0 * nm;
    IDOS_CUDA_TRY(cudaMemsetAsync(s.A, 0, sizeof(C) * (size_t)nb_mat * nm * nm, a.stream));
    IDOS_CUDA_TRY(cudaMemsetAsync(s.bar, 0, 2 * sizeof(unsigned int), a.stream));
    IDOS_CUDA_TRY(cudaMemsetAsync(s.err, 0, sizeof(int), a.stream));
    {
      const int64_t total = nb_mat * (int64_t)nm;
      const int64_t blocks = std::min<int64_t>((total + 127) / 128, 152 * 16);
      ProfScope ps(KID_LG_ASSEMBLE, a.stream);
      k_lg_assemble<T><<<(unsigned)blocks, 128, 0, a.stream>>>(
          nb_mat, m0, nm, K2, cells ? cells->n_act : nullptr, cells ? cells->act : nullptr,
          cells ? cells->inv : nullptr, cells ? cells->N : 0, a.Kside, a.t, a.eps,
          a.H ? a.H + m0 * (int64_t)nm * nm : nullptr, s.A);
      IDOS_CHECK_LAUNCH();
    }
    {
      ProfScope ps(KID_LG_TRIDIAG, a.stream);
      void* args[] = {&s};
      IDOS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(PT), args, smem, a.stream));
    }
    int herr = 0;
    IDOS_CUDA_TRY(cudaMemcpyAsync(&herr, s.err, sizeof(int), cudaMemcpyDeviceToHost, a.stream));
    IDOS_CUDA_TRY(cudaStreamSynchronize(a.stream));
    if (herr) {
      set_error("large-matrix kernel: a grid barrier wait timed out");
      return IDOS_ERR_TIMEOUT;
    }
  }
  a.ws->used = mark;
  return IDOS_OK;
}

}  // namespace

size_t large_path_bytes(int precision, int n_max, int64_t n_mat) {
  const size_t per = precision == IDOS_FP64 ? per_matrix_bytes<double>(n_max) : per_matrix_bytes<float>(n_max);
  return per * (size_t)std::max<int64_t>(n_mat, 1) + 65536 + 12 * 256;
}

int solve_large(int precision, const SolveArgs& a) {
  if (a.n_mat == 0) return IDOS_OK;
  return precision == IDOS_FP64 ? solve_large_t<double>(a) : solve_large_t<float>(a);
}

}  // namespace idos
