// k_large.cu - two-stage reduction of large Hermitian matrices (held in
// global memory, batched) to real symmetric tridiagonal form.
//
// Stage 1, dense -> band of half-width BW: for every panel of BW columns,
//   Householder QR of the block below the band, P = Q R with
//   Q = H_0 ... H_{BW-1} = I - Y T Y^H (compact WY, T upper triangular,
//   H_c = I - tau_c y_c y_c^H with real tau_c as in k_small.cu), then the
//   two-sided update of the trailing matrix  A22 <- Q^H A22 Q  as
//     W = A22 (Y T),  M = Y^H W,  Z = W - 1/2 Y (T^H M),  A22 -= Y Z^H + Z Y^H
//   (Q^H A Q = A - W Y^H - Y W^H + Y T^H Y^H W Y^H and W^H Y T = T^H Y^H W,
//   so the update is the Hermitian rank-2BW form above).  Five batched
//   launches per panel: panel QR (one cluster of CTAs per matrix), W = A22 YT
//   (tiled, split over the inner dimension), the split sum with M = Y^H W and
//   Z (two launches over row chunks), the rank-2BW update (tiled).
// Stage 2, band -> tridiagonal by bulge chasing, is in k_chase.cu.
#include <cooperative_groups.h>

#include <vector>

#include "graphene.cuh"
#include "large.cuh"
#include "tmdc.cuh"

namespace cg = cooperative_groups;

namespace idos {

namespace {

using namespace lg;

constexpr int PQ_THREADS = 512; // panel QR / Z kernels
// Tile sizes keep static shared memory under 48 KB for both element types.
template <typename T> struct Tiles;
template <> struct Tiles<float> { static constexpr int GT = 64, WR = 64, WK = 64; };
template <> struct Tiles<double> { static constexpr int GT = 32, WR = 32, WK = 32; };
// --------------------------------------------------------------- assembly --
// H(k) into global memory (rows of kept sites only; the buffer is zeroed
// beforehand).  One thread per (matrix, row).
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

// H(k) of the TMDC-shaped model into global memory, rows of kept orbitals
// only, built by tmdc_row (hops into removed pairs are skipped; the buffer is
// zeroed beforehand).  One thread per (matrix, row).
template <typename T>
__global__ void k_lg_assemble_tmdc(int64_t n_mat_batch, int64_t mat0, int n_max, int K2,
                                   const int* __restrict__ n_act_cell, const int* __restrict__ act,
                                   const int* __restrict__ inv, const uint8_t* __restrict__ pairs, int N, int K,
                                   const double* __restrict__ P, c2<T>* __restrict__ A) {
  using C = c2<T>;
  const int64_t total = n_mat_batch * (int64_t)n_max;
  const int n_orb = kTmdcOrb * N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t mat = idx / n_max;
    const int a = (int)(idx - mat * n_max);
    const int64_t gmat = mat0 + mat;
    const int64_t cell = gmat / K2;
    const int kidx = (int)(gmat - cell * K2);
    if (a >= n_act_cell[cell]) continue;
    C* row = A + mat * (int64_t)n_max * n_max + (int64_t)a * n_max;
    const int* invc = inv + cell * n_orb;
    const uint8_t* pc = pairs + cell * (N * N);
    tmdc_row(N, K, kidx, act[cell * n_orb + a], P, [&](int c) { return pc[c] != 0; },
             [&](int o2, double2 v) {
               const int col = invc[o2];
               if (col >= 0) row[col] = cadd<T>(row[col], mk<T>((T)v.x, (T)v.y));
             });
  }
}

// ------------------------------------------------------------ block sums --
template <typename T, int NT>
__device__ __forceinline__ T block_sum_t(T v, T* red) {
  v = warp_sum<T>(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = T(0);
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) s += red[w];
  return s;
}

// ------------------------------------------------------------- panel QR --
// One CTA per matrix.  Panel P[r][c] = A[k+BW+r][k+c], r < m = n-k-BW, c < BW,
// factored in place in shared memory when it fits (else in global memory).
// Outputs Y[c][r] (reflector c, zero above row c), YT = Y T, T; writes R back
// (upper triangle) and zeros below it.
template <typename T>
__global__ void __launch_bounds__(PQ_THREADS, 1)
k_ts_panel(Batch bt, int k, c2<T>* __restrict__ A, c2<T>* __restrict__ Y, c2<T>* __restrict__ YT,
           c2<T>* __restrict__ Tm, int use_smem) {
  using C = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[PQ_THREADS / 32];
  __shared__ C sw[BW];
  __shared__ C swp[PQ_THREADS / 32][BW];
  __shared__ C sG[BW][BW];
  __shared__ C sT[BW][BW];
  __shared__ T stau[BW];
  __shared__ C salpha;
  const int b = blockIdx.x;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int m = n - k - BW;
  if (m <= 0) return;
  C* Ab = A + (size_t)b * nm * nm;
  C* P;
  int ld;
  if (use_smem) {
    P = reinterpret_cast<C*>(smem_raw);
    ld = BW;
    for (int idx = threadIdx.x; idx < m * BW; idx += PQ_THREADS) {
      const int r = idx / BW, c = idx % BW;
      P[idx] = Ab[(size_t)(k + BW + r) * nm + k + c];
    }
    __syncthreads();
  } else {
    P = Ab + (size_t)(k + BW) * nm + k;
    ld = nm;
  }
  C* Yb = Y + (size_t)b * BW * nm;
  for (int c = 0; c < BW; ++c) {
    // x = P[c:, c]; rest = sum_{r > c} |x_r|^2
    T rest = T(0);
    for (int r = c + 1 + threadIdx.x; r < m; r += PQ_THREADS) rest += cabs2<T>(P[(size_t)r * ld + c]);
    rest = block_sum_t<T, PQ_THREADS>(rest, red);
    if (threadIdx.x == 0) salpha = c < m ? P[(size_t)c * ld + c] : mk<T>(T(0), T(0));
    __syncthreads();
    const C alpha = salpha;
    const bool tr = c < m && rest > tiny_rest<T>();
    T tau = T(0);
    C v0 = alpha, beta = alpha;
    if (tr) {
      C ph;
      const T aa = cabs_phase<T>(alpha, ph), sigma = sqrt(cabs2<T>(alpha) + rest);
      tau = T(1) / (sigma * (sigma + aa));
      v0 = cadd<T>(alpha, cscale<T>(ph, sigma));
      beta = cscale<T>(ph, -sigma);
    }
    if (threadIdx.x == 0) stau[c] = tau;
    // y_c: zero above row c, v below
    for (int r = threadIdx.x; r < m; r += PQ_THREADS) {
      C y = mk<T>(T(0), T(0));
      if (tr && r >= c) y = (r == c) ? v0 : P[(size_t)r * ld + c];
      Yb[(size_t)c * nm + r] = y;
    }
    if (tr) {
      // w_d = v^H P[c:, d] for all d > c at once.  Thread t works on column
      // d = t % BW over the rows r = g (mod G), g = t / BW, G = PQ_THREADS / BW;
      // lanes l and l + 16 share d, then warps are summed in a fixed order.
      constexpr int G = PQ_THREADS / BW;
      const int d = threadIdx.x % BW, g = threadIdx.x / BW;
      C acc = mk<T>(T(0), T(0));
      if (d > c) {
        for (int r = c + ((g - c % G) + G) % G; r < m; r += G) {
          const C v = (r == c) ? v0 : P[(size_t)r * ld + c];
          acc = cadd<T>(acc, cjmul<T>(v, P[(size_t)r * ld + d]));
        }
      }
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 16);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 16);
      if ((threadIdx.x & 31) < BW) swp[threadIdx.x >> 5][d] = acc;
      __syncthreads();
      if (threadIdx.x < BW) {
        C sum = mk<T>(T(0), T(0));
        for (int w2 = 0; w2 < PQ_THREADS / 32; ++w2) sum = cadd<T>(sum, swp[w2][threadIdx.x]);
        sw[threadIdx.x] = sum;
      }
      __syncthreads();
      if (d > c) {
        const C wd = cscale<T>(sw[d], tau);
        for (int r = c + ((g - c % G) + G) % G; r < m; r += G) {
          const C v = (r == c) ? v0 : P[(size_t)r * ld + c];
          P[(size_t)r * ld + d] = csub<T>(P[(size_t)r * ld + d], cmul<T>(v, wd));
        }
      }
      __syncthreads();
      // column c becomes (beta, 0, ..., 0) below the band row
      for (int r = c + threadIdx.x; r < m; r += PQ_THREADS) P[(size_t)r * ld + c] = (r == c) ? beta : mk<T>(T(0), T(0));
    }
    __syncthreads();
  }
  // Gram matrix G[q][c] = y_q^H y_c (q < c), warp per pair
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int pr = warp; pr < BW * BW; pr += PQ_THREADS / 32) {
    const int q = pr / BW, c = pr % BW;
    if (q >= c) continue;
    C acc = mk<T>(T(0), T(0));
    for (int r = c + lane; r < m; r += 32)
      acc = cadd<T>(acc, cjmul<T>(Yb[(size_t)q * nm + r], Yb[(size_t)c * nm + r]));
    acc.x = warp_sum<T>(acc.x);
    acc.y = warp_sum<T>(acc.y);
    if (lane == 0) sG[q][c] = acc;
  }
  __syncthreads();
  // T (forward, columnwise): T[c][c] = tau_c, T[0:c, c] = -tau_c T[0:c, 0:c] G[0:c, c]
  if (threadIdx.x == 0) {
    for (int c = 0; c < BW; ++c) {
      for (int q = 0; q < BW; ++q) sT[q][c] = mk<T>(T(0), T(0));
      sT[c][c] = mk<T>(stau[c], T(0));
      for (int q = 0; q < c; ++q) {
        C acc = mk<T>(T(0), T(0));
        for (int u = q; u < c; ++u) acc = cadd<T>(acc, cmul<T>(sT[q][u], sG[u][c]));
        sT[q][c] = cscale<T>(acc, -stau[c]);
      }
    }
  }
  __syncthreads();
  C* Tb = Tm + (size_t)b * BW * BW;
  for (int idx = threadIdx.x; idx < BW * BW; idx += PQ_THREADS) Tb[idx] = sT[idx / BW][idx % BW];
  // YT[c][r] = sum_{q <= c} Y[q][r] T[q][c]
  C* YTb = YT + (size_t)b * BW * nm;
  for (int r = threadIdx.x; r < m; r += PQ_THREADS) {
    C yr[BW];
#pragma unroll
    for (int q = 0; q < BW; ++q) yr[q] = Yb[(size_t)q * nm + r];
#pragma unroll 1
    for (int c = 0; c < BW; ++c) {
      C acc = mk<T>(T(0), T(0));
#pragma unroll
      for (int q = 0; q < BW; ++q)
        if (q <= c) acc = cadd<T>(acc, cmul<T>(yr[q], sT[q][c]));
      YTb[(size_t)c * nm + r] = acc;
    }
  }
  if (use_smem) {
    for (int idx = threadIdx.x; idx < m * BW; idx += PQ_THREADS) {
      const int r = idx / BW, c = idx % BW;
      Ab[(size_t)(k + BW + r) * nm + k + c] = P[idx];
    }
  }
}

// ---------------------------------------------------- panel QR (cluster) --
// The panel of one matrix spread over a cluster of PC CTAs (PC = 1: one
// CTA); CTA q holds the panel rows [q RC, (q+1) RC), RC = ceil(m / PC), in
// shared memory.  Column c needs, besides local rows, only
//   h_d = sum_{r > c} conj(P[r][c]) P[r][d]   (d >= c; Re h_c = rest)
// and row c of the panel: with v = x + ph sigma e_c,
//   w_d = v^H P[:, d] = h_d + conj(v_c) P[c][d],
// so one cluster exchange per column suffices.  Every CTA adds the PC
// partials in rank order, so all hold bit-identical reflectors.  The Gram
// matrix of Y, needed for T, is exchanged the same way once per panel.
template <typename T, bool CL>
__global__ void __launch_bounds__(PQ_THREADS, 1)
k_ts_panel_cl(Batch bt, int k, c2<T>* __restrict__ A, c2<T>* __restrict__ Y, c2<T>* __restrict__ YT,
              c2<T>* __restrict__ Tm, int rc_max) {
  using C = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ C part[2][2 * BW];   // [buffer][h_0..h_{BW-1}, row c entries]
  __shared__ C gpart[BW][BW];
  __shared__ C swp[PQ_THREADS / 32][BW];
  __shared__ C sH[BW], sRow[BW], sbeta[BW];
  __shared__ C sG[BW][BW], sT[BW][BW];
  __shared__ T stau[BW];
  const int PC = CL ? (int)cg::this_cluster().num_blocks() : 1;
  const int q = CL ? (int)cg::this_cluster().block_rank() : 0;
  const int b = blockIdx.x / PC;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int m = n - k - BW;
  if (m <= 0) return;   // the same for every CTA of the cluster
  const int RC = (m + PC - 1) / PC;
  const int rlo = q * RC, rhi = min(m, rlo + RC);
  const int nr = max(0, rhi - rlo);
  C* P = reinterpret_cast<C*>(smem_raw);   // [rc_max][BW]
  C* Yl = P + (size_t)rc_max * BW;         // [rc_max][BW]
  C* Ab = A + (size_t)b * nm * nm;
  for (int idx = threadIdx.x; idx < nr * BW; idx += PQ_THREADS) {
    const int r = idx / BW, c = idx % BW;
    P[idx] = Ab[(size_t)(k + BW + rlo + r) * nm + k + c];
  }
  __syncthreads();
  constexpr int G = PQ_THREADS / BW;
  const int d = threadIdx.x % BW, g = threadIdx.x / BW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < BW; ++c) {
    const int buf = c & 1;
    // local partial h_d over rows r > c
    C acc = mk<T>(T(0), T(0));
    if (d >= c) {
      for (int r = g; r < nr; r += G)
        if (rlo + r > c) acc = cadd<T>(acc, cjmul<T>(P[(size_t)r * BW + c], P[(size_t)r * BW + d]));
    }
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 16);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 16);
    if (lane < BW) swp[warp][d] = acc;
    __syncthreads();
    if (threadIdx.x < BW) {
      C sum = mk<T>(T(0), T(0));
      for (int w2 = 0; w2 < PQ_THREADS / 32; ++w2) sum = cadd<T>(sum, swp[w2][threadIdx.x]);
      part[buf][threadIdx.x] = sum;
    } else if (threadIdx.x < 2 * BW) {
      const int dd = threadIdx.x - BW;
      part[buf][threadIdx.x] = (c >= rlo && c < rhi && dd >= c) ? P[(size_t)(c - rlo) * BW + dd] : mk<T>(T(0), T(0));
    }
    if constexpr (CL) cg::this_cluster().sync(); else __syncthreads();
    if (threadIdx.x < 2 * BW) {
      C sum = mk<T>(T(0), T(0));
      for (int o = 0; o < PC; ++o) {
        const C* pp = &part[buf][threadIdx.x];
        if constexpr (CL) pp = cg::this_cluster().map_shared_rank(pp, o);
        sum = cadd<T>(sum, *pp);
      }
      if (threadIdx.x < BW) sH[threadIdx.x] = sum;
      else sRow[threadIdx.x - BW] = sum;
    }
    __syncthreads();
    // reflector (every thread computes the same values)
    const C alpha = sRow[c];
    const T rest = sH[c].x;
    const bool tr = c < m && rest > tiny_rest<T>();
    T tau = T(0);
    C vc = alpha, beta = alpha;
    if (tr) {
      C ph;
      const T aa = cabs_phase<T>(alpha, ph), sigma = sqrt(cabs2<T>(alpha) + rest);
      tau = T(1) / (sigma * (sigma + aa));
      vc = cadd<T>(alpha, cscale<T>(ph, sigma));
      beta = cscale<T>(ph, -sigma);
    }
    if (threadIdx.x == 0) {
      stau[c] = tau;
      sbeta[c] = beta;
    }
    if (tr && d > c) {
      const C wd = cscale<T>(cadd<T>(sH[d], cjmul<T>(vc, sRow[d])), tau);
      for (int r = g; r < nr; r += G) {
        const int rg = rlo + r;
        if (rg < c) continue;
        const C v = rg == c ? vc : P[(size_t)r * BW + c];
        P[(size_t)r * BW + d] = csub<T>(P[(size_t)r * BW + d], cmul<T>(v, wd));
      }
    } else if (d == c) {
      for (int r = g; r < nr; r += G) {
        const int rg = rlo + r;
        Yl[(size_t)r * BW + c] = (!tr || rg < c) ? mk<T>(T(0), T(0)) : (rg == c ? vc : P[(size_t)r * BW + c]);
      }
    }
    __syncthreads();
  }
  // Gram matrix G[u][c] = y_u^H y_c (u < c): local partials, one exchange
  if (threadIdx.x < BW * BW) {
    const int u = threadIdx.x / BW, c = threadIdx.x % BW;
    C a2 = mk<T>(T(0), T(0));
    if (u < c)
      for (int r = 0; r < nr; ++r) a2 = cadd<T>(a2, cjmul<T>(Yl[(size_t)r * BW + u], Yl[(size_t)r * BW + c]));
    gpart[u][c] = a2;
  }
  if constexpr (CL) cg::this_cluster().sync(); else __syncthreads();
  if (threadIdx.x < BW * BW) {
    const int u = threadIdx.x / BW, c = threadIdx.x % BW;
    C sum = mk<T>(T(0), T(0));
    for (int o = 0; o < PC; ++o) {
      const C* pp = &gpart[u][c];
      if constexpr (CL) pp = cg::this_cluster().map_shared_rank(pp, o);
      sum = cadd<T>(sum, *pp);
    }
    sG[u][c] = sum;
  }
  __syncthreads();
  // T (forward, columnwise): T[c][c] = tau_c, T[u][c] = -tau_c sum_{u <= s < c} T[u][s] G[s][c]
  if (warp == 0) {
    for (int c = 0; c < BW; ++c) {
      if (lane < BW) {
        C t = mk<T>(T(0), T(0));
        if (lane == c) {
          t = mk<T>(stau[c], T(0));
        } else if (lane < c) {
          C a3 = mk<T>(T(0), T(0));
          for (int s2 = lane; s2 < c; ++s2) a3 = cadd<T>(a3, cmul<T>(sT[lane][s2], sG[s2][c]));
          t = cscale<T>(a3, -stau[c]);
        }
        sT[lane][c] = t;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (q == 0) {
    C* Tb = Tm + (size_t)b * BW * BW;
    for (int idx = threadIdx.x; idx < BW * BW; idx += PQ_THREADS) Tb[idx] = sT[idx / BW][idx % BW];
  }
  // Y, YT = Y T and the panel (R above its diagonal, beta on it, zeros below)
  C* Yb = Y + (size_t)b * BW * nm;
  C* YTb = YT + (size_t)b * BW * nm;
  for (int idx = threadIdx.x; idx < nr * BW; idx += PQ_THREADS) {
    const int c = idx / nr, r = idx % nr;   // consecutive threads: consecutive rows
    const int rg = rlo + r;
    C a4 = mk<T>(T(0), T(0));
#pragma unroll 4
    for (int u = 0; u <= c; ++u) a4 = cadd<T>(a4, cmul<T>(Yl[(size_t)r * BW + u], sT[u][c]));
    Yb[(size_t)c * nm + rg] = Yl[(size_t)r * BW + c];
    YTb[(size_t)c * nm + rg] = a4;
  }
  for (int idx = threadIdx.x; idx < nr * BW; idx += PQ_THREADS) {
    const int r = idx / BW, c = idx % BW;
    const int rg = rlo + r;
    const C v = rg == c ? sbeta[c] : (rg > c ? mk<T>(T(0), T(0)) : P[idx]);
    Ab[(size_t)(k + BW + rg) * nm + k + c] = v;
  }
  if constexpr (CL) cg::this_cluster().sync();   // no CTA leaves while others may read its partials
}

// --------------------------------------------------------- W = A22 (Y T) --
// Wp[s][c][r] = sum over the s-th inner chunk of A22[r][x] YT[c][x].
template <typename T>
__global__ void __launch_bounds__(256)
k_ts_w(Batch bt, int k, const c2<T>* __restrict__ A, const c2<T>* __restrict__ YT, c2<T>* __restrict__ Wp,
       int nsplit) {
  using C = c2<T>;
  constexpr int WR = Tiles<T>::WR, WK = Tiles<T>::WK, RPT = WR / 16;
  __shared__ C sA[WR][WK + 1];
  __shared__ C sY[BW][WK + 1];
  const int b = blockIdx.z / nsplit, sp = blockIdx.z % nsplit;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int m = n - k - BW;
  const int r0 = blockIdx.x * WR;
  if (m <= 0 || r0 >= m) return;
  const int chunk = ((m + nsplit - 1) / nsplit + WK - 1) / WK * WK;
  const int x_lo = sp * chunk, x_hi = min(m, x_lo + chunk);
  const C* A22 = A + (size_t)b * nm * nm + (size_t)(k + BW) * nm + (k + BW);
  const C* YTb = YT + (size_t)b * BW * nm;
  const int tc = threadIdx.x % BW, tr = threadIdx.x / BW;   // 16 x 16 threads: RPT rows each
  C acc[RPT];
#pragma unroll
  for (int u = 0; u < RPT; ++u) acc[u] = mk<T>(T(0), T(0));
  for (int x0 = x_lo; x0 < x_hi; x0 += WK) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < WR * WK; idx += 256) {
      const int rr = idx / WK, xx = idx % WK;
      const int r = r0 + rr, x = x0 + xx;
      sA[rr][xx] = (r < m && x < x_hi) ? A22[(size_t)r * nm + x] : mk<T>(T(0), T(0));
    }
    for (int idx = threadIdx.x; idx < BW * WK; idx += 256) {
      const int c = idx / WK, xx = idx % WK;
      const int x = x0 + xx;
      sY[c][xx] = x < x_hi ? YTb[(size_t)c * nm + x] : mk<T>(T(0), T(0));
    }
    __syncthreads();
#pragma unroll 8
    for (int xx = 0; xx < WK; ++xx) {
      const C y = sY[tc][xx];
#pragma unroll
      for (int u = 0; u < RPT; ++u) acc[u] = cadd<T>(acc[u], cmul<T>(sA[tr * RPT + u][xx], y));
    }
  }
  C* W = Wp + ((size_t)b * nsplit + sp) * BW * nm;
#pragma unroll
  for (int u = 0; u < RPT; ++u) {
    const int r = r0 + tr * RPT + u;
    if (r < m) W[(size_t)tc * nm + r] = acc[u];
  }
}

// Float32 W = A22 (Y T) with register tiles: 128 rows x 16 columns per CTA,
// each thread 4 rows x 2 columns; A22 tiles read as 16-byte pairs of
// complex entries (row-major, rows 34 complex apart: the 4 rows a warp reads
// at once fall on distinct banks), (Y T) tiles stored x-major so a thread
// reads its column pair with one 16-byte load; the next tile is fetched into
// registers while the current one is used.  Needs an even n_max (16-byte
// alignment of every row pair); same sums as k_ts_w in a different order.
constexpr int W4R = 128, W4K = 32, W4LD = W4K + 2;

__device__ __forceinline__ float4 ld_pair(const float2* __restrict__ row, int x, int x_hi, bool row_ok) {
  if (!row_ok || x >= x_hi) return make_float4(0.f, 0.f, 0.f, 0.f);
  if (x + 1 < x_hi) return *reinterpret_cast<const float4*>(row + x);
  const float2 a = row[x];
  return make_float4(a.x, a.y, 0.f, 0.f);
}

__global__ void __launch_bounds__(256)
k_ts_w4(Batch bt, int k, const float2* __restrict__ A, const float2* __restrict__ YT, float2* __restrict__ Wp,
        int nsplit) {
  __shared__ __align__(16) float2 sA[W4R * W4LD];
  __shared__ __align__(16) float2 sY[W4K * BW];
  const int b = blockIdx.z / nsplit, sp = blockIdx.z % nsplit;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int m = n - k - BW;
  const int r0 = blockIdx.x * W4R;
  if (m <= 0 || r0 >= m) return;
  const int chunk = ((m + nsplit - 1) / nsplit + W4K - 1) / W4K * W4K;
  const int x_lo = sp * chunk, x_hi = min(m, x_lo + chunk);
  const float2* A22 = A + (size_t)b * nm * nm + (size_t)(k + BW) * nm + (k + BW);
  const float2* YTb = YT + (size_t)b * BW * nm;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cp = lane >> 2, rg = lane & 3;   // column pair (2 cp, 2 cp + 1), row group
  // tile loads: A rows tid / 16 + 16 i (i < 8), pair tid % 16; Y column tid / 16, pair tid % 16
  const int la_r = tid >> 4, la_p = tid & 15;
  float4 ra[8], ry;
  auto fetch = [&](int x0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = r0 + la_r + 16 * i;
      ra[i] = ld_pair(A22 + (size_t)r * nm, x0 + 2 * la_p, x_hi, r < m);
    }
    ry = ld_pair(YTb + (size_t)la_r * nm, x0 + 2 * la_p, x_hi, true);
  };
  float2 acc[4][2];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = make_float2(0.f, 0.f);
  if (x_lo < x_hi) fetch(x_lo);
  for (int x0 = x_lo; x0 < x_hi; x0 += W4K) {
    __syncthreads();   // the previous tile is no longer read
#pragma unroll
    for (int i = 0; i < 8; ++i)
      *reinterpret_cast<float4*>(&sA[(la_r + 16 * i) * W4LD + 2 * la_p]) = ra[i];
    sY[(2 * la_p) * BW + la_r] = make_float2(ry.x, ry.y);
    sY[(2 * la_p + 1) * BW + la_r] = make_float2(ry.z, ry.w);
    __syncthreads();
    if (x0 + W4K < x_hi) fetch(x0 + W4K);
#pragma unroll 4
    for (int xx = 0; xx < W4K; xx += 2) {
      const float4 y0 = *reinterpret_cast<const float4*>(&sY[xx * BW + 2 * cp]);         // Y[xx][2cp], Y[xx][2cp+1]
      const float4 y1 = *reinterpret_cast<const float4*>(&sY[(xx + 1) * BW + 2 * cp]);   // Y[xx+1][..]
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 a = *reinterpret_cast<const float4*>(&sA[(warp * 16 + rg + 4 * u) * W4LD + xx]);
        // acc[u][j] += A[xx] Y[xx][j] + A[xx+1] Y[xx+1][j]
        acc[u][0].x += a.x * y0.x - a.y * y0.y + a.z * y1.x - a.w * y1.y;
        acc[u][0].y += a.x * y0.y + a.y * y0.x + a.z * y1.y + a.w * y1.x;
        acc[u][1].x += a.x * y0.z - a.y * y0.w + a.z * y1.z - a.w * y1.w;
        acc[u][1].y += a.x * y0.w + a.y * y0.z + a.z * y1.w + a.w * y1.z;
      }
    }
  }
  float2* W = Wp + ((size_t)b * nsplit + sp) * BW * nm;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = r0 + warp * 16 + rg + 4 * u;
    if (r < m) {
      W[(size_t)(2 * cp) * nm + r] = acc[u][0];
      W[(size_t)(2 * cp + 1) * nm + r] = acc[u][1];
    }
  }
}

// ----------------------------------------------- Z = W - 1/2 Y (T^H M) --
// Two wide launches over row chunks of ZR rows: k_ts_wm sums the split
// partials of W (kept in Z) and forms the chunk's share of M = Y^H W;
// k_ts_zc adds the shares in chunk order, P = T^H M, Z = W - 1/2 Y P.
constexpr int ZR = 128;

template <typename T>
__global__ void __launch_bounds__(256)
k_ts_wm(Batch bt, int k, const c2<T>* __restrict__ Y, const c2<T>* __restrict__ Wp, int nsplit,
        c2<T>* __restrict__ Z, c2<T>* __restrict__ Mp, int nchunk) {
  using C = c2<T>;
  __shared__ C sY[BW][ZR + 1], sW[BW][ZR + 1];
  const int b = blockIdx.y;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int m = n - k - BW;
  const int r0 = blockIdx.x * ZR;
  C* Mb = Mp + ((size_t)b * nchunk + blockIdx.x) * BW * BW;
  if (m <= 0) return;
  if (r0 >= m) {   // chunk past this matrix's rows: a zero share
    for (int idx = threadIdx.x; idx < BW * BW; idx += 256) Mb[idx] = mk<T>(T(0), T(0));
    return;
  }
  const C* Yb = Y + (size_t)b * BW * nm;
  C* Zb = Z + (size_t)b * BW * nm;
  for (int idx = threadIdx.x; idx < BW * ZR; idx += 256) {
    const int c = idx / ZR, rr = idx % ZR;
    const int r = r0 + rr;
    C w = mk<T>(T(0), T(0)), y = mk<T>(T(0), T(0));
    if (r < m) {
      for (int sp = 0; sp < nsplit; ++sp) w = cadd<T>(w, Wp[((size_t)b * nsplit + sp) * BW * nm + (size_t)c * nm + r]);
      y = Yb[(size_t)c * nm + r];
      Zb[(size_t)c * nm + r] = w;
    }
    sW[c][rr] = w;
    sY[c][rr] = y;
  }
  __syncthreads();
  const int u = threadIdx.x / BW, c = threadIdx.x % BW;
  C acc = mk<T>(T(0), T(0));
#pragma unroll 4
  for (int rr = 0; rr < ZR; ++rr) acc = cadd<T>(acc, cjmul<T>(sY[u][rr], sW[c][rr]));
  Mb[u * BW + c] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_ts_zc(Batch bt, int k, const c2<T>* __restrict__ Y, const c2<T>* __restrict__ Tm, const c2<T>* __restrict__ Mp,
        int nchunk, c2<T>* __restrict__ Z) {
  using C = c2<T>;
  __shared__ C sM[BW][BW], sP[BW][BW];
  const int b = blockIdx.y;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int m = n - k - BW;
  const int r0 = blockIdx.x * ZR;
  if (m <= 0 || r0 >= m) return;
  {
    const int u = threadIdx.x / BW, c = threadIdx.x % BW;
    C acc = mk<T>(T(0), T(0));
    for (int ch = 0; ch < nchunk; ++ch) acc = cadd<T>(acc, Mp[((size_t)b * nchunk + ch) * BW * BW + u * BW + c]);
    sM[u][c] = acc;
  }
  __syncthreads();
  const C* Tb = Tm + (size_t)b * BW * BW;
  {
    const int u = threadIdx.x / BW, c = threadIdx.x % BW;
    C acc = mk<T>(T(0), T(0));
    for (int s2 = 0; s2 <= u; ++s2) acc = cadd<T>(acc, cjmul<T>(Tb[s2 * BW + u], sM[s2][c]));   // conj(T[s][u]) M[s][c]
    sP[u][c] = cscale<T>(acc, T(0.5));
  }
  __syncthreads();
  const C* Yb = Y + (size_t)b * BW * nm;
  C* Zb = Z + (size_t)b * BW * nm;
  for (int idx = threadIdx.x; idx < BW * ZR; idx += 256) {
    const int c = idx / ZR, r = r0 + idx % ZR;
    if (r >= m) continue;
    C acc = mk<T>(T(0), T(0));
#pragma unroll
    for (int u = 0; u < BW; ++u) acc = cadd<T>(acc, cmul<T>(Yb[(size_t)u * nm + r], sP[u][c]));
    Zb[(size_t)c * nm + r] = csub<T>(Zb[(size_t)c * nm + r], acc);
  }
}

// ----------------------------------------- A22 -= Y Z^H + Z Y^H (tiles) --
template <typename T>
__global__ void __launch_bounds__(256)
k_ts_her2k(Batch bt, int k, c2<T>* __restrict__ A, const c2<T>* __restrict__ Y, const c2<T>* __restrict__ Z) {
  using C = c2<T>;
  constexpr int GT = Tiles<T>::GT, PB = GT / 16;   // PB x PB outputs per thread
  __shared__ C sYr[BW][GT], sZr[BW][GT], sYc[BW][GT], sZc[BW][GT];
  const int b = blockIdx.z;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int m = n - k - BW;
  const int r0 = blockIdx.y * GT, c0 = blockIdx.x * GT;
  if (m <= 0 || r0 >= m || c0 >= m) return;
  const C* Yb = Y + (size_t)b * BW * nm;
  const C* Zb = Z + (size_t)b * BW * nm;
  for (int idx = threadIdx.x; idx < BW * GT; idx += 256) {
    const int q = idx / GT, x = idx % GT;
    const int r = r0 + x, c = c0 + x;
    sYr[q][x] = r < m ? Yb[(size_t)q * nm + r] : mk<T>(T(0), T(0));
    sZr[q][x] = r < m ? Zb[(size_t)q * nm + r] : mk<T>(T(0), T(0));
    sYc[q][x] = c < m ? Yb[(size_t)q * nm + c] : mk<T>(T(0), T(0));
    sZc[q][x] = c < m ? Zb[(size_t)q * nm + c] : mk<T>(T(0), T(0));
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  C acc[PB][PB];
#pragma unroll
  for (int a = 0; a < PB; ++a)
#pragma unroll
    for (int d = 0; d < PB; ++d) acc[a][d] = mk<T>(T(0), T(0));
#pragma unroll 4
  for (int q = 0; q < BW; ++q) {
    C yr[PB], zr[PB], yc[PB], zc[PB];
#pragma unroll
    for (int a = 0; a < PB; ++a) {
      yr[a] = sYr[q][ty + 16 * a];
      zr[a] = sZr[q][ty + 16 * a];
      yc[a] = sYc[q][tx + 16 * a];
      zc[a] = sZc[q][tx + 16 * a];
    }
#pragma unroll
    for (int a = 0; a < PB; ++a)
#pragma unroll
      for (int d = 0; d < PB; ++d) {
        acc[a][d] = cadd<T>(acc[a][d], cmulc<T>(yr[a], zc[d]));
        acc[a][d] = cadd<T>(acc[a][d], cmulc<T>(zr[a], yc[d]));
      }
  }
  C* A22 = A + (size_t)b * nm * nm + (size_t)(k + BW) * nm + (k + BW);
#pragma unroll
  for (int a = 0; a < PB; ++a)
#pragma unroll
    for (int d = 0; d < PB; ++d) {
      const int r = r0 + ty + 16 * a, c = c0 + tx + 16 * d;
      if (r < m && c < m) {
        C* e = A22 + (size_t)r * nm + c;
        *e = csub<T>(*e, acc[a][d]);
      }
    }
}

template <typename T>
size_t per_matrix_bytes(int nm, int nsplit) {
  using C = c2<T>;
  const size_t nchunk = (size_t)(nm + ZR - 1) / ZR;
  const size_t tc = sizeof(T) == 4 ? tc_operand_bytes(nm, 6) : 0;   // tensor-core operands (float32 only)
  return sizeof(C) * ((size_t)nm * nm + (size_t)(3 + nsplit) * BW * nm + BW * BW + (size_t)ND * nm +
                      nchunk * BW * BW) + tc + 2048;
}

constexpr int kMaxSplit = 8;

template <typename T>
int solve_large_t(const SolveArgs& a) {
  using C = c2<T>;
  const int nm = a.n_max;
  const CellSet* cells = a.cells;
  const int K2 = a.Kside * a.Kside;
  const size_t per_mat = per_matrix_bytes<T>(nm, kMaxSplit);
  const size_t room = a.ws->cap > a.ws->used ? a.ws->cap - a.ws->used : 0;
  int64_t batch = std::max<int64_t>(1, (int64_t)((room > 65536 ? room - 65536 : 0) / per_mat));
  batch = std::min<int64_t>(batch, a.n_mat);
  const size_t mark = a.ws->used;
  C* A = a.ws->take<C>((size_t)batch * nm * nm);
  C* Y = a.ws->take<C>((size_t)batch * BW * nm);
  C* YT = a.ws->take<C>((size_t)batch * BW * nm);
  C* Z = a.ws->take<C>((size_t)batch * BW * nm);
  C* Wp = a.ws->take<C>((size_t)batch * kMaxSplit * BW * nm);
  C* Tm = a.ws->take<C>((size_t)batch * BW * BW);
  C* Bd = a.ws->take<C>((size_t)batch * ND * nm);
  const int nchunk_max = (nm + ZR - 1) / ZR;
  C* Mp = a.ws->take<C>((size_t)batch * nchunk_max * BW * BW);
  if (!A || !Y || !YT || !Z || !Wp || !Tm || !Bd || !Mp) {
    set_error("large-matrix workspace does not fit");
    return IDOS_ERR_OUT_OF_MEMORY;
  }
  // tensor-core trailing update (float32 storage only)
  const bool use_tc = sizeof(T) == 4 && a.tc_np != 0 && nm % 2 == 0;
  TcPlan tcp;
  if (use_tc) {
    const size_t half = tc_operand_bytes(nm, a.tc_np) / 3;   // Aop: one third, Bop: two thirds
    void* Aop = a.ws->take<char>((size_t)batch * half);
    void* Bop = a.ws->take<char>((size_t)batch * 2 * half);
    if (!Aop || !Bop) {
      set_error("large-matrix workspace does not fit the tensor-core operands");
      return IDOS_ERR_OUT_OF_MEMORY;
    }
    IDOS_TRY(tc_plan(tcp, nm, batch, a.tc_np, Aop, Bop, A));
    tcp.lower = a.her2k_lower;
  }
  // panel QR in shared memory when the (n - BW) x BW panel fits
  const size_t panel_smem = sizeof(C) * (size_t)(nm - BW) * BW;
  const int use_smem = panel_smem <= 160 * 1024 ? 1 : 0;
  if (use_smem)
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_ts_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem));
  int dev = 0, sms = 0;
  IDOS_CUDA_TRY(cudaGetDevice(&dev));
  IDOS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // (launch shapes follow the device's SM count even inside an SM partition,
  // so that results do not depend on how the SMs are shared)
  // cluster panel QR: the smallest cluster (<= 16 CTAs, more than 8 only
  // where the level is not confined to an SM partition) whose shared memory
  // holds the first panel, grown while the batch leaves SMs idle and each CTA
  // keeps at least 64 rows; pc = 0 keeps the one-CTA kernel above (the panel
  // in global memory: n = 8192 needs 16 CTAs)
  int pc = 0, pc_rows = 0;
  for (int q = 1; q <= std::min(16, a.max_cluster); q *= 2) {
    if (q > 8 && pc != 0) break;   // 16 CTAs only when 8 cannot hold the panel
    const int rows = (nm - BW + q - 1) / q;
    const size_t smem = 2 * sizeof(C) * (size_t)rows * BW;
    if (smem > 200 * 1024) continue;
    if (pc == 0 || (a.panel_cluster > 0 ? q <= a.panel_cluster : (batch * q <= sms && rows >= 64))) {
      pc = q;
      pc_rows = rows;
    } else {
      break;
    }
  }
  const size_t pc_smem = 2 * sizeof(C) * (size_t)pc_rows * BW;
  if (pc == 1) {
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_ts_panel_cl<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pc_smem));
  } else if (pc > 1) {
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_ts_panel_cl<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pc_smem));
    if (pc > 8)
      IDOS_CUDA_TRY(cudaFuncSetAttribute(k_ts_panel_cl<T, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  }
  ChasePlan cp;
  IDOS_TRY(chase_plan<T>(nm, batch, sms, a.max_cluster, cp, a.chase_pair != 0));
  const bool own_err = a.err == nullptr;
  int* d_err = own_err ? a.ws->take<int>(1) : a.err;
  if (!d_err) {
    set_error("large-matrix workspace does not fit");
    return IDOS_ERR_OUT_OF_MEMORY;
  }
  if (own_err) IDOS_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), a.stream));
  for (int64_t m0 = 0; m0 < a.n_mat; m0 += batch) {
    const int64_t nb_mat = std::min<int64_t>(batch, a.n_mat - m0);
    Batch bt{nm, (int)nb_mat, K2, m0, cells ? cells->n_act : nullptr};
    IDOS_CUDA_TRY(cudaMemsetAsync(A, 0, sizeof(C) * (size_t)nb_mat * nm * nm, a.stream));
    {
      const int64_t total = nb_mat * (int64_t)nm;
      const int64_t blocks = std::min<int64_t>((total + 127) / 128, 152 * 16);
      ProfScope ps(KID_LG_ASSEMBLE, a.stream);
      if (a.kind == IDOS_TMDC && cells && !a.H) {
        k_lg_assemble_tmdc<T><<<(unsigned)blocks, 128, 0, a.stream>>>(nb_mat, m0, nm, K2, cells->n_act, cells->act,
                                                                      cells->inv, cells->vmask, cells->N, a.Kside,
                                                                      a.tmdc_p, A);
      } else {
        k_lg_assemble<T><<<(unsigned)blocks, 128, 0, a.stream>>>(
            nb_mat, m0, nm, K2, cells ? cells->n_act : nullptr, cells ? cells->act : nullptr,
            cells ? cells->inv : nullptr, cells ? cells->N : 0, a.Kside, a.t, a.eps,
            a.H ? a.H + m0 * (int64_t)nm * nm : nullptr, A);
      }
      IDOS_CHECK_LAUNCH();
    }
    {
      ProfScope ps(KID_LG_BAND, a.stream, 0);
      for (int k = 0; k + BW < nm; k += BW) {
        const int m = nm - k - BW;
        {
          ProfScope p1(KID_LG_PANEL, a.stream);
          if (pc == 1) {
            k_ts_panel_cl<T, false><<<(unsigned)nb_mat, PQ_THREADS, pc_smem, a.stream>>>(bt, k, A, Y, YT, Tm, pc_rows);
          } else if (pc > 1) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(nb_mat * pc));
            cfg.blockDim = dim3(PQ_THREADS);
            cfg.dynamicSmemBytes = pc_smem;
            cfg.stream = a.stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = pc;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            IDOS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_ts_panel_cl<T, true>, bt, k, A, Y, YT, Tm, pc_rows));
          } else {
            k_ts_panel<T><<<(unsigned)nb_mat, PQ_THREADS, use_smem ? panel_smem : 0, a.stream>>>(bt, k, A, Y, YT, Tm,
                                                                                              use_smem);
          }
        }
        // float32 with an even n_max: the register-tiled W (16-byte pairs) or,
        // when the autotuner picked it (w_tile 2, with the tensor-core
        // update), W on the tensor cores
        const bool wtc = use_tc && a.w_tile == 2;
        const bool w4 = sizeof(T) == 4 && (nm % 2) == 0 && a.w_tile != 0;
        const int wr = wtc ? 128 : (w4 ? W4R : Tiles<T>::WR);
        const int rt = (m + wr - 1) / wr;
        // K splits: about one CTA per SM for the tensor-core W (one resident
        // per SM), two per SM for the register-tiled kernels
        const int nsplit =
            wtc ? (int)std::max<int64_t>(1, std::min<int64_t>(std::min(kMaxSplit, (m + 31) / 32),
                                                              (sms + rt * nb_mat - 1) / (rt * nb_mat)))
                : (int)std::max<int64_t>(1, std::min<int64_t>(kMaxSplit, (2 * sms + rt * nb_mat - 1) / (rt * nb_mat)));
        {
          if (wtc) {
            ProfScope p2(KID_LG_W, a.stream, 2);
            IDOS_TRY(tc_w(tcp, bt, k, reinterpret_cast<const c2<float>*>(YT), reinterpret_cast<c2<float>*>(Wp), nsplit,
                          d_err, a.stream));
          } else {
            ProfScope p2(KID_LG_W, a.stream);
            if constexpr (sizeof(T) == 4) {
              if (w4)
                k_ts_w4<<<dim3(rt, 1, (unsigned)(nb_mat * nsplit)), 256, 0, a.stream>>>(
                    bt, k, reinterpret_cast<const float2*>(A), reinterpret_cast<const float2*>(YT),
                    reinterpret_cast<float2*>(Wp), nsplit);
              else
                k_ts_w<T><<<dim3(rt, 1, (unsigned)(nb_mat * nsplit)), 256, 0, a.stream>>>(bt, k, A, YT, Wp, nsplit);
            } else {
              k_ts_w<T><<<dim3(rt, 1, (unsigned)(nb_mat * nsplit)), 256, 0, a.stream>>>(bt, k, A, YT, Wp, nsplit);
            }
          }
          ProfScope p2z(KID_LG_Z, a.stream, 2);
          const int nchunk = (m + ZR - 1) / ZR;
          k_ts_wm<T><<<dim3(nchunk, (unsigned)nb_mat), 256, 0, a.stream>>>(bt, k, Y, Wp, nsplit, Z, Mp, nchunk);
          k_ts_zc<T><<<dim3(nchunk, (unsigned)nb_mat), 256, 0, a.stream>>>(bt, k, Y, Tm, Mp, nchunk, Z);
        }
        if (use_tc) {
          ProfScope p3(KID_LG_HER2K, a.stream, 2);
          IDOS_TRY(tc_her2k(tcp, bt, k, reinterpret_cast<const c2<float>*>(Y), reinterpret_cast<const c2<float>*>(Z),
                            d_err, a.stream));
        } else {
          ProfScope p3(KID_LG_HER2K, a.stream);
          const int gt = (m + Tiles<T>::GT - 1) / Tiles<T>::GT;
          k_ts_her2k<T><<<dim3(gt, gt, (unsigned)nb_mat), 256, 0, a.stream>>>(bt, k, A, Y, Z);
        }
      }
      IDOS_CHECK_LAUNCH();
    }
    {
      ProfScope ps(KID_LG_CHASE, a.stream, 2);
      IDOS_TRY(chase_run<T>(cp, bt, A, Bd, reinterpret_cast<T*>(a.d) + m0 * nm, reinterpret_cast<T*>(a.e2) + m0 * nm,
                            d_err, a.stream));
    }
  }
  if ((cp.csz > 0 || use_tc) && own_err) {
    int herr = 0;
    IDOS_CUDA_TRY(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, a.stream));
    IDOS_CUDA_TRY(cudaStreamSynchronize(a.stream));
    if (herr) {
      set_error("large path: a bounded wait (band chase or tensor-core pipeline) timed out");
      return IDOS_ERR_TIMEOUT;
    }
  }
  a.ws->used = mark;
  return IDOS_OK;
}

}  // namespace

size_t large_path_bytes(int precision, int n_max, int64_t n_mat) {
  const size_t per = precision == IDOS_FP64 ? per_matrix_bytes<double>(n_max, kMaxSplit)
                                            : per_matrix_bytes<float>(n_max, kMaxSplit);
  return per * (size_t)std::max<int64_t>(n_mat, 1) + 65536 + 12 * 256;
}

int solve_large(int precision, const SolveArgs& a) {
  if (a.n_mat == 0) return IDOS_OK;
  return precision == IDOS_FP64 ? solve_large_t<double>(a) : solve_large_t<float>(a);
}

}  // namespace idos

// ------------------------------------------------- trailing-update parity --
namespace {

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

extern "C" int idos_her2k(int tc_products, int n, int64_t batch, const double* A, const double* Y, const double* Z,
                          double* A_out) {
  using namespace idos;
  using namespace idos::lg;
  if (!A || !Y || !Z || !A_out) {
    set_error("null argument");
    return IDOS_ERR_INVALID_ARG;
  }
  if ((tc_products != 0 && tc_products != 3 && tc_products != 6) || n < 1 || n > 8192 || batch < 1 ||
      batch > 65535) {
    set_error("tc_products (0, 3, 6), n (1..8192) or batch (1..65535) out of range");
    return IDOS_ERR_INVALID_ARG;
  }
  int sms = 0;
  IDOS_TRY(check_device(sms));
  const size_t nn = (size_t)n * n;
  const size_t na = (size_t)batch * nn, ny = (size_t)batch * BW * n;
  std::vector<float> hA(2 * na), hY(2 * ny), hZ(2 * ny);
  for (size_t i = 0; i < 2 * na; ++i) hA[i] = (float)A[i];
  for (size_t i = 0; i < 2 * ny; ++i) {
    hY[i] = (float)Y[i];
    hZ[i] = (float)Z[i];
  }
  DevBuf dA, dY, dZ, dErr, dOp;
  IDOS_CUDA_TRY(cudaMalloc(&dA.p, sizeof(float) * 2 * na));
  IDOS_CUDA_TRY(cudaMalloc(&dY.p, sizeof(float) * 2 * ny));
  IDOS_CUDA_TRY(cudaMalloc(&dZ.p, sizeof(float) * 2 * ny));
  IDOS_CUDA_TRY(cudaMalloc(&dErr.p, sizeof(int)));
  IDOS_CUDA_TRY(cudaMemcpy(dA.p, hA.data(), sizeof(float) * 2 * na, cudaMemcpyHostToDevice));
  IDOS_CUDA_TRY(cudaMemcpy(dY.p, hY.data(), sizeof(float) * 2 * ny, cudaMemcpyHostToDevice));
  IDOS_CUDA_TRY(cudaMemcpy(dZ.p, hZ.data(), sizeof(float) * 2 * ny, cudaMemcpyHostToDevice));
  IDOS_CUDA_TRY(cudaMemset(dErr.p, 0, sizeof(int)));
  const Batch bt{n, (int)batch, 1, 0, nullptr};
  auto* cA = reinterpret_cast<c2<float>*>(dA.p);
  auto* cY = reinterpret_cast<c2<float>*>(dY.p);
  auto* cZ = reinterpret_cast<c2<float>*>(dZ.p);
  if (tc_products) {
    const size_t a_bytes = ((size_t)batch * n * tc_products * 4 * BW * 2 + 255) & ~size_t(255);
    IDOS_CUDA_TRY(cudaMalloc(&dOp.p, a_bytes * 3));
    TcPlan p;
    IDOS_TRY(tc_plan(p, n, batch, tc_products, dOp.p, static_cast<char*>(dOp.p) + a_bytes, dA.p));
    IDOS_TRY(tc_her2k(p, bt, -BW, cY, cZ, static_cast<int*>(dErr.p), 0));
  } else {
    const int gt = (n + Tiles<float>::GT - 1) / Tiles<float>::GT;
    k_ts_her2k<float><<<dim3(gt, gt, (unsigned)batch), 256>>>(bt, -BW, cA, cY, cZ);
    IDOS_CHECK_LAUNCH();
  }
  IDOS_CUDA_TRY(cudaDeviceSynchronize());
  int herr = 0;
  IDOS_CUDA_TRY(cudaMemcpy(&herr, dErr.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) {
    set_error("tensor-core trailing update: a bounded wait timed out");
    return IDOS_ERR_TIMEOUT;
  }
  IDOS_CUDA_TRY(cudaMemcpy(hA.data(), dA.p, sizeof(float) * 2 * na, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < 2 * na; ++i) A_out[i] = (double)hA[i];
  return IDOS_OK;
}

extern "C" int idos_stage1_w(int mode, int n, int64_t batch, int k, const double* A, const double* YT,
                             double* W_out) {
  using namespace idos;
  using namespace idos::lg;
  if (!A || !YT || !W_out) {
    set_error("null argument");
    return IDOS_ERR_INVALID_ARG;
  }
  if (mode < 0 || mode > 2 || n < BW + 1 || n > 8192 || batch < 1 || batch > 65535 || k < 0 || k % BW != 0 ||
      k + BW >= n || (mode != 0 && n % 2 != 0)) {
    set_error("mode (0..2), n (17..8192, even for modes 1 and 2), batch (1..65535) or k (multiple of 16 below n - 16) "
              "out of range");
    return IDOS_ERR_INVALID_ARG;
  }
  int sms = 0;
  IDOS_TRY(check_device(sms));
  const int m = n - k - BW;
  const size_t na = (size_t)batch * n * n, ny = (size_t)batch * BW * n;
  std::vector<float> hA(2 * na), hV(2 * ny);
  for (size_t i = 0; i < 2 * na; ++i) hA[i] = (float)A[i];
  for (size_t i = 0; i < 2 * ny; ++i) hV[i] = (float)YT[i];
  DevBuf dA, dV, dW, dErr, dOp;
  IDOS_CUDA_TRY(cudaMalloc(&dA.p, sizeof(float) * 2 * na));
  IDOS_CUDA_TRY(cudaMalloc(&dV.p, sizeof(float) * 2 * ny));
  IDOS_CUDA_TRY(cudaMalloc(&dW.p, sizeof(float) * 2 * ny * kMaxSplit));
  IDOS_CUDA_TRY(cudaMalloc(&dErr.p, sizeof(int)));
  IDOS_CUDA_TRY(cudaMemcpy(dA.p, hA.data(), sizeof(float) * 2 * na, cudaMemcpyHostToDevice));
  IDOS_CUDA_TRY(cudaMemcpy(dV.p, hV.data(), sizeof(float) * 2 * ny, cudaMemcpyHostToDevice));
  IDOS_CUDA_TRY(cudaMemset(dErr.p, 0, sizeof(int)));
  const Batch bt{n, (int)batch, 1, 0, nullptr};
  auto* cA = reinterpret_cast<c2<float>*>(dA.p);
  auto* cV = reinterpret_cast<c2<float>*>(dV.p);
  auto* cW = reinterpret_cast<c2<float>*>(dW.p);
  // the split rule of the solver's loop
  const int wr = mode == 2 ? 128 : (mode == 1 ? W4R : Tiles<float>::WR);
  const int rt = (m + wr - 1) / wr;
  const int nsplit =
      mode == 2 ? (int)std::max<int64_t>(1, std::min<int64_t>(std::min(kMaxSplit, (m + 31) / 32),
                                                              (sms + rt * batch - 1) / (rt * batch)))
                : (int)std::max<int64_t>(1, std::min<int64_t>(kMaxSplit, (2 * sms + rt * batch - 1) / (rt * batch)));
  if (mode == 2) {
    const size_t a_bytes = ((size_t)batch * n * 6 * 4 * BW * 2 + 255) & ~size_t(255);
    IDOS_CUDA_TRY(cudaMalloc(&dOp.p, a_bytes * 3));
    TcPlan p;
    IDOS_TRY(tc_plan(p, n, batch, 6, dOp.p, static_cast<char*>(dOp.p) + a_bytes, dA.p));
    IDOS_TRY(tc_w(p, bt, k, cV, cW, nsplit, static_cast<int*>(dErr.p), 0));
  } else if (mode == 1) {
    k_ts_w4<<<dim3(rt, 1, (unsigned)(batch * nsplit)), 256>>>(bt, k, reinterpret_cast<const float2*>(cA),
                                                              reinterpret_cast<const float2*>(cV),
                                                              reinterpret_cast<float2*>(cW), nsplit);
    IDOS_CHECK_LAUNCH();
  } else {
    k_ts_w<float><<<dim3(rt, 1, (unsigned)(batch * nsplit)), 256>>>(bt, k, cA, cV, cW, nsplit);
    IDOS_CHECK_LAUNCH();
  }
  IDOS_CUDA_TRY(cudaDeviceSynchronize());
  int herr = 0;
  IDOS_CUDA_TRY(cudaMemcpy(&herr, dErr.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) {
    set_error("tensor-core W: a bounded wait timed out");
    return IDOS_ERR_TIMEOUT;
  }
  std::vector<float> hW(2 * ny * nsplit);
  IDOS_CUDA_TRY(cudaMemcpy(hW.data(), dW.p, sizeof(float) * hW.size(), cudaMemcpyDeviceToHost));
  for (int64_t b = 0; b < batch; ++b)
    for (int c = 0; c < BW; ++c)
      for (int r = 0; r < n; ++r) {
        float re = 0.f, im = 0.f;
        if (r < m)
          for (int sp = 0; sp < nsplit; ++sp) {
            const size_t o = (((size_t)b * nsplit + sp) * BW + c) * n + r;
            re += hW[2 * o];
            im += hW[2 * o + 1];
          }
        const size_t q = ((size_t)b * BW + c) * n + r;
        W_out[2 * q] = re;
        W_out[2 * q + 1] = im;
      }
  return IDOS_OK;
}
