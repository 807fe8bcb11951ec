// k_large.cu - blocked Householder tridiagonalisation of large Hermitian
// matrices held in global memory (L2 / HBM), batched over many matrices.
//
// Same reflectors as k_small.cu (real tau, |e_j| = ||x||), organised in
// panels of NB columns (the LAPACK "LATRD" arrangement): inside a panel the
// trailing matrix is left as it was at the panel start and every column is
// corrected on the fly by the panel's earlier (v, w) pairs,
//   A_cur = A_start - V W^H - W V^H,
// so the matrix-vector product of each column is a GEMV with the panel-start
// matrix plus two thin products.  After the panel the trailing block receives
// the rank-2NB update A -= V W^H + W V^H (a Hermitian rank-2k update).
//
// Per column three launches cover every matrix of the batch at once:
//   k_lg_start   corrected column j, d_j, e_j^2, reflector v (one CTA / matrix)
//   k_lg_gemv    y = A22 v (many CTAs / matrix, column-sliced partial sums)
//   k_lg_finish  p, K, w (one CTA / matrix)
// and k_lg_her2k applies the panel update.
#include "graphene.cuh"
#include "internal.h"

namespace idos {

namespace {

constexpr int NB = 32;          // panel width
constexpr int GEMV_ROWS = 256;  // output rows per GEMV CTA
constexpr int GEMV_COLS = 256;  // columns per GEMV slice

template <typename T> __device__ __forceinline__ T tiny_pivot();
template <> __device__ __forceinline__ float tiny_pivot<float>() { return 1e-30f; }
template <> __device__ __forceinline__ double tiny_pivot<double>() { return 1e-290; }

struct LgState {
  int n_max;
  int64_t n_mat;          // matrices in this batch
  int64_t mat0;           // global index of the batch's first matrix
  const int* n_act_cell;  // may be null (all n_max)
  int K2;
};

__device__ __forceinline__ int lg_n(const LgState& s, int64_t mat) {
  return s.n_act_cell ? s.n_act_cell[(s.mat0 + mat) / s.K2] : s.n_max;
}

// Assembly of H(k) into global memory (rows of kept sites only; the buffer is
// zeroed beforehand).  One thread per (matrix, row).
template <typename T>
__global__ void k_lg_assemble(LgState s, const int* __restrict__ act, const int* __restrict__ inv,
                              int N, int K, double t_hop, double eps, const double2* __restrict__ Hin,
                              c2<T>* __restrict__ A) {
  using C = c2<T>;
  const int64_t total = s.n_mat * (int64_t)s.n_max;
  const int n_sites = 2 * N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t mat = idx / s.n_max;
    const int a = (int)(idx - mat * s.n_max);
    C* Am = A + mat * (int64_t)s.n_max * s.n_max;
    if (Hin) {
      const double2* src = Hin + mat * (int64_t)s.n_max * s.n_max + (int64_t)a * s.n_max;
      for (int c = 0; c < s.n_max; ++c) Am[(int64_t)a * s.n_max + c] = mk<T>((T)src[c].x, (T)src[c].y);
      continue;
    }
    const int64_t gmat = s.mat0 + mat;
    const int64_t cell = gmat / s.K2;
    const int kidx = (int)(gmat - cell * s.K2);
    if (a >= s.n_act_cell[cell]) continue;
    int nb[3];
    bool fromB;
    graphene_neighbours(N, act[cell * n_sites + a], nb, fromB);
    C* row = Am + (int64_t)a * s.n_max;
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

// Corrected column j (rows r >= j) of the current matrix, its reflector, and
// the tridiagonal entries d_j, e_j^2.  One CTA per matrix.
template <typename T>
__global__ void __launch_bounds__(1024)
k_lg_start(LgState s, int j0, int i, const c2<T>* __restrict__ A, c2<T>* __restrict__ V,
           c2<T>* __restrict__ W, T* __restrict__ tau_out, T* __restrict__ d_out,
           T* __restrict__ e2_out) {
  using C = c2<T>;
  __shared__ T red[32];
  __shared__ C s_wj[NB], s_vj[NB];
  __shared__ C s_alpha;
  const int64_t mat = blockIdx.x;
  const int n = lg_n(s, mat);
  const int j = j0 + i;
  const int nm = s.n_max;
  C* Vm = V + mat * (int64_t)NB * nm;
  C* Wm = W + mat * (int64_t)NB * nm;
  if (j >= n) return;
  const C* Arow = A + mat * (int64_t)nm * nm + (int64_t)j * nm;
  if (threadIdx.x < i) {
    s_wj[threadIdx.x] = Wm[(int64_t)threadIdx.x * nm + j];
    s_vj[threadIdx.x] = Vm[(int64_t)threadIdx.x * nm + j];
  }
  __syncthreads();
  // column j of A_cur: a_r = conj(A[j][r]) - sum_q V[q][r] conj(W[q][j]) + W[q][r] conj(V[q][j])
  T rest = T(0);
  for (int r = j + threadIdx.x; r < n; r += blockDim.x) {
    C a = conjg<T>(Arow[r]);
    for (int q = 0; q < i; ++q) {
      a = csub<T>(a, cmulc<T>(Vm[(int64_t)q * nm + r], s_wj[q]));
      a = csub<T>(a, cmulc<T>(Wm[(int64_t)q * nm + r], s_vj[q]));
    }
    if (r == j) d_out[mat * nm + j] = a.x;
    else if (r == j + 1) s_alpha = a;
    else rest += cabs2<T>(a);
    // keep the corrected value in V[i][r] for the reflector below
    if (r > j) Vm[(int64_t)i * nm + r] = a;
  }
  rest = block_sum<T>(rest, red);   // contains __syncthreads
  if (j == n - 1) {
    if (threadIdx.x == 0) tau_out[mat] = T(0);
    return;
  }
  const C alpha = s_alpha;
  const T aa2 = cabs2<T>(alpha), sigma2 = aa2 + rest;
  if (threadIdx.x == 0) e2_out[mat * nm + j] = sigma2;
  const bool tr = rest > tiny_pivot<T>();
  T tau = T(0);
  if (tr) {
    const T sigma = sqrt(sigma2), aa = sqrt(aa2);
    const C phs = aa > T(0) ? cscale<T>(alpha, T(1) / aa) : mk<T>(T(1), T(0));
    tau = T(1) / (sigma * (sigma + aa));
    if (threadIdx.x == 0) Vm[(int64_t)i * nm + j + 1] = cadd<T>(alpha, cscale<T>(phs, sigma));
  } else {
    for (int r = j + 1 + threadIdx.x; r < n; r += blockDim.x) Vm[(int64_t)i * nm + r] = mk<T>(T(0), T(0));
  }
  for (int r = threadIdx.x; r <= j && r < nm; r += blockDim.x) Vm[(int64_t)i * nm + r] = mk<T>(T(0), T(0));
  if (threadIdx.x == 0) tau_out[mat] = tau;
}

// Partial y = A22 v over one slice of columns: part[slice][r] = sum_c conj(A[c][r]) v_c.
template <typename T>
__global__ void __launch_bounds__(GEMV_ROWS)
k_lg_gemv(LgState s, int j, int i, const c2<T>* __restrict__ A, const c2<T>* __restrict__ V,
          const T* __restrict__ tau, c2<T>* __restrict__ part, int n_slices) {
  using C = c2<T>;
  __shared__ C sv[GEMV_COLS];
  const int64_t mat = blockIdx.z;
  const int n = lg_n(s, mat);
  const int nm = s.n_max;
  if (j >= n - 1 || tau[mat] == T(0)) return;
  const int r = blockIdx.x * GEMV_ROWS + threadIdx.x;
  const int c0 = max(j + 1, (int)blockIdx.y * GEMV_COLS);
  const int c1 = min(n, (int)(blockIdx.y + 1) * GEMV_COLS);
  const int rmin = blockIdx.x * GEMV_ROWS;
  if (rmin >= n || (int)(blockIdx.y + 1) * GEMV_COLS <= j + 1) return;
  const C* Vi = V + mat * (int64_t)NB * nm + (int64_t)i * nm;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) sv[c - c0] = Vi[c];
  __syncthreads();
  if (r <= j || r >= n) return;
  const C* Am = A + mat * (int64_t)nm * nm;
  C acc = mk<T>(T(0), T(0));
  for (int c = c0; c < c1; ++c) acc = cadd<T>(acc, cjmul<T>(Am[(int64_t)c * nm + r], sv[c - c0]));
  part[(mat * n_slices + blockIdx.y) * (int64_t)nm + r] = acc;
}

// p = tau (y - V (W^H v) - W (V^H v)), K = tau/2 Re(v^H p), w = p - K v.
template <typename T>
__global__ void __launch_bounds__(1024)
k_lg_finish(LgState s, int j0, int i, const c2<T>* __restrict__ V, c2<T>* __restrict__ W,
            const T* __restrict__ tau, const c2<T>* __restrict__ part, int n_slices) {
  using C = c2<T>;
  __shared__ C s1[NB], s2[NB];
  __shared__ T red[32];
  const int64_t mat = blockIdx.x;
  const int n = lg_n(s, mat);
  const int j = j0 + i;
  const int nm = s.n_max;
  C* Wm = W + mat * (int64_t)NB * nm;
  const C* Vm = V + mat * (int64_t)NB * nm;
  if (j >= n) return;
  const T tu = tau[mat];
  if (j == n - 1 || tu == T(0)) {
    for (int r = threadIdx.x; r < nm; r += blockDim.x) Wm[(int64_t)i * nm + r] = mk<T>(T(0), T(0));
    return;
  }
  const C* vi = Vm + (int64_t)i * nm;
  // s1_q = W_q^H v, s2_q = V_q^H v over rows > j (warp q)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < i) {
    C a1 = mk<T>(T(0), T(0)), a2 = mk<T>(T(0), T(0));
    for (int r = j + 1 + lane; r < n; r += 32) {
      const C vr = vi[r];
      a1 = cadd<T>(a1, cjmul<T>(Wm[(int64_t)warp * nm + r], vr));
      a2 = cadd<T>(a2, cjmul<T>(Vm[(int64_t)warp * nm + r], vr));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a1.x += __shfl_xor_sync(0xffffffffu, a1.x, o);
      a1.y += __shfl_xor_sync(0xffffffffu, a1.y, o);
      a2.x += __shfl_xor_sync(0xffffffffu, a2.x, o);
      a2.y += __shfl_xor_sync(0xffffffffu, a2.y, o);
    }
    if (lane == 0) { s1[warp] = a1; s2[warp] = a2; }
  }
  __syncthreads();
  T kpart = T(0);
  const int slice0 = (j + 1) / GEMV_COLS;
  for (int r = j + 1 + threadIdx.x; r < n; r += blockDim.x) {
    C y = mk<T>(T(0), T(0));
    for (int sl = slice0; sl < n_slices && sl * GEMV_COLS < n; ++sl)
      y = cadd<T>(y, part[(mat * n_slices + sl) * (int64_t)nm + r]);
    for (int q = 0; q < i; ++q) {
      y = csub<T>(y, cmul<T>(Vm[(int64_t)q * nm + r], s1[q]));
      y = csub<T>(y, cmul<T>(Wm[(int64_t)q * nm + r], s2[q]));
    }
    const C p = cscale<T>(y, tu);
    Wm[(int64_t)i * nm + r] = p;
    const C vr = vi[r];
    kpart += vr.x * p.x + vr.y * p.y;
  }
  const T Kc = T(0.5) * tu * block_sum<T>(kpart, red);
  for (int r = threadIdx.x; r < nm; r += blockDim.x) {
    if (r > j && r < n) Wm[(int64_t)i * nm + r] = csub<T>(Wm[(int64_t)i * nm + r], cscale<T>(vi[r], Kc));
    else Wm[(int64_t)i * nm + r] = mk<T>(T(0), T(0));
  }
}

// Trailing update A[r][c] -= sum_q V[q][r] conj(W[q][c]) + W[q][r] conj(V[q][c])
// for r, c >= jn.  32 x 32 output tile per CTA, (32, 8) threads.
template <typename T>
__global__ void __launch_bounds__(256)
k_lg_her2k(LgState s, int jn, c2<T>* __restrict__ A, const c2<T>* __restrict__ V,
           const c2<T>* __restrict__ W) {
  using C = c2<T>;
  __shared__ C sVr[NB][33], sWr[NB][33], sVc[NB][33], sWc[NB][33];
  const int64_t mat = blockIdx.z;
  const int n = lg_n(s, mat);
  const int nm = s.n_max;
  const int c0 = jn + blockIdx.x * 32, r0 = jn + blockIdx.y * 32;
  if (c0 >= n || r0 >= n) return;
  const C* Vm = V + mat * (int64_t)NB * nm;
  const C* Wm = W + mat * (int64_t)NB * nm;
  for (int idx = threadIdx.y * 32 + threadIdx.x; idx < NB * 32; idx += 256) {
    const int q = idx / 32, x = idx % 32;
    const int r = r0 + x, c = c0 + x;
    sVr[q][x] = r < n ? Vm[(int64_t)q * nm + r] : mk<T>(T(0), T(0));
    sWr[q][x] = r < n ? Wm[(int64_t)q * nm + r] : mk<T>(T(0), T(0));
    sVc[q][x] = c < n ? Vm[(int64_t)q * nm + c] : mk<T>(T(0), T(0));
    sWc[q][x] = c < n ? Wm[(int64_t)q * nm + c] : mk<T>(T(0), T(0));
  }
  __syncthreads();
  const int c = c0 + threadIdx.x;
  C* Am = A + mat * (int64_t)nm * nm;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int rl = threadIdx.y + 8 * k;
    const int r = r0 + rl;
    C acc = mk<T>(T(0), T(0));
#pragma unroll 8
    for (int q = 0; q < NB; ++q) {
      acc = cadd<T>(acc, cmulc<T>(sVr[q][rl], sWc[q][threadIdx.x]));
      acc = cadd<T>(acc, cmulc<T>(sWr[q][rl], sVc[q][threadIdx.x]));
    }
    if (r < n && c < n) {
      C* e = Am + (int64_t)r * nm + c;
      *e = csub<T>(*e, acc);
    }
  }
}

template <typename T>
int solve_large_t(const SolveArgs& a) {
  using C = c2<T>;
  const int nm = a.n_max;
  const int n_slices = (nm + GEMV_COLS - 1) / GEMV_COLS;
  const CellSet* cells = a.cells;
  LgState st{nm, 0, 0, cells ? cells->n_act : nullptr, a.Kside * a.Kside};
  // batch so the dense matrices stay within half the arena
  const size_t per_mat = sizeof(C) * ((size_t)nm * nm + 2 * (size_t)NB * nm + (size_t)n_slices * nm) +
                         sizeof(T) * 4;
  const size_t room = a.ws->cap > a.ws->used ? a.ws->cap - a.ws->used : 0;
  int64_t batch = std::max<int64_t>(1, (int64_t)(room / (per_mat + 1024)));
  batch = std::min<int64_t>(batch, a.n_mat);
  const size_t mark = a.ws->used;
  C* A = a.ws->take<C>((size_t)batch * nm * nm);
  C* V = a.ws->take<C>((size_t)batch * NB * nm);
  C* W = a.ws->take<C>((size_t)batch * NB * nm);
  C* part = a.ws->take<C>((size_t)batch * n_slices * nm);
  T* tau = a.ws->take<T>((size_t)batch);
  if (!A || !V || !W || !part || !tau) {
    set_error("large-matrix workspace does not fit");
    return IDOS_ERR_OUT_OF_MEMORY;
  }
  for (int64_t m0 = 0; m0 < a.n_mat; m0 += batch) {
    const int64_t nb_mat = std::min<int64_t>(batch, a.n_mat - m0);
    LgState s = st;
    s.n_mat = nb_mat;
    s.mat0 = m0;
    T* dB = reinterpret_cast<T*>(a.d) + m0 * nm;
    T* eB = reinterpret_cast<T*>(a.e2) + m0 * nm;
    IDOS_CUDA_TRY(cudaMemsetAsync(A, 0, sizeof(C) * (size_t)nb_mat * nm * nm, a.stream));
    {
      const int64_t total = nb_mat * (int64_t)nm;
      const int64_t blocks = std::min<int64_t>((total + 127) / 128, 152 * 16);
      ProfScope ps(KID_LG_ASSEMBLE, a.stream);
      k_lg_assemble<T><<<(unsigned)blocks, 128, 0, a.stream>>>(
          s, cells ? cells->act : nullptr, cells ? cells->inv : nullptr, cells ? cells->N : 0,
          a.Kside, a.t, a.eps, a.H ? a.H + m0 * (int64_t)nm * nm : nullptr, A);
      IDOS_CHECK_LAUNCH();
    }
    const dim3 ggrid((nm + GEMV_ROWS - 1) / GEMV_ROWS, n_slices, (unsigned)nb_mat);
    for (int j0 = 0; j0 < nm; j0 += NB) {
      for (int i = 0; i < NB && j0 + i < nm; ++i) {
        const int j = j0 + i;
        {
          ProfScope ps(KID_LG_START, a.stream);
          k_lg_start<T><<<(unsigned)nb_mat, 1024, 0, a.stream>>>(s, j0, i, A, V, W, tau, dB, eB);
        }
        {
          ProfScope ps(KID_LG_GEMV, a.stream);
          k_lg_gemv<T><<<ggrid, GEMV_ROWS, 0, a.stream>>>(s, j, i, A, V, tau, part, n_slices);
        }
        {
          ProfScope ps(KID_LG_FINISH, a.stream);
          k_lg_finish<T><<<(unsigned)nb_mat, 1024, 0, a.stream>>>(s, j0, i, V, W, tau, part, n_slices);
        }
      }
      const int jn = j0 + NB;
      if (jn < nm) {
        const dim3 hgrid((nm - jn + 31) / 32, (nm - jn + 31) / 32, (unsigned)nb_mat);
        ProfScope ps(KID_LG_HER2K, a.stream);
        k_lg_her2k<T><<<hgrid, dim3(32, 8), 0, a.stream>>>(s, jn, A, V, W);
      }
      IDOS_CHECK_LAUNCH();
    }
  }
  a.ws->used = mark;
  return IDOS_OK;
}

}  // namespace

int solve_large(int precision, const SolveArgs& a) {
  if (a.n_mat == 0) return IDOS_OK;
  return precision == IDOS_FP64 ? solve_large_t<double>(a) : solve_large_t<float>(a);
}

}  // namespace idos
