// k_small.cu - fused H(k) assembly + Householder tridiagonalisation of small
// Hermitian matrices held entirely in shared memory (one thread group per
// matrix, several groups per CTA).
//
// H(k) (eq. (3.2a)-(3.2b)) is built directly in shared memory on the kept
// sites only (vacancies compacted out, Sec. 3.2), so it never touches HBM.
// The reduction is the unblocked Householder method with a real scaling
// factor: for column j, with x = A[j+1:, j], sigma = ||x||, phase ph = x_1/|x_1|,
//   v = x + ph sigma e_1,  tau = 1 / (sigma (sigma + |x_1|)),  P = I - tau v v^H,
// P x = -ph sigma e_1, so the Hermitian tridiagonal has |e_j| = sigma and
// its eigenvalues are those of the real symmetric (d, |e|).  The two-sided
// update uses p = tau A22 v, K = tau/2 Re(v^H p), w = p - K v,
// A22 <- A22 - v w^H - w v^H, fused with the next step's product: each step
// reads and writes the trailing block once.
#include <algorithm>
#include <cfloat>

#include "graphene.cuh"
#include "internal.h"

namespace idos {

namespace {

// The reflector v and update vector w of one step, side by side, so the
// fused pass reads the pending pair of a row with one 16-byte (float) load.
template <typename T>
struct __align__(2 * sizeof(c2<T>)) VW {
  c2<T> v, w;
};

// sigma = sqrt(sigma2), |alpha|, the phase alpha / |alpha| (by cabs_phase,
// exact for tiny alpha) and tau = 1 / (sigma (sigma + |alpha|)) of a
// reflector (sigma2 > 0).  Float32 takes the hardware reciprocal square root
// and the fast divide for sigma and tau (a relative error of a few 1e-7, the
// size of the reduction's own rounding); float64 the correctly rounded
// operations.
template <typename T>
__device__ __forceinline__ void reflector_scalars(c2<T> alpha, T sigma2, T& sigma, T& aa, c2<T>& phs, T& tau) {
  aa = cabs_phase<T>(alpha, phs);
  if constexpr (sizeof(T) == 4) {
    sigma = sigma2 * rsqrtf(sigma2);
    tau = __fdividef(1.f, sigma * (sigma + aa));
  } else {
    sigma = sqrt(sigma2);
    tau = T(1) / (sigma * (sigma + aa));
  }
}

template <typename T>
struct SmallLayout {
  // per group: vw[2][n_max] (pending and next pair, first: 16-byte aligned),
  // A[n_max * n_max] (complex), 3 bond phases, scratch
  __host__ __device__ static size_t bytes(int n_max) {
    const size_t b = sizeof(VW<T>) * 2 * (size_t)n_max + sizeof(c2<T>) * ((size_t)n_max * n_max + 3) +
                     sizeof(T) * 64;
    return (b + 31) & ~size_t(31);
  }
};

// One matrix `mat` reduced by the NT threads of group gid (tid = rank in the
// group) in the shared-memory slot `base` of SmallLayout<T>::bytes(n_max).
template <typename T, int NT, int MPB>
__device__ __forceinline__ void small_tridiag_group(unsigned char* base, int gid, int tid,
                                                    const int* __restrict__ n_act_cell, const int* __restrict__ act,
                                                    const int* __restrict__ inv, int N, int K, int n_max, int64_t mat,
                                                    double t_hop, double eps, const double2* __restrict__ Hin,
                                                    T* __restrict__ d_out, T* __restrict__ e2_out) {
  using C = c2<T>;
  VW<T>* vwb0 = reinterpret_cast<VW<T>*>(base);
  VW<T>* vwb1 = vwb0 + n_max;
  C* A = reinterpret_cast<C*>(vwb1 + n_max);
  C* ph = A + (size_t)n_max * n_max;
  T* scratch = reinterpret_cast<T*>(ph + 3);

  const int K2 = K * K;
  const int64_t cell = mat / K2;
  const int kidx = (int)(mat - cell * K2);
  const int n = Hin ? n_max : n_act_cell[cell];
  T* dO = d_out + mat * n_max;
  T* eO = e2_out + mat * n_max;
  if (n <= 0) return;

  // ---------------------------------------------------------- assembly ---
  if (Hin) {
    const double2* src = Hin + mat * (int64_t)n * n;
    for (int i = tid; i < n * n; i += NT) A[i] = mk<T>((T)src[i].x, (T)src[i].y);
  } else {
    const int n_sites = 2 * N * N;
    if (tid < 3) {
      if constexpr (sizeof(T) == 4) {
        const float2 p = graphene_phase_f(N, K, kidx, tid);
        ph[tid] = mk<T>((T)t_hop * p.x, (T)t_hop * p.y);
      } else {
        const double2 p = graphene_phase(N, K, kidx, tid);
        ph[tid] = mk<T>((T)(t_hop * p.x), (T)(t_hop * p.y));
      }
    }
    for (int i = tid; i < n * n; i += NT) A[i] = mk<T>(T(0), T(0));
    group_sync<NT, MPB>(gid);
    const int* actc = act + cell * n_sites;
    const int* invc = inv + cell * n_sites;
    for (int a = tid; a < n; a += NT) {
      int nb[3];
      bool fromB;
      graphene_neighbours(N, actc[a], nb, fromB);
      C* row = A + (size_t)a * n;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int col = invc[nb[b]];
        if (col < 0) continue;
        const C hp = fromB ? conjg<T>(ph[b]) : ph[b];
        row[col] = cadd<T>(row[col], hp);
      }
      row[a].x += (T)eps;
    }
  }
  group_sync<NT, MPB>(gid);

  // ------------------------------------------------------ tridiagonalise ---
  VW<T>* vw = vwb0;     // pending update (v, w) of the previous step
  VW<T>* nvw = vwb1;    // this step's reflector and update vector
  bool pend = false;
  for (int j = 0; j < n - 1; ++j) {
    // (a) bring row j up to date (columns c >= j): it is conj of column j.
    if (pend) {
      const VW<T> q = vw[j];
      for (int c = j + tid; c < n; c += NT) {
        const VW<T> qc = vw[c];
        C a = A[(size_t)j * n + c];
        a = csub<T>(a, cmulc<T>(q.v, qc.w));
        a = csub<T>(a, cmulc<T>(q.w, qc.v));
        A[(size_t)j * n + c] = a;
      }
    }
    group_sync<NT, MPB>(gid);
    // (b) x_c = conj(A[j][c]), c > j.  sigma^2 = |x_{j+1}|^2 + rest.
    T rest = T(0);
    for (int c = j + 2 + tid; c < n; c += NT) rest += cabs2<T>(A[(size_t)j * n + c]);
    rest = group_sum<NT, MPB, T>(rest, scratch, gid);
    const C alpha = conjg<T>(A[(size_t)j * n + j + 1]);
    const T aa2 = cabs2<T>(alpha);
    const T sigma2 = aa2 + rest;
    if (tid == 0) {
      dO[j] = A[(size_t)j * n + j].x;
      eO[j] = sigma2;
    }
    // a column whose entries below the subdiagonal are (numerically) zero is
    // already reduced; |e_j|^2 is recorded either way
    const bool tr = rest > (sizeof(T) == 4 ? T(1e-30f) : T(1e-290));
    T tau = T(0);
    if (tr) {
      T sigma, aa;
      C phs;
      reflector_scalars<T>(alpha, sigma2, sigma, aa, phs, tau);
      for (int c = j + 1 + tid; c < n; c += NT)
        nvw[c].v = (c == j + 1) ? cadd<T>(alpha, cscale<T>(phs, sigma)) : conjg<T>(A[(size_t)j * n + c]);
    }
    group_sync<NT, MPB>(gid);
    // (c) fused pass: apply the pending update to the trailing block and
    //     accumulate p = tau A22 v with the updated entries.
    T kpart = T(0);
    if (pend && tr) {
      // the common case, without branches in the row loop
      for (int c = j + 1 + tid; c < n; c += NT) {
        const VW<T> qc = vw[c];
        // two partial sums (rows j+1, j+3, ... and j+2, j+4, ...) halve the
        // dependent accumulation chain
        C p0 = mk<T>(T(0), T(0)), p1 = mk<T>(T(0), T(0));
        C* ac = A + (size_t)(j + 1) * n + c;
        int r = j + 1;
#pragma unroll 2
        for (; r + 1 < n; r += 2, ac += 2 * n) {
          const VW<T> q0 = vw[r], q1 = vw[r + 1];
          C a0 = ac[0], a1 = ac[n];
          a0 = csub<T>(a0, cmulc<T>(q0.v, qc.w));
          a1 = csub<T>(a1, cmulc<T>(q1.v, qc.w));
          a0 = csub<T>(a0, cmulc<T>(q0.w, qc.v));
          a1 = csub<T>(a1, cmulc<T>(q1.w, qc.v));
          ac[0] = a0;
          ac[n] = a1;
          p0 = cadd<T>(p0, cjmul<T>(a0, nvw[r].v));   // (A22 v)_c = sum_r conj(A[r][c]) v_r
          p1 = cadd<T>(p1, cjmul<T>(a1, nvw[r + 1].v));
        }
        if (r < n) {
          const VW<T> q0 = vw[r];
          C a0 = ac[0];
          a0 = csub<T>(a0, cmulc<T>(q0.v, qc.w));
          a0 = csub<T>(a0, cmulc<T>(q0.w, qc.v));
          ac[0] = a0;
          p0 = cadd<T>(p0, cjmul<T>(a0, nvw[r].v));
        }
        C p = cadd<T>(p0, p1);
        p = cscale<T>(p, tau);
        nvw[c].w = p;
        const C nc = nvw[c].v;
        kpart += nc.x * p.x + nc.y * p.y;   // Re(conj(v_c) p_c)
      }
    } else if (pend || tr) {
      for (int c = j + 1 + tid; c < n; c += NT) {
        C p = mk<T>(T(0), T(0));
        const VW<T> qc = pend ? vw[c] : VW<T>{mk<T>(T(0), T(0)), mk<T>(T(0), T(0))};
        for (int r = j + 1; r < n; ++r) {
          C a = A[(size_t)r * n + c];
          if (pend) {
            const VW<T> qr = vw[r];
            a = csub<T>(a, cmulc<T>(qr.v, qc.w));
            a = csub<T>(a, cmulc<T>(qr.w, qc.v));
            A[(size_t)r * n + c] = a;
          }
          if (tr) p = cadd<T>(p, cjmul<T>(a, nvw[r].v));
        }
        if (tr) {
          p = cscale<T>(p, tau);
          nvw[c].w = p;
          const C nc = nvw[c].v;
          kpart += nc.x * p.x + nc.y * p.y;
        }
      }
    }
    if (tr) {
      const T Kc = T(0.5) * tau * group_sum<NT, MPB, T>(kpart, scratch, gid);
      for (int c = j + 1 + tid; c < n; c += NT) nvw[c].w = csub<T>(nvw[c].w, cscale<T>(nvw[c].v, Kc));
    }
    pend = tr;
    VW<T>* t = vw; vw = nvw; nvw = t;
    group_sync<NT, MPB>(gid);
  }
  if (tid == 0) {
    C a = A[(size_t)(n - 1) * n + (n - 1)];
    if (pend) {
      const VW<T> q = vw[n - 1];
      a = csub<T>(a, cmulc<T>(q.v, q.w));
      a = csub<T>(a, cmulc<T>(q.w, q.v));
    }
    dO[n - 1] = a.x;
  }
}

// Register-resident variant for float32 and n <= 32, one warp per matrix:
// lane c holds column c of A in registers (a[r] = A[r][c]).  Same method and
// step order as small_tridiag_group: row j is brought up to date with the
// pending update (v', w') of step j - 1 (by symmetry conj(row j) is the
// column below the diagonal), the reflector is formed from it, then one
// pass over the rows applies the pending update to a[r] and accumulates
// p = A22 v.  Only the vectors travel through shared memory (a 1.5 KB slot
// per warp, read as broadcasts), pre-arranged so that the pass is six packed
// float32 FMAs per row (fma.rn.f32x2):
//   a <- a - (v'_r.x, v'_r.y) w'_c.x - (v'_r.y, -v'_r.x) w'_c.y
//          - (w'_r.x, w'_r.y) v'_c.x - (w'_r.y, -w'_r.x) v'_c.y
//      = a - v'_r conj(w'_c) - w'_r conj(v'_c),
//   P1 += a (v_r.x, v_r.x),  P2 += a (v_r.y, v_r.y),
//   conj(a) v_r summed = (P1.x + P2.y, P2.x - P1.y).
// The reflector and update entries of rows <= j (reduced) and of rows >= n
// (lanes without a column) are exactly zero, so those rows are no-ops and
// the pass runs over 4-row chunks that intersect (j, n), skipping the others
// with a warp-uniform branch.
struct WarpRegSlot {
  float4 pv[32];   // pending: (v'.x, v'.y, v'.y, -v'.x) of every row
  float4 pw[32];   //          (w'.x, w'.y, w'.y, -w'.x)
  float4 vv[32];   // this step's reflector: (v.x, v.x, v.y, v.y)
};

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ unsigned long long pk2(float2 v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
// packed a b + c on (x, y) pairs
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(d);
}
// the pending rank-2 update of one entry; nw*, nv*: this lane's negated
// (w'_c.x, w'_c.x), (w'_c.y, w'_c.y), (v'_c.x, v'_c.x), (v'_c.y, v'_c.y)
__device__ __forceinline__ float2 pend_update(float2 a, float4 pv, float4 pw, float2 nwx, float2 nwy, float2 nvx,
                                              float2 nvy) {
  a = fma2(f2(pv.x, pv.y), nwx, a);
  a = fma2(f2(pv.z, pv.w), nwy, a);
  a = fma2(f2(pw.x, pw.y), nvx, a);
  a = fma2(f2(pw.z, pw.w), nvy, a);
  return a;
}

// ------------------------------------------ graphene: bidiagonal form --
// Graphene's H(k) in the basis (A sites, B sites) is eps I + [[0, T], [T^H,
// 0]]: the nearest-neighbour hopping of Sec. 3.1 couples only the two
// sublattices, and vacancies remove sites without breaking that.  Its
// eigenvalues are eps +- sigma_i(T) and, when the sublattices keep different
// numbers of sites, |n_A - n_B| more at eps.  The q x p block M between them
// (p = min(n_A, n_B) columns, q = max(n_A, n_B) rows, M[r][c] = H[row site
// r][column site c]) is reduced to upper bidiagonal form (diagonal a_j,
// superdiagonal b_j) by Householder reflectors applied from the left (column
// j) and from the right (row j) in turn (Golub-Kahan).  The tridiagonal with
// diagonal eps and off-diagonals |a_0|, |b_0|, |a_1|, ..., |a_{p-1}|, followed
// by q - p decoupled rows at eps, has exactly the eigenvalues of H(k): the
// output is its (d, e^2).  The reflectors' backward error is float32 eps |M|,
// as for the full reduction, for about a quarter of its flops.  One half-warp
// per matrix (n <= 32, so p, q <= 16): lane c holds column c of M in
// registers; a left reflector's vector lives in one lane and is broadcast,
// a right reflector's row products are summed by a reduce-scatter over the
// 16 lanes and gathered back.
// Every operation below is an explicitly rounded intrinsic: the function is
// inlined into two kernels (per cell set and persistent), and free FMA
// contraction could round them differently; pinned, both routes give the
// same bits.
__device__ __forceinline__ float2 cmul_f(float2 a, float2 b) {
  return f2(__fmaf_rn(a.x, b.x, __fmul_rn(-a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 cjmul_f(float2 a, float2 b) {   // conj(a) b
  return f2(__fmaf_rn(a.x, b.x, __fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(-a.y, b.x)));
}
__device__ __forceinline__ float2 cadd_f(float2 a, float2 b) { return f2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 csub_f(float2 a, float2 b) { return f2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)); }
__device__ __forceinline__ float cabs2_f(float2 a, float acc) { return __fmaf_rn(a.x, a.x, __fmaf_rn(a.y, a.y, acc)); }
// the same in float64 (the float64 path's bidiagonal form)
__device__ __forceinline__ double2 cmul_f(double2 a, double2 b) {
  return make_double2(__fma_rn(a.x, b.x, __dmul_rn(-a.y, b.y)), __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ double2 cjmul_f(double2 a, double2 b) {
  return make_double2(__fma_rn(a.x, b.x, __dmul_rn(a.y, b.y)), __fma_rn(a.x, b.y, __dmul_rn(-a.y, b.x)));
}
__device__ __forceinline__ double2 cadd_f(double2 a, double2 b) {
  return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ double2 csub_f(double2 a, double2 b) {
  return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y));
}
__device__ __forceinline__ double cabs2_f(double2 a, double acc) { return __fma_rn(a.x, a.x, __fma_rn(a.y, a.y, acc)); }
// Householder scalars for x = (alpha, rest): sigma = |x| (sigma2 = |x|^2),
// phs = alpha / |alpha| (1 for alpha = 0), tau = 1 / (sigma (sigma + |alpha|));
// v = x + phs sigma e_1 maps x to -phs sigma e_1.
__device__ __forceinline__ void gk_reflector(float2 al, float sigma2, float& sigma, float2& phs, float& tau) {
  const float s = fmaxf(fabsf(al.x), fabsf(al.y));
  float aa = 0.f;
  phs = f2(1.f, 0.f);
  if (s > 0.f) {
    const float up = s < 0x1p-64f ? 0x1p64f : 1.f;
    const float rs = __frcp_rn(__fmul_rn(s, up));
    const float ax = __fmul_rn(__fmul_rn(al.x, up), rs), ay = __fmul_rn(__fmul_rn(al.y, up), rs);
    const float q = __fmaf_rn(ax, ax, __fmul_rn(ay, ay));
    const float rq = rsqrtf(q);
    phs = f2(__fmul_rn(ax, rq), __fmul_rn(ay, rq));
    aa = __fmul_rn(s, __fmul_rn(q, rq));
  }
  sigma = __fmul_rn(sigma2, rsqrtf(sigma2));
  tau = __fdividef(1.f, __fmul_rn(sigma, __fadd_rn(sigma, aa)));
}
__device__ __forceinline__ void gk_reflector(double2 al, double sigma2, double& sigma, double2& phs, double& tau) {
  const double s = fmax(fabs(al.x), fabs(al.y));
  double aa = 0.0;
  phs = make_double2(1.0, 0.0);
  if (s > 0.0) {
    const double ax = __ddiv_rn(al.x, s), ay = __ddiv_rn(al.y, s);
    const double r = __dsqrt_rn(__fma_rn(ax, ax, __dmul_rn(ay, ay)));
    phs = make_double2(__ddiv_rn(ax, r), __ddiv_rn(ay, r));
    aa = __dmul_rn(s, r);
  }
  sigma = __dsqrt_rn(sigma2);
  tau = __ddiv_rn(1.0, __dmul_rn(sigma, __dadd_rn(sigma, aa)));
}

__device__ __forceinline__ float gk_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double gk_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float gk_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double gk_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float gk_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double gk_add(double a, double b) { return __dadd_rn(a, b); }

template <typename T>
__device__ __forceinline__ void small_gk_half(int hl, unsigned hmask, int hbase, const int* __restrict__ n_act_cell,
                                              const int* __restrict__ act, const int* __restrict__ inv, int N, int K,
                                              int n_max, int64_t mat, double t_hop, double eps,
                                              T* __restrict__ d_out, T* __restrict__ e2_out) {
  using C = c2<T>;
  const T tiny = sizeof(T) == 4 ? T(1e-30) : T(1e-300);
  const int K2 = K * K;
  const int64_t cell = mat / K2;
  const int kidx = (int)(mat - cell * K2);
  const int n = n_act_cell[cell];
  T* dO = d_out + mat * n_max;
  T* eO = e2_out + mat * n_max;
  if (n <= 0) return;
  const int n_sites = 2 * N * N;
  const int* ac = act + cell * n_sites;
  const int* iv = inv + cell * n_sites;
  // sublattice masks over the active indices (site parity 0: A, 1: B)
  const bool isA0 = hl < n && (ac[hl] & 1) == 0;
  const bool isA1 = hl + 16 < n && (ac[hl + 16] & 1) == 0;
  const unsigned lo = (__ballot_sync(hmask, isA0) >> hbase) & 0xFFFFu;
  const unsigned hi = (__ballot_sync(hmask, isA1) >> hbase) & 0xFFFFu;
  const unsigned live = n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const unsigned maskA = lo | (hi << 16), maskB = live & ~maskA;
  const int nA = __popc(maskA), nB = n - nA;
  const unsigned colm = nA >= nB ? maskB : maskA, rowm = live & ~colm;
  const int p = min(nA, nB), q = n - p;
  // column hl of M from the three bonds of its site (a bond to a removed
  // site is dropped; bonds to the same site add up)
  C m[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) m[r] = mk<T>(T(0), T(0));
  if (hl < p) {
    unsigned mm = colm;
    for (int t = 0; t < hl; ++t) mm &= mm - 1u;
    const int ic = __ffs(mm) - 1;
    int nb[3];
    bool fromB;
    graphene_neighbours(N, ac[ic], nb, fromB);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int ai = iv[nb[b]];
      if (ai >= 0 && ((rowm >> ai) & 1u)) {
        const int rw = __popc(rowm & ((1u << ai) - 1u));
        T hx, hy;
        if constexpr (sizeof(T) == 4) {
          const float2 ph = graphene_phase_f(N, K, kidx, b);
          hx = gk_mul((float)t_hop, ph.x);
          hy = gk_mul((float)t_hop, ph.y);
        } else {
          const double2 ph = graphene_phase(N, K, kidx, b);
          hx = __dmul_rn(t_hop, ph.x);
          hy = __dmul_rn(t_hop, ph.y);
        }
        const C hv = fromB ? mk<T>(hx, hy) : mk<T>(hx, -hy);   // H[row site][column site]
#pragma unroll
        for (int r = 0; r < 16; ++r)
          if (r == rw) m[r] = cadd_f(m[r], hv);
      }
    }
  }
  for (int j = 0; j < p; ++j) {
    // left reflector from column j (lane j), rows j .. q-1
    T rest = T(0);
    C al = mk<T>(T(0), T(0));
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (r == j) al = m[r];
      if (r > j && r < q) rest = cabs2_f(m[r], rest);
    }
    rest = __shfl_sync(hmask, rest, hbase + j);
    al.x = __shfl_sync(hmask, al.x, hbase + j);
    al.y = __shfl_sync(hmask, al.y, hbase + j);
    const T sa = cabs2_f(al, rest);
    if (hl == 0) eO[2 * j] = sa;
    if (rest > tiny) {
      T sigma, tau;
      C phs;
      gk_reflector(al, sa, sigma, phs, tau);
      C v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const T vx = __shfl_sync(hmask, m[r].x, hbase + j), vy = __shfl_sync(hmask, m[r].y, hbase + j);
        v[r] = r == j ? mk<T>(gk_fma(phs.x, sigma, al.x), gk_fma(phs.y, sigma, al.y))
                      : (r > j && r < q ? mk<T>(vx, vy) : mk<T>(T(0), T(0)));
      }
      if (hl > j && hl < p) {
        C s0 = mk<T>(T(0), T(0)), s1 = s0;
#pragma unroll
        for (int r = 0; r < 16; r += 2) {
          s0 = cadd_f(s0, cjmul_f(v[r], m[r]));
          s1 = cadd_f(s1, cjmul_f(v[r + 1], m[r + 1]));
        }
        const C sm = cadd_f(s0, s1);
        const C s = mk<T>(gk_mul(sm.x, tau), gk_mul(sm.y, tau));
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          m[r] = csub_f(m[r], cmul_f(v[r], s));
        }
      }
    }
    if (j + 1 >= p) break;
    // right reflector from row j, columns j+1 .. p-1 (lane c holds M[j][c]):
    // z = conj(row), H z = beta e_{j+1}, then M <- M H on rows j+1 .. q-1
    C mj = mk<T>(T(0), T(0));
#pragma unroll
    for (int r = 0; r < 16; ++r)
      if (r == j) mj = m[r];
    const C z = (hl > j && hl < p) ? mk<T>(mj.x, -mj.y) : mk<T>(T(0), T(0));
    T rz = hl > j + 1 ? cabs2_f(z, T(0)) : T(0);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) rz = gk_add(rz, __shfl_xor_sync(hmask, rz, o));
    C az;
    az.x = __shfl_sync(hmask, z.x, hbase + j + 1);
    az.y = __shfl_sync(hmask, z.y, hbase + j + 1);
    const T sb = cabs2_f(az, rz);
    if (hl == 0) eO[2 * j + 1] = sb;
    if (rz > tiny) {
      T sigma, tau;
      C phs;
      gk_reflector(az, sb, sigma, phs, tau);
      const C u = hl == j + 1 ? mk<T>(gk_fma(phs.x, sigma, az.x), gk_fma(phs.y, sigma, az.y)) : z;
      // x_r = sum_c M[r][c] u_c: reduce-scatter (lane hl ends with row hl)
      C k8[8];
      const bool b3 = (hl & 8) != 0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const C plo = (t > j && t < q) ? cmul_f(m[t], u) : mk<T>(T(0), T(0));
        const C phi = (t + 8 > j && t + 8 < q) ? cmul_f(m[t + 8], u) : mk<T>(T(0), T(0));
        const C snd = b3 ? plo : phi, kp = b3 ? phi : plo;
        k8[t] = cadd_f(kp, mk<T>(__shfl_xor_sync(hmask, snd.x, 8), __shfl_xor_sync(hmask, snd.y, 8)));
      }
      C k4[4];
      const bool b2 = (hl & 4) != 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const C snd = b2 ? k8[t] : k8[t + 4], kp = b2 ? k8[t + 4] : k8[t];
        k4[t] = cadd_f(kp, mk<T>(__shfl_xor_sync(hmask, snd.x, 4), __shfl_xor_sync(hmask, snd.y, 4)));
      }
      C k2[2];
      const bool b1 = (hl & 2) != 0;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const C snd = b1 ? k4[t] : k4[t + 2], kp = b1 ? k4[t + 2] : k4[t];
        k2[t] = cadd_f(kp, mk<T>(__shfl_xor_sync(hmask, snd.x, 2), __shfl_xor_sync(hmask, snd.y, 2)));
      }
      const bool b0 = (hl & 1) != 0;
      const C snd = b0 ? k2[0] : k2[1], kp = b0 ? k2[1] : k2[0];
      const C X = cadd_f(kp, mk<T>(__shfl_xor_sync(hmask, snd.x, 1), __shfl_xor_sync(hmask, snd.y, 1)));
      const C tu = mk<T>(gk_mul(tau, u.x), gk_mul(-tau, u.y));   // tau conj(u_c)
      const bool col = hl > j && hl < p;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const C x = mk<T>(__shfl_sync(hmask, X.x, hbase + r), __shfl_sync(hmask, X.y, hbase + r));
        if (col && r > j && r < q) {
          m[r] = csub_f(m[r], cmul_f(x, tu));
        }
      }
    }
  }
  for (int r = hl; r < n; r += 16) dO[r] = (T)eps;
  for (int r = max(0, 2 * p - 1) + hl; r < n - 1; r += 16) eO[r] = T(0);
}

// The same Golub-Kahan reduction for 32 < n <= 128 (graphene N = 5 .. 8, so
// p, q <= 64): 64 threads per matrix, thread c holding column c of M (64
// complex registers).  Per j: the owner of column j publishes the left
// reflector's vector in shared memory (double-buffered by the parity of j;
// one barrier) and every later column takes its dot and update against it
// (four float32 FMAs per row each);
// the right reflector's norm is two warp reductions combined in shared
// memory; its row products are written to a 64 x 65 shared array (column c
// writes its rows, thread r then sums row r over the live columns) and read
// back per row (three more barriers).  Rows outside (j, q) are skipped in
// 4-row chunks by branches uniform over the CTA.  About 170 registers and 36
// KB of shared memory per matrix: six matrices share an SM (the tridiagonal
// register CTA holds one 128 x 128 matrix per SM).
constexpr int kGkT = 64;           // threads per matrix of the CTA variant
constexpr int kGkCtasPerSm = 6;    // resident CTAs per SM it is compiled for (at most 170 registers)
struct GkCtaSlot {
  float2 v[2][64];    // left reflector's vector, by the parity of j
  float2 P[64][65];   // right reflector: row products P[r][c] (padded against bank conflicts)
  float2 X[64];       // right reflector: row sums
  float2 al[2];       // left: alpha, by parity
  float rest[2];      // left: |rows below alpha|^2, by parity
  float red[2];       // right: per-warp partial norms
  float2 az;          // right: alpha
  unsigned words[4];  // sublattice A bits of the active indices
};

__device__ __forceinline__ void small_gk_cta(GkCtaSlot* sl, const int* __restrict__ n_act_cell,
                                             const int* __restrict__ act, const int* __restrict__ inv, int N, int K,
                                             int n_max, int64_t mat, double t_hop, double eps,
                                             float* __restrict__ d_out, float* __restrict__ e2_out) {
  const int c = threadIdx.x, warp = c >> 5, lane = c & 31;
  const int K2 = K * K;
  const int64_t cell = mat / K2;
  const int kidx = (int)(mat - cell * K2);
  const int n = n_act_cell[cell];
  float* dO = d_out + mat * n_max;
  float* eO = e2_out + mat * n_max;
  if (n <= 0) return;   // uniform over the CTA
  const int n_sites = 2 * N * N;
  const int* ac = act + cell * n_sites;
  const int* iv = inv + cell * n_sites;
  // sublattice words: thread c covers active indices c and c + 64
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int idx = c + 64 * k;
    const unsigned b = __ballot_sync(0xffffffffu, idx < n && (ac[min(idx, n_sites - 1)] & 1) == 0);
    if (lane == 0) sl->words[2 * k + warp] = b;
  }
  __syncthreads();
  unsigned colm[4], rowm[4];
  int nA = 0;
#pragma unroll
  for (int w = 0; w < 4; ++w) nA += __popc(sl->words[w]);
  const int nB = n - nA;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const int cnt = min(32, max(0, n - 32 * w));
    const unsigned live = cnt >= 32 ? 0xFFFFFFFFu : ((1u << cnt) - 1u);
    const unsigned mA = sl->words[w];
    colm[w] = nA >= nB ? (live & ~mA) : mA;
    rowm[w] = live & ~colm[w];
  }
  const int p = min(nA, nB), q = n - p;
  float2 m[64];
#pragma unroll
  for (int r = 0; r < 64; ++r) m[r] = f2(0.f, 0.f);
  if (c < p) {
    int ic = -1, cum = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int pc = __popc(colm[w]);
      if (ic < 0 && c < cum + pc) {
        unsigned mm = colm[w];
        for (int t = 0; t < c - cum; ++t) mm &= mm - 1u;
        ic = 32 * w + __ffs(mm) - 1;
      }
      cum += pc;
    }
    int nb[3];
    bool fromB;
    graphene_neighbours(N, ac[ic], nb, fromB);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int ai = iv[nb[b]];
      if (ai >= 0 && ((rowm[ai >> 5] >> (ai & 31)) & 1u)) {
        int rw = __popc(rowm[ai >> 5] & ((1u << (ai & 31)) - 1u));
#pragma unroll
        for (int w = 0; w < 4; ++w)
          if (w < (ai >> 5)) rw += __popc(rowm[w]);
        const float2 ph = graphene_phase_f(N, K, kidx, b);
        const float hx = __fmul_rn((float)t_hop, ph.x), hy = __fmul_rn((float)t_hop, ph.y);
        const float2 hv = fromB ? f2(hx, hy) : f2(hx, -hy);
#pragma unroll
        for (int r = 0; r < 64; ++r)
          if (r == rw) m[r] = cadd_f(m[r], hv);
      }
    }
  }
  for (int j = 0; j < p; ++j) {
    const int bf = j & 1;
    // left reflector from column j (thread j), rows j .. q-1
    if (c == j) {
      float rest = 0.f;
      float2 al = f2(0.f, 0.f);
#pragma unroll
      for (int rb = 0; rb < 16; ++rb) {
        if (4 * rb + 3 < j || 4 * rb >= q) continue;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int r = 4 * rb + t;
          if (r == j) al = m[r];
          if (r > j && r < q) {
            rest = cabs2_f(m[r], rest);
            sl->v[bf][r] = m[r];
          }
        }
      }
      sl->al[bf] = al;
      sl->rest[bf] = rest;
    }
    __syncthreads();
    const float2 al = sl->al[bf];
    const float rest = sl->rest[bf];
    const float sa = cabs2_f(al, rest);
    if (c == 0) eO[2 * j] = sa;
    if (rest > 1e-30f) {
      float sigma, tau;
      float2 phs;
      gk_reflector(al, sa, sigma, phs, tau);
      const float2 vj = f2(__fmaf_rn(phs.x, sigma, al.x), __fmaf_rn(phs.y, sigma, al.y));
      if (c > j && c < p) {
        // conj(v)^T m = (A.x + B.y, A.y - B.x) with A = sum v.x m, B = sum v.y m
        float2 A = f2(0.f, 0.f), B = A;
#pragma unroll
        for (int rb = 0; rb < 16; ++rb) {
          if (4 * rb + 3 < j || 4 * rb >= q) continue;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int r = 4 * rb + t;
            if (r >= j && r < q) {
              const float2 vr = r == j ? vj : sl->v[bf][r];
              A = f2(__fmaf_rn(vr.x, m[r].x, A.x), __fmaf_rn(vr.x, m[r].y, A.y));
              B = f2(__fmaf_rn(vr.y, m[r].x, B.x), __fmaf_rn(vr.y, m[r].y, B.y));
            }
          }
        }
        const float2 s = f2(__fmul_rn(__fadd_rn(A.x, B.y), tau), __fmul_rn(__fsub_rn(A.y, B.x), tau));
        // m <- m - v s: re -= v.x s.x - v.y s.y, im -= v.x s.y + v.y s.x
#pragma unroll
        for (int rb = 0; rb < 16; ++rb) {
          if (4 * rb + 3 < j || 4 * rb >= q) continue;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int r = 4 * rb + t;
            if (r >= j && r < q) {
              const float2 vr = r == j ? vj : sl->v[bf][r];
              m[r] = f2(__fmaf_rn(vr.y, s.y, __fmaf_rn(-vr.x, s.x, m[r].x)),
                        __fmaf_rn(-vr.y, s.x, __fmaf_rn(-vr.x, s.y, m[r].y)));
            }
          }
        }
      }
    }
    if (j + 1 >= p) break;
    // right reflector from row j, columns j+1 .. p-1, applied to rows j+1 .. q-1
    float2 mj = f2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < 64; ++r)
      if (r == j) mj = m[r];
    const float2 z = (c > j && c < p) ? f2(mj.x, -mj.y) : f2(0.f, 0.f);
    float rz = (c > j + 1 && c < p) ? cabs2_f(z, 0.f) : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rz = __fadd_rn(rz, __shfl_xor_sync(0xffffffffu, rz, o));
    if (lane == 0) sl->red[warp] = rz;
    if (c == j + 1) sl->az = z;
    __syncthreads();
    const float rzt = __fadd_rn(sl->red[0], sl->red[1]);
    const float2 az = sl->az;
    const float sb = cabs2_f(az, rzt);
    if (c == 0) eO[2 * j + 1] = sb;
    if (rzt > 1e-30f) {
      float sigma, tau;
      float2 phs;
      gk_reflector(az, sb, sigma, phs, tau);
      const float2 u = c == j + 1 ? f2(__fmaf_rn(phs.x, sigma, az.x), __fmaf_rn(phs.y, sigma, az.y)) : z;
      // row products m[r] u of the live columns
      if (c > j && c < p) {
#pragma unroll
        for (int rb = 0; rb < 16; ++rb) {
          if (4 * rb + 3 <= j || 4 * rb >= q) continue;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int r = 4 * rb + t;
            if (r > j && r < q) sl->P[r][c] = cmul_f(m[r], u);
          }
        }
      }
      __syncthreads();
      if (c > j && c < q) {
        float2 x = f2(0.f, 0.f);
        for (int cc = j + 1; cc < p; ++cc) x = cadd_f(x, sl->P[c][cc]);
        sl->X[c] = x;
      }
      __syncthreads();
      if (c > j && c < p) {
        // m <- m - x w with w = tau conj(u_c)
        const float2 wv = f2(__fmul_rn(tau, u.x), __fmul_rn(-tau, u.y));
#pragma unroll
        for (int rb = 0; rb < 16; ++rb) {
          if (4 * rb + 3 <= j || 4 * rb >= q) continue;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int r = 4 * rb + t;
            if (r > j && r < q) {
              const float2 x = sl->X[r];
              m[r] = f2(__fmaf_rn(x.y, wv.y, __fmaf_rn(-x.x, wv.x, m[r].x)),
                        __fmaf_rn(-x.y, wv.x, __fmaf_rn(-x.x, wv.y, m[r].y)));
            }
          }
        }
      }
    }
  }
  for (int r = c; r < n; r += kGkT) dO[r] = (float)eps;
  for (int r = max(0, 2 * p - 1) + c; r < n - 1; r += kGkT) eO[r] = 0.f;
}

__device__ __forceinline__ void small_tridiag_warp_reg(WarpRegSlot* sl, int lane, const int* __restrict__ n_act_cell,
                                                       const int* __restrict__ act, const int* __restrict__ inv,
                                                       int N, int K, int n_max, int64_t mat, double t_hop,
                                                       double eps, const double2* __restrict__ Hin,
                                                       float* __restrict__ d_out, float* __restrict__ e2_out) {
  const int K2 = K * K;
  const int64_t cell = mat / K2;
  const int kidx = (int)(mat - cell * K2);
  const int n = Hin ? n_max : n_act_cell[cell];
  float* dO = d_out + mat * n_max;
  float* eO = e2_out + mat * n_max;
  if (n <= 0) return;
  const int c = lane;
  float2 a[32];
  if (Hin) {
    const double2* src = Hin + mat * (int64_t)n * n;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      a[r] = f2(0.f, 0.f);
      if (r < n && c < n) a[r] = f2((float)src[(size_t)r * n + c].x, (float)src[(size_t)r * n + c].y);
    }
  } else {
    // column c of H(k): A[col_b][c] = conj(H[c][col_b]) for the three bonds of
    // kept site c (bonds to removed sites dropped; N = 1 sums on one entry)
    int col[3] = {-1, -1, -1};
    float2 hv[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
    if (c < n) {
      const int n_sites = 2 * N * N;
      int nb[3];
      bool fromB;
      graphene_neighbours(N, act[cell * n_sites + c], nb, fromB);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float2 ph = graphene_phase_f(N, K, kidx, b);
        const float hx = (float)t_hop * ph.x, hy = (float)t_hop * ph.y;
        col[b] = inv[cell * n_sites + nb[b]];
        hv[b] = fromB ? f2(hx, hy) : f2(hx, -hy);   // conj of the row entry
      }
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      float2 s2 = f2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; ++b)
        if (col[b] == r) {
          s2.x += hv[b].x;
          s2.y += hv[b].y;
        }
      if (r == c && c < n) s2.x += (float)eps;
      a[r] = s2;
    }
  }
  // this lane's negated pending entries, packed: (-w'.x, -w'.x) ...
  float2 nwx = f2(0.f, 0.f), nwy = nwx, nvx = nwx, nvy = nwx;
  bool pend = false;
  float2 rowj = a[0];
  for (int j = 0; j < n - 1; ++j) {
    // (a) A[j][c] up to date
    if (pend) rowj = pend_update(rowj, sl->pv[j], sl->pw[j], nwx, nwy, nvx, nvy);
    // (b) x_c = conj(A[j][c]) for c > j; sigma^2 = |x_{j+1}|^2 + rest
    const float2 x = f2(rowj.x, -rowj.y);
    float rest = (c > j + 1 && c < n) ? x.x * x.x + x.y * x.y : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
    const float2 alpha = f2(__shfl_sync(0xffffffffu, x.x, j + 1), __shfl_sync(0xffffffffu, x.y, j + 1));
    const float sigma2 = alpha.x * alpha.x + alpha.y * alpha.y + rest;
    if (c == j) dO[j] = rowj.x;
    if (c == 0) eO[j] = sigma2;
    const bool tr = rest > 1e-30f;
    float tau = 0.f;
    float2 v = f2(0.f, 0.f);
    if (tr) {
      float sigma, aa;
      float2 phs;
      reflector_scalars<float>(alpha, sigma2, sigma, aa, phs, tau);
      if (c == j + 1) v = f2(alpha.x + phs.x * sigma, alpha.y + phs.y * sigma);
      else if (c > j + 1 && c < n) v = x;
    }
    sl->vv[c] = make_float4(v.x, v.x, v.y, v.y);
    __syncwarp();
    // (c) one pass over the 4-row chunks meeting (j, n)
    float2 p1a = f2(0.f, 0.f), p2a = p1a, p1b = p1a, p2b = p1a, rown = p1a;
#pragma unroll
    for (int rb = 0; rb < 8; ++rb) {
      if (4 * rb + 3 > j && 4 * rb < n) {   // warp-uniform
        const bool has_next = (j + 1) >> 2 == rb;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = 4 * rb + q;
          float2 ar = a[r];
          if (pend) ar = pend_update(ar, sl->pv[r], sl->pw[r], nwx, nwy, nvx, nvy);
          a[r] = ar;
          if (tr) {
            const float4 vr = sl->vv[r];
            if (q & 1) {
              p1b = fma2(ar, f2(vr.x, vr.y), p1b);
              p2b = fma2(ar, f2(vr.z, vr.w), p2b);
            } else {
              p1a = fma2(ar, f2(vr.x, vr.y), p1a);
              p2a = fma2(ar, f2(vr.z, vr.w), p2a);
            }
          }
          if (has_next && r == j + 1) rown = ar;
        }
      }
    }
    // (d) w = p - K v with p = tau A22 v, K = tau/2 Re(v^H p); zero on the
    //     reduced rows and on lanes without a column
    float2 w = f2(0.f, 0.f);
    if (tr) {
      const float px = (p1a.x + p1b.x) + (p2a.y + p2b.y), py = (p2a.x + p2b.x) - (p1a.y + p1b.y);
      const float2 p = f2(px * tau, py * tau);
      const bool live = c > j && c < n;
      float kp = live ? v.x * p.x + v.y * p.y : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) kp += __shfl_xor_sync(0xffffffffu, kp, o);
      const float Kc = 0.5f * tau * kp;
      if (live) w = f2(p.x - Kc * v.x, p.y - Kc * v.y);
    }
    __syncwarp();   // every lane has read the previous pending pair and v
    sl->pv[c] = make_float4(v.x, v.y, v.y, -v.x);
    sl->pw[c] = make_float4(w.x, w.y, w.y, -w.x);
    __syncwarp();
    nwx = f2(-w.x, -w.x);
    nwy = f2(-w.y, -w.y);
    nvx = f2(-v.x, -v.x);
    nvy = f2(-v.y, -v.y);
    pend = tr;
    rowj = rown;
  }
  if (c == n - 1) {
    float2 dl = rowj;
    if (pend) dl = pend_update(dl, sl->pv[n - 1], sl->pw[n - 1], nwx, nwy, nvx, nvy);
    dO[n - 1] = dl.x;
  }
}

// Register-resident variant for float32 and 32 < n <= 128, one CTA of
// 128 x (128 / RPT) threads per matrix: thread t holds rows [RPT h, RPT h +
// RPT) of column c = t & 127 (h = t >> 7) in registers.  Same method and step order as the other
// variants.  Per step: the thread holding row j of column c brings A[j][c] up
// to date and publishes x_c = conj(A[j][c]) (zero outside (j, n)); after one
// barrier every thread has sigma, tau and its column's v_c; the pass then
// applies the pending update to its rows and accumulates its half of
// p = A22 v, using x itself as v (v and x differ only in row j + 1 by
// ph sigma, added as one correction term); a second barrier combines the
// halves and the K reduction.  Packed float32 FMAs as in the warp variant.
constexpr int kCR = 128;
template <int RPT>
struct CtaRegSlot {
  static constexpr int kParts = kCR / RPT, kThreads = kCR * kParts;
  float4 xq[kCR];          // (x.x, x.x, x.y, x.y) of this step (0 outside (j, n))
  float4 pv[kCR];          // pending (v'.x, v'.y, v'.y, -v'.x)
  float4 pw[kCR];          // pending (w'.x, w'.y, w'.y, -w'.x)
  float4 pp[kParts][kCR];  // p partials of the row parts (P1, P2)
  float red_rest[kThreads / 32];
  float red_kp[kThreads / 32];
};

__device__ __forceinline__ float block_part_sum(float v, float* red) {
  // warp sums into red[warp]; the caller synchronises and adds the 8 values
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  return v;
}

template <int RPT>
__device__ __forceinline__ void small_tridiag_cta_reg(CtaRegSlot<RPT>* sl, const int* __restrict__ n_act_cell,
                                                      const int* __restrict__ act, const int* __restrict__ inv, int N,
                                                      int K, int n_max, int64_t mat, double t_hop, double eps,
                                                      const double2* __restrict__ Hin, float* __restrict__ d_out,
                                                      float* __restrict__ e2_out) {
  const int K2 = K * K;
  const int64_t cell = mat / K2;
  const int kidx = (int)(mat - cell * K2);
  const int n = Hin ? n_max : n_act_cell[cell];
  float* dO = d_out + mat * n_max;
  float* eO = e2_out + mat * n_max;
  if (n <= 0) return;   // uniform over the CTA
  constexpr int kParts = kCR / RPT, kThreads = kCR * kParts;
  const int t = threadIdx.x, c = t & (kCR - 1), hh = t >> 7, r0 = RPT * hh;
  float2 a[RPT];
  if (Hin) {
    const double2* src = Hin + mat * (int64_t)n * n;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      a[r] = f2(0.f, 0.f);
      if (r0 + r < n && c < n) a[r] = f2((float)src[(size_t)(r0 + r) * n + c].x, (float)src[(size_t)(r0 + r) * n + c].y);
    }
  } else {
    int col[3] = {-1, -1, -1};
    float2 hv[3] = {f2(0.f, 0.f), f2(0.f, 0.f), f2(0.f, 0.f)};
    if (c < n) {
      const int n_sites = 2 * N * N;
      int nb[3];
      bool fromB;
      graphene_neighbours(N, act[cell * n_sites + c], nb, fromB);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float2 ph = graphene_phase_f(N, K, kidx, b);
        const float hx = (float)t_hop * ph.x, hy = (float)t_hop * ph.y;
        col[b] = inv[cell * n_sites + nb[b]] - r0;   // row within this half
        hv[b] = fromB ? f2(hx, hy) : f2(hx, -hy);
      }
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      float2 s2 = f2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; ++b)
        if (col[b] == r) {
          s2.x += hv[b].x;
          s2.y += hv[b].y;
        }
      if (r0 + r == c && c < n) s2.x += (float)eps;
      a[r] = s2;
    }
  }
  float2 nwx = f2(0.f, 0.f), nwy = nwx, nvx = nwx, nvy = nwx;
  bool pend = false;
  float2 rowj = a[0];   // A[j][c] on the thread holding row j (row 0: part 0)
  // row j of the pending pair (v', w'), computed by every thread itself after
  // the previous step's second barrier (the shared copies of row j are
  // written after that barrier, so reading them here would race)
  float4 pvj = make_float4(0.f, 0.f, 0.f, 0.f), pwj = pvj;
  for (int j = 0; j < n - 1; ++j) {
    const bool own = j / RPT == hh;   // this thread holds row j of its column
    float rest_part = 0.f;
    if (own) {
      if (pend) rowj = pend_update(rowj, pvj, pwj, nwx, nwy, nvx, nvy);
      const bool in = c > j && c < n;
      const float2 x = in ? f2(rowj.x, -rowj.y) : f2(0.f, 0.f);
      sl->xq[c] = make_float4(x.x, x.x, x.y, x.y);
      if (c > j + 1) rest_part = x.x * x.x + x.y * x.y;
      if (c == j) dO[j] = rowj.x;
    }
    block_part_sum(rest_part, sl->red_rest);
    __syncthreads();   // x, the rest partials
    float rest = 0.f;
#pragma unroll
    for (int w2 = 0; w2 < kThreads / 32; ++w2) rest += sl->red_rest[w2];
    const float4 xa = sl->xq[j + 1];
    const float2 alpha = f2(xa.x, xa.z);
    const float sigma2 = alpha.x * alpha.x + alpha.y * alpha.y + rest;
    if (t == 0) eO[j] = sigma2;
    const bool tr = rest > 1e-30f;
    float tau = 0.f, sigma = 0.f;
    float2 phs = f2(1.f, 0.f), v = f2(0.f, 0.f);
    if (tr) {
      float aa;
      reflector_scalars<float>(alpha, sigma2, sigma, aa, phs, tau);
      const float4 xc = sl->xq[c];
      v = f2(xc.x, xc.z);
      if (c == j + 1) v = f2(alpha.x + phs.x * sigma, alpha.y + phs.y * sigma);
    }
    // pass over this half's 4-row chunks that meet (j, n)
    float2 p1 = f2(0.f, 0.f), p2 = p1, rown = p1;
#pragma unroll
    for (int rb = 0; rb < RPT / 4; ++rb) {
      if (r0 + 4 * rb + 3 > j && r0 + 4 * rb < n) {   // warp-uniform (the row part is per warp)
        const bool has_next = ((j + 1 - r0) >> 2) == rb;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = 4 * rb + q, R = r0 + r;
          float2 ar = a[r];
          if (pend) ar = pend_update(ar, sl->pv[R], sl->pw[R], nwx, nwy, nvx, nvy);
          a[r] = ar;
          if (tr) {
            const float4 xr = sl->xq[R];
            p1 = fma2(ar, f2(xr.x, xr.y), p1);
            p2 = fma2(ar, f2(xr.z, xr.w), p2);
          }
          if (has_next && R == j + 1) rown = ar;
        }
      }
    }
    float kp_part = 0.f;
    if (tr) {
      if ((j + 1) / RPT == hh) {
        // row j + 1: v - x = ph sigma there
        const float2 dv = f2(phs.x * sigma, phs.y * sigma);
        p1 = fma2(rown, f2(dv.x, dv.x), p1);
        p2 = fma2(rown, f2(dv.y, dv.y), p2);
      }
      sl->pp[hh][c] = make_float4(p1.x, p1.y, p2.x, p2.y);
      // Re(conj(v) p) of this half (linear in p): (P1.x + P2.y, P2.x - P1.y)
      if (c > j && c < n) kp_part = v.x * (p1.x + p2.y) + v.y * (p2.x - p1.y);
    }
    block_part_sum(kp_part, sl->red_kp);
    __syncthreads();   // p halves, the K partials; every pass is done
    float2 w = f2(0.f, 0.f);
    pvj = make_float4(0.f, 0.f, 0.f, 0.f);
    pwj = pvj;
    if (tr) {
      float kp = 0.f;
#pragma unroll
      for (int w2 = 0; w2 < kThreads / 32; ++w2) kp += sl->red_kp[w2];
      // tau (tau kp): tau reaches ~1e30 for a noise-level column, tau^2 would overflow
      const float Kc = 0.5f * tau * (tau * kp);
      float4 q = sl->pp[0][c], qn = sl->pp[0][j + 1];
#pragma unroll
      for (int h2 = 1; h2 < kParts; ++h2) {
        const float4 a1 = sl->pp[h2][c], b1 = sl->pp[h2][j + 1];
        q = make_float4(q.x + a1.x, q.y + a1.y, q.z + a1.z, q.w + a1.w);
        qn = make_float4(qn.x + b1.x, qn.y + b1.y, qn.z + b1.z, qn.w + b1.w);
      }
      const float px = tau * (q.x + q.w), py = tau * (q.z - q.y);
      if (c > j && c < n) w = f2(px - Kc * v.x, py - Kc * v.y);
      // row j + 1 of (v, w), the next step's pending entries of its row
      const float2 vn = f2(alpha.x + phs.x * sigma, alpha.y + phs.y * sigma);
      const float nx = tau * (qn.x + qn.w), ny = tau * (qn.z - qn.y);
      const float2 wn = f2(nx - Kc * vn.x, ny - Kc * vn.y);
      pvj = make_float4(vn.x, vn.y, vn.y, -vn.x);
      pwj = make_float4(wn.x, wn.y, wn.y, -wn.x);
    }
    if (hh == 0) {
      sl->pv[c] = make_float4(v.x, v.y, v.y, -v.x);
      sl->pw[c] = make_float4(w.x, w.y, w.y, -w.x);
    }
    nwx = f2(-w.x, -w.x);
    nwy = f2(-w.y, -w.y);
    nvx = f2(-v.x, -v.x);
    nvy = f2(-v.y, -v.y);
    pend = tr;
    if ((j + 1) / RPT == hh) rowj = rown;
    // the next step reads pv / pw after its first barrier
  }
  if (c == n - 1 && (n - 1) / RPT == hh) {
    float2 dl = rowj;
    if (pend) dl = pend_update(dl, pvj, pwj, nwx, nwy, nvx, nvy);
    dO[n - 1] = dl.x;
  }
}

template <int RPT>
__global__ void __launch_bounds__(CtaRegSlot<RPT>::kThreads, 1)
k_small_tridiag_ctareg(const int* __restrict__ n_act_cell, const int* __restrict__ act, const int* __restrict__ inv,
                       int N, int K, int n_max, int64_t n_mat, double t_hop, double eps,
                       const double2* __restrict__ Hin, float* __restrict__ d_out, float* __restrict__ e2_out) {
  __shared__ CtaRegSlot<RPT> slot;
  const int64_t mat = blockIdx.x;
  if (mat >= n_mat) return;
  small_tridiag_cta_reg(&slot, n_act_cell, act, inv, N, K, n_max, mat, t_hop, eps, Hin, d_out, e2_out);
}

constexpr int kCtaRpt = 64;   // rows per thread of the register CTA reduction (256 threads; 32 rows per thread was slower)

// graphene cell sets with 32 < n <= 128: one matrix per 64-thread CTA
__global__ void __launch_bounds__(kGkT, kGkCtasPerSm)
k_small_gk_cta(const int* __restrict__ n_act_cell, const int* __restrict__ act, const int* __restrict__ inv, int N,
               int K, int n_max, double t_hop, double eps, float* __restrict__ d_out, float* __restrict__ e2_out) {
  __shared__ GkCtaSlot slot;
  small_gk_cta(&slot, n_act_cell, act, inv, N, K, n_max, blockIdx.x, t_hop, eps, d_out, e2_out);
}
constexpr int kRegWarps = 4;   // warps (matrices) per CTA of k_small_tridiag_reg

__global__ void __launch_bounds__(32 * kRegWarps)
k_small_tridiag_reg(const int* __restrict__ n_act_cell, const int* __restrict__ act, const int* __restrict__ inv,
                    int N, int K, int n_max, int64_t n_mat, double t_hop, double eps, const double2* __restrict__ Hin,
                    float* __restrict__ d_out, float* __restrict__ e2_out) {
  __shared__ WarpRegSlot slots[kRegWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!Hin) {
    // graphene cells: one matrix per half-warp, bidiagonal form
    const int half = lane >> 4;
    const int64_t mat = ((int64_t)blockIdx.x * kRegWarps + warp) * 2 + half;
    if (mat >= n_mat) return;   // the half-warp leaves together
    small_gk_half(lane & 15, 0xFFFFu << (16 * half), 16 * half, n_act_cell, act, inv, N, K, n_max, mat, t_hop, eps,
                  d_out, e2_out);
    return;
  }
  const int64_t mat = (int64_t)blockIdx.x * kRegWarps + warp;
  if (mat >= n_mat) return;   // whole warp leaves together
  small_tridiag_warp_reg(&slots[warp], lane, n_act_cell, act, inv, N, K, n_max, mat, t_hop, eps, Hin, d_out, e2_out);
}

template <typename T, int NT, int MPB>
__global__ void __launch_bounds__(NT* MPB)
k_small_tridiag(const int* __restrict__ n_act_cell, const int* __restrict__ act,
                const int* __restrict__ inv, int N, int K, int n_max, int64_t n_mat, double t_hop,
                double eps, const double2* __restrict__ Hin, T* __restrict__ d_out,
                T* __restrict__ e2_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int gid = threadIdx.x / NT;
  const int tid = threadIdx.x % NT;
  const int64_t mat = (int64_t)blockIdx.x * MPB + gid;
  if (mat >= n_mat) return;   // whole group leaves together
  small_tridiag_group<T, NT, MPB>(smem_raw + (size_t)gid * SmallLayout<T>::bytes(n_max), gid, tid, n_act_cell, act,
                                  inv, N, K, n_max, mat, t_hop, eps, Hin, d_out, e2_out);
}

// Row-group variant for 32 < n <= NC: thread t works on column c = t / RG
// and on the rows r = j + 1 + (t % RG) (mod RG) of the trailing block, so NC
// columns keep NC * RG threads busy and every step's column loops are RG times
// shorter; the RG partial products of a column are added with shuffles (the
// RG threads of a column are consecutive lanes).  Rows are LD complex entries
// apart (LD = 8 mod 16), which spreads the RG rows a warp touches at once over
// different shared-memory banks.
template <typename T>
struct RgLayout {
  // row stride: n_max rounded up to 16, plus 8 (rows 16 banks apart)
  __host__ __device__ static int ld(int n_max) { return ((n_max + 15) & ~15) + 8; }
  // vw[2][nc] first, then A[n_max][ld], 3 bond phases, scratch
  __host__ __device__ static size_t bytes(int n_max, int nc) {
    const size_t b = sizeof(VW<T>) * 2 * (size_t)nc + sizeof(c2<T>) * ((size_t)n_max * ld(n_max) + 3) +
                     sizeof(T) * 64;
    return (b + 31) & ~size_t(31);
  }
};

// One matrix `mat` reduced by the whole CTA (NC * RG threads) in the
// shared-memory region smem_raw of RgLayout<T>::bytes(n_max, NC).
template <typename T, int NC, int RG>
__device__ __forceinline__ void small_tridiag_rg_cta(unsigned char* smem_raw, const int* __restrict__ n_act_cell,
                                                     const int* __restrict__ act, const int* __restrict__ inv, int N,
                                                     int K, int n_max, int64_t mat, double t_hop, double eps,
                                                     const double2* __restrict__ Hin, T* __restrict__ d_out,
                                                     T* __restrict__ e2_out) {
  using C = c2<T>;
  constexpr int NT = NC * RG;
  const int LD = RgLayout<T>::ld(n_max);
  const int tid = threadIdx.x;
  VW<T>* vwb0 = reinterpret_cast<VW<T>*>(smem_raw);
  VW<T>* vwb1 = vwb0 + NC;
  C* A = reinterpret_cast<C*>(vwb1 + NC);
  C* ph = A + (size_t)n_max * LD;
  T* scratch = reinterpret_cast<T*>(ph + 3);

  const int K2 = K * K;
  const int64_t cell = mat / K2;
  const int kidx = (int)(mat - cell * K2);
  const int n = Hin ? n_max : n_act_cell[cell];
  T* dO = d_out + mat * n_max;
  T* eO = e2_out + mat * n_max;
  if (n <= 0) return;

  // ---------------------------------------------------------- assembly ---
  if (Hin) {
    const double2* src = Hin + mat * (int64_t)n * n;
    for (int i = tid; i < n * n; i += NT) A[(i / n) * LD + i % n] = mk<T>((T)src[i].x, (T)src[i].y);
  } else {
    const int n_sites = 2 * N * N;
    if (tid < 3) {
      if constexpr (sizeof(T) == 4) {
        const float2 p = graphene_phase_f(N, K, kidx, tid);
        ph[tid] = mk<T>((T)t_hop * p.x, (T)t_hop * p.y);
      } else {
        const double2 p = graphene_phase(N, K, kidx, tid);
        ph[tid] = mk<T>((T)(t_hop * p.x), (T)(t_hop * p.y));
      }
    }
    for (int i = tid; i < n * LD; i += NT) A[i] = mk<T>(T(0), T(0));
    __syncthreads();
    const int* actc = act + cell * n_sites;
    const int* invc = inv + cell * n_sites;
    for (int a = tid; a < n; a += NT) {
      int nb[3];
      bool fromB;
      graphene_neighbours(N, actc[a], nb, fromB);
      C* row = A + (size_t)a * LD;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int col = invc[nb[b]];
        if (col < 0) continue;
        const C hp = fromB ? conjg<T>(ph[b]) : ph[b];
        row[col] = cadd<T>(row[col], hp);
      }
      row[a].x += (T)eps;
    }
  }
  __syncthreads();

  // ------------------------------------------------------ tridiagonalise ---
  const int c_own = tid / RG, rg = tid % RG;
  VW<T>* vw = vwb0;
  VW<T>* nvw = vwb1;
  bool pend = false;
  for (int j = 0; j < n - 1; ++j) {
    // (a) row j of the trailing block, columns c >= j
    if (pend) {
      const VW<T> q = vw[j];
      for (int c = j + tid; c < n; c += NT) {
        const VW<T> qc = vw[c];
        C a = A[(size_t)j * LD + c];
        a = csub<T>(a, cmulc<T>(q.v, qc.w));
        a = csub<T>(a, cmulc<T>(q.w, qc.v));
        A[(size_t)j * LD + c] = a;
      }
    }
    __syncthreads();
    // (b) x_c = conj(A[j][c]), c > j
    T rest = T(0);
    for (int c = j + 2 + tid; c < n; c += NT) rest += cabs2<T>(A[(size_t)j * LD + c]);
    rest = group_sum<NT, 1, T>(rest, scratch, 0);
    const C alpha = conjg<T>(A[(size_t)j * LD + j + 1]);
    const T aa2 = cabs2<T>(alpha);
    const T sigma2 = aa2 + rest;
    if (tid == 0) {
      dO[j] = A[(size_t)j * LD + j].x;
      eO[j] = sigma2;
    }
    const bool tr = rest > (sizeof(T) == 4 ? T(1e-30f) : T(1e-290));
    T tau = T(0);
    if (tr) {
      T sigma, aa;
      C phs;
      reflector_scalars<T>(alpha, sigma2, sigma, aa, phs, tau);
      for (int c = j + 1 + tid; c < n; c += NT)
        nvw[c].v = (c == j + 1) ? cadd<T>(alpha, cscale<T>(phs, sigma)) : conjg<T>(A[(size_t)j * LD + c]);
    }
    __syncthreads();
    // (c) fused pass over the trailing block: this thread's column, every
    //     RG-th row; partial products of the column's RG threads added after
    T kpart = T(0);
    {
      const int c = c_own;
      const bool act_c = c > j && c < n;
      C p = mk<T>(T(0), T(0));
      if (act_c && pend && tr) {
        // the common case, without branches in the row loop
        const VW<T> qc = vw[c];
        C* ac = A + (size_t)(j + 1 + rg) * LD + c;
#pragma unroll 2
        for (int r = j + 1 + rg; r < n; r += RG, ac += RG * LD) {
          const VW<T> qr = vw[r];
          C a = *ac;
          a = csub<T>(a, cmulc<T>(qr.v, qc.w));
          a = csub<T>(a, cmulc<T>(qr.w, qc.v));
          *ac = a;
          p = cadd<T>(p, cjmul<T>(a, nvw[r].v));
        }
      } else if (act_c && (pend || tr)) {
        const VW<T> qc = pend ? vw[c] : VW<T>{mk<T>(T(0), T(0)), mk<T>(T(0), T(0))};
        for (int r = j + 1 + rg; r < n; r += RG) {
          C a = A[(size_t)r * LD + c];
          if (pend) {
            const VW<T> qr = vw[r];
            a = csub<T>(a, cmulc<T>(qr.v, qc.w));
            a = csub<T>(a, cmulc<T>(qr.w, qc.v));
            A[(size_t)r * LD + c] = a;
          }
          if (tr) p = cadd<T>(p, cjmul<T>(a, nvw[r].v));
        }
      }
#pragma unroll
      for (int o = 1; o < RG; o <<= 1) {
        p.x += __shfl_xor_sync(0xffffffffu, p.x, o);
        p.y += __shfl_xor_sync(0xffffffffu, p.y, o);
      }
      if (tr && act_c && rg == 0) {
        p = cscale<T>(p, tau);
        nvw[c].w = p;
        const C nc = nvw[c].v;
        kpart = nc.x * p.x + nc.y * p.y;
      }
    }
    if (tr) {
      const T Kc = T(0.5) * tau * group_sum<NT, 1, T>(kpart, scratch, 0);
      for (int c = j + 1 + tid; c < n; c += NT) nvw[c].w = csub<T>(nvw[c].w, cscale<T>(nvw[c].v, Kc));
    }
    pend = tr;
    VW<T>* t = vw; vw = nvw; nvw = t;
    __syncthreads();
  }
  if (tid == 0) {
    C a = A[(size_t)(n - 1) * LD + (n - 1)];
    if (pend) {
      const VW<T> q = vw[n - 1];
      a = csub<T>(a, cmulc<T>(q.v, q.w));
      a = csub<T>(a, cmulc<T>(q.w, q.v));
    }
    dO[n - 1] = a.x;
  }
}

template <typename T, int NC, int RG>
__global__ void __launch_bounds__(NC* RG)
k_small_tridiag_rg(const int* __restrict__ n_act_cell, const int* __restrict__ act, const int* __restrict__ inv,
                   int N, int K, int n_max, int64_t n_mat, double t_hop, double eps, const double2* __restrict__ Hin,
                   T* __restrict__ d_out, T* __restrict__ e2_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t mat = blockIdx.x;
  if (mat >= n_mat) return;
  small_tridiag_rg_cta<T, NC, RG>(smem_raw, n_act_cell, act, inv, N, K, n_max, mat, t_hop, eps, Hin, d_out, e2_out);
}

template <typename T, int NC, int RG>
int run_small_rg(const SolveArgs& a) {
  const size_t smem = RgLayout<T>::bytes(a.n_max, NC);
  auto kern = k_small_tridiag_rg<T, NC, RG>;
  IDOS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const CellSet* c = a.cells;
  ProfScope ps(KID_SMALL_TRIDIAG, a.stream);
  kern<<<(unsigned)a.n_mat, NC * RG, smem, a.stream>>>(
      c ? c->n_act : nullptr, c ? c->act : nullptr, c ? c->inv : nullptr, c ? c->N : 0, a.Kside, a.n_max, a.n_mat,
      a.t, a.eps, a.H, reinterpret_cast<T*>(a.d), reinterpret_cast<T*>(a.e2));
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

template <typename T, int NT, int MPB>
int run_small(const SolveArgs& a) {
  const size_t smem = SmallLayout<T>::bytes(a.n_max) * MPB;
  auto kern = k_small_tridiag<T, NT, MPB>;
  IDOS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t blocks = (a.n_mat + MPB - 1) / MPB;
  const CellSet* c = a.cells;
  ProfScope ps(KID_SMALL_TRIDIAG, a.stream);
  kern<<<(unsigned)blocks, NT * MPB, smem, a.stream>>>(
      c ? c->n_act : nullptr, c ? c->act : nullptr, c ? c->inv : nullptr, c ? c->N : 0, a.Kside,
      a.n_max, a.n_mat, a.t, a.eps, a.H, reinterpret_cast<T*>(a.d), reinterpret_cast<T*>(a.e2));
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

constexpr size_t kSmemLimit = 227 * 1024;

// ---------------------------------------------------- persistent launch ---
// 640 threads: one matrix of n <= 160 per CTA item (160 columns x 4 row
// groups) or one matrix of n <= 32 per warp item (20 warps).
constexpr int kPNC = kPersistMaxN, kPRG = 4, kPThreads = kPNC * kPRG, kPWarps = kPThreads / 32;

struct PersistWork {
  SmallSeg seg[kMaxSmallSegs];
  int64_t end[kMaxSmallSegs];   // cumulative matrix counts, per phase
  int n_big;                    // segments [0, n_big): n_max > 128, CTA items of the 640-thread kernel
  int n_cta;                    // segments [n_big, n_cta): 32 < n_max <= 128, register CTA items;
                                // [n_cta, n_seg): warp items
  int n_seg;
  int64_t total_big, total_cta, total_warp;
};

__global__ void __launch_bounds__(kPThreads, 1)
k_small_persistent(const PersistWork w, double t_hop, double eps, unsigned long long* __restrict__ ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_item;
  // the larger matrices, one per CTA item, segments in descending n
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(&ctr[0], 1ull);
    __syncthreads();
    const long long it = s_item;
    if (it >= w.total_big) break;   // uniform over the CTA
    int g = 0;
    while (g + 1 < w.n_big && it >= w.end[g]) ++g;
    const SmallSeg& sg = w.seg[g];
    const int64_t mat = it - (g > 0 ? w.end[g - 1] : 0);
    small_tridiag_rg_cta<float, kPNC, kPRG>(smem_raw, sg.n_act, sg.act, sg.inv, sg.N, sg.Kside, sg.n_max, mat,
                                            t_hop, eps, nullptr, sg.d, sg.e2);
    __syncthreads();   // s_item and the shared region are reused
  }
}

// The 32 < n <= 128 matrices, one per 64-thread CTA item (bidiagonal form),
// taken in descending n by whichever CTA is free.
__global__ void __launch_bounds__(kGkT, kGkCtasPerSm)
k_small_persistent_cr(const PersistWork w, double t_hop, double eps, unsigned long long* __restrict__ ctr) {
  __shared__ GkCtaSlot slot;
  __shared__ long long s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(&ctr[2], 1ull);
    __syncthreads();
    const long long it = s_item;
    if (it >= w.total_cta) break;   // uniform over the CTA
    int g = w.n_big;
    while (g + 1 < w.n_cta && it >= w.end[g]) ++g;
    const SmallSeg& sg = w.seg[g];
    const int64_t mat = it - (g > w.n_big ? w.end[g - 1] : 0);
    small_gk_cta(&slot, sg.n_act, sg.act, sg.inv, sg.N, sg.Kside, sg.n_max, mat, t_hop, eps, sg.d, sg.e2);
    __syncthreads();   // s_item and the slot are reused
  }
}

// The n <= 32 matrices of every warp segment, one per warp item, taken by
// whichever warp is free (a second persistent launch after the CTA items:
// the register-resident reduction needs more registers per thread than the
// 640-thread CTA items leave).
constexpr int kPWarpCta = 16;   // warps per CTA of the warp-item launch (one CTA fills an SM's registers)

__global__ void __launch_bounds__(32 * kPWarpCta)
k_small_persistent_warps(const PersistWork w, double t_hop, double eps, unsigned long long* __restrict__ ctr) {
  // each half-warp takes matrices from the list on its own (bidiagonal form)
  const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
  const unsigned hmask = 0xFFFFu << (16 * half);
  for (;;) {
    long long it = 0;
    if (hl == 0) it = (long long)atomicAdd(&ctr[1], 1ull);
    it = __shfl_sync(hmask, it, 16 * half);
    if (it >= w.total_warp) break;
    int g = w.n_cta;
    while (g + 1 < w.n_seg && it >= w.end[g]) ++g;
    const SmallSeg& sg = w.seg[g];
    const int64_t mat = it - (g > w.n_cta ? w.end[g - 1] : 0);
    small_gk_half(hl, hmask, 16 * half, sg.n_act, sg.act, sg.inv, sg.N, sg.Kside, sg.n_max, mat, t_hop, eps, sg.d,
                  sg.e2);
    __syncwarp(hmask);
  }
}

}  // namespace

int solve_small_persistent(const SmallSeg* segs, int n_segs, double t, double eps, unsigned long long* counters,
                           int ctas, int reserve, cudaStream_t s) {
  if (n_segs <= 0) return IDOS_OK;
  if (n_segs > kMaxSmallSegs || !counters) {
    set_error("persistent launch: too many segments or no counters");
    return IDOS_ERR_INVALID_ARG;
  }
  // CTA segments first, in descending n_max; then the warp segments
  PersistWork w{};
  int order[kMaxSmallSegs], no = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < n_segs; ++i)
      if ((segs[i].n_max > 32) == (pass == 0) && segs[i].n_mat > 0) order[no++] = i;
  std::sort(order, order + no, [&](int a, int b) {
    const bool ca = segs[a].n_max > 32, cb = segs[b].n_max > 32;
    if (ca != cb) return ca;
    return segs[a].n_max > segs[b].n_max;
  });
  size_t smem = 0;
  for (int q = 0; q < no; ++q) {
    const SmallSeg& sg = segs[order[q]];
    if (sg.n_max < 1 || sg.n_max > kPersistMaxN || !sg.n_act || !sg.act || !sg.inv || !sg.d || !sg.e2) {
      set_error("persistent launch: segment with n_max outside 1..160 or a null buffer");
      return IDOS_ERR_INVALID_ARG;
    }
    w.seg[q] = sg;
    if (sg.n_max > kCR) {
      w.total_big += sg.n_mat;
      w.end[q] = w.total_big;
      w.n_big = q + 1;
      w.n_cta = q + 1;
      smem = std::max(smem, RgLayout<float>::bytes(sg.n_max, kPNC));
    } else if (sg.n_max > 32) {
      w.total_cta += sg.n_mat;
      w.end[q] = w.total_cta;
      w.n_cta = q + 1;
    } else {
      w.total_warp += sg.n_mat;
      w.end[q] = w.total_warp;
    }
  }
  w.n_seg = no;
  if (no == 0) return IDOS_OK;
  if (smem > kSmemLimit) {
    set_error("persistent launch: shared memory above the per-CTA limit");
    return IDOS_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  IDOS_CUDA_TRY(cudaGetDevice(&dev));
  IDOS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int sm_grid = std::max(1, (ctas > 0 ? std::min(ctas, sms) : sms) - std::max(0, reserve));
  IDOS_CUDA_TRY(cudaMemsetAsync(counters, 0, 3 * sizeof(unsigned long long), s));
  if (w.total_cta > 0) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_grid * kGkCtasPerSm, w.total_cta));
    ProfScope ps(KID_SMALL_TRIDIAG, s);
    k_small_persistent_cr<<<grid, kGkT, 0, s>>>(w, t, eps, counters);
    IDOS_CHECK_LAUNCH();
  }
  if (w.total_big > 0) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sm_grid, w.total_big));
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_small_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(KID_SMALL_TRIDIAG, s);
    k_small_persistent<<<grid, kPThreads, smem, s>>>(w, t, eps, counters);
    IDOS_CHECK_LAUNCH();
  }
  if (w.total_warp > 0) {
    // one 16-warp CTA per SM (the register-resident reduction's occupancy)
    const int64_t ctas_w = (w.total_warp + 2 * kPWarpCta - 1) / (2 * kPWarpCta);   // two matrices per warp
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_grid, ctas_w));
    ProfScope ps(KID_SMALL_TRIDIAG, s);
    k_small_persistent_warps<<<grid, 32 * kPWarpCta, 0, s>>>(w, t, eps, counters);
    IDOS_CHECK_LAUNCH();
  }
  return IDOS_OK;
}

bool small_path_fits(int precision, int n_max) {
  if (n_max <= 32) {
    const size_t b = precision == IDOS_FP64 ? SmallLayout<double>::bytes(n_max) : SmallLayout<float>::bytes(n_max);
    return b <= kSmemLimit;
  }
  if (n_max > 256) return false;
  const int nc = n_max <= 64 ? 64 : n_max <= 128 ? 128 : 256;
  const size_t b = precision == IDOS_FP64 ? RgLayout<double>::bytes(n_max, nc) : RgLayout<float>::bytes(n_max, nc);
  return b <= kSmemLimit;
}

int run_small_reg(const SolveArgs& a) {
  const CellSet* c = a.cells;
  const int per = a.H ? kRegWarps : 2 * kRegWarps;   // cell sets: one matrix per half-warp
  const int64_t blocks = (a.n_mat + per - 1) / per;
  ProfScope ps(KID_SMALL_TRIDIAG, a.stream);
  k_small_tridiag_reg<<<(unsigned)blocks, 32 * kRegWarps, 0, a.stream>>>(
      c ? c->n_act : nullptr, c ? c->act : nullptr, c ? c->inv : nullptr, c ? c->N : 0, a.Kside, a.n_max, a.n_mat,
      a.t, a.eps, a.H, reinterpret_cast<float*>(a.d), reinterpret_cast<float*>(a.e2));
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

int run_small_ctareg(const SolveArgs& a) {
  const CellSet* c = a.cells;
  ProfScope ps(KID_SMALL_TRIDIAG, a.stream);
  if (!a.H && c) {
    // graphene cells: bidiagonal form, 64 threads per matrix
    k_small_gk_cta<<<(unsigned)a.n_mat, kGkT, 0, a.stream>>>(c->n_act, c->act, c->inv, c->N, a.Kside, a.n_max,
                                                              a.t, a.eps, reinterpret_cast<float*>(a.d),
                                                              reinterpret_cast<float*>(a.e2));
    IDOS_CHECK_LAUNCH();
    return IDOS_OK;
  }
  k_small_tridiag_ctareg<kCtaRpt><<<(unsigned)a.n_mat, CtaRegSlot<kCtaRpt>::kThreads, 0, a.stream>>>(
      c ? c->n_act : nullptr, c ? c->act : nullptr, c ? c->inv : nullptr, c ? c->N : 0, a.Kside, a.n_max, a.n_mat,
      a.t, a.eps, a.H, reinterpret_cast<float*>(a.d), reinterpret_cast<float*>(a.e2));
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

// float64 graphene cell sets with n <= 32: the bidiagonal form, one matrix per
// half-warp (the float32 cell sets take it inside k_small_tridiag_reg)
__global__ void __launch_bounds__(32 * kRegWarps)
k_small_gk_half64(const int* __restrict__ n_act_cell, const int* __restrict__ act, const int* __restrict__ inv, int N,
                  int K, int n_max, int64_t n_mat, double t_hop, double eps, double* __restrict__ d_out,
                  double* __restrict__ e2_out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4;
  const int64_t mat = ((int64_t)blockIdx.x * kRegWarps + warp) * 2 + half;
  if (mat >= n_mat) return;   // the half-warp leaves together
  small_gk_half<double>(lane & 15, 0xFFFFu << (16 * half), 16 * half, n_act_cell, act, inv, N, K, n_max, mat, t_hop,
                        eps, d_out, e2_out);
}

template <typename T>
static int solve_small_t(const SolveArgs& a) {
  if constexpr (sizeof(T) == 4) {
    if (a.n_max <= 32) return run_small_reg(a);
    if (a.n_max <= kCR) return run_small_ctareg(a);
  } else {
    if (a.n_max <= 32 && !a.H && a.cells) {
      const CellSet* c = a.cells;
      const int64_t blocks = (a.n_mat + 2 * kRegWarps - 1) / (2 * kRegWarps);
      ProfScope ps(KID_SMALL_TRIDIAG, a.stream);
      k_small_gk_half64<<<(unsigned)blocks, 32 * kRegWarps, 0, a.stream>>>(
          c->n_act, c->act, c->inv, c->N, a.Kside, a.n_max, a.n_mat, a.t, a.eps, reinterpret_cast<double*>(a.d),
          reinterpret_cast<double*>(a.e2));
      IDOS_CHECK_LAUNCH();
      return IDOS_OK;
    }
  }
  if (a.n_max <= 32) {
    // up to 4 matrices per CTA while they fit
    if (SmallLayout<T>::bytes(a.n_max) * 4 <= kSmemLimit) return run_small<T, 32, 4>(a);
    return run_small<T, 32, 1>(a);
  }
  if (a.n_max <= 64) return run_small_rg<T, 64, 4>(a);
  if (a.n_max <= 128) return run_small_rg<T, 128, 4>(a);
  return run_small_rg<T, 256, 4>(a);
}

int solve_small(int precision, const SolveArgs& a) {
  if (a.n_mat == 0) return IDOS_OK;
  return precision == IDOS_FP64 ? solve_small_t<double>(a) : solve_small_t<float>(a);
}

}  // namespace idos
