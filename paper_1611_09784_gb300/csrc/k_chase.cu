// k_chase.cu - stage 2 of the large-matrix reduction: the band of half-width
// BW left by stage 1 (k_large.cu) is reduced to real symmetric tridiagonal
// form by bulge chasing.  Sweep i annihilates column i below the subdiagonal
// with a length-BW reflector applied two-sided to the next diagonal block;
// the reflector's right application to the block below creates a bulge
// whose first column the next reflector annihilates, and so on down the
// band.  Step k of sweep i touches only entries with rows and columns in
// [i+1+(k-1)BW, i+1+(k+1)BW) and rows below i+1+(k+1)BW, so it is
// independent of steps k+2, k+3, ... of sweep i-1 (whose entries all have
// rows >= i+(k+2)BW): sweep i may run step k once sweep i-1 has finished
// step k+1, and the lower bandwidth never exceeds 2 BW.  The tridiagonal
// comes out as d = Re diag, e^2 = |subdiag|^2.
#include <cooperative_groups.h>

#include <algorithm>

#include "large.cuh"

namespace cg = cooperative_groups;

namespace idos {
namespace lg {

namespace {

// Warps of the chase kernel (each active sweep needs one; more sweeps than
// warps are taken in turn), bounded by the kernel's register use.
template <typename T> struct Chase;
template <> struct Chase<float> { static constexpr int WARPS = 16; };
template <> struct Chase<double> { static constexpr int WARPS = 8; };


// ----------------------------------------------------------- to band --
// Bd[d][c] = A[c+d][c] for d <= BW, 0 for BW < d < ND.
template <typename T>
__global__ void k_ts_to_band(Batch bt, const c2<T>* __restrict__ A, c2<T>* __restrict__ Bd) {
  using C = c2<T>;
  const int b = blockIdx.y;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const C* Ab = A + (size_t)b * nm * nm;
  C* Bb = Bd + (size_t)b * ND * nm;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < ND * nm; idx += gridDim.x * blockDim.x) {
    const int d = idx / nm, c = idx % nm;
    C v = mk<T>(T(0), T(0));
    if (d <= BW && c + d < n) v = Ab[(size_t)(c + d) * nm + c];
    Bb[idx] = v;
  }
}

// ------------------------------------------------------------ chase --
template <typename T>
struct Band {
  c2<T>* p;
  int ld;
  __device__ __forceinline__ c2<T> get(int r, int c) const {
    return r >= c ? p[(size_t)(r - c) * ld + c] : conjg<T>(p[(size_t)(c - r) * ld + r]);
  }
  __device__ __forceinline__ void set(int r, int c, c2<T> v) const { p[(size_t)(r - c) * ld + c] = v; }
};

// Warp reflector from x (lane l < L holds x_l): tau, v_l, beta = -ph sigma.
template <typename T>
__device__ __forceinline__ bool warp_reflector(c2<T> x, int L, T& tau, c2<T>& v, c2<T>& beta) {
  const int lane = threadIdx.x & 31;
  T rest = (lane >= 1 && lane < L) ? cabs2<T>(x) : T(0);
  rest = warp_sum<T>(rest);
  const c2<T> alpha = shfl_c<T>(x, 0);
  tau = T(0);
  v = x;
  beta = alpha;
  if (!(rest > tiny_rest<T>())) return false;
  c2<T> ph;
  const T aa = cabs_phase<T>(alpha, ph), sigma = sqrt(cabs2<T>(alpha) + rest);
  tau = T(1) / (sigma * (sigma + aa));
  if (lane == 0) v = cadd<T>(alpha, cscale<T>(ph, sigma));
  beta = cscale<T>(ph, -sigma);
  return true;
}

// Per-warp scratch of the chase: the current reflector v, the vector w, the
// previous reflector, and a BW x (BW+1) buffer for column reductions.
template <typename T>
struct WarpScratch {
  c2<T> v[BW], w[BW], vp[BW];
  c2<T> m[BW][BW + 1];
};

// Two-sided D <- H D H on the Hermitian block D = A(r0.., r0..) of size L;
// lane l holds v_l, ws->v holds v.  Only the lower triangle is stored.
template <typename T>
__device__ __forceinline__ void load_block(const Band<T>& bd, int r0, int c0, int Lr, int Lc, c2<T>* out) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < BW; ++c) out[c] = (lane < Lr && c < Lc) ? bd.get(r0 + lane, c0 + c) : mk<T>(T(0), T(0));
}

template <typename T>
__device__ __forceinline__ void warp_two_sided(const Band<T>& bd, int r0, int L, T tau, c2<T> v,
                                               WarpScratch<T>* ws, const c2<T>* drow) {
  using C = c2<T>;
  const int lane = threadIdx.x & 31;
  C p = mk<T>(T(0), T(0));
#pragma unroll
  for (int c = 0; c < BW; ++c) p = cadd<T>(p, cmul<T>(drow[c], ws->v[c]));
  p = cscale<T>(p, tau);
  const T kp = lane < L ? (v.x * p.x + v.y * p.y) : T(0);
  const T K = T(0.5) * tau * warp_sum<T>(kp);
  const C w = csub<T>(p, cscale<T>(v, K));
  if (lane < BW) ws->w[lane] = lane < L ? w : mk<T>(T(0), T(0));
  __syncwarp();
  if (lane < L) {
#pragma unroll
    for (int c = 0; c < BW; ++c) {
      if (c <= lane) {
        C d = drow[c];
        d = csub<T>(d, cmulc<T>(v, ws->w[c]));
        d = csub<T>(d, cmulc<T>(w, ws->v[c]));
        if (c == lane) d.y = T(0);
        bd.set(r0 + lane, r0 + c, d);
      }
    }
  }
  __syncwarp();
}

// band_in_smem: the band is copied into shared memory first (when it fits)
// and the chase runs there; otherwise it runs on the band in global memory.
template <typename T>
__global__ void __launch_bounds__(32 * Chase<T>::WARPS)
k_ts_chase(Batch bt, c2<T>* __restrict__ Bd, T* __restrict__ d_out, T* __restrict__ e2_out,
           int slots, int band_in_smem) {
  using C = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nwarps = blockDim.x >> 5;
  WarpScratch<T>* wsc = reinterpret_cast<WarpScratch<T>*>(smem_raw);
  C* sv = reinterpret_cast<C*>(wsc + nwarps);                   // [slots][BW]
  T* stau = reinterpret_cast<T*>(sv + (size_t)slots * BW);      // [slots]
  const int b = blockIdx.x;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  C* gband = Bd + (size_t)b * ND * nm;
  C* band = gband;
  if (band_in_smem) {
    const size_t head = sizeof(WarpScratch<T>) * nwarps + (sizeof(C) * BW + sizeof(T)) * (size_t)slots;
    band = reinterpret_cast<C*>(smem_raw + ((head + 255) & ~size_t(255)));
    for (int idx = threadIdx.x; idx < ND * nm; idx += blockDim.x) band[idx] = gband[idx];
    __syncthreads();
  }
  const Band<T> bd{band, nm};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpScratch<T>* ws = wsc + warp;
  if (n >= 3) {
    const int T_total = 2 * (n - 3) + 1;
    for (int tstep = 0; tstep < T_total; ++tstep) {
      const int ihi = min(tstep / 2, n - 3);
      for (int i = ihi - warp; i >= 0; i -= nwarps) {
        const int k = tstep - 2 * i;
        const int nsteps = (n - 2 - i) / BW + 1;   // step k while row i + 1 + k BW exists
        if (k >= nsteps) break;                    // older sweeps are done too
        const int slot = i % slots;
        if (k == 0) {
          // annihilate column i below the subdiagonal within the band
          const int L = min(BW, n - 1 - i);
          const C x = lane < L ? bd.get(i + 1 + lane, i) : mk<T>(T(0), T(0));
          C drow[BW];
          load_block<T>(bd, i + 1, i + 1, L, L, drow);
          T tau;
          C v, beta;
          const bool tr = warp_reflector<T>(x, L, tau, v, beta);
          if (tr) {
            if (lane < L) bd.set(i + 1 + lane, i, lane == 0 ? beta : mk<T>(T(0), T(0)));
            if (lane < BW) ws->v[lane] = lane < L ? v : mk<T>(T(0), T(0));
            __syncwarp();
            warp_two_sided<T>(bd, i + 1, L, tau, v, ws, drow);
          }
          if (lane < BW) sv[slot * BW + lane] = (tr && lane < L) ? v : mk<T>(T(0), T(0));
          if (lane == 0) stau[slot] = tau;
        } else {
          const int j0 = i + 1 + (k - 1) * BW;
          const int Lp = min(BW, n - j0);
          const int r0 = j0 + BW;
          const int Lr = min(BW, n - r0);
          const T tprev = stau[slot];
          if (lane < BW) ws->vp[lane] = sv[slot * BW + lane];
          // E = A(r0.., j0..) and D = A(r0.., r0..), both loaded up front: lane l holds row l
          C e[BW], drow[BW];
          load_block<T>(bd, r0, j0, Lr, Lp, e);
          load_block<T>(bd, r0, r0, Lr, Lr, drow);
          __syncwarp();
          if (tprev != T(0)) {
            // E <- E H_prev
            C u = mk<T>(T(0), T(0));
#pragma unroll
            for (int c = 0; c < BW; ++c) u = cadd<T>(u, cmul<T>(e[c], ws->vp[c]));
            u = cscale<T>(u, tprev);
#pragma unroll
            for (int c = 0; c < BW; ++c) e[c] = csub<T>(e[c], cmulc<T>(u, ws->vp[c]));
          }
          // new reflector from E's first column
          T tau;
          C v, beta;
          const bool tr = warp_reflector<T>(e[0], Lr, tau, v, beta);
          if (tr) {
            // E <- H E: column sums w_c = sum_l conj(v_l) e_l[c] through the scratch matrix
            if (lane < BW) {
#pragma unroll
              for (int c = 0; c < BW; ++c) ws->m[lane][c] = lane < Lr ? cjmul<T>(v, e[c]) : mk<T>(T(0), T(0));
            }
            __syncwarp();
            if (lane < BW) {
              C acc = mk<T>(T(0), T(0));
#pragma unroll
              for (int l = 0; l < BW; ++l) acc = cadd<T>(acc, ws->m[l][lane]);
              ws->w[lane] = acc;
            }
            __syncwarp();
#pragma unroll
            for (int c = 1; c < BW; ++c) e[c] = csub<T>(e[c], cscale<T>(cmul<T>(v, ws->w[c]), tau));
            e[0] = lane == 0 ? beta : mk<T>(T(0), T(0));
          }
          if (lane < Lr) {
#pragma unroll
            for (int c = 0; c < BW; ++c)
              if (c < Lp) bd.set(r0 + lane, j0 + c, e[c]);
          }
          if (tr) {
            if (lane < BW) ws->v[lane] = lane < Lr ? v : mk<T>(T(0), T(0));
            __syncwarp();
            warp_two_sided<T>(bd, r0, Lr, tau, v, ws, drow);
          }
          if (lane < BW) sv[slot * BW + lane] = (tr && lane < Lr) ? v : mk<T>(T(0), T(0));
          if (lane == 0) stau[slot] = tau;
        }
        __syncwarp();
      }
      __syncthreads();
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    d_out[(size_t)b * nm + c] = bd.get(c, c).x;
    if (c < n - 1) e2_out[(size_t)b * nm + c] = cabs2<T>(bd.get(c + 1, c));
  }
}

// Dataflow chase on a cluster of CS CTAs (CS = 1: one CTA), owner
// computes.  CTA q holds the band columns [q CW, (q+1) CW) (CW a power of
// two) and runs every step whose anchor column (i for step 0 of sweep i,
// i + 1 + (k-1) BW for step k >= 1) it holds: a step touches only columns
// [anchor, anchor + 2 BW), so all but the steps within 2 BW of the right
// edge work on local shared memory.  Warp w of every CTA runs the sweeps
// i = w (mod NW) in order.  Instead of a barrier per time step, step k of
// sweep i starts once sweep i-1 has completed min(k+2, its steps) (the
// steps whose entries it shares; later steps of earlier sweeps touch only
// entries further down the band) and, at its first step in a CTA, once the
// CTA on the left has finished step k-1 and left its reflector in this
// CTA's mailbox.  Completion counts, tagged with the sweep (i * 1024 + steps)
// in a ring of NSL slots, are published with release stores at cluster
// scope to the owning CTA and both neighbours, which hold every step that
// waits on them; every wait is bounded and sets the error flag when it
// gives up.
template <bool CL>
__device__ __forceinline__ void st_release(int* p, int v) {
  if constexpr (CL) asm volatile("st.release.cluster.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
  else asm volatile("st.release.cta.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
template <bool CL>
__device__ __forceinline__ void st_relaxed(int* p, int v) {
  if constexpr (CL) asm volatile("st.relaxed.cluster.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
  else asm volatile("st.relaxed.cta.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
template <bool CL>
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  if constexpr (CL) asm volatile("ld.acquire.cluster.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  else asm volatile("ld.acquire.cta.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
template <bool CL>
__device__ __forceinline__ void fence_acq_rel() {
  if constexpr (CL) asm volatile("fence.acq_rel.cluster;" ::: "memory");
  else asm volatile("fence.acq_rel.cta;" ::: "memory");
}

// A CTA's band columns are stored diagonal-major with the diagonal stride
// padded to 2^cwl + kBandPad entries.  Without the pad (a power-of-two stride)
// the 16 rows of a block, which lie on 16 consecutive diagonals, fall into one
// shared-memory bank: every block load and store was a 16-way conflict.  With
// a stride of 3 (mod 16) complex entries the rows of a block below the
// diagonal (stride +S per row) are conflict-free and the mirrored entries
// above it (stride 1 - S per row) at most 2-way.
constexpr int kBandPad = 3;
__host__ __device__ constexpr int band_stride(int cwl) { return (1 << cwl) + kBandPad; }

// CL = false: the whole band is in this CTA (no distributed addressing).
template <typename T, bool CL>
struct DBand {
  c2<T>* local;   // this CTA's band storage [ND][cw]
  int cwl;        // log2 of the columns per CTA
  int rank;
  __device__ __forceinline__ c2<T>* addr(int d, int c) const {
    if constexpr (!CL) {
      return local + (size_t)d * band_stride(cwl) + c;
    } else {
      const int o = c >> cwl;
      c2<T>* p = local + (size_t)d * band_stride(cwl) + (c & ((1 << cwl) - 1));
      return o == rank ? p : cg::this_cluster().map_shared_rank(p, o);
    }
  }
  __device__ __forceinline__ c2<T> get(int r, int c) const {
    return r >= c ? *addr(r - c, c) : conjg<T>(*addr(c - r, r));
  }
  __device__ __forceinline__ void set(int r, int c, c2<T> v) const { *addr(r - c, c) = v; }
};

constexpr int HB = BW / 2;   // columns per lane

template <typename T>
struct DScratch {
  c2<T> v[BW], w[BW], vp[BW];
  c2<T> m[BW][BW + 1];
  T tau_prev;
};

// Load row (r0 + l) columns c0 + h*HB + q of a block (Lr rows, Lc columns).
template <typename T, typename BandT>
__device__ __forceinline__ void dload(const BandT& bd, int r0, int c0, int Lr, int Lc, c2<T>* out) {
  const int l = threadIdx.x & 15, h = (threadIdx.x >> 4) & 1;
#pragma unroll
  for (int q = 0; q < HB; ++q) {
    const int c = h * HB + q;
    out[q] = (l < Lr && c < Lc) ? bd.get(r0 + l, c0 + c) : mk<T>(T(0), T(0));
  }
}

// Reflector from x (lanes l < L of the first half hold x_l; both halves
// return v_l of their row).
template <typename T>
__device__ __forceinline__ bool dreflector(c2<T> x, int L, T& tau, c2<T>& v, c2<T>& beta) {
  const int lane = threadIdx.x & 31, l = lane & 15;
  T rest = (lane < 16 && l >= 1 && l < L) ? cabs2<T>(x) : T(0);
  rest = warp_sum<T>(rest);
  const c2<T> alpha = shfl_c<T>(x, 0);
  const c2<T> xl = shfl_c<T>(x, l);
  tau = T(0);
  v = xl;
  beta = alpha;
  if (!(rest > tiny_rest<T>())) return false;
  c2<T> ph;
  const T aa = cabs_phase<T>(alpha, ph), sigma = sqrt(cabs2<T>(alpha) + rest);
  tau = T(1) / (sigma * (sigma + aa));
  if (l == 0) v = cadd<T>(alpha, cscale<T>(ph, sigma));
  beta = cscale<T>(ph, -sigma);
  return true;
}

// D <- H D H on A(r0.., r0..) (L rows), lower triangle stored.  ws->v holds v.
template <typename T, typename BandT>
__device__ __forceinline__ void dtwo_sided(const BandT& bd, int r0, int L, T tau, c2<T> v, DScratch<T>* ws,
                                           const c2<T>* dr) {
  using C = c2<T>;
  const int lane = threadIdx.x & 31, l = lane & 15, h = lane >> 4;
  C p = mk<T>(T(0), T(0));
#pragma unroll
  for (int q = 0; q < HB; ++q) p = cadd<T>(p, cmul<T>(dr[q], ws->v[h * HB + q]));
  p.x += __shfl_xor_sync(0xffffffffu, p.x, 16);
  p.y += __shfl_xor_sync(0xffffffffu, p.y, 16);
  p = cscale<T>(p, tau);
  const T kp = (h == 0 && l < L) ? (v.x * p.x + v.y * p.y) : T(0);
  const T K = T(0.5) * tau * warp_sum<T>(kp);
  const C w = csub<T>(p, cscale<T>(v, K));
  if (h == 0) ws->w[l] = l < L ? w : mk<T>(T(0), T(0));
  __syncwarp();
  if (l < L) {
#pragma unroll
    for (int q = 0; q < HB; ++q) {
      const int c = h * HB + q;
      if (c <= l) {
        C d = dr[q];
        d = csub<T>(d, cmulc<T>(v, ws->w[c]));
        d = csub<T>(d, cmulc<T>(w, ws->v[c]));
        if (c == l) d.y = T(0);
        bd.set(r0 + l, r0 + c, d);
      }
    }
  }
  __syncwarp();
}

// Columns [lo, lo + 2^cwl) of the band, all in this CTA.
template <typename T>
struct LBand {
  c2<T>* local;
  int cwl;
  int lo;
  __device__ __forceinline__ c2<T>* addr(int d, int c) const { return local + (size_t)d * band_stride(cwl) + (c - lo); }
  __device__ __forceinline__ c2<T> get(int r, int c) const {
    return r >= c ? *addr(r - c, c) : conjg<T>(*addr(c - r, r));
  }
  __device__ __forceinline__ void set(int r, int c, c2<T> v) const { *addr(r - c, c) = v; }
};

// One step of the chase (k = 0: annihilate column i; k >= 1: apply the
// previous reflector to the bulge block, annihilate its first column, apply
// the new reflector two-sided to the next diagonal block).  The previous
// reflector and its tau are in ws on entry and are replaced on exit.
template <typename T, typename BandT>
__device__ __forceinline__ void chase_step(const BandT& bd, int n, int i, int k, DScratch<T>* ws) {
  using C = c2<T>;
  const int lane = threadIdx.x & 31, l = lane & 15, h = lane >> 4;
  if (k == 0) {
    const int L = min(BW, n - 1 - i);
    const C x = (h == 0 && l < L) ? bd.get(i + 1 + l, i) : mk<T>(T(0), T(0));
    C dr[HB];
    dload<T>(bd, i + 1, i + 1, L, L, dr);
    T tau;
    C v, beta;
    const bool tr = dreflector<T>(x, L, tau, v, beta);
    if (tr) {
      if (h == 0 && l < L) bd.set(i + 1 + l, i, l == 0 ? beta : mk<T>(T(0), T(0)));
      if (h == 0) ws->v[l] = l < L ? v : mk<T>(T(0), T(0));
      __syncwarp();
      dtwo_sided<T>(bd, i + 1, L, tau, v, ws, dr);
    }
    if (h == 0) ws->vp[l] = (tr && l < L) ? v : mk<T>(T(0), T(0));
    if (lane == 0) ws->tau_prev = tau;
    return;
  }
  const int j0 = i + 1 + (k - 1) * BW;
  const int Lp = min(BW, n - j0);
  const int r0 = j0 + BW;
  const int Lr = min(BW, n - r0);
  C e[HB], dr[HB];
  dload<T>(bd, r0, j0, Lr, Lp, e);
  dload<T>(bd, r0, r0, Lr, Lr, dr);
  __syncwarp();
  const T tprev = ws->tau_prev;
  if (tprev != T(0)) {
    C u = mk<T>(T(0), T(0));
#pragma unroll
    for (int q = 0; q < HB; ++q) u = cadd<T>(u, cmul<T>(e[q], ws->vp[h * HB + q]));
    u.x += __shfl_xor_sync(0xffffffffu, u.x, 16);
    u.y += __shfl_xor_sync(0xffffffffu, u.y, 16);
    u = cscale<T>(u, tprev);
#pragma unroll
    for (int q = 0; q < HB; ++q) e[q] = csub<T>(e[q], cmulc<T>(u, ws->vp[h * HB + q]));
  }
  // reflector from E's first column (held by lanes of the first half, q = 0)
  T tau;
  C v, beta;
  const bool tr = dreflector<T>(e[0], Lr, tau, v, beta);
  if (tr) {
    // E <- H E, column sums through the scratch matrix
#pragma unroll
    for (int q = 0; q < HB; ++q) ws->m[l][h * HB + q] = l < Lr ? cjmul<T>(v, e[q]) : mk<T>(T(0), T(0));
    __syncwarp();
    {
      const int c = l;   // lanes l and l + 16 sum half of the rows of column l each
      C acc = mk<T>(T(0), T(0));
#pragma unroll
      for (int rr = 0; rr < HB; ++rr) acc = cadd<T>(acc, ws->m[h * HB + rr][c]);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 16);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 16);
      __syncwarp();
      if (h == 0) ws->w[c] = acc;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < HB; ++q) e[q] = csub<T>(e[q], cscale<T>(cmul<T>(v, ws->w[h * HB + q]), tau));
    if (h == 0) e[0] = l == 0 ? beta : mk<T>(T(0), T(0));
  }
  if (l < Lr) {
#pragma unroll
    for (int q = 0; q < HB; ++q)
      if (h * HB + q < Lp) bd.set(r0 + l, j0 + h * HB + q, e[q]);
  }
  if (tr) {
    if (h == 0) ws->v[l] = l < Lr ? v : mk<T>(T(0), T(0));
    __syncwarp();
    dtwo_sided<T>(bd, r0, Lr, tau, v, ws, dr);
  }
  __syncwarp();
  if (h == 0) ws->vp[l] = (tr && l < Lr) ? v : mk<T>(T(0), T(0));
  if (lane == 0) ws->tau_prev = tau;
}

// Reflector hand-over slot of a sweep entering a CTA.
template <typename T>
struct Mailbox {
  c2<T> v[BW];
  T tau;
};
constexpr int NMB = 16;   // mailbox ring (a slot is reused only after its sweep moved two CTAs on)

__host__ __device__ constexpr int chase_ring(int cw) {
  // progress ring: a slot is reused once its sweep is three CTAs ahead
  int r = 64;
  while (r < 4 * cw / (BW - 1) + 8) r *= 2;
  return r;
}

template <typename T, bool CL>
__global__ void __launch_bounds__(32 * Chase<T>::WARPS)
k_ts_chase_flow(Batch bt, const c2<T>* __restrict__ Bd, T* __restrict__ d_out, T* __restrict__ e2_out, int cwl,
                int* __restrict__ err) {
  using C = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int CSZ = CL ? (int)cg::this_cluster().num_blocks() : 1;
  const int rank = CL ? (int)cg::this_cluster().block_rank() : 0;
  const int nwarps = blockDim.x >> 5;
  const int cw = 1 << cwl;
  const int NSL = chase_ring(cw);
  const int b = blockIdx.x / CSZ;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int lo = rank * cw, hi = lo + cw;
  DScratch<T>* wsc = reinterpret_cast<DScratch<T>*>(smem_raw);
  Mailbox<T>* mbox = reinterpret_cast<Mailbox<T>*>(wsc + nwarps);   // [NMB]
  int* prog = reinterpret_cast<int*>(mbox + NMB);                  // [NSL]
  const size_t head = sizeof(DScratch<T>) * nwarps + sizeof(Mailbox<T>) * NMB + sizeof(int) * (size_t)NSL;
  C* local = reinterpret_cast<C*>(smem_raw + ((head + 255) & ~size_t(255)));
  const C* gband = Bd + (size_t)b * ND * nm;
  for (int idx = threadIdx.x; idx < ND * cw; idx += blockDim.x) {
    const int d = idx >> cwl, c = lo + (idx & (cw - 1));
    local[(size_t)d * band_stride(cwl) + (idx & (cw - 1))] = c < nm ? gband[(size_t)d * nm + c] : mk<T>(T(0), T(0));
  }
  for (int idx = threadIdx.x; idx < NSL; idx += blockDim.x) prog[idx] = 0;
  if constexpr (CL) cg::this_cluster().sync(); else __syncthreads();
  const DBand<T, CL> bd{local, cwl, rank};
  const LBand<T> lb{local, cwl, lo};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, l = lane & 15, h = lane >> 4;
  DScratch<T>* ws = wsc + warp;
  // Bounded wait until the local counter slot reaches `want`.  Every lane
  // polls with its own acquire load (one broadcast read per poll), so each
  // lane is ordered after the release it observed; the error flag in global
  // memory is read only every 1024 polls.
  auto wait_for = [&](int slot, int want) -> bool {
    bool ok = true;
    int spins = 0;
    while (ld_acquire<CL>(prog + slot) < want) {
      ++spins;
      if ((spins & 1023) == 0 && (spins >= (1 << 25) || *(volatile int*)err)) {
        atomicExch(err, 1);
        ok = false;
        break;
      }
      if (spins > 256) __nanosleep(20);
    }
    return __all_sync(0xffffffffu, ok);
  };
  bool ok = true;
  for (int i = warp; ok && i <= n - 3 && i < hi; i += nwarps) {
    const int nsteps = (n - 2 - i) / BW + 1;
    // steps of sweep i anchored in [lo, hi): k in [klo, khi)
    const int klo = i >= lo ? 0 : (lo - i - 1 + BW - 1) / BW + 1;
    const int khi = min(nsteps, (hi - i - 1 + BW - 1) / BW + 1);
    if (klo >= khi) continue;
    const int dep_steps = i > 0 ? (n - 1 - i) / BW + 1 : 0;   // steps of sweep i-1
    for (int k = klo; k < khi; ++k) {
      if (k == klo && klo > 0) {
        // hand-over: step k-1 done in the CTA on the left, reflector in the mailbox
        ok = wait_for(i % NSL, i * 1024 + k);
        if (!ok) break;
        const Mailbox<T>* mb = mbox + (i % NMB);
        if (h == 0) ws->vp[l] = mb->v[l];
        if (lane == 0) ws->tau_prev = mb->tau;
        __syncwarp();
      }
      if (i > 0) {
        ok = wait_for((i - 1) % NSL, (i - 1) * 1024 + min(k + 2, dep_steps));
        if (!ok) break;
      }
      const int anchor = k == 0 ? i : i + 1 + (k - 1) * BW;
      if (!CL || anchor + 2 * BW <= hi) chase_step<T>(lb, n, i, k, ws);
      else chase_step<T>(bd, n, i, k, ws);
      const bool handover = CL && k == khi - 1 && k + 1 < nsteps;
      if (handover) {
        // the next step of this sweep runs in the CTA on the right
        Mailbox<T>* mb = mbox + (i % NMB);
        if constexpr (CL) mb = cg::this_cluster().map_shared_rank(mb, rank + 1);
        __syncwarp();
        if (h == 0) mb->v[l] = ws->vp[l];
        if (lane == 0) mb->tau = ws->tau_prev;
      }
      // Release: the warp barrier orders every lane's band (and mailbox)
      // writes before lane 0's fence, and the fence with the strong stores
      // after it forms one release pattern for the counter copies.  At a
      // hand-over the right copy is itself a release store, so the CTA that
      // continues the sweep also sees this CTA's earlier counter writes (its
      // own later writes to the same slots come after them).
      __syncwarp();
      if (lane == 0) {
        const int tagv = i * 1024 + k + 1;
        int* own = prog + (i % NSL);
        fence_acq_rel<CL>();
        if constexpr (CL) {
          if (rank > 0) st_relaxed<CL>(cg::this_cluster().map_shared_rank(own, rank - 1), tagv);
          st_relaxed<CL>(own, tagv);
          if (rank + 1 < CSZ) {
            int* right = cg::this_cluster().map_shared_rank(own, rank + 1);
            if (handover) st_release<CL>(right, tagv);
            else st_relaxed<CL>(right, tagv);
          }
        } else {
          st_relaxed<CL>(own, tagv);
        }
      }
    }
  }
  if constexpr (CL) cg::this_cluster().sync(); else __syncthreads();
  for (int c_ = threadIdx.x; c_ < cw; c_ += blockDim.x) {
    const int c = lo + c_;
    if (c < n) {
      d_out[(size_t)b * nm + c] = bd.get(c, c).x;
      if (c < n - 1) e2_out[(size_t)b * nm + c] = cabs2<T>(bd.get(c + 1, c));
    }
  }
  if constexpr (CL) cg::this_cluster().sync();   // no CTA leaves while others may still read its shared memory
}

// ------------------------------------------------------ warp-pair chase --
// The clustered dataflow chase with two warps per sweep.  A step's work
// splits at its reflector: the E warp waits for the step's inputs, applies
// the previous reflector to the block below the previous diagonal block (or,
// at step 0, takes column i), forms the new reflector and applies it to that
// block from the left; the D warp loads the next diagonal block meanwhile and,
// once the reflector is in shared memory, applies it two-sided.  The two
// halves write disjoint entries (E: columns [j0, j0 + BW) below row
// j0 + BW - 1; D: rows and columns from j0 + BW), and the next step of the
// sweep touches neither half's block except through the reflector, so they
// run side by side.  Both warps pass the same three pair barriers per step
// (inputs ready / reflector ready / step done) in the same order on every
// path; only the E warp polls (bounded) and hands its outcome to the D warp
// through shared memory before the first barrier, so a wait that gives up
// ends both warps' loops at the same point.
__device__ __forceinline__ void pair_bar(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// E half of step k of sweep i; wsd: the D warp's scratch, which receives the
// reflector (v in wsd->v, tau in wsd->tau_prev) before the reflector barrier.
template <typename T, typename BandT>
__device__ __forceinline__ void pair_step_e(const BandT& bd, int n, int i, int k, DScratch<T>* ws, DScratch<T>* wsd,
                                            int bar) {
  using C = c2<T>;
  const int lane = threadIdx.x & 31, l = lane & 15, h = lane >> 4;
  if (k == 0) {
    const int L = min(BW, n - 1 - i);
    const C x = (h == 0 && l < L) ? bd.get(i + 1 + l, i) : mk<T>(T(0), T(0));
    T tau;
    C v, beta;
    const bool tr = dreflector<T>(x, L, tau, v, beta);
    if (tr && h == 0 && l < L) bd.set(i + 1 + l, i, l == 0 ? beta : mk<T>(T(0), T(0)));
    if (h == 0) wsd->v[l] = (tr && l < L) ? v : mk<T>(T(0), T(0));
    if (lane == 0) wsd->tau_prev = tr ? tau : T(0);
    pair_bar(bar);   // reflector ready
    if (h == 0) ws->vp[l] = (tr && l < L) ? v : mk<T>(T(0), T(0));
    if (lane == 0) ws->tau_prev = tr ? tau : T(0);
    return;
  }
  const int j0 = i + 1 + (k - 1) * BW;
  const int Lp = min(BW, n - j0);
  const int r0 = j0 + BW;
  const int Lr = min(BW, n - r0);
  C e[HB];
  dload<T>(bd, r0, j0, Lr, Lp, e);
  __syncwarp();
  const T tprev = ws->tau_prev;
  if (tprev != T(0)) {
    C u = mk<T>(T(0), T(0));
#pragma unroll
    for (int q = 0; q < HB; ++q) u = cadd<T>(u, cmul<T>(e[q], ws->vp[h * HB + q]));
    u.x += __shfl_xor_sync(0xffffffffu, u.x, 16);
    u.y += __shfl_xor_sync(0xffffffffu, u.y, 16);
    u = cscale<T>(u, tprev);
#pragma unroll
    for (int q = 0; q < HB; ++q) e[q] = csub<T>(e[q], cmulc<T>(u, ws->vp[h * HB + q]));
  }
  T tau;
  C v, beta;
  const bool tr = dreflector<T>(e[0], Lr, tau, v, beta);
  if (h == 0) wsd->v[l] = (tr && l < Lr) ? v : mk<T>(T(0), T(0));
  if (lane == 0) wsd->tau_prev = tr ? tau : T(0);
  pair_bar(bar);   // reflector ready
  if (tr) {
#pragma unroll
    for (int q = 0; q < HB; ++q) ws->m[l][h * HB + q] = l < Lr ? cjmul<T>(v, e[q]) : mk<T>(T(0), T(0));
    __syncwarp();
    {
      const int c = l;
      C acc = mk<T>(T(0), T(0));
#pragma unroll
      for (int rr = 0; rr < HB; ++rr) acc = cadd<T>(acc, ws->m[h * HB + rr][c]);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 16);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 16);
      __syncwarp();
      if (h == 0) ws->w[c] = acc;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < HB; ++q) e[q] = csub<T>(e[q], cscale<T>(cmul<T>(v, ws->w[h * HB + q]), tau));
    if (h == 0) e[0] = l == 0 ? beta : mk<T>(T(0), T(0));
  }
  if (l < Lr) {
#pragma unroll
    for (int q = 0; q < HB; ++q)
      if (h * HB + q < Lp) bd.set(r0 + l, j0 + h * HB + q, e[q]);
  }
  __syncwarp();
  if (h == 0) ws->vp[l] = (tr && l < Lr) ? v : mk<T>(T(0), T(0));
  if (lane == 0) ws->tau_prev = tr ? tau : T(0);
}

// D half of step k of sweep i: the two-sided update of the diagonal block
// with the reflector the E warp left in ws (this warp's scratch).
template <typename T, typename BandT>
__device__ __forceinline__ void pair_step_d(const BandT& bd, int n, int i, int k, DScratch<T>* ws, int bar) {
  using C = c2<T>;
  const int l = threadIdx.x & 15;
  const int r0 = k == 0 ? i + 1 : i + 1 + k * BW;
  const int L = k == 0 ? min(BW, n - 1 - i) : min(BW, n - r0);
  C dr[HB];
  dload<T>(bd, r0, r0, L, L, dr);
  pair_bar(bar);   // reflector ready
  const T tau = ws->tau_prev;
  if (tau != T(0)) dtwo_sided<T>(bd, r0, L, tau, ws->v[l], ws, dr);
}

template <typename T>
__global__ void __launch_bounds__(32 * Chase<T>::WARPS)
k_ts_chase_pair(Batch bt, const c2<T>* __restrict__ Bd, T* __restrict__ d_out, T* __restrict__ e2_out, int cwl,
                int* __restrict__ err) {
  using C = c2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int CSZ = (int)cg::this_cluster().num_blocks();
  const int rank = (int)cg::this_cluster().block_rank();
  const int nwarps = blockDim.x >> 5, npairs = nwarps >> 1;
  const int cw = 1 << cwl;
  const int NSL = chase_ring(cw);
  const int b = blockIdx.x / CSZ;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int lo = rank * cw, hi = lo + cw;
  DScratch<T>* wsc = reinterpret_cast<DScratch<T>*>(smem_raw);
  Mailbox<T>* mbox = reinterpret_cast<Mailbox<T>*>(wsc + nwarps);   // [NMB]
  int* prog = reinterpret_cast<int*>(mbox + NMB);                  // [NSL]
  int* pok = prog + NSL;                                           // [16] per pair: inputs ready
  const size_t head =
      sizeof(DScratch<T>) * nwarps + sizeof(Mailbox<T>) * NMB + sizeof(int) * ((size_t)NSL + 16);
  C* local = reinterpret_cast<C*>(smem_raw + ((head + 255) & ~size_t(255)));
  const C* gband = Bd + (size_t)b * ND * nm;
  for (int idx = threadIdx.x; idx < ND * cw; idx += blockDim.x) {
    const int d = idx >> cwl, c = lo + (idx & (cw - 1));
    local[(size_t)d * band_stride(cwl) + (idx & (cw - 1))] = c < nm ? gband[(size_t)d * nm + c] : mk<T>(T(0), T(0));
  }
  for (int idx = threadIdx.x; idx < NSL; idx += blockDim.x) prog[idx] = 0;
  cg::this_cluster().sync();
  const DBand<T, true> bd{local, cwl, rank};
  const LBand<T> lb{local, cwl, lo};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, l = lane & 15, h = lane >> 4;
  const int pair = warp >> 1, role = warp & 1;   // role 0: E half, 1: D half
  const int bar = 1 + pair;                      // named barrier of the pair (0 is the CTA's)
  DScratch<T>* ws = wsc + warp;
  DScratch<T>* wsd = wsc + (warp | 1);           // the pair's D scratch (receives the reflector)
  auto wait_for = [&](int slot, int want) -> bool {
    bool ok = true;
    int spins = 0;
    while (ld_acquire<true>(prog + slot) < want) {
      ++spins;
      if ((spins & 1023) == 0 && (spins >= (1 << 25) || *(volatile int*)err)) {
        atomicExch(err, 1);
        ok = false;
        break;
      }
      if (spins > 256) __nanosleep(20);
    }
    return __all_sync(0xffffffffu, ok);
  };
  bool ok = true;
  for (int i = pair; ok && i <= n - 3 && i < hi; i += npairs) {
    const int nsteps = (n - 2 - i) / BW + 1;
    const int klo = i >= lo ? 0 : (lo - i - 1 + BW - 1) / BW + 1;
    const int khi = min(nsteps, (hi - i - 1 + BW - 1) / BW + 1);
    if (klo >= khi) continue;
    const int dep_steps = i > 0 ? (n - 1 - i) / BW + 1 : 0;
    for (int k = klo; k < khi; ++k) {
      // inputs: the E warp waits (bounded) and hands the outcome over
      if (role == 0) {
        bool in_ok = true;
        if (k == klo && klo > 0) {
          in_ok = wait_for(i % NSL, i * 1024 + k);
          if (in_ok) {
            const Mailbox<T>* mb = mbox + (i % NMB);
            if (h == 0) ws->vp[l] = mb->v[l];
            if (lane == 0) ws->tau_prev = mb->tau;
          }
        }
        if (in_ok && i > 0) in_ok = wait_for((i - 1) % NSL, (i - 1) * 1024 + min(k + 2, dep_steps));
        if (lane == 0) pok[pair] = in_ok ? 1 : 0;
      }
      pair_bar(bar);   // inputs ready
      ok = pok[pair] != 0;
      if (!ok) break;
      const int anchor = k == 0 ? i : i + 1 + (k - 1) * BW;
      const bool here = anchor + 2 * BW <= hi;
      if (role == 0) {
        if (here) pair_step_e<T>(lb, n, i, k, ws, wsd, bar);
        else pair_step_e<T>(bd, n, i, k, ws, wsd, bar);
      } else {
        if (here) pair_step_d<T>(lb, n, i, k, ws, bar);
        else pair_step_d<T>(bd, n, i, k, ws, bar);
      }
      const bool handover = k == khi - 1 && k + 1 < nsteps;
      if (role == 0 && handover) {
        Mailbox<T>* mb = cg::this_cluster().map_shared_rank(mbox + (i % NMB), rank + 1);
        __syncwarp();
        if (h == 0) mb->v[l] = ws->vp[l];
        if (lane == 0) mb->tau = ws->tau_prev;
      }
      pair_bar(bar);   // step done (both halves' writes before the release below)
      if (role == 0 && lane == 0) {
        const int tagv = i * 1024 + k + 1;
        int* own = prog + (i % NSL);
        fence_acq_rel<true>();
        if (rank > 0) st_relaxed<true>(cg::this_cluster().map_shared_rank(own, rank - 1), tagv);
        st_relaxed<true>(own, tagv);
        if (rank + 1 < CSZ) {
          int* right = cg::this_cluster().map_shared_rank(own, rank + 1);
          if (handover) st_release<true>(right, tagv);
          else st_relaxed<true>(right, tagv);
        }
      }
    }
  }
  cg::this_cluster().sync();
  for (int c_ = threadIdx.x; c_ < cw; c_ += blockDim.x) {
    const int c = lo + c_;
    if (c < n) {
      d_out[(size_t)b * nm + c] = bd.get(c, c).x;
      if (c < n - 1) e2_out[(size_t)b * nm + c] = cabs2<T>(bd.get(c + 1, c));
    }
  }
  cg::this_cluster().sync();   // no CTA leaves while others may still read its shared memory
}

template <typename T>
int chase_plan_t(int nm, int64_t batch, int sms, int max_cluster, ChasePlan& p, bool allow_pair) {
  using C = c2<T>;
  p = ChasePlan{};
  // barrier kernel: one warp per concurrently active sweep (at most n/(2 BW) + 2)
  const int active = nm / (2 * BW) + 2;
  p.threads = 32 * std::min(Chase<T>::WARPS, std::max(2, active));
  p.slots = 2 * active + 2;
  const size_t head_bytes = sizeof(WarpScratch<T>) * (p.threads / 32) + (sizeof(C) * BW + sizeof(T)) * (size_t)p.slots;
  const size_t slot_bytes = (head_bytes + 255) & ~size_t(255);
  const size_t band_bytes = sizeof(C) * (size_t)ND * nm;
  p.band_in_smem = slot_bytes + band_bytes <= 200 * 1024 ? 1 : 0;
  p.smem = slot_bytes + (p.band_in_smem ? band_bytes : 0) + 64;
  IDOS_CUDA_TRY(cudaFuncSetAttribute(k_ts_chase<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
  // dataflow kernel: the smallest cluster (1 .. 16 CTAs, power-of-two column
  // split) whose shared memory holds the band, grown (while the batch leaves
  // SMs idle) until its warps cover the active sweeps; a CTA of the cluster
  // sees at most CW / (2 BW) + 2 active sweeps at a time, and fewer warps
  // than active sweeps only serialise sweeps.
  auto cfg = [&](int q, int& w, int& cwl, size_t& need) {
    cwl = 0;
    while ((1 << cwl) * q < nm) ++cwl;
    w = std::min(Chase<T>::WARPS, std::max(2, std::min(active, (1 << cwl) / (2 * BW) + 2)));
    const size_t hb = (sizeof(DScratch<T>) * w + sizeof(Mailbox<T>) * NMB + sizeof(int) * (size_t)chase_ring(1 << cwl) +
                       255) & ~size_t(255);
    need = hb + sizeof(C) * (size_t)ND * band_stride(cwl) + 64;
    return need <= 200 * 1024;
  };
  auto covered = [&](int w, int cwl) { return w >= std::min(active, (1 << cwl) / (2 * BW) + 2); };
  for (int q = 1; q <= std::min(16, max_cluster); q *= 2) {
    int w, cwl;
    size_t need;
    if (!cfg(q, w, cwl, need)) continue;
    if (p.csz == 0 || (!covered(p.cwarps, p.ccwl) && batch * q <= sms)) {
      p.csz = q;
      p.cwarps = w;
      p.ccwl = cwl;
      p.csmem = need;
    } else {
      break;
    }
  }
  // Two warps per sweep when the cluster splits the band into CTAs narrow
  // enough that the pairs still cover a CTA's active sweeps (a pair leaves a
  // sweep after cw / BW steps, the next sweep starts 2 steps later).
  if (p.csz > 1 && allow_pair) {
    const int cw = 1 << p.ccwl;
    const int pairs = std::min(Chase<T>::WARPS / 2, cw / (2 * BW) + 2);
    if (pairs >= cw / (2 * BW) && pairs >= 1) {
      const size_t hb = (sizeof(DScratch<T>) * 2 * pairs + sizeof(Mailbox<T>) * NMB +
                         sizeof(int) * ((size_t)chase_ring(cw) + 16) + 255) & ~size_t(255);
      const size_t need = hb + sizeof(C) * (size_t)ND * band_stride(p.ccwl) + 64;
      if (need <= 200 * 1024) {
        p.pair = 1;
        p.cwarps = 2 * pairs;
        p.csmem = need;
        IDOS_CUDA_TRY(cudaFuncSetAttribute(k_ts_chase_pair<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.csmem));
        if (p.csz > 8)
          IDOS_CUDA_TRY(cudaFuncSetAttribute(k_ts_chase_pair<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        return IDOS_OK;
      }
    }
  }
  if (p.csz == 1) {
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_ts_chase_flow<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.csmem));
  } else if (p.csz > 1) {
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_ts_chase_flow<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.csmem));
    if (p.csz > 8)
      IDOS_CUDA_TRY(cudaFuncSetAttribute(k_ts_chase_flow<T, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  }
  return IDOS_OK;
}

template <typename T>
int chase_run_t(const ChasePlan& p, const Batch& bt, const c2<T>* A, c2<T>* Bd, T* d, T* e2, int* err, cudaStream_t s) {
  using C = c2<T>;
  const unsigned nb = (unsigned)bt.B;
  k_ts_to_band<T><<<dim3(64, nb), 256, 0, s>>>(bt, A, Bd);
  if (p.csz == 1) {
    k_ts_chase_flow<T, false><<<nb, 32 * p.cwarps, p.csmem, s>>>(bt, (const C*)Bd, d, e2, p.ccwl, err);
  } else if (p.csz > 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nb * (unsigned)p.csz);
    cfg.blockDim = dim3(32 * p.cwarps);
    cfg.dynamicSmemBytes = p.csmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.csz;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (p.pair)
      IDOS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_ts_chase_pair<T>, bt, (const C*)Bd, d, e2, p.ccwl, err));
    else
      IDOS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_ts_chase_flow<T, true>, bt, (const C*)Bd, d, e2, p.ccwl, err));
  } else {
    k_ts_chase<T><<<nb, p.threads, p.smem, s>>>(bt, Bd, d, e2, p.slots, p.band_in_smem);
  }
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

}  // namespace

template <typename T>
int chase_plan(int n_max, int64_t batch, int sms, int max_cluster, ChasePlan& p, bool allow_pair) {
  return chase_plan_t<T>(n_max, batch, sms, max_cluster, p, allow_pair);
}
template <typename T>
int chase_run(const ChasePlan& p, const Batch& bt, const c2<T>* A, c2<T>* Bd, T* d, T* e2, int* err, cudaStream_t s) {
  return chase_run_t<T>(p, bt, A, Bd, d, e2, err, s);
}
template int chase_plan<float>(int, int64_t, int, int, ChasePlan&, bool);
template int chase_plan<double>(int, int64_t, int, int, ChasePlan&, bool);
template int chase_run<float>(const ChasePlan&, const Batch&, const c2<float>*, c2<float>*, float*, float*, int*,
                              cudaStream_t);
template int chase_run<double>(const ChasePlan&, const Batch&, const c2<double>*, c2<double>*, double*, double*, int*,
                               cudaStream_t);

}  // namespace lg
}  // namespace idos
