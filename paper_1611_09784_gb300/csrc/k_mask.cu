// k_mask.cu - vacancy masks (Sec. 3.2), control-variate corner slicing
// (Sec. 3.3), compaction maps, and the dense H(k) export used for parity.
#include <cmath>

#include "graphene.cuh"
#include "internal.h"
#include "tmdc.cuh"

namespace idos {

// Site `site` of sample `sample` on `level` is removed iff word 0 of
// Philox4x64-10(counter = (site, sample, level, 0), key = (seed, 1)) is below
// floor(p 2^64); all_removed handles p = 1 (threshold 2^64).
// dyn (optional, device): [0] the seed, used in place of `seed`, and
// [1 + level] the first sample index, to which `first_sample` is then added
// as an offset (a replayed graph takes its per-call values from there).
__global__ void k_fine_masks(uint8_t* __restrict__ out, int n_sites, int64_t total, uint64_t seed,
                             int level, int64_t first_sample, uint64_t thr, int all_removed,
                             const uint64_t* __restrict__ dyn) {
  if (dyn) {
    seed = dyn[0];
    first_sample += (int64_t)dyn[1 + level];
  }
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / n_sites;
    const int site = (int)(idx - s * n_sites);
    const u64x4 r = philox4x64_10((uint64_t)site, (uint64_t)(first_sample + s), (uint64_t)level, 0ull,
                                  seed, kStreamVacancy);
    out[idx] = (all_removed || r.w[0] < thr) ? 1 : 0;
  }
}

int launch_fine_masks(uint8_t* out, int n_sites, int64_t count, uint64_t seed, int level,
                      int64_t first_sample, double p, cudaStream_t s, const uint64_t* dyn) {
  const int all_removed = p >= 1.0 ? 1 : 0;
  const uint64_t thr = all_removed ? 0ull : (uint64_t)std::ldexp(p, 64);
  const int64_t total = count * (int64_t)n_sites;
  if (total == 0) return IDOS_OK;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 152 * 32);
  ProfScope ps(KID_MASKS, s);
  k_fine_masks<<<(unsigned)blocks, threads, 0, s>>>(out, n_sites, total, seed, level, first_sample,
                                                   thr, all_removed, dyn);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

// Corner r = ri + 2 rj of a fine N x N cell: cells i in [ri h, (ri+1) h),
// j in [rj h, (rj+1) h), h = N/2; vacancy site `sub` (0 .. per-1) of local
// cell (i', j') is per (i' + h j') + sub.
__global__ void k_corner_masks(const uint8_t* __restrict__ fine, int N, int per, int64_t total,
                               uint8_t* __restrict__ out) {
  const int h = N / 2, nsc = per * h * h, nsf = per * N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t inst = idx / nsc;          // 4 s + r
    const int ml = (int)(idx - inst * nsc);
    const int64_t smp = inst >> 2;
    const int r = (int)(inst & 3), ri = r & 1, rj = r >> 1;
    const int sub = ml % per, cl = ml / per, il = cl % h, jl = cl / h;
    const int mf = per * ((il + ri * h) + N * (jl + rj * h)) + sub;
    out[idx] = fine[smp * nsf + mf];
  }
}

int launch_corner_masks(const uint8_t* fine, int N, int per, int64_t count, uint8_t* out, cudaStream_t s) {
  const int h = N / 2;
  const int64_t total = count * 4 * (int64_t)(per * h * h);
  if (total == 0) return IDOS_OK;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 152 * 32);
  ProfScope ps(KID_CORNERS, s);
  k_corner_masks<<<(unsigned)blocks, threads, 0, s>>>(fine, N, per, total, out);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

// TMDC-shaped model: orbital o = 11 c + q is removed iff q >= 5 (a pair
// orbital) and cell c's pair is removed.
__global__ void k_orbital_masks(const uint8_t* __restrict__ pairs, int nc, int64_t total, uint8_t* __restrict__ out) {
  const int no = kTmdcOrb * nc;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / no;
    const int o = (int)(idx - s * no);
    const int c = o / kTmdcOrb, q = o - c * kTmdcOrb;
    out[idx] = (q >= kTmdcM && pairs[s * nc + c]) ? 1 : 0;
  }
}

int launch_orbital_masks(const uint8_t* pairs, int N, int64_t count, uint8_t* out, cudaStream_t s) {
  const int64_t total = count * (int64_t)kTmdcOrb * N * N;
  if (total == 0) return IDOS_OK;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 152 * 32);
  ProfScope ps(KID_CORNERS, s);
  k_orbital_masks<<<(unsigned)blocks, threads, 0, s>>>(pairs, N * N, total, out);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

void tmdc_draw_params(uint64_t model_seed, double lo, double hi, double* out) {
  for (int i = 0; i < kTmdcParams; ++i) {
    const u64x4 r = philox4x64_10((uint64_t)i, 0ull, 0ull, 0ull, model_seed, kStreamParams);
    const double u = std::ldexp((double)(r.w[0] >> 11), -53);
    out[i] = lo + (hi - lo) * u;
  }
}

// One CTA per cell: ascending list of kept sites and the inverse map.
__global__ void k_cell_maps(const uint8_t* __restrict__ mask, int n_sites, int* __restrict__ n_act,
                            int* __restrict__ act, int* __restrict__ inv) {
  __shared__ int scan[1024];
  const int64_t cell = blockIdx.x;
  const uint8_t* mk = mask + cell * n_sites;
  const int nt = blockDim.x, t = threadIdx.x;
  const int per = (n_sites + nt - 1) / nt;
  const int lo = t * per, hi = min(n_sites, lo + per);
  int cnt = 0;
  for (int i = lo; i < hi; ++i) cnt += mk[i] ? 0 : 1;
  scan[t] = cnt;
  __syncthreads();
  // Hillis-Steele inclusive scan over the block
  for (int o = 1; o < nt; o <<= 1) {
    int v = (t >= o) ? scan[t - o] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  int pos = scan[t] - cnt;
  for (int i = lo; i < hi; ++i) {
    if (mk[i]) {
      inv[cell * n_sites + i] = -1;
    } else {
      inv[cell * n_sites + i] = pos;
      act[cell * n_sites + pos] = i;
      ++pos;
    }
  }
  if (t == nt - 1) n_act[cell] = scan[t];
}

int launch_cell_maps(CellSet& c, cudaStream_t s) {
  if (c.count == 0) return IDOS_OK;
  const int threads = c.n_sites >= 1024 ? 1024 : (c.n_sites >= 256 ? 256 : 32);
  ProfScope ps(KID_CELL_MAPS, s);
  k_cell_maps<<<(unsigned)c.count, threads, 0, s>>>(c.mask, c.n_sites, c.n_act, c.act, c.inv);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

// Dense H(k) of cell 0 in the full site basis (parity export): removed sites
// get zero rows/columns and `sentinel` on the diagonal.
__global__ void k_assemble_dense(const uint8_t* __restrict__ mask, int N, int K, int kidx, double t,
                                 double eps, double sentinel, double2* __restrict__ out) {
  const int n = 2 * N * N;
  __shared__ double2 ph[3];
  if (threadIdx.x < 3) ph[threadIdx.x] = graphene_phase(N, K, kidx, threadIdx.x);
  __syncthreads();
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double2* row = out + (int64_t)m * n;
    if (mask[m]) {
      row[m] = make_double2(row[m].x + sentinel, row[m].y);
      continue;
    }
    int nb[3];
    bool fromB;
    graphene_neighbours(N, m, nb, fromB);
    for (int b = 0; b < 3; ++b) {
      if (mask[nb[b]]) continue;
      const double2 p = ph[b];
      row[nb[b]].x += t * p.x;
      row[nb[b]].y += fromB ? -t * p.y : t * p.y;
    }
    row[m].x += eps;
  }
}

// TMDC-shaped model in the full orbital basis: rows built by tmdc_row (the
// function the large-path assembly uses), removed pairs' orbitals with zero
// rows and columns and `sentinel` on the diagonal.
__global__ void k_assemble_dense_tmdc(const uint8_t* __restrict__ pairs, int N, int K, int kidx,
                                      const double* __restrict__ P, double sentinel, double2* __restrict__ out) {
  const int n = kTmdcOrb * N * N;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    double2* row = out + (int64_t)o * n;
    const int c = o / kTmdcOrb, q = o % kTmdcOrb;
    if (q >= kTmdcM && pairs[c]) {
      row[o] = make_double2(sentinel, 0.0);
      continue;
    }
    tmdc_row(N, K, kidx, o, P, [&](int cell) { return pairs[cell] != 0; },
             [&](int o2, double2 v) {
               row[o2].x += v.x;
               row[o2].y += v.y;
             });
  }
}

int launch_assemble_dense(const SolveArgs& a, int k_index, double2* out, double sentinel) {
  const int N = a.cells->N, n = a.cells->n_sites;
  IDOS_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double2) * (size_t)n * n, a.stream));
  if (a.kind == IDOS_TMDC) {
    k_assemble_dense_tmdc<<<(n + 127) / 128, 128, 0, a.stream>>>(a.cells->vmask, N, a.Kside, k_index, a.tmdc_p,
                                                                 sentinel, out);
  } else {
    k_assemble_dense<<<(n + 127) / 128, 128, 0, a.stream>>>(a.cells->mask, N, a.Kside, k_index, a.t, a.eps,
                                                            sentinel, out);
  }
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

}  // namespace idos
