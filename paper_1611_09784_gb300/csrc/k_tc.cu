// k_tc.cu - the trailing update of stage 1 of the large-matrix reduction,
//   A22 <- A22 - (Y Z^H + Z Y^H)            (compact-WY two-sided update, Sec. 4.2's
//                                             dense eigensolver in two-stage form)
// on the 5th-generation tensor cores: operands staged in shared memory by TMA,
// one thread issuing tcgen05.mma, the float32 accumulator in tensor memory,
// read back with tcgen05.ld for the read-modify-write of A22.
//
// Real form.  With U = [Y | Z] and V = [Z | Y] (m x 2BW complex), C = U V^H.
// Real operand rows A'[r] = [Re U_r, Im U_r] (4BW reals) and
//   B'[2c] = [Re V_c, Im V_c],  B'[2c+1] = [-Im V_c, Re V_c]
// give (A' B'^T)[r][2c] = Re C[r][c] and (A' B'^T)[r][2c+1] = Im C[r][c]: the
// real product comes out in the interleaved (re, im) layout of A22.
//
// Split bfloat16.  Every float32 operand x is written as x_hi + x_mid + x_lo
// (bfloat16 each, x - x_hi - x_mid - x_lo below 2^-24 |x|).  The K dimension
// holds NP segments of 4BW = 64 so that one bfloat16 MMA chain with float32
// accumulation sums
//   NP = 6: hi*hi + hi*mid + mid*hi + hi*lo + lo*hi + mid*mid  (dropped terms
//           below ~3 * 2^-24 relative: float32 quality),
//   NP = 3: hi*hi + hi*lo' + lo'*hi with lo' = bf16(x - x_hi)   (lo' carries
//           8 of the 16 bits below x_hi: the products lose ~2^-16 of each
//           term, partly cancelling over the K sum).
// Measured against float64 on GB300 (n = 256, 32 rank-1 terms of size ~3):
// largest error 3e-8 (FP32 pipe), 1.5e-7 (NP = 6: the tensor cores' own
// float32 accumulation), 7e-7 (NP = 3) of the largest term.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "large.cuh"

namespace idos {
namespace lg {

namespace {

constexpr int TC_M = 128;          // tile rows (tensor-memory lanes)
constexpr int TC_N = 128;          // tile columns, real (64 complex columns)
constexpr int TC_KC = 64;          // bfloat16 per K chunk (one 128-byte swizzle row)
constexpr int TC_KS = 4 * BW;      // reals per operand row segment (= TC_KC)
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_CHUNK_BYTES = (TC_M + TC_N) * TC_KC * 2;   // A and B box of one chunk
static_assert(TC_KS == TC_KC, "one operand segment per K chunk");

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of a barrier: false when it gave up (the
// error word is then set) or when another thread already reported an error.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int* err) {
  for (int it = 0; it < (1 << 24); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 1023) == 1023 && *(volatile int*)err) return false;
    if (it > 64) __nanosleep(64);
  }
  atomicExch(err, 1);
  return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (the layout TMA writes for a box
// whose inner extent is 128 bytes under CU_TENSOR_MAP_SWIZZLE_128B).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024u >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: float32 accumulator, bfloat16 A and B,
// both K-major, M = TC_M, N = TC_N.
__host__ __device__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

// the same for M = m, N = n
__host__ __device__ constexpr uint32_t tc_idesc_n(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// -------------------------------------------------------------- operands --
// bfloat16 split segments of one real value for operand A and B.
template <int NP>
__device__ __forceinline__ void split_segments(float x, __nv_bfloat16* segA, __nv_bfloat16* segB) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(hi);
  if constexpr (NP == 3) {
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1);
    segA[0] = hi; segA[1] = hi; segA[2] = lo;
    segB[0] = hi; segB[1] = lo; segB[2] = hi;
  } else {
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    segA[0] = hi; segA[1] = hi; segA[2] = mid; segA[3] = hi; segA[4] = lo; segA[5] = mid;
    segB[0] = hi; segB[1] = mid; segB[2] = hi; segB[3] = lo; segB[4] = hi; segB[5] = mid;
  }
}

// Aop[b][r][NP * 64] and Bop[b][2c + {0,1}][NP * 64] for rows r < m_max of
// every matrix (zero rows beyond the matrix's own trailing size).  One
// thread per (row, real index j < 64).
template <int NP>
__global__ void __launch_bounds__(256)
k_tc_operands(Batch bt, int k, const float2* __restrict__ Y, const float2* __restrict__ Z,
              __nv_bfloat16* __restrict__ Aop, __nv_bfloat16* __restrict__ Bop, int m_max) {
  constexpr int KP = NP * TC_KS;
  const int b = blockIdx.y;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int m = n - k - BW;
  const float2* Yb = Y + (size_t)b * BW * nm;
  const float2* Zb = Z + (size_t)b * BW * nm;
  __nv_bfloat16* Ab = Aop + (size_t)b * nm * KP;
  __nv_bfloat16* Bb = Bop + (size_t)b * 2 * nm * KP;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m_max * TC_KS; idx += gridDim.x * blockDim.x) {
    const int r = idx / TC_KS, j = idx % TC_KS;
    float a = 0.f, b0 = 0.f, b1 = 0.f;   // A'[r][j], B'[2r][j], B'[2r+1][j]
    if (r < m) {
      const int q = j & (2 * BW - 1);
      const bool im = j >= 2 * BW;
      const float2 u = q < BW ? Yb[(size_t)q * nm + r] : Zb[(size_t)(q - BW) * nm + r];
      const float2 v = q < BW ? Zb[(size_t)q * nm + r] : Yb[(size_t)(q - BW) * nm + r];
      a = im ? u.y : u.x;
      b0 = im ? v.y : v.x;
      b1 = im ? v.x : -v.y;
    }
    __nv_bfloat16 sa[NP], sb0[NP], sb1[NP], dummy[NP];
    split_segments<NP>(a, sa, dummy);
    split_segments<NP>(b0, dummy, sb0);
    split_segments<NP>(b1, dummy, sb1);
#pragma unroll
    for (int s = 0; s < NP; ++s) {
      Ab[(size_t)r * KP + s * TC_KS + j] = sa[s];
      Bb[(size_t)(2 * r) * KP + s * TC_KS + j] = sb0[s];
      Bb[(size_t)(2 * r + 1) * KP + s * TC_KS + j] = sb1[s];
    }
  }
}

// ------------------------------------------------------------ the update --
constexpr int TC_STAGES = 3;   // operand ring (A and B box of one K chunk per stage)
constexpr uint32_t TC_STAGE_BYTES = TC_CHUNK_BYTES;
constexpr uint32_t TC_OUT_GROUP_BYTES = TC_M * 128;   // 128 rows x 32 floats (one 128-byte swizzle row each)
static_assert(TC_N / 32 * TC_OUT_GROUP_BYTES <= TC_STAGES * TC_STAGE_BYTES, "output tile fits the operand ring");

__device__ __forceinline__ void tma_reduce_add_3d(const CUtensorMap* map, int x, int y, int z, uint32_t src) {
  asm volatile("cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z), "r"(src)
               : "memory");
}

// One CTA per (64-complex-column tile tj, 128-row tile ti, matrix b).
// Thread 0 streams the NP K chunks of the A and B tiles through a ring of
// TC_STAGES stages with TMA; thread 32 issues the 4 NP tcgen05.mma of K = 16
// as chunks land and frees each stage with a commit; the four warps then move
// the accumulator (warp w: lanes 32w..32w+31) into the swizzled output tile
// in shared memory, negated, and one TMA reduce-add per 32-float column group
// subtracts it from A22 in place.  Rows and columns beyond a matrix's trailing
// size carry zero operands (their update is an exact +-0), and the tensor
// bounds clip the tile at the matrix edge.
template <int NP>
__global__ void __launch_bounds__(TC_THREADS, 2)
k_tc_her2k(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
           const __grid_constant__ CUtensorMap tmC, Batch bt, int k, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_slot;
  const int b = blockIdx.z, ti = blockIdx.y, tj = blockIdx.x;
  const int n = batch_n(bt, b);
  const int m = n - k - BW;
  const int r0 = ti * TC_M, c0 = tj * (TC_N / 2);
  if (m <= 0 || r0 >= m || c0 >= m) return;   // the same for the whole CTA, before any barrier
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(tc_smem) + 1023u) & ~1023u;
  auto stage_a = [&](int s) { return base + (uint32_t)s * TC_STAGE_BYTES; };
  auto stage_b = [&](int s) { return base + (uint32_t)s * TC_STAGE_BYTES + (uint32_t)(TC_M * TC_KC * 2); };
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)TC_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  int issued = 0;   // chunks whose loads thread 0 issued
  if (threadIdx.x == 0) {
    for (int kc = 0; kc < NP; ++kc) {
      const int s = kc % TC_STAGES;
      if (kc >= TC_STAGES && !mbar_wait_bounded(smem_u32(&empty[s]), (uint32_t)((kc / TC_STAGES - 1) & 1), err)) break;
      const uint32_t bar = smem_u32(&full[s]);
      mbar_expect_tx(bar, TC_STAGE_BYTES);
      tma_load_3d(stage_a(s), &tmA, kc * TC_KC, r0, b, bar);
      tma_load_3d(stage_b(s), &tmB, kc * TC_KC, 2 * c0, b, bar);
      issued = kc + 1;
    }
  }
  if (threadIdx.x == 32) {
    constexpr uint32_t idesc = tc_idesc();
    for (int kc = 0; kc < NP; ++kc) {
      const int s = kc % TC_STAGES;
      if (!mbar_wait_bounded(smem_u32(&full[s]), (uint32_t)((kc / TC_STAGES) & 1), err)) break;
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < TC_KC / 16; ++kk) {
        const uint64_t ad = sw128_desc(stage_a(s) + kk * 32);
        const uint64_t bd = sw128_desc(stage_b(s) + kk * 32);
        tc_mma(tmem, ad, bd, idesc, (kc | kk) != 0 ? 1u : 0u);
      }
      tc_commit(smem_u32(&empty[s]));   // the stage is free once these MMAs have read it
    }
    tc_commit(smem_u32(&done));         // and the accumulator is final once all have completed
  }
  __syncwarp();
  const bool ready = mbar_wait_bounded(smem_u32(&done), 0, err);
  tc_fence_after();
  const bool ok = __all_sync(0xffffffffu, ready && !*(volatile int*)err);   // warp-uniform (tcgen05.ld is .aligned)
  if (ok) {
    // -acc into the output tile: column group g = real columns [32 g, 32 g + 32)
    // of the 128 rows, 128 bytes per row, 16-byte chunks swizzled by row % 8
    const int row = warp * 32 + lane;
#pragma unroll 1
    for (int g = 0; g < TC_N / 32; ++g) {
      float acc[32];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * 32), acc);
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * 32 + 16), acc + 16);
      const uint32_t rbase = base + (uint32_t)g * TC_OUT_GROUP_BYTES + (uint32_t)row * 128;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint32_t addr = rbase + (uint32_t)((c ^ (row & 7)) << 4);
        asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(-acc[4 * c]), "f"(-acc[4 * c + 1]),
                     "f"(-acc[4 * c + 2]), "f"(-acc[4 * c + 3])
                     : "memory");
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the bulk copy
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ok) {
      for (int g = 0; g < TC_N / 32; ++g)
        tma_reduce_add_3d(&tmC, 2 * (k + BW + c0) + 32 * g, k + BW + r0, b, base + (uint32_t)g * TC_OUT_GROUP_BYTES);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // shared memory read before leaving
    } else {
      // a wait gave up: let the loads already issued land before leaving
      for (int kc = 0; kc < issued; ++kc) {
        const int s = kc % TC_STAGES;
        for (int it = 0; it < (1 << 20) && !mbar_try_wait(smem_u32(&full[s]), (uint32_t)((kc / TC_STAGES) & 1)); ++it)
          __nanosleep(64);
      }
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TC_N) : "memory");
  }
}

// ------------------------------------- the update, lower-triangle tiles --
// The same update on square tiles of 128 rows x 128 complex columns (MMA
// N = 256 reals), only on and below the diagonal: U = Y Z^H + Z Y^H is
// Hermitian, so tile (I, J), I > J, also gives the block (J, I) as its
// conjugate transpose.  Its epilogue subtracts U from A22[I][J] and
// conj(U)^T from A22[J][I] (the mirror, staged transposed in shared memory
// and added by 16-row TMA reduce-adds); a diagonal tile subtracts its whole
// block directly.  Every entry of A22 is updated exactly once, with about half
// the MMAs and operand loads of the full grid.
constexpr int TL_N = 256;                                        // real columns of a tile (128 complex)
constexpr int TL_STAGES = 2;
constexpr uint32_t TL_STAGE_BYTES = (TC_M + TL_N) * TC_KC * 2;   // A and B box of one K chunk
constexpr uint32_t TL_GROUP_BYTES = 2 * TC_M * 128;              // direct (128 rows) + mirror (16 x 256 floats) group
constexpr int TL_GROUPS_PER_BATCH = (int)(TL_STAGES * TL_STAGE_BYTES / TL_GROUP_BYTES);
static_assert(TL_GROUPS_PER_BATCH >= 1, "epilogue staging fits the operand ring");
constexpr int TL_THREADS = 256;   // two warps per TMEM lane quarter share the epilogue's column groups

__device__ __forceinline__ void tile_of(int t, int& I, int& J) {
  int i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  I = i;
  J = t - i * (i + 1) / 2;
}

template <int NP>
__global__ void __launch_bounds__(TL_THREADS, 2)
k_tc_her2k_lt(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmCm, Batch bt, int k,
              int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t full[TL_STAGES], empty[TL_STAGES];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_slot;
  const int b = blockIdx.z;
  int I, J;
  tile_of((int)blockIdx.x, I, J);
  const int n = batch_n(bt, b);
  const int m = n - k - BW;
  const int r0 = I * TC_M, c0 = J * TC_M;
  if (m <= 0 || r0 >= m) return;   // the same for the whole CTA, before any barrier
  const bool mirror = I > J;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(tc_smem) + 1023u) & ~1023u;
  auto stage_a = [&](int s) { return base + (uint32_t)s * TL_STAGE_BYTES; };
  auto stage_b = [&](int s) { return base + (uint32_t)s * TL_STAGE_BYTES + (uint32_t)(TC_M * TC_KC * 2); };
  if (threadIdx.x == 0) {
    for (int s = 0; s < TL_STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)TL_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  int issued = 0;
  if (threadIdx.x == 0) {
    for (int kc = 0; kc < NP; ++kc) {
      const int s = kc % TL_STAGES;
      if (kc >= TL_STAGES && !mbar_wait_bounded(smem_u32(&empty[s]), (uint32_t)((kc / TL_STAGES - 1) & 1), err)) break;
      const uint32_t bar = smem_u32(&full[s]);
      mbar_expect_tx(bar, TL_STAGE_BYTES);
      tma_load_3d(stage_a(s), &tmA, kc * TC_KC, r0, b, bar);
      tma_load_3d(stage_b(s), &tmB, kc * TC_KC, 2 * c0, b, bar);
      issued = kc + 1;
    }
  }
  if (threadIdx.x == 32) {
    constexpr uint32_t idesc = tc_idesc_n(TC_M, TL_N);
    for (int kc = 0; kc < NP; ++kc) {
      const int s = kc % TL_STAGES;
      if (!mbar_wait_bounded(smem_u32(&full[s]), (uint32_t)((kc / TL_STAGES) & 1), err)) break;
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < TC_KC / 16; ++kk) {
        const uint64_t ad = sw128_desc(stage_a(s) + kk * 32);
        const uint64_t bd = sw128_desc(stage_b(s) + kk * 32);
        tc_mma(tmem, ad, bd, idesc, (kc | kk) != 0 ? 1u : 0u);
      }
      tc_commit(smem_u32(&empty[s]));
    }
    tc_commit(smem_u32(&done));
  }
  __syncwarp();
  const bool ready = mbar_wait_bounded(smem_u32(&done), 0, err);
  tc_fence_after();
  // block-uniform: every thread takes part in the staging barriers below
  const bool ok = __syncthreads_and(ready && !*(volatile int*)err) != 0;
  const int q4 = warp & 3, half = warp >> 2;   // TMEM lane quarter; which groups of a batch
  const int row = q4 * 32 + lane;               // tile row = TMEM lane
  if (ok) {
    for (int g0 = 0; g0 < TL_N / 32; g0 += TL_GROUPS_PER_BATCH) {
      const int g1 = min(TL_N / 32, g0 + TL_GROUPS_PER_BATCH);
      for (int g = g0 + half; g < g1; g += 2) {
        // complex columns 16 g .. 16 g + 15 of the tile
        float acc[32];
        tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(g * 32), acc);
        tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(g * 32 + 16), acc + 16);
        const uint32_t dbase = base + (uint32_t)(g - g0) * TL_GROUP_BYTES;
        const uint32_t rbase = dbase + (uint32_t)row * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const uint32_t addr = rbase + (uint32_t)((c ^ (row & 7)) << 4);
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(-acc[4 * c]), "f"(-acc[4 * c + 1]),
                       "f"(-acc[4 * c + 2]), "f"(-acc[4 * c + 3])
                       : "memory");
        }
        if (mirror) {
          // mirror block: rows = the group's 16 complex columns j, columns =
          // the tile's 128 rows, as 8 boxes of 16 rows x 16 complex
          const uint32_t mbase = dbase + (uint32_t)(TC_M * 128) + (uint32_t)(row >> 4) * 2048;
          const int cc = row & 15;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const uint32_t addr =
                mbase + (uint32_t)j * 128 + (uint32_t)((((cc >> 1) ^ (j & 7))) << 4) + (uint32_t)((cc & 1) * 8);
            asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(-acc[2 * j]), "f"(acc[2 * j + 1])
                         : "memory");
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the bulk copies
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int g = g0; g < g1; ++g) {
          const uint32_t dbase = base + (uint32_t)(g - g0) * TL_GROUP_BYTES;
          tma_reduce_add_3d(&tmC, 2 * (k + BW + c0) + 32 * g, k + BW + r0, b, dbase);
          if (mirror)
            for (int bx = 0; bx < TC_M / 16; ++bx)
              tma_reduce_add_3d(&tmCm, 2 * (k + BW + r0) + 32 * bx, k + BW + c0 + 16 * g, b,
                                dbase + (uint32_t)(TC_M * 128) + (uint32_t)bx * 2048);
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // staging read before it is reused
      }
      __syncthreads();
    }
  } else if (threadIdx.x == 0) {
    // a wait gave up: let the loads still in flight land before leaving
    for (int kc = max(0, issued - TL_STAGES); kc < issued; ++kc) {
      const int s = kc % TL_STAGES;
      for (int it = 0; it < (1 << 20) && !mbar_try_wait(smem_u32(&full[s]), (uint32_t)((kc / TL_STAGES) & 1)); ++it)
        __nanosleep(64);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TL_N) : "memory");
  }
}

// ------------------------------------------------------ W = A22 (Y T) --
// The product W = A22 V (V = Y T, m x BW complex) of every stage-1 step on
// the tensor cores.  Real form: row r of A22 is 2m interleaved reals
// a[2x + t] (t = 0: Re, 1: Im of A22[r][x]); with the operand rows
//   B'[2c][2x] = Re V[x][c],  B'[2c][2x+1] = -Im V[x][c],
//   B'[2c+1][2x] = Im V[x][c], B'[2c+1][2x+1] = Re V[x][c]
// (a B'^T)[2c] = Re W[r][c] and (a B'^T)[2c+1] = Im W[r][c].  K runs over
// x-chunks of 32 complex columns (64 reals, one 128-byte bfloat16 row); for
// each chunk the six split products of the trailing update are accumulated,
// hi*hi into one TMEM accumulator and the five smaller terms (hi*mid, mid*hi,
// hi*lo, lo*hi, mid*mid) into a second, added in float32 at the end: summed
// into the large hi*hi partial sums, the small terms lost low bits in the
// tensor cores' accumulation (about 10x the FP32 pipe's error, measured).
// B' is split once per step into three bfloat16 planes in global memory; A22
// stays float32 and is split in shared memory: TMA brings the float32 tile of
// a chunk, eight converter warps write its hi, mid and lo planes in the
// 128-byte swizzled K-major layout, one thread issues the MMAs (M = 128 rows,
// N = 32 reals).  A CTA covers 128 rows and a range of chunks (a K split: its
// partial W goes to its own slice, summed later in split order).
constexpr int TW_N = 2 * BW;                                   // real output columns
constexpr int TW_CONV_WARPS = 8;
constexpr int TW_THREADS = 32 * (2 + TW_CONV_WARPS);           // TMA warp, MMA warp, converters
constexpr uint32_t TW_BOX_A = TC_M * 32 * 4;                   // one float32 box: 128 rows x 32 floats
constexpr uint32_t TW_A_BYTES = 2 * TW_BOX_A;                  // the chunk's 64 reals per row
constexpr uint32_t TW_BOX_B = TW_N * TC_KC * 2;                // one B' plane box: 32 rows x 64 bfloat16
constexpr uint32_t TW_B_BYTES = 3 * TW_BOX_B;
constexpr uint32_t TW_PLANE = TC_M * TC_KC * 2;                // one A plane: 128 rows x 64 bfloat16
constexpr uint32_t TW_STAGE_BYTES = TW_A_BYTES + TW_B_BYTES + 3 * TW_PLANE;
constexpr int TW_STAGES = 2;
constexpr uint32_t TW_TMEM_COLS = 2 * TW_N;                    // large-term and small-term accumulators
static_assert(TW_A_BYTES % 1024 == 0 && TW_B_BYTES % 1024 == 0 && TW_STAGE_BYTES % 1024 == 0, "1024-byte alignment");

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bw[b][plane][2c + e][j] (plane 0, 1, 2 = hi, mid, lo of B' above), j < kw,
// zero for x = j / 2 >= m.  One thread per (row, j).
__global__ void __launch_bounds__(256)
k_tc_w_operands(Batch bt, int k, const float2* __restrict__ YT, __nv_bfloat16* __restrict__ Bw, int kw) {
  const int b = blockIdx.y;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int m = n - k - BW;
  const float2* Vb = YT + (size_t)b * BW * nm;
  __nv_bfloat16* out = Bw + (size_t)b * 3 * TW_N * kw;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < TW_N * kw; idx += gridDim.x * blockDim.x) {
    const int row = idx / kw, j = idx % kw;
    const int c = row >> 1, e = row & 1, x = j >> 1, t = j & 1;
    float v = 0.f;
    if (x < m) {
      const float2 y = Vb[(size_t)c * nm + x];
      v = e == 0 ? (t == 0 ? y.x : -y.y) : (t == 0 ? y.y : y.x);
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
    out[(size_t)(0 * TW_N + row) * kw + j] = hi;
    out[(size_t)(1 * TW_N + row) * kw + j] = mid;
    out[(size_t)(2 * TW_N + row) * kw + j] = lo;
  }
}

// hi, mid, lo bfloat16 pairs of two floats (the same splits as split_segments)
__device__ __forceinline__ void split3_pair(float x0, float x1, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const float r0 = x0 - hf.x, r1 = x1 - hf.y;
  const __nv_bfloat162 md = __floats2bfloat162_rn(r0, r1);
  const float2 mf = __bfloat1622float2(md);
  const __nv_bfloat162 l = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  mid = *reinterpret_cast<const uint32_t*>(&md);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__global__ void __launch_bounds__(TW_THREADS, 1)
k_tc_w(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Batch bt, int k, int nsplit,
       float2* __restrict__ Wp, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) uint64_t a_full[TW_STAGES], a_empty[TW_STAGES], p_full[TW_STAGES], p_empty[TW_STAGES];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_slot;
  const int b = blockIdx.z, sp = blockIdx.y, ti = blockIdx.x;
  const int n = batch_n(bt, b);
  const int nm = bt.n_max;
  const int m = n - k - BW;
  const int r0 = ti * TC_M;
  if (m <= 0 || r0 >= m) return;   // the same for the whole CTA, before any barrier
  const int nxc = (m + 31) / 32;
  const int per = (nxc + nsplit - 1) / nsplit;
  const int xc_lo = sp * per;
  const int nit = max(0, min(nxc, xc_lo + per) - xc_lo);
  float2* W = Wp + ((size_t)b * nsplit + sp) * BW * nm;
  if (nit == 0) {   // an empty split: its slice of W is zero
    for (int idx = threadIdx.x; idx < BW * TC_M; idx += blockDim.x) {
      const int c = idx / TC_M, r = r0 + idx % TC_M;
      if (r < m) W[(size_t)c * nm + r] = make_float2(0.f, 0.f);
    }
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(tc_smem) + 1023u) & ~1023u;
  auto st_a = [&](int s) { return base + (uint32_t)s * TW_STAGE_BYTES; };
  auto st_b = [&](int s) { return st_a(s) + TW_A_BYTES; };
  auto st_p = [&](int s) { return st_a(s) + TW_A_BYTES + TW_B_BYTES; };
  if (threadIdx.x == 0) {
    for (int s = 0; s < TW_STAGES; ++s) {
      mbar_init(smem_u32(&a_full[s]), 1);
      mbar_init(smem_u32(&a_empty[s]), TW_CONV_WARPS + 1);
      mbar_init(smem_u32(&p_full[s]), TW_CONV_WARPS);
      mbar_init(smem_u32(&p_empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TW_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  int issued = 0;
  if (threadIdx.x == 0) {
    // producer: the float32 tile (two boxes) and the three B' plane boxes of each chunk
    for (int it = 0; it < nit; ++it) {
      const int s = it % TW_STAGES;
      if (it >= TW_STAGES &&
          !mbar_wait_bounded(smem_u32(&a_empty[s]), (uint32_t)((it / TW_STAGES - 1) & 1), err))
        break;
      const uint32_t bar = smem_u32(&a_full[s]);
      mbar_expect_tx(bar, TW_A_BYTES + TW_B_BYTES);
      const int xc = xc_lo + it;
      const int x0 = 2 * (k + BW) + 64 * xc;
      tma_load_3d(st_a(s), &tmA, x0, k + BW + r0, b, bar);
      tma_load_3d(st_a(s) + TW_BOX_A, &tmA, x0 + 32, k + BW + r0, b, bar);
      for (int q = 0; q < 3; ++q) tma_load_3d(st_b(s) + (uint32_t)q * TW_BOX_B, &tmB, 64 * xc, TW_N * q, b, bar);
      issued = it + 1;
    }
  }
  if (threadIdx.x == 32) {
    // MMA issuer: per chunk hi*hi into accumulator 0, the five smaller split
    // products into accumulator 1, four K = 16 steps each
    constexpr uint32_t idesc = tc_idesc_n(TC_M, TW_N);
    constexpr int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
    for (int it = 0; it < nit; ++it) {
      const int s = it % TW_STAGES;
      if (!mbar_wait_bounded(smem_u32(&a_full[s]), (uint32_t)((it / TW_STAGES) & 1), err)) break;
      if (!mbar_wait_bounded(smem_u32(&p_full[s]), (uint32_t)((it / TW_STAGES) & 1), err)) break;
      tc_fence_after();
#pragma unroll
      for (int pr = 0; pr < 6; ++pr) {
        const uint32_t acc = pr == 0 ? tmem : tmem + (uint32_t)TW_N;
        const bool first = it == 0 && pr <= 1;   // the first product into each accumulator
#pragma unroll
        for (int kk = 0; kk < TC_KC / 16; ++kk) {
          const uint64_t ad = sw128_desc(st_p(s) + (uint32_t)pa[pr] * TW_PLANE + kk * 32);
          const uint64_t bd = sw128_desc(st_b(s) + (uint32_t)pb[pr] * TW_BOX_B + kk * 32);
          tc_mma(acc, ad, bd, idesc, (first && kk == 0) ? 0u : 1u);
        }
      }
      tc_commit(smem_u32(&p_empty[s]));   // planes free once these MMAs have read them
      tc_commit(smem_u32(&a_empty[s]));   // and the B' boxes of the stage
    }
    tc_commit(smem_u32(&done));
  }
  if (warp >= 2) {
    // converters: row 32 (warp % 4) + lane (the TMEM lanes this warp may read
    // in the epilogue), reals [32 h, 32 h + 32) of the chunk, h = (warp - 2) / 4
    const int q4 = warp & 3, h = (warp - 2) >> 2;
    const int rl = 32 * q4 + lane;
    for (int it = 0; it < nit; ++it) {
      const int s = it % TW_STAGES;
      // every lane observes the phases itself; the warp leaves together
      bool ok = mbar_wait_bounded(smem_u32(&a_full[s]), (uint32_t)((it / TW_STAGES) & 1), err);
      if (ok && it >= TW_STAGES) ok = mbar_wait_bounded(smem_u32(&p_empty[s]), (uint32_t)((it / TW_STAGES - 1) & 1), err);
      if (!__all_sync(0xffffffffu, ok)) break;
      const uint32_t src = st_a(s) + (uint32_t)h * TW_BOX_A + (uint32_t)rl * 128;
      const uint32_t dst = st_p(s) + (uint32_t)rl * 128;
#pragma unroll
      for (int pq = 0; pq < 4; ++pq) {
        // plane chunk 4 h + pq (8 reals) = float32 chunks 2 pq, 2 pq + 1 of box h
        float f[8];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const uint32_t a = src + (uint32_t)(((2 * pq + u) ^ (rl & 7)) << 4);
          asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                       : "=f"(f[4 * u]), "=f"(f[4 * u + 1]), "=f"(f[4 * u + 2]), "=f"(f[4 * u + 3])
                       : "r"(a));
        }
        uint32_t hi[4], md[4], lo[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) split3_pair(f[2 * v], f[2 * v + 1], hi[v], md[v], lo[v]);
        const uint32_t off = (uint32_t)(((4 * h + pq) ^ (rl & 7)) << 4);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + off), "r"(hi[0]), "r"(hi[1]), "r"(hi[2]),
                     "r"(hi[3])
                     : "memory");
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + TW_PLANE + off), "r"(md[0]), "r"(md[1]),
                     "r"(md[2]), "r"(md[3])
                     : "memory");
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + 2 * TW_PLANE + off), "r"(lo[0]), "r"(lo[1]),
                     "r"(lo[2]), "r"(lo[3])
                     : "memory");
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the MMAs
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&p_full[s]));
        mbar_arrive(smem_u32(&a_empty[s]));
      }
    }
    // epilogue: W[c][r] for complex columns c in [8 h, 8 h + 8), the sum of
    // the two accumulators
    const bool ready = mbar_wait_bounded(smem_u32(&done), 0, err);
    tc_fence_after();
    if (__all_sync(0xffffffffu, ready && !*(volatile int*)err)) {
      float big[16], small[16];
      const uint32_t t = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(16 * h);
      tmem_ld16(t, big);
      tmem_ld16(t + (uint32_t)TW_N, small);
      const int r = r0 + rl;
      if (r < m) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          W[(size_t)(8 * h + j) * nm + r] = make_float2(big[2 * j] + small[2 * j], big[2 * j + 1] + small[2 * j + 1]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && issued > 0 && *(volatile int*)err) {
    // a wait gave up: let the loads still in flight (at most one per stage,
    // the last ones issued) land before leaving
    for (int it = max(0, issued - TW_STAGES); it < issued; ++it) {
      const int s = it % TW_STAGES;
      for (int w = 0; w < (1 << 20) && !mbar_try_wait(smem_u32(&a_full[s]), (uint32_t)((it / TW_STAGES) & 1)); ++w)
        __nanosleep(64);
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TW_TMEM_COLS) : "memory");
  }
}

// ----------------------------------------------------------- host side --
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_fn(EncodeTiled* out) {
  static std::mutex mu;
  static EncodeTiled fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return IDOS_ERR_CUDA;
    }
    fn = reinterpret_cast<EncodeTiled>(p);
  }
  *out = fn;
  return IDOS_OK;
}

// 3-D map over a [batch][rows][KP] bfloat16 buffer, box 64 x box_rows x 1,
// 128-byte swizzle (rows beyond `rows` read as zeros).
int make_map(CUtensorMap* map, void* ptr, int KP, int64_t rows, int64_t batch, int box_rows) {
  EncodeTiled fn;
  IDOS_TRY(encode_fn(&fn));
  const cuuint64_t dims[3] = {(cuuint64_t)KP, (cuuint64_t)rows, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)KP * 2, (cuuint64_t)KP * 2 * (cuuint64_t)rows};
  const cuuint32_t box[3] = {(cuuint32_t)TC_KC, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ptr, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed for the trailing-update operands");
    return IDOS_ERR_CUDA;
  }
  return IDOS_OK;
}

// 3-D map over the dense float32 batch A [batch][n][n] complex seen as
// [batch][n][2n] floats, box 32 floats x box_rows rows x 1 (one 128-byte
// swizzle row per tile row): the target of the reduce-add.  Needs 2n floats
// per row to be a multiple of 16 bytes, i.e. n even.
int make_map_c(CUtensorMap* map, void* A, int n, int64_t batch, int box_rows = TC_M) {
  EncodeTiled fn;
  IDOS_TRY(encode_fn(&fn));
  const cuuint64_t dims[3] = {(cuuint64_t)2 * n, (cuuint64_t)n, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)8 * n, (cuuint64_t)8 * n * (cuuint64_t)n};
  const cuuint32_t box[3] = {32, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, A, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed for the trailing block");
    return IDOS_ERR_CUDA;
  }
  return IDOS_OK;
}

size_t tc_smem_bytes() { return (size_t)TC_STAGES * TC_STAGE_BYTES + 1024; }
size_t tw_smem_bytes() { return (size_t)TW_STAGES * TW_STAGE_BYTES + 1024; }
size_t tl_smem_bytes() { return (size_t)TL_STAGES * TL_STAGE_BYTES + 1024; }

// bfloat16 reals of one B' plane row of W's operand: 64 per chunk of 32
// complex columns, enough chunks for n_max columns
int tw_kw(int n_max) { return 64 * ((n_max + 31) / 32); }

// 3-D map over B' [batch][3 planes x 32 rows][kw] bfloat16, box 64 x 32 x 1.
int make_map_wb(CUtensorMap* map, void* ptr, int kw, int64_t batch) {
  EncodeTiled fn;
  IDOS_TRY(encode_fn(&fn));
  const cuuint64_t dims[3] = {(cuuint64_t)kw, (cuuint64_t)3 * TW_N, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)kw * 2, (cuuint64_t)kw * 2 * 3 * TW_N};
  const cuuint32_t box[3] = {(cuuint32_t)TC_KC, (cuuint32_t)TW_N, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, ptr, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed for the W operand");
    return IDOS_ERR_CUDA;
  }
  return IDOS_OK;
}

}  // namespace

size_t tc_operand_bytes(int n_max, int np) { return (size_t)3 * n_max * np * TC_KS * 2 + 2 * 1024; }

int tc_plan(TcPlan& p, int n_max, int64_t batch, int np, void* Aop, void* Bop, void* A) {
  if (np != 3 && np != 6) {
    set_error("split-bfloat16 products must be 3 or 6");
    return IDOS_ERR_INVALID_ARG;
  }
  if (n_max % 2 != 0) {
    set_error("the tensor-core trailing update needs an even matrix dimension");
    return IDOS_ERR_UNSUPPORTED;
  }
  p.np = np;
  p.n_max = n_max;
  p.Aop = Aop;
  p.Bop = Bop;
  const int KP = np * TC_KS;
  IDOS_TRY(make_map(&p.mapA, Aop, KP, n_max, batch, TC_M));
  IDOS_TRY(make_map(&p.mapB, Bop, KP, 2 * (int64_t)n_max, batch, TC_N));
  IDOS_TRY(make_map(&p.mapB2, Bop, KP, 2 * (int64_t)n_max, batch, TL_N));
  IDOS_TRY(make_map_c(&p.mapC, A, n_max, batch));
  IDOS_TRY(make_map_c(&p.mapCm, A, n_max, batch, 16));
  // W's operand B' (three planes of 32 x kw bfloat16 per matrix) lives in
  // the trailing update's B buffer: each step builds and uses it before the
  // update's operands overwrite it
  p.kw = tw_kw(n_max);
  if ((size_t)3 * TW_N * p.kw * 2 > tc_operand_bytes(n_max, np) / 3 * 2) {
    set_error("W operand does not fit the trailing update's operand buffer");
    return IDOS_ERR_INVALID_ARG;
  }
  IDOS_TRY(make_map_wb(&p.mapWB, Bop, p.kw, batch));
  IDOS_CUDA_TRY(cudaFuncSetAttribute(k_tc_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tw_smem_bytes()));
  if (np == 3) {
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_tc_her2k<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes()));
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_tc_her2k_lt<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tl_smem_bytes()));
  } else {
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_tc_her2k<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes()));
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_tc_her2k_lt<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tl_smem_bytes()));
  }
  return IDOS_OK;
}

int tc_her2k(const TcPlan& p, const Batch& bt, int k, const c2<float>* Y, const c2<float>* Z, int* err,
             cudaStream_t s) {
  const int m_max = bt.n_max - k - BW;
  if (m_max <= 0) return IDOS_OK;
  const unsigned nb = (unsigned)bt.B;
  const int rows_threads = m_max * TC_KS;
  const dim3 og((unsigned)std::min(1024, (rows_threads + 255) / 256), nb);
  const dim3 tg((unsigned)((m_max + TC_N / 2 - 1) / (TC_N / 2)), (unsigned)((m_max + TC_M - 1) / TC_M), nb);
  const int T = (m_max + TC_M - 1) / TC_M;
  const dim3 tl((unsigned)(T * (T + 1) / 2), 1, nb);
  auto* ab = reinterpret_cast<__nv_bfloat16*>(p.Aop);
  auto* bb = reinterpret_cast<__nv_bfloat16*>(p.Bop);
  if (p.np == 3) {
    k_tc_operands<3><<<og, 256, 0, s>>>(bt, k, Y, Z, ab, bb, m_max);
    if (p.lower)
      k_tc_her2k_lt<3><<<tl, TL_THREADS, tl_smem_bytes(), s>>>(p.mapA, p.mapB2, p.mapC, p.mapCm, bt, k, err);
    else
      k_tc_her2k<3><<<tg, TC_THREADS, tc_smem_bytes(), s>>>(p.mapA, p.mapB, p.mapC, bt, k, err);
  } else {
    k_tc_operands<6><<<og, 256, 0, s>>>(bt, k, Y, Z, ab, bb, m_max);
    if (p.lower)
      k_tc_her2k_lt<6><<<tl, TL_THREADS, tl_smem_bytes(), s>>>(p.mapA, p.mapB2, p.mapC, p.mapCm, bt, k, err);
    else
      k_tc_her2k<6><<<tg, TC_THREADS, tc_smem_bytes(), s>>>(p.mapA, p.mapB, p.mapC, bt, k, err);
  }
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

int tc_w(const TcPlan& p, const Batch& bt, int k, const c2<float>* YT, c2<float>* Wp, int nsplit, int* err,
         cudaStream_t s) {
  const int m_max = bt.n_max - k - BW;
  if (m_max <= 0) return IDOS_OK;
  const unsigned nb = (unsigned)bt.B;
  const int opn = TW_N * p.kw;
  const dim3 og((unsigned)std::min(1024, (opn + 255) / 256), nb);
  k_tc_w_operands<<<og, 256, 0, s>>>(bt, k, reinterpret_cast<const float2*>(YT),
                                     reinterpret_cast<__nv_bfloat16*>(p.Bop), p.kw);
  const dim3 g((unsigned)((m_max + TC_M - 1) / TC_M), (unsigned)nsplit, nb);
  k_tc_w<<<g, TW_THREADS, tw_smem_bytes(), s>>>(p.mapC, p.mapWB, bt, k, nsplit, reinterpret_cast<float2*>(Wp), err);
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

}  // namespace lg
}  // namespace idos
