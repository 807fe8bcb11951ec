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
  const bool ok = ready && !*(volatile int*)err;
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
// [batch][n][2n] floats, box 32 floats x 128 rows x 1 (one 128-byte swizzle
// row per tile row): the target of the reduce-add.  Needs 2n floats per row
// to be a multiple of 16 bytes, i.e. n even.
int make_map_c(CUtensorMap* map, void* A, int n, int64_t batch) {
  EncodeTiled fn;
  IDOS_TRY(encode_fn(&fn));
  const cuuint64_t dims[3] = {(cuuint64_t)2 * n, (cuuint64_t)n, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)8 * n, (cuuint64_t)8 * n * (cuuint64_t)n};
  const cuuint32_t box[3] = {32, (cuuint32_t)TC_M, 1};
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
  IDOS_TRY(make_map_c(&p.mapC, A, n_max, batch));
  if (np == 3) {
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_tc_her2k<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes()));
  } else {
    IDOS_CUDA_TRY(cudaFuncSetAttribute(k_tc_her2k<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes()));
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
  auto* ab = reinterpret_cast<__nv_bfloat16*>(p.Aop);
  auto* bb = reinterpret_cast<__nv_bfloat16*>(p.Bop);
  if (p.np == 3) {
    k_tc_operands<3><<<og, 256, 0, s>>>(bt, k, Y, Z, ab, bb, m_max);
    k_tc_her2k<3><<<tg, TC_THREADS, tc_smem_bytes(), s>>>(p.mapA, p.mapB, p.mapC, bt, k, err);
  } else {
    k_tc_operands<6><<<og, 256, 0, s>>>(bt, k, Y, Z, ab, bb, m_max);
    k_tc_her2k<6><<<tg, TC_THREADS, tc_smem_bytes(), s>>>(p.mapA, p.mapB, p.mapC, bt, k, err);
  }
  IDOS_CHECK_LAUNCH();
  return IDOS_OK;
}

}  // namespace lg
}  // namespace idos
