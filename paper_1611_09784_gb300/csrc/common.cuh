// common.cuh - shared device helpers of libidos (sm_103a): complex arithmetic
// on float2/double2, the Philox4x64-10 generator, group reductions, and the
// host-side error plumbing used by every translation unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/idos.h"

namespace idos {

// ---------------------------------------------------------------- errors ---
void set_error(const std::string& msg);
const char* get_error();

#define IDOS_CUDA_TRY(call)                                                        \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ::idos::set_error(std::string(#call) + ": " + cudaGetErrorString(e_) + " (" + \
                        __FILE__ + ":" + std::to_string(__LINE__) + ")");          \
      return (e_ == cudaErrorMemoryAllocation) ? IDOS_ERR_OUT_OF_MEMORY : IDOS_ERR_CUDA; \
    }                                                                              \
  } while (0)

#define IDOS_TRY(expr)        \
  do {                        \
    int s_ = (expr);          \
    if (s_ != IDOS_OK) return s_; \
  } while (0)

#define IDOS_CHECK_LAUNCH() IDOS_CUDA_TRY(cudaGetLastError())

// ---------------------------------------------------------------- complex --
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using c2 = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ c2<T> mk(T re, T im) {
  c2<T> z; z.x = re; z.y = im; return z;
}
template <typename T> __device__ __forceinline__ c2<T> cadd(c2<T> a, c2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ c2<T> csub(c2<T> a, c2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ c2<T> cmul(c2<T> a, c2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ c2<T> cmulc(c2<T> a, c2<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// conj(a) * b
template <typename T> __device__ __forceinline__ c2<T> cjmul(c2<T> a, c2<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename T> __device__ __forceinline__ c2<T> cscale(c2<T> a, T s) { return mk<T>(a.x * s, a.y * s); }

// |a| and the phase a / |a| (1 for a = 0) of a reflector's leading entry,
// computed on a scaled by its larger component.  Forming |a|^2 first loses
// the phase when a is tiny: below about 1e-19 in float32 (1e-154 in float64)
// the square is subnormal and keeps only a few bits, so a / sqrt(|a|^2) is
// not of unit modulus and I - tau v v^H is not unitary.  Such entries are
// rounding noise where the exact value is 0 (the bipartite lattice makes
// many), so they do occur.
template <typename T>
__device__ __forceinline__ T cabs_phase(c2<T> a, c2<T>& ph) {
  const T s = fmax(fabs(a.x), fabs(a.y));
  if (!(s > T(0))) {
    ph = mk<T>(T(1), T(0));
    return T(0);
  }
  const T ax = a.x / s, ay = a.y / s;
  const T r = sqrt(ax * ax + ay * ay);
  ph = mk<T>(ax / r, ay / r);
  return s * r;
}
// float32: one correctly rounded reciprocal and one hardware reciprocal
// square root (|ph| = 1 to a few float32 ulp), short on the latency path of
// the band chase's reflectors.  A subnormal s is first scaled by 2^64 (exact):
// its reciprocal would overflow to infinity and the phase become inf * 0.
template <>
__device__ __forceinline__ float cabs_phase<float>(float2 a, float2& ph) {
  const float s = fmaxf(fabsf(a.x), fabsf(a.y));
  if (!(s > 0.f)) {
    ph = make_float2(1.f, 0.f);
    return 0.f;
  }
  const float up = s < 0x1p-64f ? 0x1p64f : 1.f;
  const float rs = __frcp_rn(s * up);
  const float ax = a.x * up * rs, ay = a.y * up * rs;
  const float q = ax * ax + ay * ay;   // in [1, 2]
  const float rq = rsqrtf(q);
  ph = make_float2(ax * rq, ay * rq);
  return s * (q * rq);
}
template <typename T> __device__ __forceinline__ T cabs2(c2<T> a) { return a.x * a.x + a.y * a.y; }
template <typename T> __device__ __forceinline__ c2<T> conjg(c2<T> a) { return mk<T>(a.x, -a.y); }

// ---------------------------------------------------------------- philox ---
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): each round multiplies
// counter words 0 and 2 by fixed odd constants, swaps and xors the high
// halves with the other words and the key; the key follows a Weyl sequence.
struct u64x4 { uint64_t w[4]; };

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ u64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2_,
                                                        uint64_t c3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t lo0 = M0 * c0, hi0 = mulhi64(M0, c0);
    const uint64_t lo1 = M1 * c2_, hi1 = mulhi64(M1, c2_);
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2_ = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  u64x4 o; o.w[0] = c0; o.w[1] = c1; o.w[2] = c2_; o.w[3] = c3; return o;
}

constexpr uint64_t kStreamVacancy = 1;
constexpr uint64_t kStreamParams = 2;

// ---------------------------------------------------------------- groups ---
// A "group" is NT consecutive threads (NT a multiple of 32, or 16: half a
// warp) working on one matrix; MPB groups share a CTA.  Groups synchronise
// with a named barrier (warp or half-warp groups: __syncwarp over their lanes).
template <int NT, int MPB>
__device__ __forceinline__ void group_sync(int gid) {
  if constexpr (NT == 16) {
    __syncwarp(0xFFFFu << (16 * (gid & 1)));
  } else if constexpr (NT == 32) {
    __syncwarp();
  } else if constexpr (MPB == 1) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(NT) : "memory");
  }
}

// Sum of v over the NT threads of the group, identical in every thread and
// independent of timing (fixed order).  scratch: >= NT/32 entries per group.
template <int NT, int MPB, typename T>
__device__ __forceinline__ T group_sum(T v, T* scratch, int gid) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if constexpr (NT == 32) {
    return v;
  } else {
    const int lane = threadIdx.x & 31, w = (threadIdx.x % NT) >> 5;
    if (lane == 0) scratch[w] = v;
    group_sync<NT, MPB>(gid);
    T s = T(0);
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) s += scratch[i];
    group_sync<NT, MPB>(gid);
    return s;
  }
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch /* >= 32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  T s = T(0);
  for (int i = 0; i < nw; ++i) s += scratch[i];
  __syncthreads();
  return s;
}

}  // namespace idos
