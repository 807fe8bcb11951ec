// noalloc.cu - idos_eval_idos_noalloc: the single-configuration IDoS
// evaluation of idos_eval_idos, for callers that must not allocate device
// memory.  Its scratch (kept-site maps, tridiagonals, eigenvalues) lives in
// one file-scope static device array instead of a model's workspace, so the
// call itself performs no cudaMalloc / cudaFree and needs no model handle.
#include <cmath>
#include <mutex>
#include <string>

#include "internal.h"

namespace idos {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;   // 1 MiB on every device that loads the library
constexpr int kMaxDevices = 64;

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (host code may
// not use the symbol's host-side stand-in).  It is looked up again on every
// call whose stream is not being captured, so an address cached before a
// cudaDeviceReset (which unloads the module and may place the array
// elsewhere when it is loaded again) is never reused; a call on a capturing
// stream uses the address of the last uncaptured call on that device.
int scratch_address(cudaStream_t s, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return IDOS_ERR_NO_DEVICE;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal above the supported count");
    return IDOS_ERR_NO_DEVICE;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) {
    set_error(std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    return IDOS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
      return IDOS_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  } else if (!g_scratch_ptr[dev]) {
    set_error("idos_eval_idos_noalloc: the first call on a device must come before any stream capture");
    return IDOS_ERR_INVALID_ARG;
  }
  *out = g_scratch_ptr[dev];
  return IDOS_OK;
}

// Bump placement inside the static array (256-byte aligned pieces).
struct Carve {
  char* base;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    const size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    return reinterpret_cast<T*>(base + off);
  }
};

size_t scratch_need(int precision, int n_sites, int K2, bool own_mask, bool own_eigs) {
  Carve c{nullptr};
  const size_t ts = precision == IDOS_FP64 ? 8 : 4;
  if (own_mask) c.take<uint8_t>(n_sites);
  c.take<int>(1);
  c.take<int>(n_sites);
  c.take<int>(n_sites);
  c.take<char>(ts * (size_t)K2 * n_sites);
  c.take<char>(ts * (size_t)K2 * n_sites);
  if (own_eigs) c.take<double>((size_t)K2 * n_sites);
  return c.used;
}

int check_desc(const idos_model_desc* d) {
  auto bad = [](const char* m) { set_error(m); return IDOS_ERR_INVALID_ARG; };
  if (!d) return bad("null descriptor");
  if (d->kind != IDOS_GRAPHENE) {
    set_error("the allocation-free entry point takes the graphene model only");
    return IDOS_ERR_UNSUPPORTED;
  }
  if (d->precision != IDOS_FP64 && d->precision != IDOS_FP32_REFINE64) return bad("precision");
  if (d->smoothing != IDOS_SMOOTH_GAUSS && d->smoothing != IDOS_SMOOTH_POLY) return bad("smoothing");
  if (!(d->p >= 0.0 && d->p <= 1.0)) return bad("p must lie in [0, 1]");
  if (!(d->delta > 0.0) || !(d->e_max > d->e_min) || !(d->a > 0.0)) return bad("delta, energy range or a");
  if (d->n_E < 2 || d->n_E > 1024) return bad("n_E must lie in 2..1024");
  if (d->refine64_iters < 0 || d->refine64_iters > 64) return bad("refine64_iters must lie in 0..64");
  if (!(std::fabs(d->overlap_s) < 1.0 / 3.0) || (d->overlap_s != 0.0 && d->t == 0.0))
    return bad("overlap_s must satisfy |s| < 1/3 with a nonzero t");
  return IDOS_OK;
}

}  // namespace
}  // namespace idos

using namespace idos;

extern "C" int idos_eval_idos_noalloc(const idos_model_desc* d, int N, int Kside, const uint8_t* mask_dev,
                                      uint64_t seed, int level, int64_t sample, double* idos_dev_out,
                                      double* eigs_dev_out, void* cuda_stream) {
  IDOS_TRY(check_desc(d));
  if (!idos_dev_out) { set_error("null output"); return IDOS_ERR_INVALID_ARG; }
  if (N < 1 || N > 64 || Kside < 1 || Kside > 64 || sample < 0 || level < 0) {
    set_error("N, Kside, level or sample out of range");
    return IDOS_ERR_INVALID_ARG;
  }
  const int n_sites = 2 * N * N;
  const int K2 = Kside * Kside;
  if (!small_path_fits(d->precision, n_sites)) {
    set_error("idos_eval_idos_noalloc handles only matrices that fit the shared-memory path "
              "(2N^2 <= 160 in float32, <= 112 in float64); use idos_eval_idos");
    return IDOS_ERR_INVALID_ARG;
  }
  const size_t need = scratch_need(d->precision, n_sites, K2, mask_dev == nullptr, eigs_dev_out == nullptr);
  if (need > kNoAllocScratchBytes) {
    set_error("idos_eval_idos_noalloc needs " + std::to_string(need) + " bytes of scratch for N = " +
              std::to_string(N) + ", Kside = " + std::to_string(Kside) + "; the static scratch holds " +
              std::to_string(kNoAllocScratchBytes));
    return IDOS_ERR_INVALID_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  void* base = nullptr;
  IDOS_TRY(scratch_address(s, &base));
  Carve c{reinterpret_cast<char*>(base)};
  CellSet cells;
  cells.N = N;
  cells.n_sites = n_sites;
  cells.count = 1;
  cells.mask = mask_dev ? const_cast<uint8_t*>(mask_dev) : c.take<uint8_t>(n_sites);
  cells.n_act = c.take<int>(1);
  cells.act = c.take<int>(n_sites);
  cells.inv = c.take<int>(n_sites);
  const size_t ts = d->precision == IDOS_FP64 ? 8 : 4;
  void* dd = c.take<char>(ts * (size_t)K2 * n_sites);
  void* e2 = c.take<char>(ts * (size_t)K2 * n_sites);
  double* eigs = eigs_dev_out ? eigs_dev_out : c.take<double>((size_t)K2 * n_sites);
  if (!mask_dev) IDOS_TRY(launch_fine_masks(cells.mask, n_sites, 1, seed, level, sample, d->p, s));
  IDOS_TRY(launch_cell_maps(cells, s));
  SolveArgs a;
  a.cells = &cells;
  a.Kside = Kside;
  a.n_max = n_sites;
  a.n_mat = K2;
  a.t = d->t;
  a.eps = d->overlap_s != 0.0 ? 0.0 : d->eps_onsite;
  a.d = dd;
  a.e2 = e2;
  a.stream = s;
  IDOS_TRY(solve_small(d->precision, a));
  IDOS_TRY(launch_bisect(d->precision, d->refine64_iters, dd, e2, cells.n_act, K2, n_sites, K2, eigs, s));
  if (d->overlap_s != 0.0) IDOS_TRY(launch_overlap_map(eigs, cells.n_act, K2, n_sites, K2, d->eps_onsite, d->overlap_s / d->t, s));
  const double area = (double)N * N * cell_area(d->a);
  const EnergyGrid g{d->e_min, d->e_max, d->delta, d->n_E, d->smoothing, d->precision == IDOS_FP32_REFINE64 ? 1 : 0};
  IDOS_TRY(launch_idos(eigs, cells.n_act, K2, n_sites, 1, area, g, idos_dev_out, s));
  return IDOS_OK;
}
