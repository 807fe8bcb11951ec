// partition.cu - a spatial split of the GPU's SMs into two green contexts
// (CUDA driver API, resolved through the runtime's driver entry-point query,
// so the library does not link libcuda).  idos_sample_levels runs the finest
// level, whose few large matrices form long chains of small latency-bound
// launches, on one partition and the many-matrix levels on the other, so that
// the finest level's launches never wait for SMs the other levels hold.
#include <cuda.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace idos {

namespace {

struct GreenApi {
  CUresult (*device_get)(CUdevice*, int) = nullptr;
  CUresult (*get_resource)(CUdevice, CUdevResource*, CUdevResourceType) = nullptr;
  CUresult (*split)(CUdevResource*, unsigned int*, const CUdevResource*, CUdevResource*, unsigned int,
                    unsigned int) = nullptr;
  CUresult (*gen_desc)(CUdevResourceDesc*, CUdevResource*, unsigned int) = nullptr;
  CUresult (*ctx_create)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned int) = nullptr;
  CUresult (*ctx_destroy)(CUgreenCtx) = nullptr;
  CUresult (*stream_create)(CUstream*, CUgreenCtx, unsigned int, int) = nullptr;
  bool ok = false;
  const char* missing = "";
};

template <typename F>
bool resolve(const char* name, F& fn, const char*& missing) {
  missing = name;
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion(name, &p, CUDART_VERSION, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p)
    return false;
  fn = reinterpret_cast<F>(p);
  return true;
}

const GreenApi& api() {
  static std::once_flag once;
  static GreenApi g;
  std::call_once(once, [] {
    const char*& w = g.missing;
    g.ok = resolve("cuDeviceGet", g.device_get, w) && resolve("cuDeviceGetDevResource", g.get_resource, w) &&
           resolve("cuDevSmResourceSplitByCount", g.split, w) && resolve("cuDevResourceGenerateDesc", g.gen_desc, w) &&
           resolve("cuGreenCtxCreate", g.ctx_create, w) && resolve("cuGreenCtxDestroy", g.ctx_destroy, w) &&
           resolve("cuGreenCtxStreamCreate", g.stream_create, w);
    if (g.ok) w = "";
  });
  return g;
}

int fail(const char* what, CUresult r) {
  set_error(std::string("SM partition: ") + what + " failed (CUresult " + std::to_string((int)r) + ")");
  return IDOS_ERR_CUDA;
}

}  // namespace

int partition_create_new(int big_sms, SmPartition& p) {
  p = SmPartition{};
  const GreenApi& g = api();
  if (!g.ok) {
    set_error(std::string("SM partition: green-context entry points are not available from the driver (missing ") +
              g.missing + ")");
    return IDOS_ERR_UNSUPPORTED;
  }
  int ordinal = 0;
  IDOS_CUDA_TRY(cudaGetDevice(&ordinal));
  CUdevice dev;
  CUresult r = g.device_get(&dev, ordinal);
  if (r != CUDA_SUCCESS) return fail("cuDeviceGet", r);
  CUdevResource all;
  r = g.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM);
  if (r != CUDA_SUCCESS) return fail("cuDeviceGetDevResource", r);
  const int align = (int)std::max(1u, all.sm.smCoscheduledAlignment);
  int want = (big_sms + align - 1) / align * align;
  want = std::max<int>(want, (int)all.sm.minSmPartitionSize);
  if (want >= (int)all.sm.smCount) {
    set_error("SM partition: the reserved part must leave SMs for the rest");
    return IDOS_ERR_INVALID_ARG;
  }
  CUdevResource grp[1], rest;
  unsigned int nb = 1;
  r = g.split(grp, &nb, &all, &rest, 0, (unsigned int)want);
  if (r != CUDA_SUCCESS || nb != 1) return fail("cuDevSmResourceSplitByCount", r);
  CUdevResourceDesc d0, d1;
  r = g.gen_desc(&d0, grp, 1);
  if (r != CUDA_SUCCESS) return fail("cuDevResourceGenerateDesc", r);
  r = g.gen_desc(&d1, &rest, 1);
  if (r != CUDA_SUCCESS) return fail("cuDevResourceGenerateDesc", r);
  CUgreenCtx c0 = nullptr, c1 = nullptr;
  r = g.ctx_create(&c0, d0, dev, CU_GREEN_CTX_DEFAULT_STREAM);
  if (r != CUDA_SUCCESS) return fail("cuGreenCtxCreate", r);
  r = g.ctx_create(&c1, d1, dev, CU_GREEN_CTX_DEFAULT_STREAM);
  if (r != CUDA_SUCCESS) {
    g.ctx_destroy(c0);
    return fail("cuGreenCtxCreate", r);
  }
  p.ctx[0] = c0;
  p.ctx[1] = c1;
  p.sms[0] = (int)grp[0].sm.smCount;
  p.sms[1] = (int)rest.sm.smCount;
  return IDOS_OK;
}

// The SM count a partition of `big_sms` SMs rounds up to on this device (the
// driver's co-scheduling alignment and minimum partition size); big_sms when
// green contexts are not available.
int partition_rounded(int big_sms) {
  const GreenApi& g = api();
  if (!g.ok || big_sms <= 0) return big_sms;
  int ordinal = 0;
  if (cudaGetDevice(&ordinal) != cudaSuccess) return big_sms;
  CUdevice dev;
  CUdevResource all;
  if (g.device_get(&dev, ordinal) != CUDA_SUCCESS || g.get_resource(dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS)
    return big_sms;
  const int align = (int)std::max(1u, all.sm.smCoscheduledAlignment);
  return std::max<int>((big_sms + align - 1) / align * align, (int)all.sm.minSmPartitionSize);
}

// One partition per (device, reserved SM count), created on first use and
// kept for the life of the process: kernels are loaded into a context on
// their first launch there, so models created later reuse warm contexts.
int partition_create(int big_sms, SmPartition& p) {
  struct Entry {
    int dev, sms;
    SmPartition part;
  };
  static std::mutex mu;
  static Entry cache[64];
  static int n_cached = 0;
  int dev = 0;
  IDOS_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < n_cached; ++i) {
    if (cache[i].dev == dev && cache[i].sms == big_sms) {
      p = cache[i].part;
      return IDOS_OK;
    }
  }
  IDOS_TRY(partition_create_new(big_sms, p));
  if (n_cached < 64) {
    p.shared = true;   // the cache keeps it; a full cache leaves it to the model
    cache[n_cached++] = Entry{dev, big_sms, p};
  }
  return IDOS_OK;
}

int partition_stream(const SmPartition& p, int which, int priority, cudaStream_t* out) {
  CUstream s = nullptr;
  const CUresult r =
      api().stream_create(&s, reinterpret_cast<CUgreenCtx>(p.ctx[which]), CU_STREAM_NON_BLOCKING, priority);
  if (r != CUDA_SUCCESS) return fail("cuGreenCtxStreamCreate", r);
  *out = reinterpret_cast<cudaStream_t>(s);
  return IDOS_OK;
}

void partition_destroy(SmPartition& p) {
  for (int i = 0; i < 2; ++i) {
    if (p.ctx[i] && !p.shared) api().ctx_destroy(reinterpret_cast<CUgreenCtx>(p.ctx[i]));
    p.ctx[i] = nullptr;
  }
}

}  // namespace idos
