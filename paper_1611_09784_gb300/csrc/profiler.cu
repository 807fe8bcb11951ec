// profiler.cu - event-pair pool behind profiler.h.
#include "profiler.h"

namespace idos {

static thread_local Profiler* g_active = nullptr;

// Inside a stream capture a plain event record only orders streams; the
// external flag makes it a node of the graph that records a timestamp.
static cudaError_t record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t err = cudaStreamIsCapturing(s, &cs);
  if (err != cudaSuccess) return err;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                             : cudaEventRecord(e, s);
}
Profiler* active_profiler() { return g_active; }
void set_active_profiler(Profiler* p) { g_active = p; }

const char* kernel_name(int kid) {
  static const char* names[KID_COUNT] = {
      "k_fine_masks", "k_corner_masks", "k_cell_maps", "k_small_tridiag", "k_lg_assemble", "k_lg_band (stage 1, all)", "k_ts_panel", "k_ts_w", "k_ts_z", "k_ts_her2k", "k_ts_chase",
      "k_bisect", "k_idos", "k_level_stats"};
  return (kid >= 0 && kid < KID_COUNT) ? names[kid] : "?";
}

int Profiler::begin(int kid, cudaStream_t s, int n_launch) {
  const size_t pair = pending_kid.size();
  while (pool.size() < 2 * (pair + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    pool.push_back(e);
  }
  if (record_event(pool[2 * pair], s) != cudaSuccess) return -1;
  pending_kid.push_back(kid);
  pending_n.push_back(n_launch);
  pending_stream.push_back(s);
  return (int)pair;
}

int Profiler::mark_origin(cudaStream_t s) {
  if (!origin && cudaEventCreate(&origin) != cudaSuccess) {
    origin = nullptr;
    return -1;
  }
  trace.clear();
  origin_set = cudaEventRecord(origin, s) == cudaSuccess;
  return origin_set ? 0 : -1;
}

void Profiler::end(int pair, cudaStream_t s) { record_event(pool[2 * pair + 1], s); }

void Profiler::resolve() {
  std::vector<cudaStream_t> lanes;
  for (size_t i = 0; i < pending_kid.size(); ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) == cudaSuccess) {
      ms[pending_kid[i]] += t;
      launches[pending_kid[i]] += pending_n[i];
    }
    float a = 0.f, b = 0.f;
    if (origin_set && cudaEventElapsedTime(&a, origin, pool[2 * i]) == cudaSuccess &&
        cudaEventElapsedTime(&b, origin, pool[2 * i + 1]) == cudaSuccess) {
      int lane = 0;
      while (lane < (int)lanes.size() && lanes[lane] != pending_stream[i]) ++lane;
      if (lane == (int)lanes.size()) lanes.push_back(pending_stream[i]);
      trace.push_back(TraceEntry{pending_kid[i], lane, pending_n[i], a, b});
    }
  }
  origin_set = false;
  pending_kid.clear();
  pending_n.clear();
  pending_stream.clear();
}

void Profiler::clear() {
  pending_kid.clear();
  pending_n.clear();
  pending_stream.clear();
  trace.clear();
  for (int k = 0; k < KID_COUNT; ++k) { ms[k] = 0; launches[k] = 0; }
}

Profiler::~Profiler() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
  if (origin) cudaEventDestroy(origin);
}

}  // namespace idos
