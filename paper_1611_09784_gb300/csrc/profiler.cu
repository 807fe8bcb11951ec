// profiler.cu - event-pair pool behind profiler.h.
#include "profiler.h"

namespace idos {

static thread_local Profiler* g_active = nullptr;
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
  if (cudaEventRecord(pool[2 * pair], s) != cudaSuccess) return -1;
  pending_kid.push_back(kid);
  pending_n.push_back(n_launch);
  return (int)pair;
}

void Profiler::end(int pair, cudaStream_t s) { cudaEventRecord(pool[2 * pair + 1], s); }

void Profiler::resolve() {
  for (size_t i = 0; i < pending_kid.size(); ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) == cudaSuccess) {
      ms[pending_kid[i]] += t;
      launches[pending_kid[i]] += pending_n[i];
    }
  }
  pending_kid.clear();
  pending_n.clear();
}

void Profiler::clear() {
  pending_kid.clear();
  pending_n.clear();
  for (int k = 0; k < KID_COUNT; ++k) { ms[k] = 0; launches[k] = 0; }
}

Profiler::~Profiler() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

}  // namespace idos
