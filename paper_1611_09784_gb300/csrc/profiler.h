// profiler.h - optional per-kernel timing with CUDA events.  When a model has
// profiling enabled, every launch site brackets its kernel with an event pair
// on the launching stream; the pairs are resolved after the API call's final
// synchronisation and accumulated per kernel family.
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace idos {

enum KernelId {
  KID_MASKS = 0, KID_CORNERS, KID_CELL_MAPS, KID_SMALL_TRIDIAG, KID_LG_ASSEMBLE, KID_LG_BAND, KID_LG_PANEL, KID_LG_W, KID_LG_Z, KID_LG_HER2K, KID_LG_CHASE,
  KID_BISECT, KID_IDOS, KID_LEVEL_STATS, KID_COUNT
};

const char* kernel_name(int kid);

struct Profiler {
  bool enabled = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> pending_kid;     // kid of pair i (events 2i, 2i+1)
  std::vector<int> pending_n;       // kernel launches inside pair i
  double ms[KID_COUNT] = {};
  long long launches[KID_COUNT] = {};   // kernel launches (not scopes)
  int begin(int kid, cudaStream_t s, int n_launch);   // returns the pair index or -1
  void end(int pair, cudaStream_t s);
  void resolve();                    // call after the stream has been synchronised
  void clear();
  ~Profiler();
};

// The profiler of the model whose API call is running on this thread (or null).
Profiler* active_profiler();
void set_active_profiler(Profiler* p);

// Times the launches issued while it lives; n_launch = how many kernels they
// are (0 for a scope that only aggregates scopes nested inside it).
struct ProfScope {
  int pair = -1;
  cudaStream_t s;
  ProfScope(int kid, cudaStream_t st, int n_launch = 1) : s(st) {
    Profiler* p = active_profiler();
    if (p && p->enabled) pair = p->begin(kid, st, n_launch);
  }
  ~ProfScope() {
    Profiler* p = active_profiler();
    if (p && pair >= 0) p->end(pair, s);
  }
};

}  // namespace idos
