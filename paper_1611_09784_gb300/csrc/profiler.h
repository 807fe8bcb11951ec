// profiler.h - optional per-kernel timing with CUDA events.  When a model has
// profiling enabled, every launch site brackets its kernel with an event pair
// on the launching stream; the pairs are resolved after the API call's final
// synchronisation and accumulated per kernel family.  In timeline mode the
// levels keep their own streams and SM partitions, and every pair is also kept
// as a trace entry (start and end relative to an origin event recorded when the
// call was issued, and the stream it ran on).
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace idos {

enum KernelId {
  KID_MASKS = 0, KID_CORNERS, KID_CELL_MAPS, KID_SMALL_TRIDIAG, KID_LG_ASSEMBLE, KID_LG_BAND, KID_LG_PANEL, KID_LG_W, KID_LG_Z, KID_LG_HER2K, KID_LG_CHASE,
  KID_BISECT, KID_IDOS, KID_LEVEL_STATS, KID_COUNT
};

const char* kernel_name(int kid);

struct TraceEntry {
  int kid;        // kernel family
  int lane;       // index of the stream in order of first use within the call
  int launches;   // kernel launches inside the pair (0: an aggregating scope)
  float t0, t1;   // ms after the call's origin event
};

struct Profiler {
  bool enabled = false;
  bool timeline = false;            // concurrent streams + trace (else one serial stream)
  cudaEvent_t origin = nullptr;     // recorded when a traced call is issued
  bool origin_set = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> pending_kid;     // kid of pair i (events 2i, 2i+1)
  std::vector<int> pending_n;       // kernel launches inside pair i
  std::vector<cudaStream_t> pending_stream;
  std::vector<TraceEntry> trace;    // entries of the last traced call
  double ms[KID_COUNT] = {};
  long long launches[KID_COUNT] = {};   // kernel launches (not scopes)
  int begin(int kid, cudaStream_t s, int n_launch);   // returns the pair index or -1
  void end(int pair, cudaStream_t s);
  int mark_origin(cudaStream_t s);   // starts a traced call (clears the trace)
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
