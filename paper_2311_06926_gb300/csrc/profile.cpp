#include "profile.h"

#include <atomic>
#include <vector>

namespace shp {

namespace {
std::atomic<int64_t> g_launches{0};
thread_local Profiler* t_active = nullptr;
}  // namespace

struct Profiler {
  struct Rec {
    int cls;
    cudaEvent_t start, stop;
    double flops, bytes;
  };
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  std::vector<Rec> recs;
  cudaEvent_t pending_start = nullptr;
  int pending_cls = -1;

  cudaEvent_t take() {
    if (next == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[next++];
  }
};

Profiler* profiler_create() { return new Profiler(); }

void profiler_destroy(Profiler* p) {
  if (!p) return;
  if (t_active == p) t_active = nullptr;
  for (cudaEvent_t e : p->pool) cudaEventDestroy(e);
  delete p;
}

void profiler_activate(Profiler* p) {
  t_active = p;
  if (p) {
    p->next = 0;
    p->recs.clear();
  }
}

thread_local bool t_capturing = false;

void set_capturing(bool on) { t_capturing = on; }

void launch_begin(int cls, cudaStream_t s) {
  if (!t_capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
  Profiler* p = t_active;
  if (!p) return;
  p->pending_start = p->take();
  p->pending_cls = cls;
  cudaEventRecord(p->pending_start, s);
}

void launch_end(int cls, cudaStream_t s, double flops, double bytes) {
  Profiler* p = t_active;
  if (!p || p->pending_cls != cls) return;
  cudaEvent_t stop = p->take();
  cudaEventRecord(stop, s);
  p->recs.push_back({cls, p->pending_start, stop, flops, bytes});
  p->pending_cls = -1;
}

int64_t launch_count() { return g_launches.load(); }

void launch_add(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void profiler_collect(Profiler* p, int64_t* launches, double* ms, double* flops, double* bytes) {
  for (int c = 0; c < kNumClasses; ++c) {
    launches[c] = 0;
    ms[c] = flops[c] = bytes[c] = 0.0;
  }
  if (!p) return;
  for (const auto& r : p->recs) {
    cudaEventSynchronize(r.stop);
    float t = 0.f;
    cudaEventElapsedTime(&t, r.start, r.stop);
    launches[r.cls] += 1;
    ms[r.cls] += t;
    flops[r.cls] += r.flops;
    bytes[r.cls] += r.bytes;
  }
}

}  // namespace shp
