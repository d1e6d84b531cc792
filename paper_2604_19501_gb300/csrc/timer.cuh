// Launch timer: CUDA event pairs around the launches of selected kernel classes, read
// back after the work completes (helm_timer_enable / helm_timer_read).
#pragma once
#include <vector>
#include "common.cuh"

namespace helm {

struct LaunchTimer {
  unsigned mask = 0;
  struct Pending { int cls; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double total_ms[HELM_K_COUNT] = {};
  long long count[HELM_K_COUNT] = {};
  cudaEvent_t get();
  void resolve();       // waits for every pending pair and accumulates it
  void reset();
  ~LaunchTimer();
};

extern thread_local LaunchTimer* g_timer;

// Records an event on s; while s is being captured into a CUDA graph the record becomes
// a graph node (an external record), so the graph's replays record the event.
inline void record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

// Records an event pair around the launches issued during its lifetime.
struct KernelTimer {
  LaunchTimer* t;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  KernelTimer(int cls_, cudaStream_t s_) : t(g_timer), cls(cls_), s(s_) {
    if (t && (t->mask >> cls & 1u)) {
      a = t->get();
      record_event(a, s);
    } else {
      t = nullptr;
    }
  }
  ~KernelTimer() {
    if (!t) return;
    cudaEvent_t b = t->get();
    record_event(b, s);
    t->pending.push_back({cls, a, b});
    if (t->pending.size() >= 4096) t->resolve();
  }
};

}  // namespace helm
