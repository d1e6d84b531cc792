#include "timer.cuh"

namespace helm {

thread_local LaunchTimer* g_timer = nullptr;

cudaEvent_t LaunchTimer::get() {
  if (pool.empty()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  cudaEvent_t e = pool.back();
  pool.pop_back();
  return e;
}

void LaunchTimer::resolve() {
  for (auto& p : pending) {
    float ms = 0.f;
    cudaEventSynchronize(p.b);
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      total_ms[p.cls] += ms;
      count[p.cls] += 1;
    }
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
}

void LaunchTimer::reset() {
  resolve();
  for (int i = 0; i < HELM_K_COUNT; ++i) { total_ms[i] = 0; count[i] = 0; }
}

LaunchTimer::~LaunchTimer() {
  resolve();
  for (auto e : pool) cudaEventDestroy(e);
}

}  // namespace helm
