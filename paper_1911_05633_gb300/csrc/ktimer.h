// Optional per-kernel device timing of a plan's launches.  When a plan's timer is on,
// every kernel launch of the library is bracketed by two CUDA events recorded on the
// launching stream; `collect` waits for the recorded pairs and adds each elapsed time
// to that kernel's total.  Off by default; the launches themselves are unchanged.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace gw {

class KernelTimer {
 public:
  struct Total {
    std::string name;
    double ms = 0.0;
    long long launches = 0;
  };
  bool on = false;
  std::vector<Total> totals;

  ~KernelTimer() { release(); }
  // Waits for what is pending and destroys every event (call with the plan's device current).
  void release() {
    collect();
    for (cudaEvent_t e : pool_) cudaEventDestroy(e);
    pool_.clear();
  }
  void begin(cudaStream_t st) {
    a_ = get();
    if (a_ && cudaEventRecord(a_, st) != cudaSuccess) {
      pool_.push_back(a_);
      a_ = nullptr;
    }
  }
  void end(const char* name, cudaStream_t st) {
    if (!a_) return;
    cudaEvent_t b = get();
    if (!b || cudaEventRecord(b, st) != cudaSuccess) {
      pool_.push_back(a_);
      if (b) pool_.push_back(b);
      a_ = nullptr;
      return;
    }
    pending_.push_back({name, a_, b});
    a_ = nullptr;
  }
  // Waits for every recorded pair and adds it to the totals.
  cudaError_t collect() {
    cudaError_t err = cudaSuccess;
    for (const Pending& p : pending_) {
      float ms = 0.0f;
      cudaError_t e = cudaEventSynchronize(p.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
      if (e != cudaSuccess && err == cudaSuccess) err = e;
      add(p.name, e == cudaSuccess ? ms : 0.0);
      pool_.push_back(p.a);
      pool_.push_back(p.b);
    }
    pending_.clear();
    return err;
  }
  void reset() {
    collect();
    totals.clear();
  }

 private:
  struct Pending {
    const char* name;  // a string literal at the launch site
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending_;
  std::vector<cudaEvent_t> pool_;
  cudaEvent_t a_ = nullptr;

  cudaEvent_t get() {
    if (!pool_.empty()) {
      cudaEvent_t e = pool_.back();
      pool_.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
  }
  void add(const char* name, double ms) {
    for (Total& t : totals)
      if (t.name == name) {
        t.ms += ms;
        ++t.launches;
        return;
      }
    totals.push_back({name, ms, 1});
  }
};

// The timer of the plan whose entry point runs on this thread (null when timing is off).
KernelTimer*& current_timer();

// Makes a plan's timer the current one for the scope of one entry point.
struct ActiveTimer {
  KernelTimer* prev;
  explicit ActiveTimer(KernelTimer* t) : prev(current_timer()) { current_timer() = (t && t->on) ? t : nullptr; }
  ~ActiveTimer() { current_timer() = prev; }
};

// Brackets one launch: `{ TimedLaunch tl("k_name", st); k_name<<<...>>>(...); }`.
struct TimedLaunch {
  KernelTimer* t;
  const char* name;
  cudaStream_t st;
  TimedLaunch(const char* n, cudaStream_t s) : t(current_timer()), name(n), st(s) {
    if (t) t->begin(st);
  }
  ~TimedLaunch() {
    if (t) t->end(name, st);
  }
};

}  // namespace gw
