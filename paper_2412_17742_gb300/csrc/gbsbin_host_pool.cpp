// A small persistent pool of host threads for the FP64 state algebra (the per-state work of
// gbsbin_plan_create / gbsbin_plan_set_state: the output covariance, two Cholesky
// factorisations, a triangular inverse and a Gram product, O(n^3) each).  Portable C++
// threads only.  Workers spin for a short while after each job (the algebra dispatches a
// few dozen jobs back to back) and then sleep on a condition variable; one job runs at a
// time (callers from several threads take turns).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include <unistd.h>

#include "gbsbin_host_state.h"

namespace gbsbin {
namespace {

class Pool {
 public:
  explicit Pool(int workers) {
    for (int t = 0; t < workers; ++t) threads_.emplace_back([this, t] { loop(t + 1); });
  }
  int size() const { return (int)threads_.size() + 1; }

  void run(int nthreads, const std::function<void(int, int)>& fn) {
    std::lock_guard<std::mutex> turn(run_m_);
    nthreads = std::max(1, std::min(nthreads, size()));
    if (nthreads == 1 || getpid() != pid_) {        // a forked child has no workers
      fn(0, 1);
      return;
    }
    {
      std::lock_guard<std::mutex> lk(m_);
      job_ = &fn;
      active_ = nthreads;
      pending_.store(nthreads - 1);
      gen_.fetch_add(1);
    }
    cv_.notify_all();
    fn(0, nthreads);
    while (pending_.load(std::memory_order_acquire) != 0) std::this_thread::yield();
  }

 private:
  void loop(int t) {
    unsigned long long seen = 0;                     // the generation at construction: a job
                                                     // posted before this thread started still runs
    for (;;) {
      // spin briefly for the next job, then sleep
      const auto t0 = std::chrono::steady_clock::now();
      while (gen_.load(std::memory_order_acquire) == seen &&
             std::chrono::steady_clock::now() - t0 < std::chrono::microseconds(300))
        std::this_thread::yield();
      if (gen_.load(std::memory_order_acquire) == seen) {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_.load() != seen; });
      }
      const std::function<void(int, int)>* job;
      int active;
      {
        std::lock_guard<std::mutex> lk(m_);
        seen = gen_.load();
        job = job_;
        active = active_;
      }
      if (t < active) {
        (*job)(t, active);
        pending_.fetch_sub(1, std::memory_order_release);
      }
    }
  }

  std::vector<std::thread> threads_;
  const pid_t pid_ = getpid();
  std::mutex m_, run_m_;
  std::condition_variable cv_;
  std::atomic<unsigned long long> gen_{0};
  std::atomic<int> pending_{0};
  const std::function<void(int, int)>* job_ = nullptr;
  int active_ = 0;
};

// Never destroyed: its workers are blocked or spinning when the process exits, and a
// destructor would have to join threads that a forked child does not have.
Pool& pool() {
  static Pool* p = new Pool(host_threads() - 1);
  return *p;
}

}  // namespace

int host_threads() {
  static const int n = [] {
    int v = (int)std::thread::hardware_concurrency();
    if (const char* e = std::getenv("GBSBIN_HOST_THREADS")) v = std::atoi(e);
    return std::max(1, std::min(v, 16));
  }();
  return n;
}

void parallel_run(int nthreads, const std::function<void(int, int)>& fn) { pool().run(nthreads, fn); }

}  // namespace gbsbin
