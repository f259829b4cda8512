// Persistent worker threads behind dgl::parallel_ranges (see host_pool.hpp).
//
// A regrid runs about ten short loops back to back.  After each job a helper polls the job
// counter for a short while before it sleeps on the condition variable, so the loops after the
// first find the helpers awake; the first loop of a regrid pays the wake-up.
#include "host_pool.hpp"

#include <pthread.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>

namespace dgl {
namespace {

constexpr auto kPollTime = std::chrono::microseconds(300);

class WorkerPool {
 public:
  explicit WorkerPool(int helpers) : pid_(getpid()), helpers_(helpers) {
    // detached: the pool lives until the process ends and is never destroyed, so no thread
    // object needs joining at exit
    for (int i = 0; i < helpers_; ++i) std::thread([this, i] { loop(i); }).detach();
  }
  pid_t pid() const { return pid_; }
  int helpers() const { return helpers_; }

  // Runs job(t) for t in [0, nt) with t = 0 on the calling thread; false if the pool is busy.
  bool run(int nt, const std::function<void(int)>& job) {
    std::unique_lock<std::mutex> busy(run_mu_, std::try_to_lock);
    if (!busy.owns_lock()) return false;
    {
      std::lock_guard<std::mutex> lk(mu_);
      job_ = &job;
      active_ = nt - 1;
      // every helper acknowledges every job, so job_ and active_ stay fixed until the last
      // helper is done reading them
      pending_.store(helpers_, std::memory_order_relaxed);
      gen_.fetch_add(1, std::memory_order_release);   // publishes job_ and active_
    }
    cv_.notify_all();
    job(0);
    if (!poll([this] { return pending_.load(std::memory_order_acquire) == 0; })) {
      std::unique_lock<std::mutex> lk(mu_);
      done_.wait(lk, [this] { return pending_.load(std::memory_order_acquire) == 0; });
    }
    return true;
  }

 private:
  // Polls `ready` for up to kPollTime; true once it holds.
  template <class F>
  static bool poll(F ready) {
    const auto t0 = std::chrono::steady_clock::now();
    for (int i = 1;; ++i) {
      if (ready()) return true;
      if ((i & 255) == 0 && std::chrono::steady_clock::now() - t0 > kPollTime) return false;
    }
  }

  void loop(int id) {
    uint64_t seen = 0;
    for (;;) {
      if (!poll([&] { return gen_.load(std::memory_order_acquire) != seen; })) {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != seen; });
      }
      seen = gen_.load(std::memory_order_acquire);
      if (id < active_) (*job_)(id + 1);
      if (pending_.fetch_sub(1, std::memory_order_acq_rel) == 1) {
        // taking the mutex orders this wake-up after the caller's last check of pending_
        { std::lock_guard<std::mutex> lk(mu_); }
        done_.notify_one();
      }
    }
  }

  const pid_t pid_;
  const int helpers_;
  std::mutex run_mu_;            // one job at a time
  std::mutex mu_;                // sleeping on cv_ / done_
  std::condition_variable cv_, done_;
  const std::function<void(int)>* job_ = nullptr;
  int active_ = 0;
  std::atomic<uint64_t> gen_{0};
  std::atomic<int> pending_{0};
};

std::mutex g_pool_mu;
WorkerPool* g_pool = nullptr;

// fork() copies g_pool_mu in whatever state it has at that moment: were another thread inside
// pool(), the child would inherit a mutex that no thread of its own ever releases.  The handlers
// take it around fork(), so both processes resume with it free.  (The child never touches the
// parent's pool object or its mutexes: it builds a pool of its own.)
void fork_prepare() { g_pool_mu.lock(); }
void fork_release() { g_pool_mu.unlock(); }
const int g_atfork = pthread_atfork(fork_prepare, fork_release, fork_release);

WorkerPool* pool() {
  (void)g_atfork;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  // a forked child inherits the pool object but none of its threads: it starts a new one (the
  // parent's copy is left in place, unused)
  if (!g_pool || g_pool->pid() != getpid()) {
    const unsigned hc = std::max(1u, std::thread::hardware_concurrency());
    g_pool = new WorkerPool((int)std::min(16u, hc) - 1);
  }
  return g_pool;
}

}  // namespace

void parallel_ranges(int64_t n, int64_t grain, const std::function<void(int64_t, int64_t)>& fn) {
  if (n <= 0) return;
  grain = std::max<int64_t>(grain, 1);
  WorkerPool* p = pool();
  const int64_t want = std::min<int64_t>(p->helpers() + 1, (n + grain - 1) / grain);
  const int nt = (int)std::max<int64_t>(want, 1);
  if (nt > 1) {
    auto part = [&](int t) { fn(n * t / nt, n * (t + 1) / nt); };
    if (p->run(nt, part)) return;
  }
  fn(0, n);
}

int64_t exclusive_scan(int64_t* cnt, int64_t n) {
  int64_t s = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t c = cnt[i];
    cnt[i] = s;
    s += c;
  }
  return s;
}

}  // namespace dgl
