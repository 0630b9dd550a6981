#include "host_pool.hpp"

#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <exception>
#include <mutex>
#include <thread>
#include <vector>

namespace dmrg {
namespace {

class Pool {
 public:
  Pool() : pid_(getpid()) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned nw = std::min(16u, hw) - 1;
    for (unsigned w = 0; w < nw; ++w) workers_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> lk(m_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : workers_) t.join();
  }
  unsigned threads() const { return (unsigned)workers_.size() + 1; }

  void run(size_t n, const std::function<void(size_t)>& fn) {
    if (n == 0) return;
    // one job at a time; a concurrent caller, a caller inside a job, or a
    // forked child (whose copy of the pool has no threads) runs serially
    bool idle = false;
    if (workers_.empty() || getpid() != pid_ || n == 1 || !busy_.compare_exchange_strong(idle, true)) {
      for (size_t i = 0; i < n; ++i) fn(i);
      return;
    }
    struct Release {
      std::atomic<bool>& b;
      ~Release() { b.store(false); }
    } release{busy_};
    {
      std::lock_guard<std::mutex> lk(m_);
      fn_ = &fn;
      n_ = n;
      next_.store(0);
      active_ = (int)workers_.size();
      err_ = nullptr;
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> lk(m_);
    done_cv_.wait(lk, [this] { return active_ == 0; });
    fn_ = nullptr;
    if (err_) std::rethrow_exception(err_);
  }

 private:
  void work() {
    for (;;) {
      const size_t i = next_.fetch_add(1);
      if (i >= n_) return;
      try {
        (*fn_)(i);
      } catch (...) {
        std::lock_guard<std::mutex> lk(m_);
        if (!err_) err_ = std::current_exception();
        next_.store(n_);
      }
    }
  }
  void loop() {
    unsigned long long seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
      }
      work();
      {
        std::lock_guard<std::mutex> lk(m_);
        if (--active_ == 0) done_cv_.notify_one();
      }
    }
  }

  const pid_t pid_;
  std::vector<std::thread> workers_;
  std::mutex m_;
  std::atomic<bool> busy_{false};
  std::condition_variable cv_, done_cv_;
  const std::function<void(size_t)>* fn_ = nullptr;
  size_t n_ = 0;
  std::atomic<size_t> next_{0};
  int active_ = 0;
  unsigned long long gen_ = 0;
  bool stop_ = false;
  std::exception_ptr err_;
};

// Created on first use and never destroyed: idle workers end with the
// process, and a forked child (whose copy of the pool has no threads, see
// run) never joins threads it does not have.
Pool& pool() {
  static Pool* p = new Pool();
  return *p;
}

}  // namespace

void host_parallel_for(size_t n, const std::function<void(size_t)>& fn) { pool().run(n, fn); }

unsigned host_threads() { return pool().threads(); }

}  // namespace dmrg
