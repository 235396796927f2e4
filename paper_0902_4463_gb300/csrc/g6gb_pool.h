// g6gb_pool.h -- one persistent pool of host threads for the library's
// per-particle and per-cluster host loops (prediction of the active
// i-particles, correction, staging, copies of large blocks).  Internal to the
// library.
#pragma once

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdlib>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace g6 {

// Persistent host worker pool: run(n, f) calls f(0..n-1) on the workers and
// the calling thread and returns when all calls have finished.  A job is
// published by writing it and then advancing the generation counter
// (release); a worker that sees the new generation (acquire) reads the job
// without a lock.  Workers wait for the next job by spinning on the counter
// for a short while (a block step posts several jobs tens of microseconds
// apart), then by yielding, then sleep on a condition variable; the caller
// wakes sleepers only when there are any.  A job of a few pieces posted
// while workers sleep runs on the caller alone: the job is complete only
// when every worker has seen it, so it would wait for all of them to wake.
class HostPool {
public:
    explicit HostPool(int threads)
    {
        for (int i = 1; i < threads; ++i)
            th_.emplace_back([this] { worker(); });
    }
    ~HostPool()
    {
        quit_.store(true, std::memory_order_seq_cst);
        gen_.fetch_add(1, std::memory_order_seq_cst);
        {
            std::lock_guard<std::mutex> lk(mu_);
        }
        cv_.notify_all();
        for (std::thread &t : th_)
            t.join();
    }
    int size() const { return (int)th_.size() + 1; }
    void run(int n, const std::function<void(int)> &f)
    {
        if (th_.empty() || n <= 1
            || (n < WAKE_MIN && sleepers_.load(std::memory_order_relaxed) > 0)) {
            for (int i = 0; i < n; ++i)
                f(i);
            return;
        }
        // every worker has finished the previous job (busy_ reached 0), so
        // none still reads job_ or count_
        job_ = &f;
        count_ = n;
        grab_ = std::max(1, n / (8 * size()));     // indices taken per claim
        next_.store(0, std::memory_order_relaxed);
        busy_.store((int)th_.size(), std::memory_order_relaxed);
        gen_.fetch_add(1, std::memory_order_seq_cst);
        if (sleepers_.load(std::memory_order_seq_cst) > 0) {
            std::lock_guard<std::mutex> lk(mu_);
            cv_.notify_all();
        }
        take(f, n, grab_);
        for (int spins = 0; busy_.load(std::memory_order_acquire) != 0;)
            if (++spins > SPIN_TIGHT)
                std::this_thread::yield();
    }

private:
    static constexpr int SPIN_TIGHT = 20000;   // polls before yielding (tens of us)
    static constexpr int SPIN_YIELD = 2000;    // yields before sleeping
    static constexpr int WAKE_MIN = 8;         // pieces worth waking sleepers for

    // claim indices `grab` at a time until none are left
    void take(const std::function<void(int)> &f, int n, int grab)
    {
        for (int i; (i = next_.fetch_add(grab, std::memory_order_relaxed)) < n;)
            for (int k = i, ke = std::min(n, i + grab); k < ke; ++k)
                f(k);
    }

    // Workers are started before any run(), when the generation is 0.
    void worker()
    {
        unsigned seen = 0;
        for (;;) {
            unsigned g;
            int spins = 0;
            while ((g = gen_.load(std::memory_order_acquire)) == seen) {
                ++spins;
                if (spins <= SPIN_TIGHT)
                    continue;
                if (spins <= SPIN_TIGHT + SPIN_YIELD) {
                    std::this_thread::yield();
                    continue;
                }
                // sleep until the generation moves (the caller notifies when
                // it sees a sleeper; the predicate is checked after the
                // sleeper count is raised, so no wake-up is lost)
                sleepers_.fetch_add(1, std::memory_order_seq_cst);
                {
                    std::unique_lock<std::mutex> lk(mu_);
                    cv_.wait(lk, [&] { return gen_.load(std::memory_order_seq_cst) != seen; });
                }
                sleepers_.fetch_sub(1, std::memory_order_seq_cst);
                spins = 0;
            }
            seen = g;
            if (quit_.load(std::memory_order_acquire))
                return;
            take(*job_, count_, grab_);
            busy_.fetch_sub(1, std::memory_order_release);
        }
    }
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_;
    std::atomic<unsigned> gen_{0};
    std::atomic<int> next_{0}, busy_{0}, sleepers_{0};
    std::atomic<bool> quit_{false};
    const std::function<void(int)> *job_ = nullptr;
    int count_ = 0, grab_ = 1;
};

inline int host_threads()
{
    if (const char *e = std::getenv("G6GB_HOST_THREADS")) {
        const int n = std::atoi(e);
        if (n >= 1)
            return std::min(n, 256);
    }
    const unsigned hw = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(hw, 16u));
}

// The process-wide pool (started on first use; NULL if threads cannot be
// started).
inline HostPool *shared_pool()
{
    static std::unique_ptr<HostPool> pool;
    static std::once_flag once;
    std::call_once(once, [] {
        try {
            pool.reset(new HostPool(host_threads()));
        } catch (...) {
            pool.reset();
        }
    });
    return pool.get();
}

// f(0 .. n-1) on the process-wide pool; serially when the pool is in use by
// another caller (or by this one: nested calls), has no threads, or n < 2.
inline void parallel_run(int n, const std::function<void(int)> &f)
{
    static std::mutex busy;
    std::unique_lock<std::mutex> lk(busy, std::try_to_lock);
    HostPool *p = n > 1 && lk.owns_lock() ? shared_pool() : nullptr;
    if (!p) {
        for (int i = 0; i < n; ++i)
            f(i);
        return;
    }
    p->run(n, f);
}

}  // namespace g6
