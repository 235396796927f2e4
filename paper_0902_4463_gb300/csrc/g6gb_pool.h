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
// the calling thread and returns when all calls have finished.  Workers spin
// briefly for the next job, then sleep on a condition variable.
class HostPool {
public:
    explicit HostPool(int threads)
    {
        for (int i = 1; i < threads; ++i)
            th_.emplace_back([this] { worker(); });
    }
    ~HostPool()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            quit_ = true;
            gen_.fetch_add(1);
        }
        cv_.notify_all();
        for (std::thread &t : th_)
            t.join();
    }
    int size() const { return (int)th_.size() + 1; }
    void run(int n, const std::function<void(int)> &f)
    {
        if (th_.empty() || n <= 1) {
            for (int i = 0; i < n; ++i)
                f(i);
            return;
        }
        {
            std::lock_guard<std::mutex> lk(mu_);
            job_ = &f;
            count_ = n;
            next_.store(0);
            busy_.store((int)th_.size());
            gen_.fetch_add(1);
        }
        cv_.notify_all();
        for (int i; (i = next_.fetch_add(1)) < n;)
            f(i);
        while (busy_.load() != 0)
            std::this_thread::yield();
    }

private:
    // Workers are started before any run(), when the generation is 0.
    void worker()
    {
        unsigned seen = 0;
        for (;;) {
            int spins = 0;
            while (gen_.load() == seen && ++spins < 4096)
                std::this_thread::yield();
            if (gen_.load() == seen) {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return gen_.load() != seen; });
            }
            seen = gen_.load();
            const std::function<void(int)> *f;
            int n;
            {
                std::lock_guard<std::mutex> lk(mu_);
                if (quit_)
                    return;
                f = job_;
                n = count_;
            }
            for (int i; (i = next_.fetch_add(1)) < n;)
                (*f)(i);
            busy_.fetch_sub(1);
        }
    }
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_;
    std::atomic<unsigned> gen_{0};
    std::atomic<int> next_{0}, busy_{0};
    const std::function<void(int)> *job_ = nullptr;
    int count_ = 0;
    bool quit_ = false;
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
