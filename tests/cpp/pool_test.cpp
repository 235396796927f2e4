// Unit test of the library's host thread pool (g6gb_pool.h): every index of
// every run is processed exactly once, for pool sizes 1 .. 16 and for long
// series of back-to-back runs; nested and concurrent parallel_run calls fall
// back to serial loops without deadlock; a pool whose workers have gone to
// sleep on its condition variable still runs jobs (small ones on the caller
// alone) and joins on destruction.
// Exit status 0 on success; the first failure is printed.
#include "g6gb_pool.h"

#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <thread>
#include <vector>

#define CHECK(c)                                                      \
    do {                                                              \
        if (!(c)) {                                                   \
            std::fprintf(stderr, "%s:%d: %s\n", __FILE__, __LINE__, #c); \
            std::exit(1);                                             \
        }                                                             \
    } while (0)

static void once_each(g6::HostPool &p, int n)
{
    std::vector<std::atomic<int>> hit(n > 0 ? n : 1);
    for (auto &h : hit)
        h.store(0);
    p.run(n, [&](int i) {
        CHECK(i >= 0 && i < n);
        hit[i].fetch_add(1);
    });
    for (int i = 0; i < n; ++i)
        CHECK(hit[i].load() == 1);
}

int main()
{
    for (int threads : {1, 2, 4, 16}) {
        g6::HostPool p(threads);
        CHECK(p.size() == threads);
        for (int n : {0, 1, 2, 3, 17, 1000, 100000})
            once_each(p, n);
        for (int r = 0; r < 20000; ++r)          // back-to-back generations
            once_each(p, 1 + r % 7);
    }
    {
        // workers asleep on the condition variable (past their spin) wake
        // for the next job
        g6::HostPool p(4);
        once_each(p, 64);
        std::this_thread::sleep_for(std::chrono::milliseconds(100));
        once_each(p, 64);
        // a job of a few pieces posted while they sleep runs on the caller
        // alone, each index once; a larger one wakes them and still runs
        // every index once, and the pool joins afterwards
        std::this_thread::sleep_for(std::chrono::milliseconds(300));
        const std::thread::id me = std::this_thread::get_id();
        std::atomic<int> others{0};
        p.run(3, [&](int) {
            if (std::this_thread::get_id() != me)
                others.fetch_add(1);
        });
        CHECK(others.load() == 0);
        once_each(p, 3);
        std::this_thread::sleep_for(std::chrono::milliseconds(100));
        once_each(p, 1000);
    }
    {
        // nested use of the process-wide pool runs serially inside
        std::atomic<long> sum{0};
        g6::parallel_run(64, [&](int i) {
            g6::parallel_run(10, [&](int k) { sum.fetch_add(1000L * i + k); });
        });
        long want = 0;
        for (int i = 0; i < 64; ++i)
            for (int k = 0; k < 10; ++k)
                want += 1000L * i + k;
        CHECK(sum.load() == want);
    }
    {
        // two callers at once: one gets the pool, the other runs serially
        std::atomic<long> a{0}, b{0};
        std::thread t([&] {
            for (int r = 0; r < 200; ++r)
                g6::parallel_run(500, [&](int i) { a.fetch_add(i); });
        });
        for (int r = 0; r < 200; ++r)
            g6::parallel_run(500, [&](int i) { b.fetch_add(i); });
        t.join();
        CHECK(a.load() == 200L * 499 * 500 / 2);
        CHECK(b.load() == 200L * 499 * 500 / 2);
    }
    CHECK(g6::host_threads() >= 1 && g6::host_threads() <= 256);
    std::puts("pool ok");
    return 0;
}
