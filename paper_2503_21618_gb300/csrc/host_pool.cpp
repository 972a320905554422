// Process-wide host worker pools for the setup steps.
#include "host_pool.h"

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdlib>
#include <exception>
#include <mutex>
#include <thread>
#include <vector>

#include <unistd.h>

namespace slrf {

namespace {

int thread_cap() {
    static const int cap = [] {
        const unsigned hc = std::thread::hardware_concurrency();
        int t = (int)std::min<unsigned>(hc ? hc : 1, 16u);
        if (const char *env = std::getenv("SLRF_HOST_THREADS")) {
            const int v = std::atoi(env);
            if (v >= 1) t = std::min(v, 64);
        }
        return t;
    }();
    return cap;
}

// Iterations of a waiting loop before it sleeps: a few tens of microseconds,
// about the gap between two steps of a setup.
constexpr int kSpin = 20000;

// Workers 1 .. size()-1 wait for a job (a generation number, the function and
// the team size, published together under the mutex), run their member of
// it and count down; the caller runs member 0 and waits for the count.
class Pool {
  public:
    explicit Pool(int workers) {
        for (int i = 0; i < workers; ++i) {
            try {
                std::thread([this, id = i + 1] { loop(id); }).detach();
                ++size_;
            } catch (...) {   // fewer workers: larger teams start their own threads
                break;
            }
        }
    }
    int size() const { return size_; }
    bool try_acquire() { return busy_.try_lock(); }
    void release() { busy_.unlock(); }

    void run(int nt, const std::function<void(int)> &fn) {
        {
            std::lock_guard<std::mutex> lk(m_);
            job_ = &fn;
            nt_ = nt;
            left_.store(nt - 1, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_release);
        }
        cv_work_.notify_all();
        try {   // a member that fails: the others still finish first
            fn(0);
        } catch (...) {
            keep(std::current_exception());
        }
        for (int i = 0; left_.load(std::memory_order_acquire) != 0; ++i)
            if (i >= kSpin) {
                std::unique_lock<std::mutex> lk(m_);
                cv_done_.wait(lk, [&] { return left_.load(std::memory_order_acquire) == 0; });
                break;
            }
        std::exception_ptr ex;
        {
            std::lock_guard<std::mutex> lk(m_);
            ex = ex_;
            ex_ = nullptr;
        }
        if (ex) std::rethrow_exception(ex);
    }

  private:
    void keep(std::exception_ptr e) {   // the first failure of a job
        std::lock_guard<std::mutex> lk(m_);
        if (!ex_) ex_ = e;
    }

    void loop(int id) {
        int64_t seen = 0;
        for (;;) {
            for (int i = 0; i < kSpin && gen_.load(std::memory_order_acquire) == seen; ++i) {
            }
            const std::function<void(int)> *f;
            int nt;
            {
                std::unique_lock<std::mutex> lk(m_);
                cv_work_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != seen; });
                seen = gen_.load(std::memory_order_acquire);
                f = job_;
                nt = nt_;
            }
            if (id >= nt) continue;
            try {
                (*f)(id);
            } catch (...) {
                keep(std::current_exception());
            }
            if (left_.fetch_sub(1, std::memory_order_acq_rel) == 1) {
                std::lock_guard<std::mutex> lk(m_);
                cv_done_.notify_all();
            }
        }
    }

    std::mutex busy_;   // held by the caller whose job the pool runs
    std::mutex m_;
    std::condition_variable cv_work_, cv_done_;
    std::atomic<int64_t> gen_{0};
    std::atomic<int> left_{0};
    const std::function<void(int)> *job_ = nullptr;
    std::exception_ptr ex_;
    int nt_ = 0;
    int size_ = 1;
};

// Two pools (the multigrid setup thread and the thread that creates the
// handle run steps at the same time), created on first use and again in a
// forked child, whose copies have no workers.  Pools are never destroyed:
// their workers wait for the life of the process.
constexpr int kPools = 2;
std::mutex g_pools_m;
Pool *g_pools[kPools] = {nullptr, nullptr};
pid_t g_pools_pid = 0;

Pool *acquire_pool(int nt) {
    std::lock_guard<std::mutex> lk(g_pools_m);
    const pid_t pid = getpid();
    if (pid != g_pools_pid) {
        for (auto &p : g_pools) p = nullptr;   // a forked child: the parent's workers are not here
        g_pools_pid = pid;
    }
    for (auto &p : g_pools) {
        if (!p) p = new Pool(thread_cap() - 1);
        if (p->size() >= nt && p->try_acquire()) return p;
    }
    return nullptr;
}

}  // namespace

int host_threads(int64_t work) { return work < 32768 ? 1 : thread_cap(); }

void host_team(int nt, const std::function<void(int)> &fn) {
    if (nt <= 1) {
        fn(0);
        return;
    }
    if (Pool *p = acquire_pool(nt)) {
        struct Release {
            Pool *p;
            ~Release() { p->release(); }
        } rel{p};
        p->run(nt, fn);
        return;
    }
    // threads of the caller's own: they start the job together once all of
    // them exist (a team whose members wait on one another must not start
    // short of a member); a failure to start one, or of any member, is
    // rethrown here after every started thread has returned
    std::atomic<int> go{0};   // 0 wait, 1 run, 2 give up
    std::mutex em;
    std::exception_ptr ex;
    auto keep = [&](std::exception_ptr e) {
        std::lock_guard<std::mutex> lk(em);
        if (!ex) ex = e;
    };
    std::vector<std::thread> th;
    try {
        for (int t = 1; t < nt; ++t)
            th.emplace_back([&, t] {
                int g;
                while ((g = go.load(std::memory_order_acquire)) == 0) std::this_thread::yield();
                if (g != 1) return;
                try {
                    fn(t);
                } catch (...) {
                    keep(std::current_exception());
                }
            });
    } catch (...) {
        keep(std::current_exception());
    }
    const bool all = (int)th.size() == nt - 1;
    go.store(all ? 1 : 2, std::memory_order_release);
    if (all) {
        try {
            fn(0);
        } catch (...) {
            keep(std::current_exception());
        }
    }
    for (auto &x : th) x.join();
    if (ex) std::rethrow_exception(ex);
}

}  // namespace slrf
