// Test harness (host only) for the setup worker pools (host_pool.cpp), which
// it links directly.  Exit status 0 when every check passes; a check that
// fails prints its name.  Waits inside the checks are bounded, so a pool that
// lost a member fails instead of hanging.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <stdexcept>
#include <thread>
#include <vector>

#include "host_pool.h"

using namespace slrf;

namespace {

bool g_ok = true;
void check(bool c, const char *what) {
    if (!c) {
        std::printf("FAILED: %s\n", what);
        g_ok = false;
    }
}

// Every member arrives, then waits (at most ~10 s) until all have arrived:
// only a team whose members really run at the same time gets through.
bool team_meets(int nt) {
    std::atomic<int> arrived{0};
    std::atomic<int> timeouts{0};
    host_team(nt, [&](int) {
        arrived.fetch_add(1);
        const auto t0 = std::chrono::steady_clock::now();
        while (arrived.load() < nt)
            if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(10)) {
                timeouts.fetch_add(1);
                return;
            }
    });
    return timeouts.load() == 0 && arrived.load() == nt;
}

}  // namespace

int main() {
    // 1. every member runs once, with its own index
    for (int nt : {1, 2, 7, 16}) {
        std::vector<std::atomic<int>> hits(nt);
        for (auto &h : hits) h = 0;
        host_team(nt, [&](int t) { hits[t].fetch_add(1); });
        bool once = true;
        for (auto &h : hits) once = once && h.load() == 1;
        check(once, "each member runs exactly once");
    }
    // 2. members run at the same time (a barrier inside the team)
    check(team_meets(16), "16 members meet at a barrier");
    // 3. row ranges cover [0, n) once, for row counts below and above the team size
    for (int n : {0, 1, 5, 16, 1000, 100003}) {
        std::vector<int> cover(n, 0);
        host_parallel_rows(n, 16, [&](int r0, int r1, int) {
            for (int r = r0; r < r1; ++r) cover[r]++;
        });
        bool ok = true;
        for (int c : cover) ok = ok && c == 1;
        check(ok, "row ranges cover every row once");
    }
    // 4. three callers at once (two pools, then threads of the caller's own),
    //    each with teams that meet at a barrier, many times over
    {
        std::atomic<int> fails{0};
        std::vector<std::thread> callers;
        for (int c = 0; c < 3; ++c)
            callers.emplace_back([&] {
                for (int rep = 0; rep < 200; ++rep)
                    if (!team_meets(8)) fails.fetch_add(1);
            });
        for (auto &t : callers) t.join();
        check(fails.load() == 0, "concurrent callers each get a whole team");
    }
    // 5. a member that throws (the caller's own, then a worker's): the others
    //    finish, the exception reaches the caller, and the pool takes the next job
    {
        std::atomic<int> others{0};
        bool caught = false;
        try {
            host_team(8, [&](int t) {
                if (t == 0) throw std::runtime_error("member 0");
                others.fetch_add(1);
            });
        } catch (const std::runtime_error &) {
            caught = true;
        }
        check(caught && others.load() == 7, "an exception of member 0 reaches the caller after the others");
        check(team_meets(16), "the pool works after an exception");
        others = 0;
        caught = false;
        try {
            host_team(8, [&](int t) {
                if (t == 5) throw std::runtime_error("member 5");
                others.fetch_add(1);
            });
        } catch (const std::runtime_error &) {
            caught = true;
        }
        check(caught && others.load() == 7, "an exception of another member reaches the caller");
        check(team_meets(16), "the pool works after a member's exception");
    }
    // 6. thread counts: one below the threshold, at least one above it
    check(host_threads(100) == 1, "small work runs on one thread");
    check(host_threads(1 << 24) >= 1, "large work gets a team");
    std::printf(g_ok ? "host pool checks passed\n" : "host pool checks FAILED\n");
    return g_ok ? 0 : 1;
}
