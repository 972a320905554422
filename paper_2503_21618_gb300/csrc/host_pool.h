// Host worker threads for the setup steps (multigrid hierarchy, row groups,
// dense host eigensolver).  A setup runs a few dozen parallel steps of a
// millisecond or less each; starting fresh threads for every step cost about
// as much as the step itself, so the workers are started once per process
// and wait between steps.
#pragma once

#include <cstdint>
#include <functional>

namespace slrf {

// Host threads for a step of the given work (stored entries touched, or
// flops): up to 16 (or SLRF_HOST_THREADS, read once), one below 32 768 (a
// team of waiting workers starts in tens of microseconds).  No result of the
// setup depends on the count.
int host_threads(int64_t work);

// Runs fn(t) for t = 0 .. nt-1 at the same time on nt threads; the calling
// thread is member 0, so members may wait on one another (a barrier).  The
// other members come from one of two process-wide pools of waiting workers;
// a caller that finds both pools busy (a third concurrent setup), or asks
// for more members than a pool has, starts threads of its own.  Returns when
// every member has returned; the first exception of any member is rethrown
// then (a member that throws before a barrier the others wait at leaves them
// waiting: members that wait on one another must not throw).
void host_team(int nt, const std::function<void(int)> &fn);

// fn(r0, r1, t) over nt contiguous row ranges of [0, nrows) on a team.
template <class Fn>
void host_parallel_rows(int nrows, int nt, Fn fn) {
    if (nt <= 1 || nrows <= 1) {
        fn(0, nrows, 0);
        return;
    }
    host_team(nt, [&](int t) {
        const int r0 = (int)((int64_t)nrows * t / nt), r1 = (int)((int64_t)nrows * (t + 1) / nt);
        fn(r0, r1, t);
    });
}

}  // namespace slrf
