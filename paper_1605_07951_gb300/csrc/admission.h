// Admission policy of the request server (continuous batching): which queued
// request a free worker takes next.  Header-only and free of CUDA so that the
// host tests compile it on their own.
#pragma once
#include <cstddef>

namespace rsrr {

// Index of the queued request to admit, or -1.  A request is admitted only
// while fewer than `slots` run; the queue is scanned in arrival order and the
// first request whose byte estimate fits in `budget - used` is taken.  A
// request that has already been passed over `max_bypass` times blocks every
// request behind it until it fits, so no request waits for ever behind a
// stream of smaller ones.  `bytes(q)` and `bypassed(q)` read queue entry q.
template <typename Bytes, typename Bypassed>
inline int admit_index(int count, Bytes bytes, Bypassed bypassed, size_t used, size_t budget,
                       int active, int slots, int max_bypass) {
    if (active >= slots) return -1;
    for (int q = 0; q < count; ++q) {
        const size_t b = bytes(q);
        if (used <= budget && b <= budget - used) return q;
        if (bypassed(q) >= max_bypass) return -1;
    }
    return -1;
}

}  // namespace rsrr
