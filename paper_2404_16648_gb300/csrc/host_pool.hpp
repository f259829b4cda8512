// Persistent host worker threads for the integer mesh work of a regrid (neighbour tables,
// buffer dilation, leaf emission, face lists, connectivity).  At 10^4 - 10^5 leaves each loop
// takes tens to hundreds of microseconds, the same order as creating a thread, so the helpers
// are created once per process and woken per loop.
#pragma once
#include <cstdint>
#include <functional>

namespace dgl {

// Runs fn(i0, i1) over [0, n) cut into contiguous ranges, one per thread: the caller's thread
// and up to 15 helpers, with no range shorter than `grain` items.  Every caller writes outputs
// indexed by i only, so results do not depend on how [0, n) is cut.  A call made while another
// is in flight (from a helper, or from a second host thread) runs fn(0, n) on its own thread.
// fn must not throw.
void parallel_ranges(int64_t n, int64_t grain, const std::function<void(int64_t, int64_t)>& fn);

// Exclusive prefix sum in place over cnt[0..n) (serial; n is the leaf count); returns the total.
int64_t exclusive_scan(int64_t* cnt, int64_t n);

}  // namespace dgl
