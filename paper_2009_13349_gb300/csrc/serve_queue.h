// serve_queue.h -- the request server's host-side scheduling (no CUDA): where
// a new request goes in the inbox ring, and which waiting requests form the
// next batch of a lane.  Used by serve.cu; the CPU tests build it on its own.
#ifndef CCD_GB300_SERVE_QUEUE_H
#define CCD_GB300_SERVE_QUEUE_H

#include <stddef.h>
#include <stdint.h>

namespace ccd_serve {

enum { WAITING = 0, RUNNING = 1, DONE = 2, CANCELLED = 3 };

// A request's place in the inbox and its scheduling state.
struct Entry {
    int64_t ticket;
    int64_t off;      // first record in the inbox ring
    int64_t n;        // records it holds
    int state;
    int cls;          // cost class (1: ms > delta, batched apart)
    bool reported;    // its completion was returned to the caller
};

// Inbox position for `want` records after the entries of `order` (oldest
// first, in ring order), in a ring of `cap` records, or -1 if there is no
// room now.  The entries occupy [first, end) or, once wrapped, [first, cap)
// and [0, end); a request never straddles the ring's end.
template <class Q>
int64_t inbox_alloc(const Q &order, int64_t cap, int64_t want)
{
    if (want > cap || want < 1) return -1;
    if (order.empty()) return 0;
    const int64_t first = order.front()->off;
    const int64_t end = order.back()->off + order.back()->n;
    if (order.back()->off >= first) {            // not wrapped
        if (end + want <= cap) return end;
        return want <= first ? 0 : -1;
    }
    return end + want <= first ? end : -1;
}

// The next batch for a lane: a high-priority lane takes the oldest waiting
// request of class 0, any other lane the oldest waiting request; the batch
// extends over the following requests while they wait, share its class, lie
// right after it in the inbox and fit max_batch records (class 1: at most
// max_batch_1, but at least one request) and max_segments requests.
// Returns false when nothing waits for this lane; otherwise the batch is
// order[*first .. *first + *count).
template <class Q>
bool select_batch(const Q &order, bool high, int64_t max_batch, int max_segments, size_t *first,
                  size_t *count, int64_t max_batch_1 = -1)
{
    size_t i = 0;
    for (; i < order.size(); ++i)
        if (order[i]->state == WAITING && (!high || order[i]->cls == 0)) break;
    if (i == order.size()) return false;
    const int cls = order[i]->cls;
    const int64_t limit = cls == 1 && max_batch_1 >= 0 ? max_batch_1 : max_batch;
    const size_t i0 = i;
    int64_t n = 0;
    for (; i < order.size(); ++i) {
        const auto *r = order[i];
        if (r->state != WAITING || r->cls != cls) break;
        if (i > i0 && r->off != order[i - 1]->off + order[i - 1]->n) break;   // ring wrapped
        if ((i > i0 && n + r->n > limit) || n + r->n > max_batch ||
            (int64_t)(i - i0) >= max_segments)
            break;
        n += r->n;
    }
    if (i == i0) return false;
    *first = i0;
    *count = i - i0;
    return true;
}

// How many of the oldest entries can give their space back: those finished
// (or cancelled) and reported, up to the first that is not.
template <class Q>
size_t releasable(const Q &order)
{
    size_t k = 0;
    while (k < order.size() && (order[k]->state == DONE || order[k]->state == CANCELLED) &&
           order[k]->reported)
        ++k;
    return k;
}

}  // namespace ccd_serve

#endif
