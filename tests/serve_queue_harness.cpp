// C entry points over the request server's host scheduling (serve_queue.h)
// for the CPU tests: each call builds the queue from plain arrays.
#include <deque>
#include <vector>

#include "serve_queue.h"

using ccd_serve::Entry;

static std::deque<Entry *> build(std::vector<Entry> &e, const long long *off, const long long *n,
                                 const int *state, const int *cls, const unsigned char *rep,
                                 int count)
{
    std::deque<Entry *> d;
    e.resize(count);
    for (int i = 0; i < count; ++i) {
        e[i] = Entry{i, off[i], n[i], state ? state[i] : 0, cls ? cls[i] : 0,
                     rep ? rep[i] != 0 : false};
        d.push_back(&e[i]);
    }
    return d;
}

extern "C" long long h_alloc(const long long *off, const long long *n, int count, long long cap,
                             long long want)
{
    std::vector<Entry> e;
    return ccd_serve::inbox_alloc(build(e, off, n, nullptr, nullptr, nullptr, count), cap, want);
}

extern "C" int h_select(const long long *off, const long long *n, const int *state,
                        const int *cls, int count, int high, long long max_batch, int max_segs,
                        long long *first, long long *k)
{
    std::vector<Entry> e;
    size_t f = 0, c = 0;
    const bool ok = ccd_serve::select_batch(build(e, off, n, state, cls, nullptr, count),
                                            high != 0, max_batch, max_segs, &f, &c);
    *first = (long long)f;
    *k = (long long)c;
    return ok ? 1 : 0;
}

extern "C" long long h_releasable(const int *state, const unsigned char *rep, int count)
{
    std::vector<long long> z(count, 0);
    std::vector<Entry> e;
    return (long long)ccd_serve::releasable(build(e, z.data(), z.data(), state, nullptr, rep, count));
}
