// internal.h -- interface between the solver (ccd.cu) and the request server
// (serve.cu, the served form of the C ABI).  Not part of the public ABI.
#ifndef CCD_GB300_INTERNAL_H
#define CCD_GB300_INTERNAL_H

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "ccd.h"

namespace ccd_internal {

// A pool of deep-frontier pages shared by the deep stages of several batches
// (they take and free pages with atomics on the bitmap; nothing waits).
struct FrontierPool {
    void *pages;                 // npages pages of page_bytes() each
    unsigned long long *bits;    // free bitmap, one bit per page
    int nwords;                  // (npages + 63) / 64
    long long npages;
    int *counters;               // 2 ints: pages held now, the most held at once
    int deep_threads;            // deep-solver block size of the batches on the pool
    int sharers;                 // deep launches that may use the pool at once
};

size_t page_bytes();
// bitmap (rounded to 256 bytes) + pages
size_t pool_bytes(long long npages);
// marks every page free and clears the counters (on `st`)
ccd_status pool_init(const FrontierPool &pool, cudaStream_t st);

// One segmented batch (the arguments of ccd_multi_batch, default launch
// shapes) whose deep stage draws on a shared pool; the workspace holds the
// per-query lists, the small-frontier slots and two full-size slots.
struct ServedBatch {
    const double *verts;
    int64_t n;
    const ccd_segment *segs;
    int32_t nseg;
    int64_t max_itr_bound;
    uint8_t *collides;
    double *toi;
    double *out_tol;
    int64_t *checks;
    void *workspace;
    size_t ws_bytes;
};

size_t served_workspace_bytes(int64_t n, int64_t max_itr_bound);
size_t header_bytes();
// deep-solver block size for a server with npages pool pages and `lanes` lanes
int served_deep_threads(long long npages, int lanes);
// header reset, validation, level 0, pooled and one-warp stages, deep list
ccd_status served_front(const ServedBatch &b, const FrontierPool &pool, cudaStream_t st);
// one deep round: until the deep list is empty, slice_ns has passed (> 0)
// or *yield (device-readable host memory, may be NULL) is set
ccd_status served_deep_round(const ServedBatch &b, const FrontierPool &pool, long long slice_ns,
                             const volatile int *yield, cudaStream_t st);
// the deferred queries in the full-size slots
ccd_status served_finish(const ServedBatch &b, const FrontierPool &pool, cudaStream_t st);
// from a host copy of the batch's header: deep queries not yet taken, and
// the status the kernels recorded
long long served_deep_left(const void *header);
int served_status(const void *header);

}  // namespace ccd_internal

#endif
