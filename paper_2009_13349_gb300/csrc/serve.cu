// serve.cu -- the served form of the C ABI: a request server doing continuous
// batching over the segmented solver (ccd_batch_begin / submit / poll /
// cancel / end).
//
// Requests -- a set of queries of one kind with their own delta, ms and m_I,
// as the line searches of many simulations issue them (Algorithm 4 calls CCD
// with a per-step d, delta and m_I) -- arrive at any time.  The server holds
// one device arena of the caller's budget:
//   - the inbox: a ring of query records (24 doubles each) into which every
//     request is copied when it is submitted, and a ring of request
//     descriptors (one ccd_segment each) beside it: the queue lives on the
//     device, the host keeps only bookkeeping;
//   - per lane (a CUDA stream) the region of one batch: its queries as
//     planes, outputs, segment table and workspace;
//   - a pool of deep-frontier pages shared by every lane's deep stage, so
//     memory goes to the batches whose frontiers need it.
// A free lane takes a batch: the oldest run of waiting requests of one cost
// class (requests whose minimum separation exceeds their tolerance subdivide
// whole |F| <= d regions and are batched apart), contiguous in the inbox.  On
// its stream the descriptors are gathered into the batch's segment table and
// the records turned into planes (both on the device), eps is taken from each
// request's own bounds (Sec. 6), and the solver stages run.  Expensive
// batches run one at a time, in arrival order, on the last lane, at the low
// stream priority; the others run on the remaining lanes at the high one.
// The deep stage runs in rounds: when a cheap batch starts while an
// expensive one is in its deep stage, the latter's blocks are asked (a flag
// in mapped host memory) to take no new query, which frees the SMs for the
// cheap batch's kernels, and poll() launches the next round; optionally
// rounds also end after a fixed slice.  Nothing on the device waits for
// anything.  Each request's answer is the one a call of its own would give:
// the solver's results do not depend on batching, launch shapes, pool size
// or round boundaries.

#include "ccd.h"
#include "internal.h"
#include "serve_queue.h"

#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <new>
#include <thread>
#include <vector>

using namespace ccd_internal;

namespace {

constexpr int MAX_LANES = 16;
constexpr size_t QUERY_BYTES = 24 * sizeof(double);

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

using ccd_serve::WAITING;
using ccd_serve::RUNNING;
using ccd_serve::DONE;
using ccd_serve::CANCELLED;

// A request: its scheduling entry (ticket, inbox place, state, cost class)
// and what the caller gave.
struct Req : ccd_serve::Entry {
    ccd_request r;        // the caller's description (host pointers)
    int status;
    cudaEvent_t uploaded;
};

struct Lane {
    cudaStream_t st;
    bool high;            // high stream priority (cheap batches)
    int state;            // 0 idle, 1 deep rounds, 2 finishing
    std::vector<Req *> reqs;
    int64_t n;
    ServedBatch b;
    // device region
    double *verts;
    uint8_t *col;
    double *toi, *tol;
    int64_t *chk;
    ccd_segment *segs;
    // pinned host staging
    uint8_t *h_col;
    double *h_toi, *h_tol;
    int64_t *h_chk;
    unsigned char *h_hdr;
    cudaEvent_t ev;
    volatile int *yield;      // mapped host memory: set to end the running deep round
    int *d_yield;             // its device address
};

// descriptors of requests first_slot .. first_slot + k - 1 (ring order) into
// the batch's segment table, offsets relative to the batch's first query
__global__ void gather_segments_kernel(const ccd_segment *ring, int ring_cap, int first_slot,
                                       int k, long long base, ccd_segment *out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    int s = first_slot + j;
    if (s >= ring_cap) s -= ring_cap;
    ccd_segment g = ring[s];
    g.offset -= base;
    out[j] = g;
}

int cost_class(const ccd_request &r) { return r.ms > 0.0 && r.delta < r.ms ? 1 : 0; }

}  // namespace

struct ccd_server {
    ccd_server_config cfg;
    int device;
    char *arena;
    size_t arena_bytes;
    double *inbox;            // inbox_queries records
    ccd_segment *ring;        // max_requests descriptors
    ccd_segment *h_ring;      // pinned staging of the descriptors
    FrontierPool pool;
    cudaStream_t upload;
    Lane lanes[MAX_LANES];
    std::deque<Req *> order;  // requests holding inbox space, in inbox order
    int64_t next_ticket;
    std::vector<Req *> finished;
    ccd_server_stats stats;
};

namespace {

void fill_defaults(ccd_server_config &c)
{
    if (c.budget_bytes == 0) c.budget_bytes = (size_t)40 << 30;
    if (c.lanes == 0) c.lanes = 4;
    if (c.max_batch == 0) c.max_batch = 1 << 20;
    if (c.inbox_queries == 0) c.inbox_queries = 4 * c.max_batch;
    if (c.max_requests == 0) c.max_requests = 4096;
    if (c.max_segments == 0) c.max_segments = 1024;
    if (c.max_itr_bound == 0) c.max_itr_bound = 1000000;
}

// An expensive batch (class 1) holds up to this many queries: enough deep
// queries to fill the GPU, few enough that its first request is not kept long
// waiting for the others.
constexpr int64_t MAX_BATCH_EXPENSIVE = 65536;

size_t lane_bytes(const ccd_server_config &c)
{
    const size_t n = (size_t)c.max_batch;
    return al256(QUERY_BYTES * n) + al256(n) + 2 * al256(8 * n) + al256(8 * n) +
           al256(sizeof(ccd_segment) * (size_t)c.max_segments) +
           al256(served_workspace_bytes(c.max_batch, c.max_itr_bound));
}

// the oldest requests, once reported finished (or cancelled), give their
// inbox space and descriptor slot back
void release_front(ccd_server *S)
{
    for (size_t k = ccd_serve::releasable(S->order); k > 0; --k) {
        Req *r = S->order.front();
        S->order.pop_front();
        cudaEventDestroy(r->uploaded);
        delete r;
    }
}

// A batch for an idle lane (see ccd_serve::select_batch), launched on its
// stream up to the first deep round.
bool form_batch(ccd_server *S, Lane &L)
{
    size_t first = 0, count = 0;
    if (!ccd_serve::select_batch(S->order, L.high, S->cfg.max_batch, S->cfg.max_segments, &first,
                                 &count, MAX_BATCH_EXPENSIVE))
        return false;
    std::vector<Req *> take(S->order.begin() + first, S->order.begin() + first + count);
    int64_t n = 0;
    for (Req *r : take) n += r->n;
    const int64_t base = take.front()->off;
    const int first_slot = (int)(take.front()->ticket % S->cfg.max_requests);
    cudaStream_t st = L.st;
    for (Req *r : take) {
        r->state = RUNNING;
        cudaStreamWaitEvent(st, r->uploaded, 0);
    }
    L.reqs = take;
    L.n = n;
    ServedBatch &b = L.b;
    b.verts = L.verts;
    b.n = n;
    b.segs = L.segs;
    b.nseg = (int32_t)take.size();
    b.max_itr_bound = S->cfg.max_itr_bound;
    b.collides = L.col;
    b.toi = L.toi;
    b.out_tol = L.tol;
    b.checks = L.chk;
    const int k = (int)take.size();
    gather_segments_kernel<<<(k + 127) / 128, 128, 0, st>>>(S->ring, S->cfg.max_requests,
                                                            first_slot, k, base, L.segs);
    ccd_status r = ccd_aos_to_soa(S->inbox + (size_t)base * 24, n, L.verts, n, st);
    if (r == CCD_OK) r = ccd_segments_err_from_bounds(L.verts, n, L.segs, k, st);
    if (r == CCD_OK) r = served_front(b, S->pool, st);
    *L.yield = 0;
    if (r == CCD_OK)
        r = served_deep_round(b, S->pool, S->cfg.deep_slice_us * 1000LL, L.d_yield, st);
    if (r == CCD_OK &&
        cudaMemcpyAsync(L.h_hdr, b.workspace, header_bytes(), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        r = CCD_ERR_CUDA;
    if (r == CCD_OK && cudaEventRecord(L.ev, st) != cudaSuccess) r = CCD_ERR_CUDA;
    if (r != CCD_OK) {   // nothing more can be done on this batch: report it
        for (Req *q : take) {
            q->state = DONE;
            q->status = r;
            S->finished.push_back(q);
        }
        L.reqs.clear();
        return true;
    }
    L.state = 1;
    S->stats.batches += 1;
    S->stats.deep_rounds += 1;
    return true;
}

// Moves a lane's batch along when its last step finished on the device.
void advance(ccd_server *S, Lane &L)
{
    if (L.state == 0 || cudaEventQuery(L.ev) != cudaSuccess) return;
    cudaStream_t st = L.st;
    if (L.state == 1) {
        ccd_status r = CCD_OK;
        if (served_deep_left(L.h_hdr) > 0) {   // another round for the rest of the deep list
            *L.yield = 0;
            r = served_deep_round(L.b, S->pool, S->cfg.deep_slice_us * 1000LL, L.d_yield, st);
            if (r == CCD_OK &&
                cudaMemcpyAsync(L.h_hdr, L.b.workspace, header_bytes(), cudaMemcpyDeviceToHost,
                                st) != cudaSuccess)
                r = CCD_ERR_CUDA;
            if (r == CCD_OK) {
                cudaEventRecord(L.ev, st);
                S->stats.deep_rounds += 1;
                return;
            }
        } else {
            r = served_finish(L.b, S->pool, st);
            const size_t n = (size_t)L.n;
            if (r == CCD_OK &&
                (cudaMemcpyAsync(L.h_col, L.col, n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                 cudaMemcpyAsync(L.h_toi, L.toi, 8 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                 cudaMemcpyAsync(L.h_tol, L.tol, 8 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                 cudaMemcpyAsync(L.h_chk, L.chk, 8 * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                 cudaMemcpyAsync(L.h_hdr, L.b.workspace, header_bytes(), cudaMemcpyDeviceToHost,
                                 st) != cudaSuccess))
                r = CCD_ERR_CUDA;
            if (r == CCD_OK) {
                cudaEventRecord(L.ev, st);
                L.state = 2;
                return;
            }
        }
        for (Req *q : L.reqs) {
            q->state = DONE;
            q->status = r;
            S->finished.push_back(q);
        }
        L.reqs.clear();
        L.state = 0;
        return;
    }
    // finished: hand every request its part of the outputs
    const int status = served_status(L.h_hdr);
    int64_t at = 0;
    for (Req *q : L.reqs) {
        const size_t n = (size_t)q->n;
        memcpy(q->r.collides, L.h_col + at, n);
        memcpy(q->r.toi, L.h_toi + at, 8 * n);
        memcpy(q->r.out_tol, L.h_tol + at, 8 * n);
        if (q->r.checks) memcpy(q->r.checks, L.h_chk + at, 8 * n);
        at += q->n;
        q->state = DONE;
        q->status = status;
        S->finished.push_back(q);
    }
    L.reqs.clear();
    L.state = 0;
}

void progress(ccd_server *S)
{
    for (int l = 0; l < S->cfg.lanes; ++l) advance(S, S->lanes[l]);
    release_front(S);
    // high-priority lanes first: cheap requests should not queue behind
    // expensive ones.  A new cheap batch asks the deep rounds running on the
    // low-priority lane to end, so that its kernels get SMs (the next round
    // follows at the next poll, at low priority).
    bool cheap_started = false, running[MAX_LANES];
    for (int l = 0; l < S->cfg.lanes; ++l) running[l] = S->lanes[l].state == 1;
    for (int pass = 0; pass < 2; ++pass)
        for (int l = 0; l < S->cfg.lanes; ++l) {
            Lane &L = S->lanes[l];
            if (L.state == 0 && L.high == (pass == 0) && form_batch(S, L) && L.high)
                cheap_started = true;
        }
    if (cheap_started)
        for (int l = 0; l < S->cfg.lanes; ++l) {
            Lane &L = S->lanes[l];
            if (!L.high && running[l] && L.state == 1 && !*L.yield) {
                *L.yield = 1;
                S->stats.yields += 1;
            }
        }
    int busy = 0;
    for (int l = 0; l < S->cfg.lanes; ++l) busy += S->lanes[l].state != 0;
    if (busy > S->stats.lanes_busy_peak) S->stats.lanes_busy_peak = busy;
}

void destroy(ccd_server *S)
{
    if (!S) return;
    cudaDeviceSynchronize();
    for (Req *r : S->order) {
        cudaEventDestroy(r->uploaded);
        delete r;
    }
    for (int l = 0; l < MAX_LANES; ++l) {
        Lane &L = S->lanes[l];
        if (L.st) cudaStreamDestroy(L.st);
        if (L.ev) cudaEventDestroy(L.ev);
        if (L.h_col) cudaFreeHost(L.h_col);
        if (L.yield) cudaFreeHost((void *)L.yield);
    }
    if (S->upload) cudaStreamDestroy(S->upload);
    if (S->h_ring) cudaFreeHost(S->h_ring);
    if (S->arena) cudaFree(S->arena);
    delete S;
}

}  // namespace

extern "C" {

ccd_status ccd_batch_begin(const ccd_server_config *config, ccd_server **out)
{
    if (!out) return CCD_ERR_ARG;
    *out = nullptr;
    ccd_server_config c{};
    if (config) c = *config;
    fill_defaults(c);
    if (c.lanes < 1 || c.lanes > MAX_LANES || c.max_batch < 1 || c.max_batch >= 0x7fffffffLL ||
        c.inbox_queries < c.max_batch || c.max_requests < 1 || c.max_segments < 1 ||
        c.max_itr_bound < 1 || c.deep_slice_us < 0)
        return CCD_ERR_ARG;
    ccd_server *S = new (std::nothrow) ccd_server();
    if (!S) return CCD_ERR_CUDA;
    S->cfg = c;
    if (cudaGetDevice(&S->device) != cudaSuccess) { delete S; return CCD_ERR_CUDA; }
    // the arena: inbox, descriptors, pool counters, lanes, then the pages
    const size_t lb = lane_bytes(c);
    const size_t fixed = al256(QUERY_BYTES * (size_t)c.inbox_queries) +
                         al256(sizeof(ccd_segment) * (size_t)c.max_requests) + 256 +
                         (size_t)c.lanes * lb;
    if (lb == 0 || c.budget_bytes <= fixed + pool_bytes(2)) { delete S; return CCD_ERR_WORKSPACE; }
    long long np = (long long)((c.budget_bytes - fixed) / page_bytes());
    while (np > 2 && fixed + pool_bytes(np) > c.budget_bytes) --np;
    if (np > (1LL << 30)) np = 1LL << 30;
    S->arena_bytes = fixed + pool_bytes(np);
    if (cudaMalloc(&S->arena, S->arena_bytes) != cudaSuccess) {
        S->arena = nullptr;
        destroy(S);
        return CCD_ERR_WORKSPACE;
    }
    char *a = S->arena;
    S->inbox = (double *)a; a += al256(QUERY_BYTES * (size_t)c.inbox_queries);
    S->ring = (ccd_segment *)a; a += al256(sizeof(ccd_segment) * (size_t)c.max_requests);
    int *counters = (int *)a; a += 256;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    const size_t n = (size_t)c.max_batch;
    for (int l = 0; l < c.lanes; ++l) {
        Lane &L = S->lanes[l];
        L.high = l < c.lanes - 1;   // the last lane takes expensive batches, one at a time
        if (cudaStreamCreateWithPriority(&L.st, cudaStreamNonBlocking, L.high ? hi : lo) !=
                cudaSuccess ||
            cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming) != cudaSuccess) {
            destroy(S);
            return CCD_ERR_CUDA;
        }
        char *b = a + (size_t)l * lb;
        L.verts = (double *)b; b += al256(QUERY_BYTES * n);
        L.col = (uint8_t *)b; b += al256(n);
        L.toi = (double *)b; b += al256(8 * n);
        L.tol = (double *)b; b += al256(8 * n);
        L.chk = (int64_t *)b; b += al256(8 * n);
        L.segs = (ccd_segment *)b; b += al256(sizeof(ccd_segment) * (size_t)c.max_segments);
        L.b.workspace = b;
        L.b.ws_bytes = al256(served_workspace_bytes(c.max_batch, c.max_itr_bound));
        void *h = nullptr;
        const size_t hb = al256(n) + 3 * al256(8 * n) + al256(header_bytes());
        if (cudaHostAlloc(&h, hb, cudaHostAllocDefault) != cudaSuccess) { destroy(S); return CCD_ERR_CUDA; }
        char *hc = (char *)h;
        L.h_col = (uint8_t *)hc; hc += al256(n);
        L.h_toi = (double *)hc; hc += al256(8 * n);
        L.h_tol = (double *)hc; hc += al256(8 * n);
        L.h_chk = (int64_t *)hc; hc += al256(8 * n);
        L.h_hdr = (unsigned char *)hc;
        void *y = nullptr;
        if (cudaHostAlloc(&y, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&L.d_yield, y, 0) != cudaSuccess) {
            if (y) cudaFreeHost(y);
            destroy(S);
            return CCD_ERR_CUDA;
        }
        L.yield = (volatile int *)y;
        *L.yield = 0;
    }
    a += (size_t)c.lanes * lb;
    S->pool.bits = (unsigned long long *)a;
    S->pool.nwords = (int)((np + 63) / 64);
    S->pool.pages = a + al256(sizeof(unsigned long long) * (size_t)S->pool.nwords);
    S->pool.npages = np;
    S->pool.counters = counters;
    S->pool.sharers = 2 * c.lanes;   // each lane's two deep launches (VF, EE)
    S->pool.deep_threads = served_deep_threads(np, c.lanes);
    if (cudaStreamCreateWithFlags(&S->upload, cudaStreamNonBlocking) != cudaSuccess ||
        cudaHostAlloc((void **)&S->h_ring, sizeof(ccd_segment) * (size_t)c.max_requests,
                      cudaHostAllocDefault) != cudaSuccess) {
        destroy(S);
        return CCD_ERR_CUDA;
    }
    ccd_status r = pool_init(S->pool, S->upload);
    if (r == CCD_OK && cudaStreamSynchronize(S->upload) != cudaSuccess) r = CCD_ERR_CUDA;
    if (r != CCD_OK) { destroy(S); return r; }
    S->stats.arena_bytes = S->arena_bytes;
    S->stats.pages = np;
    *out = S;
    return CCD_OK;
}

ccd_status ccd_batch_submit(ccd_server *S, const ccd_request *req, int64_t *ticket)
{
    if (!S || !req || !ticket) return CCD_ERR_ARG;
    const ccd_request &q = *req;
    if ((q.kind != CCD_KIND_VF && q.kind != CCD_KIND_EE) || q.n < 0 || !(q.delta > 0.0) ||
        !(q.ms >= 0.0) || q.max_itr < 1 || q.max_itr > S->cfg.max_itr_bound ||
        q.n > S->cfg.max_batch || (q.n > 0 && (!q.verts || !q.collides || !q.toi || !q.out_tol)))
        return CCD_ERR_ARG;
    progress(S);
    if ((int64_t)S->order.size() >= S->cfg.max_requests) {
        S->stats.busy_rejections += 1;
        return CCD_ERR_BUSY;
    }
    const int64_t off = ccd_serve::inbox_alloc(S->order, S->cfg.inbox_queries, q.n > 0 ? q.n : 1);
    if (off < 0) {
        S->stats.busy_rejections += 1;
        return CCD_ERR_BUSY;
    }
    Req *r = new (std::nothrow) Req();
    if (!r) return CCD_ERR_CUDA;
    r->ticket = S->next_ticket++;
    r->r = q;
    r->off = off;
    r->n = q.n > 0 ? q.n : 1;     // an empty request keeps one record until released
    r->reported = false;
    r->cls = cost_class(q);
    r->status = CCD_OK;
    if (cudaEventCreateWithFlags(&r->uploaded, cudaEventDisableTiming) != cudaSuccess) {
        delete r;
        return CCD_ERR_CUDA;
    }
    if (q.n == 0) {                       // nothing to solve
        r->state = DONE;
        S->order.push_back(r);
        S->finished.push_back(r);
        *ticket = r->ticket;
        S->stats.submitted += 1;
        return CCD_OK;
    }
    const int slot = (int)(r->ticket % S->cfg.max_requests);
    ccd_segment &d = S->h_ring[slot];
    memset(&d, 0, sizeof(d));
    d.offset = off;
    d.count = q.n;
    d.kind = q.kind;
    d.group = 0;
    d.ms = q.ms;
    d.delta = q.delta;
    d.max_itr = q.max_itr;
    d.t_max = 1.0;
    // the caller's buffer may be pageable: the copy returns once it is staged
    if (cudaMemcpyAsync(S->inbox + (size_t)off * 24, q.verts, QUERY_BYTES * (size_t)q.n,
                        cudaMemcpyHostToDevice, S->upload) != cudaSuccess ||
        cudaMemcpyAsync(S->ring + slot, &d, sizeof(d), cudaMemcpyHostToDevice, S->upload) !=
            cudaSuccess ||
        cudaEventRecord(r->uploaded, S->upload) != cudaSuccess) {
        cudaEventDestroy(r->uploaded);
        delete r;
        return CCD_ERR_CUDA;
    }
    r->state = WAITING;
    S->order.push_back(r);
    const Req *f = S->order.front();
    const int64_t end = r->off + r->n;
    const int64_t used = end >= f->off ? end - f->off : S->cfg.inbox_queries - f->off + end;
    if (used > S->stats.inbox_peak_queries) S->stats.inbox_peak_queries = used;
    S->stats.submitted += 1;
    *ticket = r->ticket;
    progress(S);
    return CCD_OK;
}

ccd_status ccd_batch_poll(ccd_server *S, int64_t *done, int32_t *status, int32_t cap,
                          int32_t *ndone, int32_t wait_us)
{
    if (!S || !ndone || cap < 0 || (cap > 0 && !done)) return CCD_ERR_ARG;
    *ndone = 0;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        progress(S);
        while (*ndone < cap && !S->finished.empty()) {
            Req *r = S->finished.front();
            S->finished.erase(S->finished.begin());
            r->reported = true;
            done[*ndone] = r->ticket;
            if (status) status[*ndone] = r->status;
            *ndone += 1;
            if (r->state == DONE) S->stats.completed += 1;
        }
        if (*ndone > 0 || wait_us <= 0) break;
        const auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                            std::chrono::steady_clock::now() - t0).count();
        if (us >= wait_us) break;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    release_front(S);
    return CCD_OK;
}

ccd_status ccd_batch_cancel(ccd_server *S, int64_t ticket)
{
    if (!S) return CCD_ERR_ARG;
    for (Req *r : S->order) {
        if (r->ticket != ticket) continue;
        if (r->state != WAITING) return CCD_ERR_BUSY;
        r->state = CANCELLED;
        r->status = CCD_ERR_CANCELLED;
        S->finished.push_back(r);
        S->stats.cancelled += 1;
        return CCD_OK;
    }
    return CCD_ERR_ARG;
}

ccd_status ccd_batch_stats(ccd_server *S, ccd_server_stats *out)
{
    if (!S || !out) return CCD_ERR_ARG;
    int peak[2] = {0, 0};
    if (cudaMemcpy(peak, S->pool.counters, sizeof(peak), cudaMemcpyDeviceToHost) != cudaSuccess)
        return CCD_ERR_CUDA;
    S->stats.pages_peak = peak[1];
    *out = S->stats;
    return CCD_OK;
}

ccd_status ccd_batch_end(ccd_server *S)
{
    if (!S) return CCD_ERR_ARG;
    destroy(S);
    return CCD_OK;
}

}  // extern "C"
