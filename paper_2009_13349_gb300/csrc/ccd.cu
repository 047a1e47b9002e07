// ccd.cu -- sm_103a kernels and C ABI of the batched inclusion-based CCD root
// finder (Wang et al. 2021, Sec. 4, Algorithm 2; minimum separation Sec. 5.1).
//
// Execution plan of one batch (all launches on the caller's stream, no host
// synchronisation, no allocation):
//   1. root_kernel      one thread per query: loads the 192-byte record,
//                       checks the level-0 box [0,1]^3 (Eq. box, Eq.
//                       ccd-error).  Queries rejected there, or terminating
//                       there, are answered; the rest get kappa (Eq. kappas)
//                       and join the survivor list.
//   2. pool_kernel      persistent; one warp holds up to 32 survivor queries
//                       and packs the next boxes of all of them into its
//                       lanes; a query whose level outgrows its slot (64
//                       boxes by default) moves to the next list.
//   3. solve_kernel<32> persistent; one warp per query, frontiers up to 1024
//                       boxes per level; a query that outgrows it moves to the
//                       deep list with the level it reached.
//   4. order_by_level_kernel  sorts the deep list shallowest level first (the
//                       longest queries first).
//   5. solve_kernel<256> persistent; one 256-thread block per deep query (three
//                       resident per SM), frontier slot sized for 2 m_I boxes
//                       (the most any level can hold, see solve_query); a
//                       chunk of 256 boxes shares its t-quantities and partials
//                       (a chunk too varied for the tables goes as sub-chunks
//                       of 128 boxes).
// A query that moves on restarts from level 0 in the next stage; its result
// does not depend on the stage that answers it.
//
// Level-synchronous form of Algorithm 2.  Q is ordered by (level, left end
// of I_t); ties keep insertion order, children inserted left then right.
// All boxes of one level have the same widths, hence the same split
// dimension.  A level is therefore an array in Q order: for u and v splits
// the children of box j are adjacent (left, right); for t splits, each run of
// boxes sharing I_t emits all left children, then all right children.  The
// check counter of the box at array position i is n_before + i + 1, so the
// first colliding box, the m_I cut-off and the termination test are decided
// block-wide exactly as the sequential loop would.
//
// Boxes are stored as integer numerators (a_t, a_u, a_v) of dyadic
// endpoints a 2^-k, k <= 53 per dimension, converted to doubles exactly.
// F is evaluated in a fixed fused order: positions fma(x1 - x0, t, x0)
// first; VF F = fma(-v, e2, fma(-u, e1, q)) with q = p - v1, e1 = v2 - v1,
// e2 = v3 - v1; EE F = fma(u, d1, p1 - fma(v, d2, p3)), d1 = p2 - p1,
// d2 = p4 - p3.  Every add, multiply and fused multiply-add is an explicit
// round-to-nearest intrinsic (nothing else is contracted).  Per axis and t
// value, the minimum and maximum of B_F's corners are taken from the two
// extreme corners (corner_range), which give the same bits as all four.

#include "ccd.h"
#include "internal.h"

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

namespace {

constexpr int KMAX = 53;              // deepest dyadic level per dimension
constexpr int ROOT_THREADS = 256;
constexpr int SMALL_THREADS = 32;     // one warp per query
constexpr int SMALL_BLOCKS_PER_SM = 16;
constexpr long long SMALL_CAP = 256;  // boxes per small-frontier slot
constexpr int POOL_SLOTS = 32;        // pooled solver: queries held by one warp ...
constexpr int POOL_CAP = 64;          // ... boxes per level per query (default) ...
constexpr int POOL_CAP_MAX = 4096;
constexpr int POOL_PCAP = 62;         // shared partials per pooled iteration (more: direct;
                                      // 62 keeps the vertex-face block at 24 per SM)
constexpr int POOL_BLOCKS_PER_SM = 24; // ... and at most this many one-warp blocks per SM (the
                                       // launch takes what the occupancy calculator allows)
constexpr int POOL_BLOCKS_EE = 20;     // edge-edge: 96 registers without spills (21 would cap it at 80)
// Resident deep-solver blocks (queries) per SM by block size, at 80
// registers without spills: one 512-thread block, three of 256, six of 128;
// a segmented kernel compiled for both kinds needs more registers (two of
// 256, four of 128).
constexpr int deep_blocks_per_sm(int bs, bool both_kinds = false)
{
    return bs == 256 ? (both_kinds ? 2 : 3) : bs == 128 ? (both_kinds ? 4 : 6) : 1;
}
// Single-kind batches run 128-thread deep blocks, six per SM: more queries
// in flight per SM and barriers over four warps instead of eight (the
// degenerate-heavy step took 4.71 s against 5.46 s with 256-thread blocks,
// the simulation-mixed one 93 ms against 103; 64-thread blocks, eleven per
// SM, took 4.66 s and 117 ms: a query's block width shows in the tail of
// the simulation workload's few deep queries).  Segmented batches default to
// 256 threads: their few deep queries (about 5,000 of 20M) end in a tail
// where each query's block width counts more (deep stage 33 vs 47 ms).
constexpr int DEEP_THREADS = 128;
constexpr int DEEP_BLOCKS_PER_SM = deep_blocks_per_sm(DEEP_THREADS);
constexpr int SEG_DEEP_THREADS = 256;
// The default page pool holds one full-size level for at most this many deep
// blocks per SM; more blocks share it (pages are taken per level as needed,
// and a block that finds none defers its query, so the size changes speed
// only).  Peak use on the degenerate-heavy workload is about a quarter.
constexpr int DEEP_POOL_BLOCKS_PER_SM = 3;
constexpr long long DEEP_MIN_PAGES = 3;   // pages per deep block a launch can count on
constexpr long long BIGL = 0x7fffffffffffffffLL;

struct Box {
    unsigned long long a[3];          // numerators of (t_L, u_L, v_L)
};

struct Header {
    int survivors;   // queries in the survivor list
    int head_small;  // work counter of the small-frontier solver
    int overflow;    // queries in the deep list (one-warp solver hand-offs)
    int head_deep;   // work counter of the deep solver
    int status;      // CCD_OK or CCD_ERR_CAPACITY
    int fallbacks;   // queries answered by the capacity fallback
    int mid;         // queries handed from the pooled solver to the one-warp solver
    int head_pool;   // work counter of the pooled solver
    unsigned long long checks_small;  // sum of n over queries finished by the small solver
    unsigned long long checks_deep;   // sum of n over queries finished by the deep solver
    unsigned long long evals_small;   // box evaluations executed by the small solver
    unsigned long long evals_deep;    // box evaluations executed by the deep solver
    unsigned long long tq_small;      // t-quantity evaluations by the small solver
    unsigned long long tq_deep;       // t-quantity evaluations by the deep solver
    unsigned long long a_tasks_deep;  // shared partials (one per t value and u / v), deep solver
    unsigned long long split_chunks_deep;  // deep chunks evaluated as sub-chunks
    unsigned long long evals_shared_deep;  // deep box evaluations from shared partials
    unsigned long long checks_pool;   // sum of n over queries finished by the pooled solver
    unsigned long long evals_pool;    // box evaluations executed by the pooled solver
    int head_pool_ee;                 // work counter of the EE pooled solver (segmented batches)
    int pad0;
    unsigned long long tq_deep_ee;      // the part of tq_deep spent on edge-edge queries
    unsigned long long a_tasks_deep_ee; // the part of a_tasks_deep spent on edge-edge queries
    unsigned long long evals_pool_ee;   // the part of evals_pool spent on edge-edge queries
    unsigned long long tq_small_ee;     // the part of tq_small spent on edge-edge queries
    unsigned long long evals_small_ee;  // the part of evals_small spent on edge-edge queries
    int jumbo;        // queries the paged deep solver deferred to the full-size slots
    int head_jumbo;   // work counter of the full-size (jumbo) stage
    int pages_used;   // deep frontier pages held now (pools owned by the workspace)
    int pages_peak;   // the most held at once
    unsigned long long tq_pool;     // t-quantity evaluations (t values) by the pooled solver
    unsigned long long tq_pool_ee;  // the part of tq_pool spent on edge-edge queries
    unsigned long long round_start; // %globaltimer at the start of a time-sliced deep round
    unsigned long long pool_iters;  // iterations of the pooled solver's warps
    unsigned long long pool_serial; // sum over those of the most boxes one slot placed
    int overflow_ee;  // segmented batches: edge-edge queries in the deep list ...
    int head_deep_ee; // ... and their work counter (vertex-face: overflow, head_deep)
    unsigned long long a_tasks_pool;          // shared partials computed by the pooled solver
    unsigned long long a_tasks_pool_ee;       // the part of a_tasks_pool spent on edge-edge queries
    unsigned long long evals_pool_shared;     // pooled box evaluations from shared partials
    unsigned long long evals_pool_shared_ee;  // the part of those on edge-edge queries
    unsigned long long evals_deep_ee;         // the part of evals_deep on edge-edge queries
    unsigned long long evals_shared_deep_ee;  // the part of evals_shared_deep on edge-edge queries
    unsigned long long pad[5];
};
static_assert(sizeof(Header) == 320, "header is five 64-byte lines");

struct Layout {
    size_t off_surv, off_mid, off_over, off_level, off_dlist, off_jlist, off_kappa, off_pool,
        off_meta, off_small, off_deep, total;
    int nb_pool, nb_small;
    long long cap_small;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---- exact dyadic conversion and small helpers -----------------------------

// a * 2^-k as a double, exact for 0 <= a <= 2^53 and 0 <= k <= 53 (integer
// construction of the bit pattern; the FP64 pipe is not used).
__device__ __forceinline__ double dyadic(unsigned long long a, int k)
{
    if (a == 0ull) return 0.0;
    int lz = __clzll((long long)a);
    int sh = lz - 11;                  // puts the leading one at bit 52
    unsigned long long m = sh >= 0 ? (a << sh) : (a >> (-sh));
    unsigned long long e = (unsigned long long)(1023 + (63 - lz) - k);
    return __longlong_as_double((long long)((e << 52) | (m & 0x000FFFFFFFFFFFFFull)));
}

__device__ __forceinline__ double pow2neg(int k)
{
    return __longlong_as_double((long long)((unsigned long long)(1023 - k) << 52));
}

// GB300 issues FP64 compares and sign changes on the same scarce FP64 pipe
// as add and multiply (about two operations per SM per clock), so the
// per-box tests take them from the bits instead.  The bits pass through a
// one-instruction move that the compiler cannot see through; a plain
// reinterpretation lets it turn integer tests of the bits back into
// floating-point compares.
__device__ __forceinline__ long long dbits(double x)
{
    long long b;
    asm("mov.b64 %0, %1;" : "=l"(b) : "d"(x));
    return b;
}
__device__ __forceinline__ double dfrombits(long long b)
{
    double x;
    asm("mov.b64 %0, %1;" : "=d"(x) : "l"(b));
    return x;
}

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// 2^-k x when the result is not normal (or x is not finite): one rounded
// multiply, out of line so that the common case never issues it
__device__ __noinline__ double scale2neg_slow(double x, int k) { return dmul(pow2neg(k), x); }
// 2^-k x, exact: by exponent arithmetic while the result stays normal
__device__ __forceinline__ double scale2neg(double x, int k)
{
    const long long b = dbits(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e > k && e < 0x7ff) return dfrombits(b - ((long long)k << 52));
    return scale2neg_slow(x, k);
}

// x == +-0
__device__ __forceinline__ bool dzero(double x) { return (dbits(x) << 1) == 0; }
// -x (the sign bit flipped, as IEEE negation does)
__device__ __forceinline__ double dneg(double x)
{
    return dfrombits(dbits(x) ^ (long long)0x8000000000000000ULL);
}
// t = t_max * s for s = a 2^-k in [0, 1]: the product is s itself when
// t_max == 1 (the whole-step interval), so the multiply is skipped then
__device__ __forceinline__ bool tmax_one(double t_max) { return dbits(t_max) == 0x3FF0000000000000LL; }
__device__ __forceinline__ double tscale(double t_max, double s)
{
    return tmax_one(t_max) ? s : dmul(t_max, s);
}

// The split dimension of Algorithm 2: the largest of c_d = 2^-k_d kappa_d,
// ties to t, then u, then v.  The c_d are +0, positive or +inf (kappa is a
// maximum of absolute values), where the order of the bits as signed
// integers is the numeric order.
__device__ __forceinline__ int split_dim(double ct, double cu, double cv)
{
    const long long bt = dbits(ct), bu = dbits(cu), bv = dbits(cv);
    long long bm = bt;
    if (bu > bm) bm = bu;
    if (bv > bm) bm = bv;
    return (bt == bm) ? 0 : (bu == bm) ? 1 : 2;
}

// ---- per-query data ---------------------------------------------------------

struct Query {
    double x0[12];   // points at t0
    double dx[12];   // x1 - x0
};

__device__ __forceinline__ void load_query(const double *__restrict__ verts, long long n,
                                           long long i, Query &Q)
{
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double a = __ldg(verts + (size_t)k * n + i);
        double b = __ldg(verts + (size_t)(12 + k) * n + i);
        Q.x0[k] = a;
        Q.dx[k] = dsub(b, a);
    }
}

// ---- order-preserving integer keys of doubles --------------------------------
// On GB300 FP64 min/max/compare issue on the same scarce FP64 pipe as add and
// multiply, so the box test orders doubles through integer keys instead:
// key(x) flips the magnitude bits of negative x, making signed 64-bit order
// equal to numeric order for finite x (only -0 < +0 differs from IEEE, which
// the thresholds below absorb).
__device__ __forceinline__ long long dkey(double x)
{
    const long long b = dbits(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dkey_inv(long long k)
{
    return dfrombits(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
// thresholds: x <= c  <=>  dkey(x) <= key_le(c);  x >= c  <=>  dkey(x) >= key_ge(c)
__device__ __forceinline__ long long key_le(double c) { return dzero(c) ? 0LL : dkey(c); }
__device__ __forceinline__ long long key_ge(double c) { return dzero(c) ? -1LL : dkey(c); }

struct Thresholds {
    long long le_eps[3];   // x <= eps_c
    long long ge_neps[3];  // x >= -eps_c
    long long delta;       // w < delta (w >= +0, delta > 0)
};

__device__ __forceinline__ void make_thresholds(const double (&eps)[3], double delta,
                                                Thresholds &T)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T.le_eps[c] = key_le(eps[c]);
        T.ge_neps[c] = key_ge(dneg(eps[c]));
    }
    T.delta = dkey(delta);
}

// Quantities of F that depend on t only, for one value of t (fixed order):
// VF: q = p - v1, e1 = v2 - v1, e2 = v3 - v1;  EE: p1, d1 = p2 - p1, p3, d2 = p4 - p3.
template <int KIND>
struct TWidth { static constexpr int W = KIND == CCD_KIND_VF ? 9 : 12; };

template <int KIND>
__device__ __forceinline__ void t_quantities(const Query &Q, double t, double *out)
{
    // Q lives in shared memory (one copy per block)
    double P[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) P[j] = dfma(Q.dx[j], t, Q.x0[j]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (KIND == CCD_KIND_VF) {
            out[c] = dsub(P[c], P[3 + c]);
            out[3 + c] = dsub(P[6 + c], P[3 + c]);
            out[6 + c] = dsub(P[9 + c], P[3 + c]);
        } else {
            out[c] = P[c];
            out[3 + c] = dsub(P[3 + c], P[c]);
            out[6 + c] = P[6 + c];
            out[9 + c] = dsub(P[9 + c], P[6 + c]);
        }
    }
}

// The same quantities for one axis c only (out[c], out[3 + c], out[6 + c]
// and, for EE, out[9 + c]), with the same operations: lets three threads
// share one t value.
template <int KIND>
__device__ __forceinline__ void t_quantities_axis(const Query &Q, double t, int c, double *out)
{
    double P[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) P[i] = dfma(Q.dx[3 * i + c], t, Q.x0[3 * i + c]);
    if (KIND == CCD_KIND_VF) {
        out[c] = dsub(P[0], P[1]);
        out[3 + c] = dsub(P[2], P[1]);
        out[6 + c] = dsub(P[3], P[1]);
    } else {
        out[c] = P[0];
        out[3 + c] = dsub(P[1], P[0]);
        out[6 + c] = P[2];
        out[9 + c] = dsub(P[3], P[2]);
    }
}

// Keys of the min and max over the four corners fma(x, g, p) of one axis at
// one t, x in {x_lo, x_hi} (x_lo < x_hi) and p in {p0, p1}.  The exact value
// x g + p is non-decreasing in p, and in x when g > 0 (non-increasing when g
// < 0; for g = +-0 both x give the same result, as x_lo and x_hi have one
// sign), and rounding is monotone, so the extreme corners are fma at the
// smaller p with the x that makes x g smallest, and at the larger p with the
// other x.  Two fmas give the same bits as the min and max of all four, in
// key order (-0 before +0) too: for a fixed x the result is key-monotone in
// p, including zero results.  (Finite g and p; no NaN arises from them.)
//
// NEG: x = -y for y in {y_lo, y_hi} (VF's -v), else x = y (EE's u); the
// negation goes into the fma's operand, fma(-y, g, p).
template <bool NEG>
__device__ __forceinline__ void corner_range(double y_lo, double y_hi, double g, double p0,
                                             double p1, long long &lo, long long &hi)
{
    const bool sw = dkey(p1) < dkey(p0);
    const double pmin = sw ? p1 : p0, pmax = sw ? p0 : p1;
    // x g smallest: x_lo = (NEG ? -y_hi : y_lo) when g's sign bit is clear
    const bool hi_y = (dbits(g) < 0) != NEG;
    const double ymin = hi_y ? y_hi : y_lo, ymax = hi_y ? y_lo : y_hi;
    lo = dkey(dfma(NEG ? -ymin : ymin, g, pmin));
    hi = dkey(dfma(NEG ? -ymax : ymax, g, pmax));
}

// B_F(I) from the t-quantities of t_L (TL) and t_R (TR): per-axis integer
// keys of the min and max over the 8 corners.
template <int KIND>
__device__ __forceinline__ void corners_keys(const double *TL, const double *TR, double ul,
                                             double ur, double vl, double vr, long long (&km)[3],
                                             long long (&kM)[3])
{
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const double *T = side ? TR : TL;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            long long lo, hi;
            if (KIND == CCD_KIND_VF) {   // F = fma(-v, e2, fma(-u, e1, q))
                const double q = T[c], e1 = T[3 + c], e2 = T[6 + c];
                const double al = dfma(-ul, e1, q), ar = dfma(-ur, e1, q);
                corner_range<true>(vl, vr, e2, al, ar, lo, hi);
            } else {                     // F = fma(u, d1, p1 - fma(v, d2, p3))
                const double a = T[c], d1 = T[3 + c], b = T[6 + c], d2 = T[9 + c];
                const double cl = dsub(a, dfma(vl, d2, b)), cr = dsub(a, dfma(vr, d2, b));
                corner_range<false>(ul, ur, d1, cl, cr, lo, hi);
            }
            if (side == 0) { km[c] = lo; kM[c] = hi; }
            else { km[c] = min(km[c], lo); kM[c] = max(kM[c], hi); }
        }
    }
}

// The box test of Algorithm 2 on integer keys (Sec. 5.1 enlargement by ms).
__device__ __forceinline__ void box_test_keys(const long long (&km)[3], const long long (&kM)[3],
                                              const Thresholds &T, double ms, bool &hit,
                                              bool &term, double &w)
{
    long long lo[3], hi[3];
    double wmax = 0.0;
    long long kw = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double m = dkey_inv(km[c]), M = dkey_inv(kM[c]);
        const double wc = dsub(M, m);           // >= +0
        const long long kc = dbits(wc);
        if (c == 0 || kc > kw) { kw = kc; wmax = wc; }
        if (!dzero(ms)) {
            lo[c] = dkey(dsub(m, ms));
            hi[c] = dkey(dadd(M, ms));
        } else {
            lo[c] = km[c];
            hi[c] = kM[c];
        }
    }
    hit = (lo[0] <= T.le_eps[0]) & (hi[0] >= T.ge_neps[0]) & (lo[1] <= T.le_eps[1]) &
          (hi[1] >= T.ge_neps[1]) & (lo[2] <= T.le_eps[2]) & (hi[2] >= T.ge_neps[2]);
    const bool inside = (lo[0] >= T.ge_neps[0]) & (hi[0] <= T.le_eps[0]) &
                        (lo[1] >= T.ge_neps[1]) & (hi[1] <= T.le_eps[1]) &
                        (lo[2] >= T.ge_neps[2]) & (hi[2] <= T.le_eps[2]);
    term = (kw < T.delta) | inside;
    w = wmax;
}

// The box test of Algorithm 2 with the Sec. 5.1 enlargement by ms.
struct BoxTest {
    bool hit;      // B (enlarged by ms) meets C_eps
    bool term;     // w(B) < delta or enlarged B inside C_eps
    double w;      // w(B), un-enlarged
};

__device__ __forceinline__ BoxTest box_test(const double (&m)[3], const double (&M)[3],
                                            const double (&eps)[3], double ms, double delta)
{
    BoxTest r;
    double lo[3], hi[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = ms != 0.0 ? dsub(m[c], ms) : m[c];   // m - 0 == m
        hi[c] = ms != 0.0 ? dadd(M[c], ms) : M[c];
    }
    r.hit = (lo[0] <= eps[0]) & (hi[0] >= -eps[0]) & (lo[1] <= eps[1]) & (hi[1] >= -eps[1]) &
            (lo[2] <= eps[2]) & (hi[2] >= -eps[2]);
    r.w = fmax(fmax(dsub(M[0], m[0]), dsub(M[1], m[1])), dsub(M[2], m[2]));
    bool inside = (lo[0] >= -eps[0]) & (hi[0] <= eps[0]) & (lo[1] >= -eps[1]) &
                  (hi[1] <= eps[1]) & (lo[2] >= -eps[2]) & (hi[2] <= eps[2]);
    r.term = (r.w < delta) | inside;
    return r;
}

// ---- block primitives (BS = 32: warp only; BS > 32: warp + shared) ---------

template <int BS>
__device__ __forceinline__ void bsync()
{
    if (BS == 32) __syncwarp(); else __syncthreads();
}


// Per-warp summary of one chunk's box tests, published before one barrier.
struct WarpDecision {
    int count;                 // colliding boxes in the warp
    int first;                 // lane of the first colliding box (32: none)
    int first_cut;             // lane of the first colliding box with n >= m_I
    int term;                  // termination test of the first colliding box
    unsigned long long at;     // a_t of the first colliding box
    double w;                  // w(B) of the first colliding box
    double w_cut;              // w(B) of the first cut box
};

template <int BS>
struct Smem {
    Query query;                     // the query being solved
    WarpDecision dec[BS / 32];
    int scan_a[BS / 32], scan_b[BS / 32];
    unsigned long long at[BS];       // a_t of each thread's box in the chunk
    unsigned long long run_at[BS];   // a_t of each run of equal t_L
    int ired[BS / 32 + 1];
    long long lred[BS / 32 + 1];
};

// exclusive prefix sum of v over the block (thread order); *total = sum
template <int BS>
__device__ __forceinline__ int block_excl_scan(int v, int *total, Smem<BS> &s)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (BS == 32) {
        *total = __shfl_sync(0xffffffffu, inc, 31);
        return inc - v;
    }
    if (lane == 31) s.ired[warp] = inc;
    __syncthreads();
    int ws = lane < BS / 32 ? s.ired[lane] : 0;
    int wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
    }
    int before = __shfl_sync(0xffffffffu, wi - ws, warp);
    *total = __shfl_sync(0xffffffffu, wi, BS / 32 - 1);
    __syncthreads();
    return before + inc - v;
}

// exclusive prefix sum with one barrier: `arr` must not be written again
// before every thread has passed another barrier
template <int BS>
__device__ __forceinline__ int block_scan_1sync(int v, int *total, int *arr)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (BS == 32) {
        *total = __shfl_sync(0xffffffffu, inc, 31);
        return inc - v;
    }
    if (lane == 31) arr[warp] = inc;
    __syncthreads();
    int before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < BS / 32; ++w) {
        const int x = arr[w];
        before += (w < warp) ? x : 0;
        tot += x;
    }
    *total = tot;
    return before + inc - v;
}

// inclusive max-scan over thread order (values >= -1); *all = the block's
// maximum (the same pass, no further barrier)
template <int BS>
__device__ __forceinline__ long long block_incl_maxscan(long long v, Smem<BS> &s, long long *all)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = max(inc, y);
    }
    if (BS == 32) {
        *all = __shfl_sync(0xffffffffu, inc, 31);
        return inc;
    }
    if (lane == 31) s.lred[warp] = inc;
    __syncthreads();
    long long prev = -1, tot = -1;
#pragma unroll
    for (int w = 0; w < BS / 32; ++w) {
        const long long x = s.lred[w];
        if (w < warp) prev = max(prev, x);
        tot = max(tot, x);
    }
    *all = tot;
    __syncthreads();
    return max(prev, inc);
}

// inclusive min-scan over reversed thread order: min over threads >= me;
// *all = the block's minimum
template <int BS>
__device__ __forceinline__ long long block_suffix_min(long long v, Smem<BS> &s, long long *all)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_down_sync(0xffffffffu, inc, o);
        if (lane + o < 32) inc = min(inc, y);
    }
    if (BS == 32) {
        *all = __shfl_sync(0xffffffffu, inc, 0);
        return inc;
    }
    if (lane == 0) s.lred[warp] = inc;
    __syncthreads();
    long long nxt = BIGL, tot = BIGL;
#pragma unroll
    for (int w = 0; w < BS / 32; ++w) {
        const long long x = s.lred[w];
        if (w > warp) nxt = min(nxt, x);
        tot = min(tot, x);
    }
    *all = tot;
    __syncthreads();
    return min(nxt, inc);
}

// ---- kernel parameters ------------------------------------------------------


struct Params {
    const double *verts;
    long long n;
    const double *err;
    int err_stride;
    double ms, delta;
    long long max_itr;
    unsigned char *collides;
    double *toi, *out_tol;
    long long *checks;
    Header *hdr;
    int *surv;       // level-0 survivors           -> pooled solver
    int *mid;        // pooled solver hand-offs     -> one-warp solver
    int *over;       // one-warp solver hand-offs   -> deep solver
    unsigned char *over_level;   // level at which each hand-off outgrew its slot
    int *deep_list;  // `over` ordered by that level, shallowest first
    int *over_ee;    // segmented batches: the edge-edge hand-offs, apart
    unsigned char *over_level_ee;
    int *deep_list_ee;
    int *jumbo;      // deep queries deferred for lack of frontier pages
    double *kappa;
};

// Per-query parameters of Algorithm 2: eps (Eq. ccd-error), ms, delta, m_I.
struct QP {
    double eps[3];
    double ms, delta;
    long long max_itr;
    double t_max;    // time interval [0, t_max]: t = t_max * s (Sec. 6, SolveMSCCD)
};

__device__ __forceinline__ QP qp_single(const Params &p, long long i)
{
    QP q;
#pragma unroll
    for (int c = 0; c < 3; ++c) q.eps[c] = __ldg(p.err + (size_t)p.err_stride * i + c);
    q.ms = p.ms;
    q.delta = p.delta;
    q.max_itr = p.max_itr;
    q.t_max = 1.0;
    return q;
}

__device__ __forceinline__ void write_result(const Params &p, long long qi, int c, double toi,
                                             double tol, long long n)
{
    p.collides[qi] = (unsigned char)c;
    p.toi[qi] = toi;
    p.out_tol[qi] = tol;
    if (p.checks) p.checks[qi] = n;
}

// ---- 1. level-0 filter ------------------------------------------------------

template <int KIND>
__device__ __forceinline__ void root_query(const Params &p, long long i, const QP &q)
{
    Query Q;
    load_query(p.verts, p.n, i, Q);
    const double(&eps)[3] = q.eps;

    // Corners of [0,t_max] x [0,1]^2.  At t = 0 the position fma(dx, 0, x0)
    // equals x0 (up to the sign of a zero, which no comparison sees); at
    // t = t_max it is fma(dx, t_max, x0); with u, v in {0, 1} the fused steps
    // fma(-u, e1, q) etc. reduce to q or one rounded subtraction, so these are
    // the fixed-order values of F.
    double F[2][2][2][3];
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        double P[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) P[j] = it ? dfma(Q.dx[j], q.t_max, Q.x0[j]) : Q.x0[j];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (KIND == CCD_KIND_VF) {
                double q = dsub(P[c], P[3 + c]);
                double e1 = dsub(P[6 + c], P[3 + c]);
                double e2 = dsub(P[9 + c], P[3 + c]);
                double a1 = dsub(q, e1);
                F[it][0][0][c] = q;
                F[it][1][0][c] = a1;
                F[it][0][1][c] = dsub(q, e2);
                F[it][1][1][c] = dsub(a1, e2);
            } else {
                double d1 = dsub(P[3 + c], P[c]);
                double d2 = dsub(P[9 + c], P[6 + c]);
                double c0 = dsub(P[c], P[6 + c]);                 // v = 0: p1 - p3
                double c1 = dsub(P[c], dadd(d2, P[6 + c]));       // v = 1: p1 - (p3 + d2)
                F[it][0][0][c] = c0;
                F[it][0][1][c] = c1;
                F[it][1][0][c] = dadd(d1, c0);
                F[it][1][1][c] = dadd(d1, c1);
            }
        }
    }
    double m[3], M[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double lo = F[0][0][0][c], hi = lo;
#pragma unroll
        for (int k = 1; k < 8; ++k) {
            double f = F[k >> 2][(k >> 1) & 1][k & 1][c];
            lo = fmin(lo, f);
            hi = fmax(hi, f);
        }
        m[c] = lo;
        M[c] = hi;
    }
    BoxTest bt = box_test(m, M, eps, q.ms, q.delta);
    if (!bt.hit) {
        write_result(p, i, 0, __longlong_as_double(0x7ff0000000000000LL), 0.0, 1);
        return;
    }
    if (1 >= q.max_itr || bt.term) {      // first colliding box of level 0
        write_result(p, i, 1, 0.0, bt.w, 1);
        return;
    }
    // Eq. (kappas) over the corners of [0,1]^3.
    double kt = 0.0, ku = 0.0, kv = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                kt = fmax(kt, fabs(dsub(F[0][a][b][c], F[1][a][b][c])));
                ku = fmax(ku, fabs(dsub(F[a][0][b][c], F[a][1][b][c])));
                kv = fmax(kv, fabs(dsub(F[a][b][0][c], F[a][b][1][c])));
            }
    p.kappa[3 * i + 0] = dmul(3.0, kt);
    p.kappa[3 * i + 1] = dmul(3.0, ku);
    p.kappa[3 * i + 2] = dmul(3.0, kv);
    // warp-aggregated append to the survivor list
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&p.hdr->survivors, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    p.surv[base + __popc(mask & ((1u << lane) - 1u))] = (int)i;
}

template <int KIND>
__global__ void __launch_bounds__(ROOT_THREADS) root_kernel(Params p)
{
    const long long i = (long long)blockIdx.x * ROOT_THREADS + threadIdx.x;
    if (i >= p.n) return;
    root_query<KIND>(p, i, qp_single(p, i));
}

// ---- 3./5. per-query level-synchronous solver (one-warp and deep) ------------

// Runs Algorithm 2 for query qi with BS cooperating threads.  Returns false
// if a level needed more than `cap` boxes (nothing is written then unless
// `fallback` is set, in which case the query is answered as at the check
// limit and the capacity status is recorded).
//
// Bound used to size the deep slots: every box of level l+1 is a child of a
// colliding box of level l whose check index n was below m_I (otherwise the
// query returned), so a level never holds more than 2 (m_I - 1) boxes.
template <int KIND>
__device__ __forceinline__ void count_done(const Params &p, bool deep, long long n,
                                           unsigned long long evals, unsigned long long tqs,
                                           unsigned long long atasks = 0,
                                           unsigned long long split_chunks = 0,
                                           unsigned long long shared_evals = 0)
{
    atomicAdd(deep ? &p.hdr->checks_deep : &p.hdr->checks_small, (unsigned long long)n);
    atomicAdd(deep ? &p.hdr->evals_deep : &p.hdr->evals_small, evals);
    atomicAdd(deep ? &p.hdr->tq_deep : &p.hdr->tq_small, tqs);
    if (KIND == CCD_KIND_EE) {
        atomicAdd(deep ? &p.hdr->tq_deep_ee : &p.hdr->tq_small_ee, tqs);
        atomicAdd(deep ? &p.hdr->evals_deep_ee : &p.hdr->evals_small_ee, evals);
    }
    if (atasks | split_chunks | shared_evals) {
        atomicAdd(&p.hdr->a_tasks_deep, atasks);
        atomicAdd(&p.hdr->split_chunks_deep, split_chunks);
        atomicAdd(&p.hdr->evals_shared_deep, shared_evals);
        if (KIND == CCD_KIND_EE) {
            atomicAdd(&p.hdr->a_tasks_deep_ee, atasks);
            atomicAdd(&p.hdr->evals_shared_deep_ee, shared_evals);
        }
    }
}

// ---- shared partials for the deep solver ----------------------------------------
//
// Within one chunk of a level, boxes of a run share t, and neighbouring boxes
// share u or v values.  The corner expression splits into a partial of one
// parameter at one t and a fused step with the other, each the same rounded
// operations the per-box evaluation performs, so computing every distinct
// partial once per chunk gives bit-identical corners:
//   VF  partial a(t,u) = fma(-u, e1, q),        corner F = fma(-v, e2(t), a);
//   EE  partial c(t,v) = p1 - fma(v, d2, p3),   corner F = fma(u, d1(t), c);
// e2 and d1 are t-quantities, so each kind needs one partial table, keyed by
// (t value, numerator of u for VF / of v for EE).  The chunk's boxes are in
// Q order (ascending t_L), so its distinct t values are the runs' left ends
// plus the right ends that are not the next run's left end, and their dense
// ids follow from one block scan (t_L of run r has id r + gaps up to r; t_R
// has that id + 1).  Distinct keys are found with a shared-memory hash
// table; dense partial ids come from a second block scan; tasks are packed
// into consecutive lanes.  A chunk with more than RUN runs or ENTRY
// distinct partials is evaluated as sub-chunks of SUB boxes, which always fit
// (a box adds at most one run, two t values and four partials); every box
// gets the same rounded operations either way.  The tables scale with the
// block: 128-thread blocks (six per SM) take half of a 256-thread block's.
template <int BS>
struct ShCaps {
    static constexpr int RUN = BS >= 256 ? 128 : BS / 2;     // runs of equal t_L per chunk
    static constexpr int TV = 2 * RUN;                       // distinct t values per chunk
    static constexpr int ENTRY = BS >= 256 ? 512 : 2 * BS;   // partials (one t value each)
    static constexpr int SUB = RUN;
    static constexpr int SLOTS = BS >= 256 ? 2048 : 8 * BS;  // hash slots, power of two
    static_assert(SUB <= RUN && 2 * SUB <= TV && 4 * SUB <= ENTRY,
                  "a sub-chunk always fits the tables");
    static_assert(4 * BS <= SLOTS, "every insert finds its key or an empty slot");
};
constexpr unsigned long long SH_EMPTY = ~0ull;
constexpr unsigned long long SH_VAL_MASK = (1ull << 54) - 1;

template <int BS>
struct SharedUV {
    unsigned long long key[ShCaps<BS>::SLOTS];
    int id[ShCaps<BS>::SLOTS];
    unsigned long long key_by_id[ShCaps<BS>::ENTRY];
    double part[ShCaps<BS>::ENTRY][3];
    double tq[ShCaps<BS>::TV][12];
};

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

template <int SLOTS>
__device__ __forceinline__ int sh_insert(unsigned long long *tab, unsigned long long key,
                                         bool *inserted)
{
    // at most 4 * blockDim.x <= SLOTS distinct keys per chunk (half full for
    // 128- and 256-thread blocks), so probing always ends at the key or at
    // an empty slot
    constexpr int SHIFT = 64 - ilog2(SLOTS);   // the product's top log2(SLOTS) bits
    static_assert((1 << (64 - SHIFT)) == SLOTS, "hash range");
    unsigned h = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> SHIFT);
    for (;;) {
        const unsigned long long old = atomicCAS(&tab[h], SH_EMPTY, key);
        if (old == SH_EMPTY) { *inserted = true; return (int)h; }
        if (old == key) { *inserted = false; return (int)h; }
        h = (h + 1) & (SLOTS - 1);
    }
}

// One chunk, or one sub-chunk, through shared partials: threads v_begin ..
// v_end - 1 hold its boxes (`valid`, one box per thread).
// Returns false, having set nothing, when the chunk exceeds a table (the
// caller then evaluates it as sub-chunks).
template <int KIND, int BS>
__device__ __forceinline__ bool eval_chunk_shared(const Query &Q, const QP &q,
                                                  const Thresholds &TH, const int (&k)[3],
                                                  bool valid, const Box &b, int v_begin,
                                                  int v_end,
                                                  Smem<BS> &s, SharedUV<BS> &sh, BoxTest &bt,
                                                  unsigned long long &tqs,
                                                  unsigned long long &ptasks,
                                                  unsigned long long &shared_evals)
{
    using C = ShCaps<BS>;
    constexpr int PD = KIND == CCD_KIND_VF ? 1 : 2;   // the partial's parameter: u or v
    constexpr int FD = 3 - PD;                        // the fused one: v or u
    const int tid = threadIdx.x;
    s.at[tid] = valid ? b.a[0] : ~0ull;
    for (int j = tid; j < C::SLOTS; j += BS) sh.key[j] = SH_EMPTY;
    __syncthreads();
    // runs of equal t_L, and gaps between consecutive runs' t values (a box
    // outside the (sub-)chunk has a_t = ~0 here)
    const bool start = valid && (tid == 0 || s.at[tid - 1] != b.a[0]);
    const bool gap = start && tid > 0 && s.at[tid - 1] != ~0ull && s.at[tid - 1] + 1 != b.a[0];
    const bool open_r = valid && (tid + 1 >= v_end || (s.at[tid + 1] != b.a[0] &&
                                                         s.at[tid + 1] != b.a[0] + 1));
    int tot;
    const int pk = block_scan_1sync<BS>((start ? 1 : 0) | ((gap ? 1 : 0) << 16), &tot, s.scan_a);
    const int nrun = tot & 0xffff, ntv = nrun + (tot >> 16) + 1;
    if (nrun > C::RUN) return false;               // block-uniform
    const int tl = (pk & 0xffff) + (start ? 0 : -1) + (pk >> 16) + (gap ? 1 : 0);   // id of t_L
    if (start) s.run_at[tl] = b.a[0];
    if (open_r) s.run_at[tl + 1] = b.a[0] + 1;     // t_R not shared with the next run
    int sk[4] = {0, 0, 0, 0};
    unsigned ins = 0;
    unsigned long long kk[4] = {0, 0, 0, 0};
    if (valid) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {   // j = 2 * side + d
            bool fresh;
            kk[j] = ((unsigned long long)(tl + (j >> 1)) << 54) | (b.a[PD] + (j & 1));
            sk[j] = sh_insert<C::SLOTS>(sh.key, kk[j], &fresh);
            if (fresh) ins |= 1u << j;
        }
    }
    __syncthreads();
    const int pack = block_scan_1sync<BS>(__popc(ins), &tot, s.scan_b);
    const int NP = tot;
    const bool share = NP <= C::ENTRY;      // block-uniform
    if (share) {
        int ip = pack;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ins & (1u << j)) { sh.id[sk[j]] = ip; sh.key_by_id[ip] = kk[j]; ++ip; }
        // one task per (t value, axis): the FP64 work of this phase spreads
        // over 3x the warps (and so over all four SM sub-partitions)
        tqs += (unsigned long long)ntv;
        for (int task = tid; task < 3 * ntv; task += BS) {
            const int tv = task / 3;
            t_quantities_axis<KIND>(Q, tscale(q.t_max, dyadic(s.run_at[tv], k[0])), task - 3 * tv,
                                    sh.tq[tv]);
        }
    }
    __syncthreads();
    if (!share) return false;
    ptasks += (unsigned long long)NP;
    shared_evals += (unsigned long long)(v_end - v_begin);
    // this box's partial ids (final since the barrier above), loaded ahead of
    // the partial tasks so that the corners need one shared load, not two
    if (valid) {
#pragma unroll
        for (int j = 0; j < 4; ++j) sk[j] = sh.id[sk[j]];
    }
    for (int task = tid; task < NP; task += BS) {
        const unsigned long long key = sh.key_by_id[task];
        const double x = dyadic(key & SH_VAL_MASK, k[PD]);
        const double *T = sh.tq[(int)(key >> 54)];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            sh.part[task][c] = KIND == CCD_KIND_VF ? dfma(-x, T[3 + c], T[c])
                                                   : dsub(T[c], dfma(x, T[9 + c], T[6 + c]));
    }
    __syncthreads();
    if (valid) {
        long long km[3], kM[3];
        const double yl = dyadic(b.a[FD], k[FD]), yr = dyadic(b.a[FD] + 1, k[FD]);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int i0 = sk[2 * side], i1 = sk[2 * side + 1];
            const double *T = sh.tq[tl + side];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double p0 = sh.part[i0][c], p1 = sh.part[i1][c];
                // VF: fma(-v, e2, a); EE: fma(u, d1, c)
                const double g = KIND == CCD_KIND_VF ? T[6 + c] : T[3 + c];
                long long lo, hi;
                corner_range<KIND == CCD_KIND_VF>(yl, yr, g, p0, p1, lo, hi);
                if (side == 0) { km[c] = lo; kM[c] = hi; }
                else { km[c] = min(km[c], lo); kM[c] = max(kM[c], hi); }
            }
        }
        box_test_keys(km, kM, TH, q.ms, bt.hit, bt.term, bt.w);
    }
    return true;
}

// ---- frontier storage of the level-synchronous solver ---------------------------
//
// Contiguous: two arrays of `cap` boxes owned by the block (one-warp slots and
// the full-size slots, 2 m_I + 64 boxes, which no level can outgrow).
//
// Paged (deep tier): the two level arrays are lists of pages of PAGE_BOXES
// boxes taken from a pool shared by every deep block (of one call, or of all
// calls of a server): memory follows the frontiers actually reached instead
// of the worst case.  Before building a level the block reserves pages for
// 2 ncol children (the most a level of ncol colliding boxes can have) and
// afterwards frees the consumed level and the surplus.  Pages are taken from
// a free bitmap with bounded scans and atomics; nothing waits.  A query that
// cannot get pages is handed back (the caller defers it to a full-size slot,
// where it restarts), so the pool's size changes speed, never results.
constexpr int PAGE_SHIFT = 15;
constexpr long long PAGE_BOXES = 1LL << PAGE_SHIFT;   // 768 KB of boxes
constexpr long long PAGE_MASK = PAGE_BOXES - 1;
constexpr int PT_CAP = 128;                           // pages per level (4.19M boxes)

struct PagePool {
    Box *base;                  // npages pages
    unsigned long long *bits;   // bit set = page free (bits past npages stay clear)
    int nwords;
    int *used, *peak;           // pages held now / at most (may be null)
};

struct PageTables {             // one deep block's page lists (shared memory)
    int pt[2][PT_CAP];
    int got;
};

template <int BS>
struct ContigFrontier {
    Box *cur, *nxt;
    long long cap;
    __device__ __forceinline__ bool init() { return true; }
    __device__ __forceinline__ Box &c(long long i) const { return cur[i]; }
    __device__ __forceinline__ Box &x(long long i) const { return nxt[i]; }
    __device__ __forceinline__ long long room(long long) const { return cap; }
    __device__ __forceinline__ void swap(long long)
    {
        bsync<BS>();
        Box *t = cur;
        cur = nxt;
        nxt = t;
    }
    __device__ __forceinline__ void release() {}
};

// Frees entries [from, to) of page list t (called after a barrier: every
// read of those pages is done).  Each freeing thread fences first, so the
// block's writes to a page are visible before another block can take it.
template <int BS>
__device__ __noinline__ void pages_give(const PagePool &P, PageTables *T, int t, int from, int to)
{
    for (int i = from + (int)threadIdx.x; i < to; i += BS) {
        const int pg = T->pt[t][i];
        __threadfence();
        atomicOr(&P.bits[pg >> 6], 1ull << (pg & 63));
    }
    if (threadIdx.x == 0 && P.used && to > from) atomicSub(P.used, to - from);
}

// Takes `want` pages into page list t; every thread of the block calls it.
// Warp 0 scans the bitmap from a block-dependent word, each lane over its
// own words, clearing set bits with atomicAnd (a bit it cleared is a page
// taken); every loop is bounded.  On failure the pages taken are returned.
template <int BS>
__device__ __noinline__ bool pages_take(const PagePool &P, PageTables *T, int t, int want)
{
    __syncthreads();
    if (threadIdx.x == 0) T->got = 0;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x, nw = P.nwords;
        const int s0 = (int)(((unsigned)blockIdx.x * 2654435761u) % (unsigned)nw);
        for (int k = lane; k < nw; k += 32) {
            if (*(volatile int *)&T->got >= want) break;
            int w = s0 + k;
            if (w >= nw) w -= nw;
            unsigned long long v = *(volatile unsigned long long *)&P.bits[w];
            for (int tries = 0; v != 0ull && tries < 128; ++tries) {
                const int b = __ffsll((long long)v) - 1;
                const unsigned long long m = 1ull << b;
                const unsigned long long old = atomicAnd(&P.bits[w], ~m);
                if (old & m) {
                    const int slot = atomicAdd(&T->got, 1);
                    if (slot < want) T->pt[t][slot] = w * 64 + b;
                    else { atomicOr(&P.bits[w], m); break; }
                }
                if (*(volatile int *)&T->got >= want) break;
                v = old & ~m;
            }
        }
    }
    __syncthreads();
    const int got = min(T->got, want);
    if (got < want) {
        for (int i = (int)threadIdx.x; i < got; i += BS) {
            const int pg = T->pt[t][i];
            atomicOr(&P.bits[pg >> 6], 1ull << (pg & 63));
        }
        return false;
    }
    if (threadIdx.x == 0 && P.used) {
        const int u = atomicAdd(P.used, want) + want;
        if (P.peak) atomicMax(P.peak, u);
    }
    return true;
}

template <int BS>
struct PagedFrontier {
    const PagePool &P;
    PageTables *T;
    int ic = 0;               // page list of the current level
    int ncur = 0, nnxt = 0;   // pages held (block-uniform)

    __device__ __forceinline__ Box &c(long long i) const
    {
        return P.base[((size_t)T->pt[ic][i >> PAGE_SHIFT] << PAGE_SHIFT) | (size_t)(i & PAGE_MASK)];
    }
    __device__ __forceinline__ Box &x(long long i) const
    {
        return P.base[((size_t)T->pt[ic ^ 1][i >> PAGE_SHIFT] << PAGE_SHIFT) |
                      (size_t)(i & PAGE_MASK)];
    }
    __device__ __forceinline__ bool init()
    {
        ic = 0;
        ncur = nnxt = 0;
        if (!pages_take<BS>(P, T, 0, 1)) return false;
        ncur = 1;
        return true;
    }
    // room for the children of ncol colliding boxes, or -1 without pages
    __device__ __forceinline__ long long room(long long ncol)
    {
        const long long want = (2 * ncol + PAGE_BOXES - 1) >> PAGE_SHIFT;
        if (want > PT_CAP || !pages_take<BS>(P, T, ic ^ 1, (int)want)) return -1;
        nnxt = (int)want;
        return want << PAGE_SHIFT;
    }
    __device__ __forceinline__ void swap(long long nchild)
    {
        __syncthreads();   // every read of the current level is done
        const int keep = (int)((nchild + PAGE_BOXES - 1) >> PAGE_SHIFT);
        pages_give<BS>(P, T, ic, 0, ncur);
        pages_give<BS>(P, T, ic ^ 1, keep, nnxt);
        ncur = keep;
        nnxt = 0;
        ic ^= 1;
        __syncthreads();
    }
    __device__ __forceinline__ void release()
    {
        __syncthreads();
        pages_give<BS>(P, T, ic, 0, ncur);
        pages_give<BS>(P, T, ic ^ 1, 0, nnxt);
        ncur = nnxt = 0;
        __syncthreads();
    }
};

// Marks the pool's npages pages free (bits past npages stay clear).
__global__ void pool_init_kernel(unsigned long long *bits, int nwords, int npages)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    const int lo = w * 64;
    const int k = npages - lo >= 64 ? 64 : (npages - lo > 0 ? npages - lo : 0);
    bits[w] = k == 64 ? ~0ull : ((1ull << k) - 1ull);
}

template <int KIND, int BS, class FR>
__device__ bool solve_query(const Params &p, const QP &q, long long qi, FR &F, bool fallback,
                            Smem<BS> &s, double *tq, int &hand_level)
{
    const int tid = threadIdx.x;
    unsigned long long evals = 0;   // boxes evaluated (thread 0's tally)
    unsigned long long tqs = 0;     // t-quantity evaluations (thread 0's tally)
    unsigned long long atasks = 0, split_chunks = 0, shared_evals = 0;
    Query &Q = s.query;             // shared: only the per-run tasks read it
    if (tid < 12) {
        const double a = __ldg(p.verts + (size_t)tid * p.n + qi);
        const double b = __ldg(p.verts + (size_t)(12 + tid) * p.n + qi);
        Q.x0[tid] = a;
        Q.dx[tid] = dsub(b, a);
    }
    double kap[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) kap[c] = p.kappa[3 * qi + c];
    Thresholds TH;
    make_thresholds(q.eps, q.delta, TH);
    constexpr int W = TWidth<KIND>::W;
    int k[3] = {0, 0, 0};
    long long size = 1;
    if (!F.init()) {                 // no frontier page: deferred
        hand_level = -1;
        return false;
    }
    if (tid == 0) F.c(0) = Box{{0ull, 0ull, 0ull}};
    bsync<BS>();
    long long n_before = 0;

    for (;;) {
        // split(): c_d = w(I_d) kappa_d, ties t > u > v.  Same for the level.
        const int sd = split_dim(scale2neg(kap[0], k[0]), scale2neg(kap[1], k[1]),
                                 scale2neg(kap[2], k[2]));
        // (the deep solver uses selects where the one-warp solver indexes by sd: a
        // dynamic index there puts k and the child boxes in local memory, which
        // kept the VF deep solver from three blocks per SM)
        const bool can_split = (BS > 32 ? (sd == 0 ? k[0] : sd == 1 ? k[1] : k[2]) : k[sd]) < KMAX;

        bool found = false;
        unsigned long long if_at = 0;
        double first_w = 0.0;
        long long ncol = 0;
        for (long long base = 0; base < size; base += BS) {
            const long long i = base + tid;
            const bool valid = i < size;
            Box b = Box{{0ull, 0ull, 0ull}};
            BoxTest bt{false, false, 0.0};
            if (valid) b = F.c(i);
            if (BS > 32) {
                // the whole chunk, else its sub-chunks in turn (block-uniform;
                // a sub-chunk always fits, so each pass makes progress)
                const int nv = (int)min((long long)BS, size - base);
                int h = 0, he = nv;
                for (;;) {
                    const bool done = eval_chunk_shared<KIND, BS>(
                        Q, q, TH, k, valid && tid >= h && tid < he, b, h, he, s,
                        *(SharedUV<BS> *)tq, bt, tqs, atasks, shared_evals);
                    if (done && he >= nv) break;
                    if (done) h = he;
                    else if (he - h <= ShCaps<BS>::SUB) break;   // unreachable: see ShCaps
                    else ++split_chunks;
                    he = min(nv, h + ShCaps<BS>::SUB);
                }
            } else {
            // Boxes are in Q order, so equal t_L form contiguous runs: the
            // t-quantities at t_L and t_R are computed once per run.
            s.at[tid] = valid ? b.a[0] : ~0ull;
            bsync<BS>();
            const bool start = valid && (tid == 0 || s.at[tid - 1] != b.a[0]);
            int nrun;
            const int before = block_excl_scan<BS>(start ? 1 : 0, &nrun, s);
            const int run = before + (start ? 0 : -1);
            if (start) s.run_at[before] = b.a[0];
            bsync<BS>();
            tqs += 2 * (unsigned long long)nrun;
            for (int task = tid; task < 2 * nrun; task += BS)
                t_quantities<KIND>(Q, tscale(q.t_max, dyadic(s.run_at[task >> 1] + (task & 1), k[0])),
                                   tq + task * W);
            bsync<BS>();
            if (valid) {
                long long km[3], kM[3];
                corners_keys<KIND>(tq + (2 * run) * W, tq + (2 * run + 1) * W,
                                   dyadic(b.a[1], k[1]), dyadic(b.a[1] + 1, k[1]),
                                   dyadic(b.a[2], k[2]), dyadic(b.a[2] + 1, k[2]), km, kM);
                box_test_keys(km, kM, TH, q.ms, bt.hit, bt.term, bt.w);
            }
            }
            evals += (unsigned long long)min((long long)BS, size - base);
            const long long nb = n_before + i + 1;
            // one barrier: each warp publishes its colliding count, its first
            // colliding box (a_t, w(B), termination) and its first box past the
            // check limit; every thread then derives the block-wide answers
            {
                const int lane = tid & 31, warp = tid >> 5;
                const unsigned mh = __ballot_sync(0xffffffffu, bt.hit);
                const unsigned mc = __ballot_sync(0xffffffffu, bt.hit && nb >= q.max_itr);
                const int fh = mh ? __ffs(mh) - 1 : 32, fcl = mc ? __ffs(mc) - 1 : 32;
                if (lane == 0) {
                    s.dec[warp].count = __popc(mh);
                    s.dec[warp].first = fh;
                    s.dec[warp].first_cut = fcl;
                }
                if (lane == fh) {
                    s.dec[warp].at = b.a[0];
                    s.dec[warp].w = bt.w;
                    s.dec[warp].term = bt.term;
                }
                if (lane == fcl) s.dec[warp].w_cut = bt.w;
                bsync<BS>();
                int before = 0, total = 0, wf = -1, wc = -1;
#pragma unroll
                for (int w = 0; w < BS / 32; ++w) {
                    const int c = s.dec[w].count;
                    before += (w < warp) ? c : 0;
                    total += c;
                    if (wf < 0 && c > 0) wf = w;
                    if (wc < 0 && s.dec[w].first_cut < 32) wc = w;
                }
                if (!found && wf >= 0) {
                    found = true;
                    if_at = s.dec[wf].at;
                    first_w = s.dec[wf].w;
                    const long long nfc = n_before + base + wf * 32 + s.dec[wf].first + 1;
                    if (nfc >= q.max_itr || s.dec[wf].term || !can_split) {
                        if (tid == 0) {
                            write_result(p, qi, 1, dmul(q.t_max, dyadic(if_at, k[0])), first_w,
                                         nfc);
                            count_done<KIND>(p, BS > 32, nfc, evals, tqs, atasks, split_chunks,
                                       shared_evals);
                        }
                        F.release();
                        return true;
                    }
                }
                if (wc >= 0) {   // a later colliding box reached the check limit
                    const long long ncut = n_before + base + wc * 32 + s.dec[wc].first_cut + 1;
                    if (tid == 0) {
                        write_result(p, qi, 1, dmul(q.t_max, dyadic(if_at, k[0])),
                                     s.dec[wc].w_cut, ncut);
                        count_done<KIND>(p, BS > 32, ncut, evals, tqs, atasks, split_chunks, shared_evals);
                    }
                    F.release();
                    return true;
                }
                const int pre = before + __popc(mh & ((1u << lane) - 1u));
                if (bt.hit) F.c(ncol + pre) = b;   // in-place compaction, ncol + pre <= i
                ncol += total;
            }
            bsync<BS>();
        }
        if (!found) {
            if (tid == 0) {
                write_result(p, qi, 0, __longlong_as_double(0x7ff0000000000000LL), 0.0,
                             n_before + size);
                count_done<KIND>(p, BS > 32, n_before + size, evals, tqs, atasks, split_chunks, shared_evals);
            }
            F.release();
            return true;
        }
        n_before += size;

        // children of the ncol colliding boxes, in Q order
        const long long cap = F.room(ncol);
        if (cap < 0) {                  // no pages for the next level: deferred
            if (tid == 0) count_done<KIND>(p, true, 0, evals, tqs, atasks, split_chunks, shared_evals);
            F.release();
            hand_level = -1;
            return false;
        }
        long long nchild;
        if (sd == 0) {
            nchild = 2 * ncol;
            if (nchild <= cap) {
                long long carry = -1;   // start of the open group of equal I_t
                for (long long base = 0; base < ncol; base += BS) {
                    const long long j = base + tid;
                    const bool valid = j < ncol;
                    Box b = Box{{0ull, 0ull, 0ull}};
                    long long v = -1;
                    if (valid) {
                        b = F.c(j);
                        if (j == 0 || F.c(j - 1).a[0] != b.a[0]) v = j;
                    }
                    long long blk;
                    const long long gs = max(carry, block_incl_maxscan<BS>(v, s, &blk));
                    if (valid) F.x(j + gs) = Box{{2 * b.a[0], b.a[1], b.a[2]}};
                    carry = max(carry, blk);
                }
                long long carry_e = ncol;   // end of the open group, scanning backwards
                const long long last = ((ncol - 1) / BS) * BS;
                for (long long base = last; base >= 0; base -= BS) {
                    const long long j = base + tid;
                    const bool valid = j < ncol;
                    Box b = Box{{0ull, 0ull, 0ull}};
                    long long v = BIGL;
                    if (valid) {
                        b = F.c(j);
                        if (j + 1 == ncol || F.c(j + 1).a[0] != b.a[0]) v = j + 1;
                    }
                    long long blk;
                    const long long ge = min(carry_e, block_suffix_min<BS>(v, s, &blk));
                    if (valid) F.x(j + ge) = Box{{2 * b.a[0] + 1, b.a[1], b.a[2]}};
                    carry_e = min(carry_e, blk);
                }
            }
        } else {
            long long carry = 0;        // right children kept so far
            for (long long base = 0; base < ncol; base += BS) {
                const long long j = base + tid;
                const bool valid = j < ncol;
                Box b = Box{{0ull, 0ull, 0ull}};
                bool keep_r = false;
                if (valid) {
                    b = F.c(j);
                    keep_r = true;
                    if (KIND == CCD_KIND_VF) {
                        // right child meets the prism iff u_L + v_L <= 1 (exact)
                        const int ku = k[1] + (sd == 1), kv = k[2] + (sd == 2);
                        const unsigned long long au = sd == 1 ? 2 * b.a[1] + 1 : b.a[1];
                        const unsigned long long av = sd == 2 ? 2 * b.a[2] + 1 : b.a[2];
                        const int K = ku > kv ? ku : kv;
                        keep_r = (au << (K - ku)) + (av << (K - kv)) <= (1ull << K);
                    }
                }
                int total;
                const int pre = block_excl_scan<BS>(keep_r ? 1 : 0, &total, s);
                if (valid) {
                    const long long pos = j + carry + pre;
                    Box l = b, r = b;
                    if (BS > 32) {
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            l.a[d] = d == sd ? 2 * b.a[d] : b.a[d];
                            r.a[d] = d == sd ? 2 * b.a[d] + 1 : b.a[d];
                        }
                    } else {
                        l.a[sd] = 2 * b.a[sd];
                        r.a[sd] = 2 * b.a[sd] + 1;
                    }
                    if (pos < cap) F.x(pos) = l;
                    if (keep_r && pos + 1 < cap) F.x(pos + 1) = r;
                }
                carry += total;
            }
            nchild = ncol + carry;
        }
        if (nchild > cap) {
            if (!fallback) {
                if (tid == 0) count_done<KIND>(p, false, 0, evals, tqs);
                hand_level = k[0] + k[1] + k[2];
                F.release();
                return false;
            }
            // answered as at the check limit: conservative, flagged
            if (tid == 0) {
                write_result(p, qi, 1, dmul(q.t_max, dyadic(if_at, k[0])), first_w, n_before);
                atomicExch(&p.hdr->status, (int)CCD_ERR_CAPACITY);
                atomicAdd(&p.hdr->fallbacks, 1);
                count_done<KIND>(p, true, n_before, evals, tqs, atasks, split_chunks, shared_evals);
            }
            F.release();
            return true;
        }
        F.swap(nchild);
        size = nchild;
        if (BS > 32) {
#pragma unroll
            for (int d = 0; d < 3; ++d) k[d] += d == sd;
        } else {
            k[sd] += 1;
        }
    }
}

// Persistent: blocks take queries from `list` (length *count, work counter
// *head); a query whose frontier outgrows `cap` goes to out_list, with the
// level it reached in out_level when that is not null (one-warp tier only;
// the deep tier answers it through the capacity fallback).
//
// PAGED (deep tier): frontier pages come from `pool`; a query that cannot get
// them goes to out_list (the full-size stage), where it restarts.
template <int KIND, int BS, bool PAGED = false>
__global__ void __launch_bounds__(BS, deep_blocks_per_sm(BS))
    solve_kernel(Params p, int deep, Box *slots, long long cap, PagePool pool, const int *list,
                 const int *count, int *head, int *out_list, unsigned char *out_level,
                 int *out_count)
{
    __shared__ Smem<BS> s;
    __shared__ int s_idx;
    extern __shared__ double tq[];   // [2 * BS][TWidth<KIND>::W] t-quantities
    Box *cur = slots + (size_t)blockIdx.x * 2 * (size_t)cap;
    Box *nxt = cur + cap;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(head, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= *(volatile const int *)count) return;
        const long long qi = list[idx];
        int level = 0;
        bool done;
        if constexpr (PAGED) {
            __shared__ PageTables pt;
            PagedFrontier<BS> F{pool, &pt};
            done = solve_query<KIND, BS>(p, qp_single(p, qi), qi, F, false, s, tq, level);
        } else {
            ContigFrontier<BS> F{cur, nxt, cap};
            done = solve_query<KIND, BS>(p, qp_single(p, qi), qi, F, deep != 0, s, tq, level);
        }
        if (!done && threadIdx.x == 0 && out_count) {
            const int j = atomicAdd(out_count, 1);
            out_list[j] = (int)qi;
            if (out_level) out_level[j] = (unsigned char)level;
        }
        __syncthreads();
    }
}

// Deep-tier schedule.  The level at which a query's frontier outgrew the
// one-warp slot predicts its remaining work closely (the shallower, the
// wider the colliding region and the more boxes it takes), so the deep
// solver takes them shallowest first (longest-first scheduling shortens the
// tail where blocks run out of queries).  One block, counting sort over the
// levels (at most 3 * KMAX < 256); the order within a level is arbitrary.
// Results do not depend on the order.
__global__ void __launch_bounds__(1024)
    order_by_level_kernel(const int *in, const unsigned char *level, const int *count, int *out)
{
    __shared__ int hist[256];
    const int n = *count;
    const int tid = threadIdx.x;
    if (tid < 256) hist[tid] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) atomicAdd(&hist[level[i]], 1);
    __syncthreads();
    if (tid < 32) {   // exclusive scan of the 256 bins, 8 per lane
        int v[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) { v[j] = hist[tid * 8 + j]; sum += v[j]; }
        int inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (tid >= o) inc += y;
        }
        int run = inc - sum;
#pragma unroll
        for (int j = 0; j < 8; ++j) { hist[tid * 8 + j] = run; run += v[j]; }
    }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) out[atomicAdd(&hist[level[i]], 1)] = in[i];
}

// ---- segment tables ------------------------------------------------------------

static_assert(sizeof(ccd_segment) == 80, "ccd_segment layout");

// Segment of query i: the last segment whose offset is <= i.
__device__ __forceinline__ int find_segment(const ccd_segment *segs, int nseg, long long i)
{
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].offset <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ QP qp_segment(const ccd_segment &sg)
{
    QP q;
#pragma unroll
    for (int c = 0; c < 3; ++c) q.eps[c] = sg.err[c];
    q.ms = sg.ms;
    q.delta = sg.delta;
    q.max_itr = sg.max_itr;
    q.t_max = sg.t_max;
    return q;
}

// ---- pooled solver (small frontiers, many queries per warp) -------------------
//
// An FP64 warp-instruction costs the same for 1 or 32 active lanes, and most
// surviving queries have only a few boxes per level.  A warp here holds up
// to POOL_SLOTS queries ("slots") and, every iteration, packs the next boxes
// of all its slots' current levels into its 32 lanes (slot priority rotates
// so that no slot waits long), evaluates them with the same code path, then
// lets each slot's owner lane apply Algorithm 2's sequential bookkeeping to
// its boxes in Q order: first colliding box, check limit, termination,
// children appended in Q order (u and v splits: left then right; t splits: the
// right children of a run of equal t_L wait in a pending list flushed when
// the run ends).  A level with more children than the slot capacity hands the
// query to the one-warp solver, which restarts it.
struct PoolSlot {
    int qi;                                      // query index (batches hold < 2^31)
    int n_before;                                // checks before this level: at most
                                                 // 3 KMAX levels of pool_cap boxes
    unsigned long long if_at, pend_at;
    int size, pos, nn, np;                       // at most pool_cap (<= 4096)
    unsigned char k[3], sd, can_split, found, buf, t_one;   // t_one: t_max == 1
};

// A slot's query record lives in global memory (one per slot of the
// workspace) and is read through L1; keeping it out of shared memory lets
// about twice as many pooled warps reside on an SM.
struct PoolMeta {
    Query Q;
    QP qp;
    double kap[3];
};

// What a slot's lanes decided in one iteration, for the slot's owner lane.
struct PoolAgg {
    unsigned long long at_fh;     // t_L numerator of the first colliding box
    unsigned long long at_k;      // ... of the last run
    unsigned char outcome;        // 0 continue, 1 answered, 2 handed over
    unsigned char fh;             // a colliding box in the iteration (0 / 1)
    unsigned char runs;           // t split: runs of equal t_L that start here
    unsigned char cnt0, cntk;     // t split: colliding boxes of the first / last run
    unsigned char hits;           // colliding boxes
    unsigned char children;       // u / v split: children written
    unsigned char pad;
};

constexpr int TV_SLOT_SHIFT = 58;     // numerators stay below 2^54
constexpr unsigned long long TV_A_MASK = (1ull << TV_SLOT_SHIFT) - 1;

template <int KIND>
struct PoolShared {
    PoolSlot st[POOL_SLOTS];
    unsigned char seg_slot[32];   // slot of the segment of lanes starting at a lane
    // distinct t values of an iteration (at most 32 runs + 31 gaps + 1):
    // t-quantities, and slot << TV_SLOT_SHIFT | t_L numerator
    double tq[64][TWidth<KIND>::W];
    unsigned long long tv_a[64];
    union {
        // distinct partials of an iteration (box evaluation): key (t value
        // id << 56 | endpoint numerator) and value per axis
        struct {
            unsigned long long pk[POOL_PCAP];
            double part[POOL_PCAP][3];
        } sp;
        PoolAgg agg[POOL_SLOTS];  // the slots' decisions (bookkeeping, after it)
    };
};

__device__ __forceinline__ void pool_split_dim(PoolSlot &S, const double (&kap)[3])
{
    S.sd = split_dim(scale2neg(kap[0], S.k[0]), scale2neg(kap[1], S.k[1]),
                     scale2neg(kap[2], S.k[2]));
    S.can_split = S.k[S.sd] < KMAX;
}

// Queries come from `list` (length *count, work counter *head).  With a
// segment table (segs != nullptr) each query takes its tolerances from its
// segment and queries of the other kind are skipped (one launch per kind).
template <int KIND>
__global__ void __launch_bounds__(32, KIND == 0 ? POOL_BLOCKS_PER_SM : POOL_BLOCKS_EE)
    pool_kernel(Params p, Box *mem, PoolMeta *metas, int cap, const int *list, const int *count_p,
                int *head, const ccd_segment *segs, int nseg)
{
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ PoolShared<KIND> sh;
    const int lane = threadIdx.x;
    PoolSlot &S = sh.st[lane];                     // the slot this lane owns
    PoolMeta *const meta = metas + (size_t)blockIdx.x * POOL_SLOTS;   // the warp's slots
    Box *const mine = mem + ((size_t)blockIdx.x * POOL_SLOTS + lane) * 3 * (size_t)cap;
    const int count = *(volatile const int *)count_p;
    bool drained = false;
    unsigned long long evals = 0, checks_done = 0, tqs = 0, iters = 0, serial = 0;
    unsigned long long ptasks = 0, shared_evals = 0;
    int rot = 0;
    S.qi = -1;
    __syncwarp();

    for (;;) {
        // 1. empty slots take the next survivors (warp-aggregated)
        const bool empty = S.qi < 0;
        const unsigned want = __ballot_sync(FULL, empty && !drained);
        if (want) {
            const int leader = __ffs(want) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(head, __popc(want));
            base = __shfl_sync(FULL, base, leader);
            if (empty && !drained) {
                const int idx = base + __popc(want & ((1u << lane) - 1u));
                long long qi = -1;
                bool mine_kind = true;
                if (idx < count) {
                    qi = list[idx];
                    if (segs) {
                        const ccd_segment sg = segs[find_segment(segs, nseg, qi)];
                        mine_kind = sg.kind == KIND;
                        if (mine_kind) meta[lane].qp = qp_segment(sg);
                    } else {
                        meta[lane].qp = qp_single(p, qi);
                    }
                }
                if (idx < count && mine_kind) {
                    load_query(p.verts, p.n, qi, meta[lane].Q);
#pragma unroll
                    for (int c = 0; c < 3; ++c) meta[lane].kap[c] = p.kappa[3 * qi + c];
                    S.qi = (int)qi;
                    S.size = 1;
                    S.pos = 0;
                    S.n_before = 0;
                    S.found = 0;
                    S.nn = S.np = 0;
                    S.buf = 0;
                    S.k[0] = S.k[1] = S.k[2] = 0;
                    S.t_one = tmax_one(meta[lane].qp.t_max);
                    pool_split_dim(S, meta[lane].kap);
                    mine[0] = Box{{0ull, 0ull, 0ull}};
                } else if (idx >= count) {
                    drained = true;
                }   // a query of the other kind: this slot takes another next time
            }
        }
        __syncwarp();
        const bool active = S.qi >= 0;
        if (!__any_sync(FULL, active) && __all_sync(FULL, drained)) break;

        // 2. place the slots' next boxes in the lanes, rotating the priority:
        // slot s takes lanes [E_s, E_s + take_s); a lane finds its slot from
        // the mask of segment starts
        const int rem = active ? min(S.size - S.pos, 32) : 0;
        const int rrem = __shfl_sync(FULL, rem, (lane + rot) & 31);
        int inc = rrem;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        const int total = __shfl_sync(FULL, inc, 31);
        const int E = __shfl_sync(FULL, inc - rrem, (lane - rot) & 31);
        const int take = (active && E < 32) ? min(rem, 32 - E) : 0;
        rot = (rot + 1) & 31;
        const unsigned starts = __reduce_or_sync(FULL, take > 0 ? (1u << E) : 0u);
        if (take > 0) sh.seg_slot[E] = lane;
        __syncwarp();
        const int nbox = min(total, 32);
        const bool have = lane < nbox;
        const unsigned below = 0xffffffffu >> (31 - lane);          // lanes <= this one
        const int st0 = have ? 31 - __clz(starts & below) : lane;    // first lane of my segment
        const unsigned later = starts & ~below;
        const int en0 = have ? (later ? __ffs(later) - 1 : nbox) : lane + 1;
        const unsigned segmask = have ? ((en0 == 32 ? 0xffffffffu : ((1u << en0) - 1u)) &
                                         ~((1u << st0) - 1u))
                                      : 0u;
        const int so = have ? sh.seg_slot[st0] : 0;
        const int off = lane - st0;
        iters += 1;
        serial += (unsigned long long)__reduce_max_sync(FULL, (unsigned)take);

        // 3. one box per lane.  A slot's boxes sit in consecutive lanes in Q
        // order (ascending t_L), so the iteration's distinct t values get
        // dense ids from one warp scan (t_L of a run: run + gaps so far; t_R:
        // that id + 1; a slot change counts as a gap); their t-quantities are
        // computed once, one task per (t value, axis), then every lane takes
        // the corners of its box from them.
        BoxTest bt{false, false, 0.0};
        Box b = Box{{0ull, 0ull, 0ull}};
        Box *const sbase = mem + ((size_t)blockIdx.x * POOL_SLOTS + so) * 3 * (size_t)cap;
        const PoolSlot &T = sh.st[so];
        if (have) {
            b = sbase[(T.buf ? cap : 0) + T.pos + off];
            evals += 1;
        }
        const unsigned long long at = b.a[0];
        const int so_prev = __shfl_up_sync(FULL, so, 1), so_next = __shfl_down_sync(FULL, so, 1);
        const unsigned long long at_prev = __shfl_up_sync(FULL, at, 1);
        const unsigned long long at_next = __shfl_down_sync(FULL, at, 1);
        const bool start = have && (lane == 0 || so_prev != so || at_prev != at);
        const bool gap = start && lane > 0 && !(so_prev == so && at_prev + 1 == at);
        const bool open_r = have && (lane + 1 >= nbox ||
                                     !(so_next == so && (at_next == at || at_next == at + 1)));
        int pk = (start ? 1 : 0) | ((gap ? 1 : 0) << 8);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, pk, o);
            if (lane >= o) pk += y;
        }
        const int tl = (pk & 0xff) - 1 + (pk >> 8);
        const int last = __shfl_sync(FULL, pk, 31);
        const int ntv = nbox > 0 ? (last & 0xff) + (last >> 8) + 1 : 0;
        tqs += (unsigned long long)ntv;   // warp-uniform: every lane's tally is the warp's
        if (start) sh.tv_a[tl] = ((unsigned long long)so << TV_SLOT_SHIFT) | at;
        if (open_r) sh.tv_a[tl + 1] = ((unsigned long long)so << TV_SLOT_SHIFT) | (at + 1);
        __syncwarp();
        // t = t_max s, where t_max == 1 (the whole step) needs no multiply: a
        // warp-uniform branch, so that the multiply is not issued at all
        if (__all_sync(FULL, S.qi < 0 || S.t_one)) {
            for (int task = lane; task < 3 * ntv; task += 32) {
                const int tv = task / 3;
                const unsigned long long ta = sh.tv_a[tv];
                const int s2 = (int)(ta >> TV_SLOT_SHIFT);
                t_quantities_axis<KIND>(meta[s2].Q, dyadic(ta & TV_A_MASK, sh.st[s2].k[0]),
                                        task - 3 * tv, sh.tq[tv]);
            }
        } else {
            for (int task = lane; task < 3 * ntv; task += 32) {
                const int tv = task / 3;
                const unsigned long long ta = sh.tv_a[tv];
                const int s2 = (int)(ta >> TV_SLOT_SHIFT);
                t_quantities_axis<KIND>(meta[s2].Q,
                                        dmul(meta[s2].qp.t_max, dyadic(ta & TV_A_MASK, sh.st[s2].k[0])),
                                        task - 3 * tv, sh.tq[tv]);
            }
        }
        __syncwarp();                  // the t-quantities, for every lane
        // Partials shared by the iteration's boxes, per axis: VF a(t, u) =
        // fma(-u, e1, q), EE c(t, v) = p1 - fma(v, d2, p3), keyed by (t value
        // id, endpoint numerator; a slot's boxes share one level, so one k).
        // A box needs four: its two t values times its two endpoints.  Of
        // {tl, tl + 1} one is even and one odd, and so are the endpoints a and
        // a + 1, so each of a box's keys has its own class (t parity, endpoint
        // parity) and equal keys always meet in the same class: one match per
        // class finds every repeat.  The distinct partials are computed once
        // each, as a dense task list, and the boxes read them from shared
        // memory (the same fused operations as evaluating the corners
        // directly, so the same bits).
        constexpr int PD = KIND == CCD_KIND_VF ? 1 : 2;   // the partial's parameter
        constexpr int FD = 3 - PD;                        // the fused one
        const unsigned hmask = __ballot_sync(FULL, have);
        const unsigned long long e0 = b.a[PD];
        const int pt = tl & 1, pe = (int)(e0 & 1);
        int pid[4];       // id of this box's key of class (t parity << 1 | endpoint parity)
        int np = 0;
#pragma unroll
        for (int cls = 0; cls < 4; ++cls) {
            const int tv = ((cls >> 1) == pt) ? tl : tl + 1;
            const unsigned long long key =
                ((unsigned long long)tv << 56) | (((cls & 1) == pe) ? e0 : e0 + 1);
            unsigned m = 0;
            if (have) m = __match_any_sync(hmask, key);
            const int lead = have ? __ffs(m) - 1 : lane;
            const unsigned L = __ballot_sync(FULL, have && lead == lane);
            pid[cls] = np + __popc(L & ((1u << lead) - 1u));
            if (have && lead == lane && pid[cls] < POOL_PCAP) sh.sp.pk[pid[cls]] = key;
            np += __popc(L);
        }
        const bool shared_p = np <= POOL_PCAP;           // warp-uniform
        if (shared_p) {
            ptasks += (unsigned long long)np;             // warp-uniform tally
            shared_evals += (unsigned long long)nbox;
            __syncwarp();              // the keys
            for (int task = lane; task < np; task += 32) {
                const unsigned long long key = sh.sp.pk[task];
                const int tv = (int)(key >> 56);
                const double x = dyadic(key & ((1ull << 56) - 1),
                                        sh.st[(int)(sh.tv_a[tv] >> TV_SLOT_SHIFT)].k[PD]);
                const double *Tq = sh.tq[tv];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    sh.sp.part[task][c] = KIND == CCD_KIND_VF
                                           ? dfma(-x, Tq[3 + c], Tq[c])
                                           : dsub(Tq[c], dfma(x, Tq[9 + c], Tq[6 + c]));
            }
            __syncwarp();
        }
        if (have) {
            long long km[3], kM[3];
            if (shared_p) {
                const double yl = dyadic(b.a[FD], T.k[FD]), yr = dyadic(b.a[FD] + 1, T.k[FD]);
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    // classes of (tl + side, a) and (tl + side, a + 1)
                    const int c0 = ((pt ^ side) << 1) | pe, c1 = c0 ^ 1;
                    const int i0 = c0 == 0 ? pid[0] : c0 == 1 ? pid[1] : c0 == 2 ? pid[2] : pid[3];
                    const int i1 = c1 == 0 ? pid[0] : c1 == 1 ? pid[1] : c1 == 2 ? pid[2] : pid[3];
                    const double *Tq = sh.tq[tl + side];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        // VF: fma(-v, e2, a); EE: fma(u, d1, c)
                        const double g = KIND == CCD_KIND_VF ? Tq[6 + c] : Tq[3 + c];
                        long long lo, hi;
                        corner_range<KIND == CCD_KIND_VF>(yl, yr, g, sh.sp.part[i0][c],
                                                          sh.sp.part[i1][c], lo, hi);
                        if (side == 0) { km[c] = lo; kM[c] = hi; }
                        else { km[c] = min(km[c], lo); kM[c] = max(kM[c], hi); }
                    }
                }
            } else {
                corners_keys<KIND>(sh.tq[tl], sh.tq[tl + 1], dyadic(b.a[1], T.k[1]),
                                   dyadic(b.a[1] + 1, T.k[1]), dyadic(b.a[2], T.k[2]),
                                   dyadic(b.a[2] + 1, T.k[2]), km, kM);
            }
            Thresholds TH;   // a few integer operations: cheaper than keeping 32 in shared memory
            make_thresholds(meta[so].qp.eps, meta[so].qp.delta, TH);
            box_test_keys(km, kM, TH, meta[so].qp.ms, bt.hit, bt.term, bt.w);
        }

        __syncwarp();   // the partials are read: their space takes the decisions next
        // 4. Algorithm 2's bookkeeping for every slot at once, with the
        // results of the sequential loop over the slot's boxes in Q order.
        // Box at lane L is check n = n_before + pos + (L - E) + 1.  Ballots
        // over the slot's lanes give its first colliding box fh, the first
        // box that returns (A: n >= m_I, or the level's first colliding box
        // terminating or unsplittable) and the first whose children would
        // not fit (O); the query returns at A if A <= O, is handed on at O
        // otherwise, else every colliding box writes its children where the
        // loop would: u / v splits at the slot's count plus a segmented
        // prefix count; t splits in runs of equal t_L, all left children of
        // a run, then its right children, where a run still open at the end
        // of the iteration keeps its right children in the pending list.
        const long long n_L = (long long)T.n_before + T.pos + off + 1;
        const bool hit = have && bt.hit;
        const unsigned Hs = __ballot_sync(FULL, hit) & segmask;
        const int fh = Hs ? __ffs(Hs) - 1 : -1;
        const int sd = T.sd;
        const bool ans = hit && (n_L >= meta[so].qp.max_itr ||
                                 (lane == fh && !T.found && (bt.term || !T.can_split)));
        bool keep_r = true;
        if (KIND == CCD_KIND_VF && hit && sd != 0) {   // right child meets the prism iff u_L + v_L <= 1
            const int ku = T.k[1] + (sd == 1), kv = T.k[2] + (sd == 2);
            const unsigned long long au = sd == 1 ? 2 * b.a[1] + 1 : b.a[1];
            const unsigned long long av = sd == 2 ? 2 * b.a[2] + 1 : b.a[2];
            const int K = ku > kv ? ku : kv;
            keep_r = (au << (K - ku)) + (av << (K - kv)) <= (1ull << K);
        }
        const int c = hit ? (sd == 0 ? 2 : 1 + (keep_r ? 1 : 0)) : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {   // segmented inclusive scan of the children
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane - o >= st0) incl += y;
        }
        const bool ov = hit && (T.nn + T.np + incl > cap);
        const unsigned As = __ballot_sync(FULL, ans) & segmask;
        const unsigned Os = __ballot_sync(FULL, ov) & segmask;
        const int A = As ? __ffs(As) - 1 : 32, O = Os ? __ffs(Os) - 1 : 32;
        const int outcome = (A < 32 && A <= O) ? 1 : (O < 32 ? 2 : 0);
        const unsigned long long at_fh = __shfl_sync(FULL, at, fh < 0 ? lane : fh);
        // t split: runs of equal t_L among the slot's colliding boxes; the
        // first may continue the run left open by the previous iteration
        const unsigned hb = Hs & ((1u << lane) - 1u);             // colliding boxes before me
        const int ph = hb ? 31 - __clz(hb) : -1;
        const unsigned long long at_ph = __shfl_sync(FULL, at, ph < 0 ? lane : ph);
        const bool run_start = hit && (ph >= 0 ? at_ph != at : !(T.np > 0 && T.pend_at == at));
        const unsigned Rs = __ballot_sync(FULL, run_start) & segmask;
        const int lh = Hs ? 31 - __clz(Hs) : lane;
        const unsigned long long at_lh = __shfl_sync(FULL, at, lh);
        if (have && lane == A && outcome == 1) {
            const unsigned long long if_at = T.found ? T.if_at : at_fh;
            write_result(p, T.qi, 1, dmul(meta[so].qp.t_max, dyadic(if_at, T.k[0])), bt.w, n_L);
            checks_done += (unsigned long long)n_L;
        }
        if (have && lane == en0 - 1) {   // the slot's last lane tells the owner
            PoolAgg &G = sh.agg[so];
            G.outcome = outcome;
            G.fh = fh >= 0;
            G.at_fh = at_fh;
            G.hits = __popc(Hs);
            G.children = incl;
            G.runs = __popc(Rs);
            G.cnt0 = Rs ? __popc(Hs & ((1u << (__ffs(Rs) - 1)) - 1u)) : G.hits;
            G.cntk = Rs ? __popc(Hs & ~((1u << (31 - __clz(Rs))) - 1u)) : G.hits;
            G.at_k = at_lh;
        }
        __syncwarp();
        // the owner moves the previous iteration's pending right children of
        // a run that closes now into the level (before anyone writes pend)
        const bool level_end = take > 0 && S.pos + take == S.size;
        if (take > 0 && S.sd == 0 && S.np > 0 && sh.agg[lane].outcome == 0 &&
            (sh.agg[lane].runs > 0 || level_end)) {
            Box *nx = mine + (S.buf ? 0 : cap);
            const Box *pd = mine + 2 * (size_t)cap;
            for (int x = 0; x < S.np; ++x) nx[S.nn + sh.agg[lane].cnt0 + x] = pd[x];
        }
        __syncwarp();
        if (hit && outcome == 0) {   // my children
            Box *nx = sbase + (T.buf ? 0 : cap);
            if (sd == 0) {
                const unsigned upto = Rs & below;
                const int j = __popc(upto);                               // my run (0: continued)
                const int rs = upto ? 31 - __clz(upto) : st0;             // its first lane
                const unsigned nxt_rs = Rs & ~below;
                const int re = nxt_rs ? __ffs(nxt_rs) - 1 : 32;           // the next run's first lane
                const unsigned runmask = (re == 32 ? 0xffffffffu : ((1u << re) - 1u)) &
                                         ~((1u << rs) - 1u);
                const int cnt = __popc(Hs & runmask);
                const int i = __popc(hb & ~((1u << rs) - 1u));           // my rank in the run
                const int h = __popc(hb);                                 // colliding boxes before me
                const int P = T.np;
                const bool closed = j < __popc(Rs) || (T.pos + (en0 - st0) == T.size);
                nx[T.nn + (j > 0 ? P : 0) + 2 * h - i] = Box{{2 * at, b.a[1], b.a[2]}};
                const Box r = Box{{2 * at + 1, b.a[1], b.a[2]}};
                if (closed) nx[T.nn + P + 2 * (h - i) + cnt + i] = r;
                else sbase[2 * (size_t)cap + (j == 0 ? P : 0) + i] = r;
            } else {
                Box l = b, r = b;
#pragma unroll
                for (int d = 1; d < 3; ++d) {
                    l.a[d] = d == sd ? 2 * b.a[d] : b.a[d];
                    r.a[d] = d == sd ? 2 * b.a[d] + 1 : b.a[d];
                }
                const long long pos = T.nn + incl - c;
                nx[pos] = l;
                if (keep_r) nx[pos + 1] = r;
            }
        }
        __syncwarp();
        // the owner updates its slot
        if (take > 0) {
            const PoolAgg G = sh.agg[lane];
            if (!S.found && G.fh && G.outcome != 2) {
                S.found = 1;
                S.if_at = G.at_fh;
            }
            if (G.outcome == 1) {
                S.qi = -1;
            } else if (G.outcome == 2) {
                p.mid[atomicAdd(&p.hdr->mid, 1)] = (int)S.qi;
                S.qi = -1;
            } else {
                if (S.sd == 0) {
                    if (level_end) {
                        S.nn += S.np + 2 * G.hits;
                        S.np = 0;
                    } else if (G.runs == 0) {
                        S.nn += G.hits;
                        S.np += G.hits;
                    } else {
                        S.nn += S.np + 2 * G.hits - G.cntk;
                        S.np = G.cntk;
                        S.pend_at = G.at_k;
                    }
                } else {
                    S.nn += G.children;
                }
                S.pos += take;
                if (S.pos == S.size) {
                    if (!S.found) {
                        write_result(p, S.qi, 0, __longlong_as_double(0x7ff0000000000000LL), 0.0,
                                     S.n_before + S.size);
                        checks_done += (unsigned long long)(S.n_before + S.size);
                        S.qi = -1;
                    } else {
                        S.n_before += S.size;
                        S.buf ^= 1;
                        S.size = S.nn;
                        S.nn = 0;
                        S.np = 0;
                        S.k[S.sd] += 1;
                        S.pos = 0;
                        S.found = 0;
                        pool_split_dim(S, meta[lane].kap);
                    }
                }
            }
        }
        __syncwarp();
    }
    atomicAdd(&p.hdr->evals_pool, evals);
    if (KIND == CCD_KIND_EE) atomicAdd(&p.hdr->evals_pool_ee, evals);
    if (lane == 0) {
        atomicAdd(&p.hdr->tq_pool, tqs);
        if (KIND == CCD_KIND_EE) atomicAdd(&p.hdr->tq_pool_ee, tqs);
        atomicAdd(&p.hdr->pool_iters, iters);
        atomicAdd(&p.hdr->pool_serial, serial);
        atomicAdd(&p.hdr->a_tasks_pool, ptasks);
        atomicAdd(&p.hdr->evals_pool_shared, shared_evals);
        if (KIND == CCD_KIND_EE) {
            atomicAdd(&p.hdr->a_tasks_pool_ee, ptasks);
            atomicAdd(&p.hdr->evals_pool_shared_ee, shared_evals);
        }
    }
    atomicAdd(&p.hdr->checks_pool, checks_done);
}

// Resident pooled blocks per SM (its shared memory and registers decide),
// at most POOL_BLOCKS_PER_SM, times the SM count.
template <typename K>
int pool_blocks(K kernel, int sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (per_sm > POOL_BLOCKS_PER_SM) per_sm = POOL_BLOCKS_PER_SM;
    return per_sm * sms;
}

// ---- multi-instance (segmented) kernels ---------------------------------------

__global__ void seg_validate_kernel(const ccd_segment *segs, int nseg, long long n,
                                    long long max_itr_bound, Header *hdr)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const ccd_segment g = segs[s];
    const long long start = s == 0 ? 0 : segs[s - 1].offset + segs[s - 1].count;
    bool ok = g.offset == start && g.count >= 0 && (g.kind == CCD_KIND_VF || g.kind == CCD_KIND_EE) &&
              g.delta > 0.0 && g.ms >= 0.0 && g.max_itr >= 1 && g.max_itr <= max_itr_bound &&
              g.t_max > 0.0 && g.t_max <= 1.0 && g.group >= 0;
    if (s == nseg - 1) ok = ok && g.offset + g.count == n;
    if (!ok) atomicExch(&hdr->status, (int)CCD_ERR_ARG);
}

__global__ void __launch_bounds__(ROOT_THREADS)
    root_kernel_seg(Params p, const ccd_segment *segs, int nseg)
{
    if (*(volatile int *)&p.hdr->status == (int)CCD_ERR_ARG) return;
    const long long i = (long long)blockIdx.x * ROOT_THREADS + threadIdx.x;
    if (i >= p.n) return;
    const ccd_segment sg = segs[find_segment(segs, nseg, i)];
    const QP q = qp_segment(sg);
    if (sg.kind == CCD_KIND_VF) root_query<CCD_KIND_VF>(p, i, q);
    else root_query<CCD_KIND_EE>(p, i, q);
}

// deep: 0 = one-warp stage (list `mid`; hand-offs go to the deep list of
// their kind), 1 = deep stage (PAGED: frontier pages from `pool`, queries
// without pages deferred to `jumbo`), 2 = full-size stage (the deferred
// queries).  KS >= 0: the kernel solves queries of that kind only (the deep
// stage runs one launch per kind, each with the registers of one kind and
// so three blocks per SM); KS < 0: either kind.
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Rounds of a served batch's deep stage: a block takes no new query once
// slice_ns has passed since the round's first block started (slice_ns > 0),
// or once the host has set *yield (mapped host memory, read between
// queries).  The SMs then come free for other batches' kernels, and the host
// launches another round for the queries left in the list; no query is
// interrupted and nothing waits.
template <int BS, bool PAGED = false, int KS = -1>
__global__ void __launch_bounds__(BS, deep_blocks_per_sm(BS, KS < 0))
    solve_kernel_seg(Params p, const ccd_segment *segs, int nseg, int deep, Box *slots,
                     long long cap, PagePool pool, long long slice_ns = 0,
                     const volatile int *yield = nullptr)
{
    __shared__ Smem<BS> s;
    __shared__ int s_idx;
    __shared__ unsigned long long s_t0;
    extern __shared__ double tq[];   // [2 * BS][TWidth<EE>::W]: sized for either kind
    Box *cur = slots + (size_t)blockIdx.x * 2 * (size_t)cap;
    Box *nxt = cur + cap;
    const bool ee = KS == CCD_KIND_EE;
    const int *list = deep == 2 ? p.jumbo : deep ? (ee ? p.deep_list_ee : p.deep_list) : p.mid;
    const int *count = deep == 2 ? &p.hdr->jumbo
                       : deep    ? (ee ? &p.hdr->overflow_ee : &p.hdr->overflow)
                                 : &p.hdr->mid;
    int *head = deep == 2 ? &p.hdr->head_jumbo
                : deep    ? (ee ? &p.hdr->head_deep_ee : &p.hdr->head_deep)
                          : &p.hdr->head_small;
    if (slice_ns > 0 && threadIdx.x == 0) {
        const unsigned long long now = global_ns();
        const unsigned long long t0 = atomicCAS(&p.hdr->round_start, 0ull, now);
        s_t0 = t0 ? t0 : now;
    }
    for (;;) {
        if (threadIdx.x == 0) {
            if ((slice_ns > 0 && global_ns() - s_t0 > (unsigned long long)slice_ns) ||
                (yield && *yield))
                s_idx = 0x7fffffff;   // the round is over: leave the rest for the next one
            else
                s_idx = atomicAdd(head, 1);
        }
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= *(volatile const int *)count) return;
        const long long qi = list[idx];
        // the query's parameters, block-uniform, in shared memory (they
        // would otherwise hold registers through the whole solve)
        __shared__ QP q;
        __shared__ int s_kind;
        if (threadIdx.x == 0) {
            const ccd_segment &sg = segs[find_segment(segs, nseg, qi)];
            q = qp_segment(sg);
            s_kind = sg.kind;
        }
        __syncthreads();
        const int kind = s_kind;
        int level = 0;
        bool done;
        if constexpr (PAGED) {
            __shared__ PageTables pt;
            PagedFrontier<BS> F{pool, &pt};
            if constexpr (KS >= 0)
                done = solve_query<(KS >= 0 ? KS : 0), BS>(p, q, qi, F, false, s, tq, level);
            else
                done = kind == CCD_KIND_VF
                           ? solve_query<CCD_KIND_VF, BS>(p, q, qi, F, false, s, tq, level)
                           : solve_query<CCD_KIND_EE, BS>(p, q, qi, F, false, s, tq, level);
        } else {
            ContigFrontier<BS> F{cur, nxt, cap};
            if constexpr (KS >= 0)
                done = solve_query<(KS >= 0 ? KS : 0), BS>(p, q, qi, F, deep != 0, s, tq, level);
            else
                done = kind == CCD_KIND_VF
                           ? solve_query<CCD_KIND_VF, BS>(p, q, qi, F, deep != 0, s, tq, level)
                           : solve_query<CCD_KIND_EE, BS>(p, q, qi, F, deep != 0, s, tq, level);
        }
        if (!done && threadIdx.x == 0) {
            if (KS >= 0 || deep) {       // paged deep stage: deferred to a full-size slot
                p.jumbo[atomicAdd(&p.hdr->jumbo, 1)] = (int)qi;
            } else if (kind == CCD_KIND_EE) {
                const int j = atomicAdd(&p.hdr->overflow_ee, 1);
                p.over_ee[j] = (int)qi;
                p.over_level_ee[j] = (unsigned char)level;
            } else {
                const int j = atomicAdd(&p.hdr->overflow, 1);
                p.over[j] = (int)qi;
                p.over_level[j] = (unsigned char)level;
            }
        }
        __syncthreads();
    }
}

// Per candidate set (segment group): alpha = min toi, tol = max out_tol
// (Algorithm 4: alpha <- min(t, alpha), delta_i <- max(delta_bar, delta_i)).
// toi and out_tol are >= 0 (or +inf), so their bit patterns order like the
// values and 64-bit atomicMin/atomicMax apply.
__global__ void group_init_kernel(double *alpha, double *tol, int ngroups)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ngroups) {
        alpha[g] = __longlong_as_double(0x7ff0000000000000LL);
        tol[g] = 0.0;
    }
}

__global__ void group_reduce_kernel(const double *__restrict__ toi,
                                    const double *__restrict__ out_tol, long long n,
                                    const ccd_segment *segs, int nseg, int ngroups,
                                    double *alpha, double *tol)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + threadIdx.x;
        const bool valid = i < n;
        int grp = -1;
        unsigned long long a = 0x7ff0000000000000ull, w = 0ull;
        if (valid) {
            grp = segs[find_segment(segs, nseg, i)].group;
            if (grp >= ngroups) grp = -1;
            a = (unsigned long long)__double_as_longlong(toi[i]);
            w = (unsigned long long)__double_as_longlong(out_tol[i]);
        }
        const int g0 = __shfl_sync(FULL, grp, 0);
        if (__all_sync(FULL, grp == g0)) {
            for (int o = 16; o; o >>= 1) {
                a = min(a, (unsigned long long)__shfl_xor_sync(FULL, a, o));
                w = max(w, (unsigned long long)__shfl_xor_sync(FULL, w, o));
            }
            if (lane == 0 && g0 >= 0) {
                atomicMin((unsigned long long *)&alpha[g0], a);
                atomicMax((unsigned long long *)&tol[g0], w);
            }
        } else if (grp >= 0) {
            atomicMin((unsigned long long *)&alpha[grp], a);
            atomicMax((unsigned long long *)&tol[grp], w);
        }
    }
}

// ---- L-infinity distance at t = 0 (Sec. 5.1 norm; Algorithm 4's d_i) ---------
//
// f(u,v) = F(0,u,v) = A + u B + v C, each component one rounded subtraction
// of t = 0 coordinates (VF: A = p - v1, B = v1 - v2, C = v1 - v3; EE:
// A = p1 - p3, B = p2 - p1, C = p3 - p4).  The distance min over the domain
// of g = max_c |(A_c + u B_c) + v C_c| is a linear program in (u, v, s); its
// optimum is at a vertex, so g is taken at every candidate vertex (domain
// corners; points of a domain edge where two of the lines +-f_c cross;
// interior points where two axes vanish or three signed lines meet) and the
// smallest value is the answer.  The operation sequence of every candidate is
// fixed (include/ccd.h states it), so the result is reproducible bit for bit.
struct LinfQ {
    double A[3], B[3], C[3];
    int vf;
};

__device__ __forceinline__ double linf_at(const LinfQ &L, double u, double v)
{
    double g = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double f = fabs(dadd(dadd(L.A[c], dmul(u, L.B[c])), dmul(v, L.C[c])));
        g = f > g ? f : g;
    }
    return g;
}

__device__ __forceinline__ bool linf_inside(const LinfQ &L, double u, double v)
{
    if (!(u >= 0.0) || !(v >= 0.0)) return false;
    return L.vf ? dadd(u, v) <= 1.0 : (u <= 1.0 && v <= 1.0);
}

// the candidate (u, v) = (b1 a22 - a12 b2, a11 b2 - b1 a21) / det of a 2x2 system
__device__ __forceinline__ void linf_solve2(const LinfQ &L, double a11, double a12, double b1,
                                            double a21, double a22, double b2, double &best)
{
    const double det = dsub(dmul(a11, a22), dmul(a12, a21));
    if (det == 0.0) return;
    const double u = __ddiv_rn(dsub(dmul(b1, a22), dmul(a12, b2)), det);
    const double v = __ddiv_rn(dsub(dmul(a11, b2), dmul(b1, a21)), det);
    if (linf_inside(L, u, v)) best = fmin(best, linf_at(L, u, v));
}

__device__ double linf_distance(const double *__restrict__ verts, long long n, long long i,
                                int kind)
{
    LinfQ L;
    L.vf = kind == CCD_KIND_VF;
    double x[4][3];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) x[j][c] = verts[(size_t)(3 * j + c) * n + i];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (L.vf) {
            L.A[c] = dsub(x[0][c], x[1][c]);
            L.B[c] = dsub(x[1][c], x[2][c]);
            L.C[c] = dsub(x[1][c], x[3][c]);
        } else {
            L.A[c] = dsub(x[0][c], x[2][c]);
            L.B[c] = dsub(x[1][c], x[0][c]);
            L.C[c] = dsub(x[2][c], x[3][c]);
        }
    }
    double best = __longlong_as_double(0x7ff0000000000000LL);
    // corners (0,0), (1,0), (0,1) and, for EE, (1,1)
    best = fmin(best, linf_at(L, 0.0, 0.0));
    best = fmin(best, linf_at(L, 1.0, 0.0));
    best = fmin(best, linf_at(L, 0.0, 1.0));
    if (!L.vf) best = fmin(best, linf_at(L, 1.0, 1.0));
    // edges (u, v) = (pu, pv) + tau (du, dv), tau in [0, 1]:
    // VF v = 0, u = 0, u + v = 1;  EE v = 0, u = 0, u = 1, v = 1
    const int nedge = L.vf ? 3 : 4;
    for (int e = 0; e < nedge; ++e) {
        double pu, pv, du, dv;
        if (e == 0) { pu = 0.0; pv = 0.0; du = 1.0; dv = 0.0; }
        else if (e == 1) { pu = 0.0; pv = 0.0; du = 0.0; dv = 1.0; }
        else if (e == 2) {
            if (L.vf) { pu = 1.0; pv = 0.0; du = -1.0; dv = 1.0; }
            else { pu = 1.0; pv = 0.0; du = 0.0; dv = 1.0; }
        } else { pu = 0.0; pv = 1.0; du = 1.0; dv = 0.0; }
        double al[3], be[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            al[c] = dadd(dadd(L.A[c], dmul(pu, L.B[c])), dmul(pv, L.C[c]));
            be[c] = dadd(dmul(du, L.B[c]), dmul(dv, L.C[c]));
        }
        // 3 zero crossings, then f_c1 = +-f_c2 for the 3 axis pairs
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double num, den;
            if (k < 3) {
                num = -al[k];
                den = be[k];
            } else {
                const int pair = (k - 3) >> 1;               // (0,1), (0,2), (1,2)
                const int c1 = pair == 2 ? 1 : 0, c2 = pair == 0 ? 1 : 2;
                const double sg = ((k - 3) & 1) ? -1.0 : 1.0;
                num = dsub(dmul(sg, al[c2]), al[c1]);
                den = dsub(be[c1], dmul(sg, be[c2]));
            }
            if (den == 0.0) continue;
            const double t = __ddiv_rn(num, den);
            if (!(t >= 0.0 && t <= 1.0)) continue;
            best = fmin(best, linf_at(L, dadd(pu, dmul(t, du)), dadd(pv, dmul(t, dv))));
        }
    }
    // interior: two axes zero
    linf_solve2(L, L.B[0], L.C[0], -L.A[0], L.B[1], L.C[1], -L.A[1], best);
    linf_solve2(L, L.B[0], L.C[0], -L.A[0], L.B[2], L.C[2], -L.A[2], best);
    linf_solve2(L, L.B[1], L.C[1], -L.A[1], L.B[2], L.C[2], -L.A[2], best);
    // interior: s1 f_1 = s2 f_2 = s3 f_3, patterns (+,+,+), (+,+,-), (+,-,+), (-,+,+)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double s1 = k == 3 ? -1.0 : 1.0, s2 = k == 2 ? -1.0 : 1.0, s3 = k == 1 ? -1.0 : 1.0;
        linf_solve2(L, dsub(dmul(s1, L.B[0]), dmul(s2, L.B[1])),
                    dsub(dmul(s1, L.C[0]), dmul(s2, L.C[1])),
                    dsub(dmul(s2, L.A[1]), dmul(s1, L.A[0])),
                    dsub(dmul(s2, L.B[1]), dmul(s3, L.B[2])),
                    dsub(dmul(s2, L.C[1]), dmul(s3, L.C[2])),
                    dsub(dmul(s3, L.A[2]), dmul(s2, L.A[1])), best);
    }
    return best;
}

__global__ void linf_group_init_kernel(double *gmin, int ngroups)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ngroups) gmin[g] = __longlong_as_double(0x7ff0000000000000LL);
}

// per query (optional) and per segment group (minimum, through the bit
// patterns: distances are >= +0, so their bits order like their values)
__global__ void linf_distance_kernel(const double *__restrict__ verts, long long n,
                                     const ccd_segment *segs, int nseg, int ngroups,
                                     double *dist, double *gmin)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + threadIdx.x;
        const bool valid = i < n;
        int grp = -1;
        unsigned long long bits = 0x7ff0000000000000ull;
        if (valid) {
            const ccd_segment sg = segs[find_segment(segs, nseg, i)];
            const double d = linf_distance(verts, n, i, sg.kind);
            if (dist) dist[i] = d;
            bits = (unsigned long long)__double_as_longlong(d);
            grp = sg.group < ngroups ? sg.group : -1;
        }
        const int g0 = __shfl_sync(FULL, grp, 0);
        if (__all_sync(FULL, grp == g0)) {
            for (int o = 16; o; o >>= 1)
                bits = min(bits, (unsigned long long)__shfl_xor_sync(FULL, bits, o));
            if (lane == 0 && g0 >= 0) atomicMin((unsigned long long *)&gmin[g0], bits);
        } else if (grp >= 0) {
            atomicMin((unsigned long long *)&gmin[grp], bits);
        }
    }
}

// per-segment eps from the segment's own points
__global__ void seg_err_init_kernel(ccd_segment *segs, int nseg)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nseg)
        for (int c = 0; c < 3; ++c) segs[s].err[c] = 1.0;
}

__global__ void seg_err_reduce_kernel(const double *__restrict__ verts, long long n,
                                      ccd_segment *segs, int nseg)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + threadIdx.x;
        const bool valid = i < n;
        double mx[3] = {0.0, 0.0, 0.0};
        int sid = -1;
        if (valid) {
            sid = find_segment(segs, nseg, i);
#pragma unroll
            for (int k = 0; k < 24; ++k)
                mx[k % 3] = fmax(mx[k % 3], fabs(verts[(size_t)k * n + i]));
        }
        const int s0 = __shfl_sync(FULL, sid, 0);
        const bool same = __all_sync(FULL, !valid || sid == s0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            unsigned long long *dst = (unsigned long long *)&segs[valid ? sid : 0].err[c];
            if (same) {
                double v = mx[c];
                for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
                if (lane == 0 && s0 >= 0)
                    atomicMax((unsigned long long *)&segs[s0].err[c],
                              (unsigned long long)__double_as_longlong(v));
            } else if (valid) {
                atomicMax(dst, (unsigned long long)__double_as_longlong(mx[c]));
            }
        }
    }
}

__global__ void seg_err_finish_kernel(ccd_segment *segs, int nseg)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const bool ms = segs[s].ms > 0.0;
    const double K = segs[s].kind == CCD_KIND_VF ? (ms ? 7.549516567451064e-15 : 6.661338147750939e-15)
                                                 : (ms ? 7.105427357601002e-15 : 6.217248937900877e-15);
    for (int c = 0; c < 3; ++c) {
        const double g = segs[s].err[c];
        segs[s].err[c] = dmul(K, dmul(dmul(g, g), g));
    }
}

// ---- layout helper: array of structures -> structure of arrays ---------------

// Block of 256 queries: coalesced load of 256 x 24 doubles into shared
// memory, then 24 coalesced plane writes.
__global__ void __launch_bounds__(256) aos_to_soa_kernel(const double *__restrict__ aos,
                                                         long long n, double *soa, long long ld)
{
    __shared__ double tile[256 * 25];   // padded rows against bank conflicts
    const long long q0 = (long long)blockIdx.x * 256;
    const int m = (int)min(256LL, n - q0);
    for (int e = threadIdx.x; e < m * 24; e += 256) {
        const int qi = e / 24, k = e - qi * 24;
        tile[qi * 25 + k] = aos[(q0 + qi) * 24 + k];
    }
    __syncthreads();
    if (threadIdx.x < m)
        for (int k = 0; k < 24; ++k) soa[(size_t)k * ld + q0 + threadIdx.x] = tile[threadIdx.x * 25 + k];
}

// ---- eps from bounds (Eq. ccd-error / msccd-error) ---------------------------

__global__ void err_init_kernel(unsigned long long *g)
{
    if (threadIdx.x < 3) g[threadIdx.x] = (unsigned long long)__double_as_longlong(1.0);
}

// scene-wide: atomicMax on the bit pattern (monotone for non-negative doubles)
__global__ void err_reduce_kernel(const double *__restrict__ verts, long long n,
                                  unsigned long long *g)
{
    double mx[3] = {0.0, 0.0, 0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int k = 0; k < 24; ++k) mx[k % 3] = fmax(mx[k % 3], fabs(verts[(size_t)k * n + i]));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double v = mx[c];
        for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0) atomicMax(g + c, (unsigned long long)__double_as_longlong(v));
    }
}

__global__ void err_finish_kernel(const unsigned long long *g, double K, double *out)
{
    if (threadIdx.x < 3) {
        double gm = __longlong_as_double((long long)g[threadIdx.x]);
        out[threadIdx.x] = dmul(K, dmul(dmul(gm, gm), gm));
    }
}

__global__ void err_per_query_kernel(const double *__restrict__ verts, long long n, double K,
                                     double *out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double g[3] = {1.0, 1.0, 1.0};
#pragma unroll
    for (int k = 0; k < 24; ++k) g[k % 3] = fmax(g[k % 3], fabs(verts[(size_t)k * n + i]));
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * i + c] = dmul(K, dmul(dmul(g[c], g[c]), g[c]));
}

// ---- FP64 pipe probe ---------------------------------------------------------

__device__ double g_probe_sink;

__global__ void __launch_bounds__(256) fp64_probe_kernel(int iters)
{
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    const double b = 0.9999999, c = 1e-7;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = __fma_rn(a[j], b, c);
    double r = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) r += a[j];
    if (r != r) g_probe_sink = r;   // never true; keeps the chains live
}

// ---- host side ----------------------------------------------------------------

int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

long long deep_cap(long long max_itr) { return 2 * max_itr + 64; }

// Fixed part of the workspace for n queries.
Layout layout_fixed(long long n, int sms)
{
    Layout L{};
    size_t off = align256(sizeof(Header));
    L.off_surv = off; off = align256(off + sizeof(int) * (size_t)n);
    L.off_mid = off; off = align256(off + sizeof(int) * (size_t)n);
    L.off_over = off; off = align256(off + sizeof(int) * (size_t)n);
    L.off_level = off; off = align256(off + (size_t)n);
    L.off_dlist = off; off = align256(off + sizeof(int) * (size_t)n);
    L.off_jlist = off; off = align256(off + sizeof(int) * (size_t)n);
    L.off_kappa = off; off = align256(off + 3 * sizeof(double) * (size_t)n);
    L.nb_pool = sms * POOL_BLOCKS_PER_SM;
    L.off_pool = off;
    off = align256(off + sizeof(Box) * 3 * (size_t)POOL_CAP * POOL_SLOTS * (size_t)L.nb_pool);
    L.off_meta = off;
    off = align256(off + sizeof(PoolMeta) * POOL_SLOTS * (size_t)L.nb_pool);
    L.nb_small = sms * SMALL_BLOCKS_PER_SM;
    L.cap_small = SMALL_CAP;
    L.off_small = off; off = align256(off + sizeof(Box) * 2 * (size_t)SMALL_CAP * L.nb_small);
    L.off_deep = off;
    L.total = off;
    return L;
}

// ---- the deep tier's part of a workspace -------------------------------------
//
// Paged: J full-size slots (two arrays of 2 m_I + 64 boxes each, for the
// queries the deep stage defers), a free bitmap and a pool of frontier pages
// shared by the deep blocks.  Contiguous (only when the room cannot hold one
// full-size slot and two pages): as many slots as fit, each of `cap` boxes
// per level; a level beyond it is answered by the capacity fallback.
constexpr size_t PAGE_BYTES = sizeof(Box) * (size_t)PAGE_BOXES;
constexpr int JUMBO_SLOTS = 2;

struct DeepLayout {
    bool paged;
    int nb_deep;                  // deep blocks (paged) / contiguous slots
    long long cap_deep;           // boxes per level of a contiguous or full-size slot
    int nb_jumbo;                 // full-size slots (paged)
    size_t off_slots;             // contiguous or full-size slots
    size_t off_bits, off_pages;   // paged
    int nwords;
    long long npages;
    size_t total;
};

long long pages_for(long long boxes) { return (boxes + PAGE_BOXES - 1) / PAGE_BOXES; }

// Pages a default workspace provides: one level of the largest size any
// level can reach (2 m_I boxes), and at least two, for every deep block up to
// DEEP_POOL_BLOCKS_PER_SM per SM; and at least DEEP_MIN_PAGES per deep block.
long long default_pages(long long nb_deep, long long max_itr)
{
    const int sms = device_sms();
    const long long cap_blocks = (long long)DEEP_POOL_BLOCKS_PER_SM * (sms > 0 ? sms : 1);
    const long long per = pages_for(deep_cap(max_itr));
    const long long full = (nb_deep < cap_blocks ? nb_deep : cap_blocks) * (per < 2 ? 2 : per);
    return full > DEEP_MIN_PAGES * nb_deep ? full : DEEP_MIN_PAGES * nb_deep;
}

// Deep blocks a launch runs on a pool of npages shared by `sharers` deep
// launches at once: every block holds a page for its current level and
// reserves pages for the next, so a block per DEEP_MIN_PAGES pages at most
// (a block that finds the pool empty defers its query to the full-size
// slots, which take deferred queries two at a time).
int page_limited_blocks(int nb, long long npages, int sharers)
{
    const long long lim = npages / (DEEP_MIN_PAGES * (long long)(sharers > 0 ? sharers : 1));
    if (lim < (long long)nb) nb = (int)(lim > 1 ? lim : 1);
    return nb;
}

size_t pool_bytes(long long npages)
{
    return align256(sizeof(unsigned long long) * (size_t)((npages + 63) / 64)) +
           PAGE_BYTES * (size_t)npages;
}

bool deep_layout(size_t off, size_t ws_bytes, long long max_itr, int nb_deep_max, DeepLayout *D)
{
    if (ws_bytes < off) return false;
    const size_t room = ws_bytes - off;
    const size_t slot = align256(sizeof(Box) * 2 * (size_t)deep_cap(max_itr));
    DeepLayout d{};
    d.off_slots = off;
    d.cap_deep = deep_cap(max_itr);
    for (int J = JUMBO_SLOTS; J >= 1; --J) {
        if (room < J * slot + 256 + 2 * PAGE_BYTES) continue;
        const size_t rest = room - J * slot;
        long long np = (long long)(rest / PAGE_BYTES);
        const size_t bits = align256(sizeof(unsigned long long) * (size_t)((np + 63) / 64));
        np = (long long)((rest - bits) / PAGE_BYTES);
        if (np > (1LL << 30)) np = 1LL << 30;
        if (np < 2) continue;
        d.paged = true;
        d.nb_deep = nb_deep_max;
        d.nb_jumbo = J;
        d.off_bits = off + J * slot;
        d.nwords = (int)((np + 63) / 64);
        d.off_pages = d.off_bits + align256(sizeof(unsigned long long) * (size_t)d.nwords);
        d.npages = np;
        d.total = d.off_pages + PAGE_BYTES * (size_t)np;
        *D = d;
        return true;
    }
    const long long nb = (long long)(room / slot);
    if (nb >= 1) {
        d.nb_deep = (int)(nb < nb_deep_max ? nb : nb_deep_max);
    } else {
        d.nb_deep = 1;
        d.cap_deep = (long long)(room / (sizeof(Box) * 2));
        if (d.cap_deep < 1024) return false;
    }
    d.total = off + sizeof(Box) * 2 * (size_t)d.cap_deep * d.nb_deep;
    *D = d;
    return true;
}

size_t default_deep_bytes(long long max_itr, int nb_deep)
{
    return JUMBO_SLOTS * align256(sizeof(Box) * 2 * (size_t)deep_cap(max_itr)) +
           pool_bytes(default_pages(nb_deep, max_itr));
}

PagePool make_pool(char *ws, const DeepLayout &D, Header *h)
{
    PagePool pool{};
    if (D.paged) {
        pool.base = (Box *)(ws + D.off_pages);
        pool.bits = (unsigned long long *)(ws + D.off_bits);
        pool.nwords = D.nwords;
        pool.used = &h->pages_used;
        pool.peak = &h->pages_peak;
    }
    return pool;
}

cudaEvent_t g_stage_events[5];
int g_stage_events_on = 0;

// Inside a stream capture a plain event record only orders the captured
// work; the external flag makes it a node of the graph, so that every replay
// records the event (and the stages of a replayed batch can be timed).
inline void stage_mark(int i, cudaStream_t st)
{
    if (!g_stage_events_on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(g_stage_events[i], st, cudaEventRecordExternal);
    else
        cudaEventRecord(g_stage_events[i], st);
}

template <int KIND>
ccd_status run_batch(const double *verts, int64_t n, const double *err, int err_stride,
                     double ms, double delta, int64_t max_itr, uint8_t *collides, double *toi,
                     double *out_tol, int64_t *checks, void *workspace, size_t ws_bytes,
                     void *stream)
{
    if (n < 0 || n >= 0x7fffffffLL || !(delta > 0.0) || max_itr <= 0 || !(ms >= 0.0) ||
        (err_stride != 0 && err_stride != 3))
        return CCD_ERR_ARG;
    if (n > 0 && (!verts || !err || !collides || !toi || !out_tol)) return CCD_ERR_ARG;
    if (!workspace) return CCD_ERR_WORKSPACE;
    const int sms = device_sms();
    if (sms <= 0) return CCD_ERR_CUDA;
    const Layout L = layout_fixed(n, sms);
    DeepLayout D;
    if (!deep_layout(L.off_deep, ws_bytes, max_itr, DEEP_BLOCKS_PER_SM * sms, &D))
        return CCD_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    if (cudaMemsetAsync(ws, 0, sizeof(Header), st) != cudaSuccess) return CCD_ERR_CUDA;
    if (n == 0) return CCD_OK;

    Params p;
    p.verts = verts; p.n = n; p.err = err; p.err_stride = err_stride;
    p.ms = ms; p.delta = delta; p.max_itr = max_itr;
    p.collides = collides; p.toi = toi; p.out_tol = out_tol; p.checks = (long long *)checks;
    p.hdr = (Header *)ws;
    p.surv = (int *)(ws + L.off_surv);
    p.mid = (int *)(ws + L.off_mid);
    p.over = (int *)(ws + L.off_over);
    p.over_level = (unsigned char *)(ws + L.off_level);
    p.deep_list = (int *)(ws + L.off_dlist);
    p.over_ee = nullptr;
    p.over_level_ee = nullptr;
    p.deep_list_ee = nullptr;
    p.jumbo = (int *)(ws + L.off_jlist);
    p.kappa = (double *)(ws + L.off_kappa);
    Header *h = p.hdr;
    const PagePool pool = make_pool(ws, D, h);

    const long long blocks = (n + ROOT_THREADS - 1) / ROOT_THREADS;
    stage_mark(0, st);
    if (D.paged)
        pool_init_kernel<<<(D.nwords + 255) / 256, 256, 0, st>>>(pool.bits, D.nwords,
                                                                 (int)D.npages);
    root_kernel<KIND><<<(unsigned)blocks, ROOT_THREADS, 0, st>>>(p);
    stage_mark(1, st);
    const int nb_pool = pool_blocks(pool_kernel<KIND>, sms);
    pool_kernel<KIND><<<nb_pool, 32, 0, st>>>(p, (Box *)(ws + L.off_pool),
                                              (PoolMeta *)(ws + L.off_meta), POOL_CAP, p.surv,
                                              &h->survivors, &h->head_pool, nullptr, 0);
    stage_mark(2, st);
    const size_t tq_small = sizeof(double) * 2 * SMALL_THREADS * TWidth<KIND>::W;
    const size_t tq_deep = sizeof(SharedUV<DEEP_THREADS>);   // deep tier: shared partials
    auto *deep_paged = solve_kernel<KIND, DEEP_THREADS, true>;
    auto *deep_contig = solve_kernel<KIND, DEEP_THREADS, false>;
    for (auto *k : {deep_paged, deep_contig})
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tq_deep) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) !=
                cudaSuccess)
            return CCD_ERR_CUDA;
    int nb_deep = D.nb_deep;
    {   // resident deep blocks per SM: the persistent grid must fit at once
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, D.paged ? deep_paged : deep_contig,
                                                          DEEP_THREADS, tq_deep) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        if (per_sm > DEEP_BLOCKS_PER_SM) per_sm = DEEP_BLOCKS_PER_SM;
        if (nb_deep > per_sm * sms) nb_deep = per_sm * sms;
        if (D.paged) nb_deep = page_limited_blocks(nb_deep, D.npages, 1);
    }
    solve_kernel<KIND, SMALL_THREADS><<<L.nb_small, SMALL_THREADS, tq_small, st>>>(
        p, 0, (Box *)(ws + L.off_small), L.cap_small, PagePool{}, p.mid, &h->mid, &h->head_small,
        p.over, p.over_level, &h->overflow);
    order_by_level_kernel<<<1, 1024, 0, st>>>(p.over, p.over_level, &h->overflow, p.deep_list);
    stage_mark(3, st);
    if (D.paged) {
        // deep queries on frontier pages; those that find no pages restart
        // in the full-size slots
        deep_paged<<<nb_deep, DEEP_THREADS, tq_deep, st>>>(
            p, 1, nullptr, 0, pool, p.deep_list, &h->overflow, &h->head_deep, p.jumbo, nullptr,
            &h->jumbo);
        deep_contig<<<D.nb_jumbo, DEEP_THREADS, tq_deep, st>>>(
            p, 1, (Box *)(ws + D.off_slots), D.cap_deep, PagePool{}, p.jumbo, &h->jumbo,
            &h->head_jumbo, nullptr, nullptr, nullptr);
    } else {
        deep_contig<<<nb_deep, DEEP_THREADS, tq_deep, st>>>(
            p, 1, (Box *)(ws + D.off_slots), D.cap_deep, PagePool{}, p.deep_list, &h->overflow,
            &h->head_deep, nullptr, nullptr, nullptr);
    }
    stage_mark(4, st);
    if (cudaGetLastError() != cudaSuccess) return CCD_ERR_CUDA;
    return CCD_OK;
}

}  // namespace

extern "C" {

size_t ccd_workspace_bytes(int64_t n, int64_t max_itr)
{
    if (n < 0 || n >= 0x7fffffffLL || max_itr <= 0) return 0;
    const int sms = device_sms();
    if (sms <= 0) return 0;
    const Layout L = layout_fixed(n, sms);
    return L.off_deep + default_deep_bytes(max_itr, DEEP_BLOCKS_PER_SM * sms);
}

ccd_status ccd_vf_batch(const double *verts, int64_t n, const double *err, int err_stride,
                        double ms, double delta, int64_t max_itr, uint8_t *collides, double *toi,
                        double *out_tol, int64_t *checks, void *workspace, size_t ws_bytes,
                        void *stream)
{
    return run_batch<CCD_KIND_VF>(verts, n, err, err_stride, ms, delta, max_itr, collides, toi,
                                  out_tol, checks, workspace, ws_bytes, stream);
}

ccd_status ccd_ee_batch(const double *verts, int64_t n, const double *err, int err_stride,
                        double ms, double delta, int64_t max_itr, uint8_t *collides, double *toi,
                        double *out_tol, int64_t *checks, void *workspace, size_t ws_bytes,
                        void *stream)
{
    return run_batch<CCD_KIND_EE>(verts, n, err, err_stride, ms, delta, max_itr, collides, toi,
                                  out_tol, checks, workspace, ws_bytes, stream);
}

size_t ccd_workspace_bytes_pages(int64_t n, int64_t max_itr, int64_t pages)
{
    if (n < 0 || n >= 0x7fffffffLL || max_itr <= 0 || pages < 2 || pages > (1LL << 30)) return 0;
    const int sms = device_sms();
    if (sms <= 0) return 0;
    const Layout L = layout_fixed(n, sms);
    return L.off_deep + JUMBO_SLOTS * align256(sizeof(Box) * 2 * (size_t)deep_cap(max_itr)) +
           pool_bytes(pages);
}

ccd_status ccd_workspace_layout(int64_t n, int64_t max_itr, size_t ws_bytes,
                                ccd_workspace_info *info)
{
    if (n < 0 || n >= 0x7fffffffLL || max_itr <= 0 || !info) return CCD_ERR_ARG;
    const int sms = device_sms();
    if (sms <= 0) return CCD_ERR_CUDA;
    const Layout L = layout_fixed(n, sms);
    DeepLayout D;
    if (!deep_layout(L.off_deep, ws_bytes, max_itr, DEEP_BLOCKS_PER_SM * sms, &D))
        return CCD_ERR_WORKSPACE;
    info->paged = D.paged ? 1 : 0;
    info->deep_blocks = D.nb_deep;
    info->full_slots = D.paged ? D.nb_jumbo : D.nb_deep;
    info->pages = D.paged ? D.npages : 0;
    info->slot_boxes = D.cap_deep;
    info->fixed_bytes = L.off_deep;
    info->used_bytes = D.total;
    return CCD_OK;
}

ccd_status ccd_err_from_bounds(int kind, const double *verts, int64_t n, int ms_nonzero,
                               int per_query, double *err_out, void *stream)
{
    if ((kind != CCD_KIND_VF && kind != CCD_KIND_EE) || n < 0 || n >= 0x7fffffffLL || !err_out ||
        (n > 0 && !verts))
        return CCD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const double K = kind == CCD_KIND_VF ? (ms_nonzero ? 7.549516567451064e-15 : 6.661338147750939e-15)
                                         : (ms_nonzero ? 7.105427357601002e-15 : 6.217248937900877e-15);
    if (per_query) {
        if (n > 0)
            err_per_query_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(verts, n, K, err_out);
    } else {
        // the 3 output doubles double as the reduction scratch
        unsigned long long *g = (unsigned long long *)err_out;
        err_init_kernel<<<1, 32, 0, st>>>(g);
        if (n > 0) {
            const int sms = device_sms();
            long long blocks = (n + 255) / 256;
            if (blocks > 8LL * sms) blocks = 8LL * sms;
            err_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(verts, n, g);
        }
        err_finish_kernel<<<1, 32, 0, st>>>(g, K, err_out);
    }
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}

ccd_status ccd_workspace_status(const void *workspace, int32_t *status, int32_t *fallbacks,
                                void *stream)
{
    if (!workspace || !status) return CCD_ERR_ARG;
    Header h;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, workspace, sizeof(Header), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return CCD_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CCD_ERR_CUDA;
    *status = h.status;
    if (fallbacks) *fallbacks = h.fallbacks;
    return CCD_OK;
}

ccd_status ccd_workspace_counters(const void *workspace, int64_t *counters, int32_t count,
                                  void *stream)
{
    if (!workspace || !counters || count < 0) return CCD_ERR_ARG;
    Header h;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, workspace, sizeof(Header), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return CCD_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CCD_ERR_CUDA;
    const int64_t all[CCD_NUM_COUNTERS] = {
        h.survivors, h.overflow, h.fallbacks, (int64_t)h.checks_small, (int64_t)h.checks_deep,
        (int64_t)h.evals_small, (int64_t)h.evals_deep, h.status, (int64_t)h.tq_small,
        (int64_t)h.tq_deep, (int64_t)h.a_tasks_deep, (int64_t)h.split_chunks_deep,
        (int64_t)h.evals_shared_deep, h.mid, (int64_t)h.checks_pool, (int64_t)h.evals_pool,
        (int64_t)h.tq_deep_ee, (int64_t)h.a_tasks_deep_ee, (int64_t)h.evals_pool_ee,
        (int64_t)h.tq_small_ee, (int64_t)h.evals_small_ee, h.jumbo, h.pages_peak,
        (int64_t)h.tq_pool, (int64_t)h.tq_pool_ee, (int64_t)h.pool_iters,
        (int64_t)h.pool_serial, (int64_t)h.a_tasks_pool, (int64_t)h.a_tasks_pool_ee,
        (int64_t)h.evals_pool_shared, (int64_t)h.evals_pool_shared_ee,
        (int64_t)h.evals_deep_ee, (int64_t)h.evals_shared_deep_ee};
    for (int i = 0; i < count && i < CCD_NUM_COUNTERS; ++i) counters[i] = all[i];
    return CCD_OK;
}

ccd_status ccd_set_stage_events(void *const *events, int count)
{
    if (count == 0) {
        g_stage_events_on = 0;
        return CCD_OK;
    }
    if (count != 5 || !events) return CCD_ERR_ARG;
    for (int i = 0; i < 5; ++i) {
        if (!events[i]) return CCD_ERR_ARG;
        g_stage_events[i] = (cudaEvent_t)events[i];
    }
    g_stage_events_on = 1;
    return CCD_OK;
}

const char *ccd_status_str(int status)
{
    switch (status) {
    case CCD_OK: return "ok";
    case CCD_ERR_ARG: return "invalid argument";
    case CCD_ERR_WORKSPACE: return "workspace missing or too small";
    case CCD_ERR_TIMEOUT: return "bounded device wait gave up";
    case CCD_ERR_CUDA: return "CUDA launch or copy failed";
    case CCD_ERR_CAPACITY: return "frontier exceeded its slot; conservative fallback used";
    case CCD_ERR_BUSY: return "no room for the request now, or it already runs";
    case CCD_ERR_CANCELLED: return "request cancelled";
    default: return "unknown status";
    }
}

ccd_status ccd_fp64_peak_probe(int blocks, int iters, float *ms_out, void *stream)
{
    if (blocks <= 0 || iters <= 0 || !ms_out) return CCD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return CCD_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return CCD_ERR_CUDA; }
    fp64_probe_kernel<<<blocks, 256, 0, st>>>(iters);   // warm-up
    cudaEventRecord(e0, st);
    fp64_probe_kernel<<<blocks, 256, 0, st>>>(iters);
    cudaEventRecord(e1, st);
    ccd_status r = CCD_OK;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms_out, e0, e1) != cudaSuccess)
        r = CCD_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) r = CCD_ERR_CUDA;
    return r;
}

}  // extern "C"


namespace {

// ---- multi-instance host side ---------------------------------------------------

struct Tuned {
    int deep_threads, deep_slots, small_blocks_per_sm, pool_cap;
    long long small_cap;
};

bool resolve_tuning(const ccd_tuning *t, int sms, Tuned *out)
{
    Tuned r{SEG_DEEP_THREADS, deep_blocks_per_sm(SEG_DEEP_THREADS) * sms, SMALL_BLOCKS_PER_SM,
            POOL_CAP, SMALL_CAP};
    if (t) {
        if (t->deep_threads) {   // resident blocks of that size, unless slots are given
            r.deep_threads = t->deep_threads;
            r.deep_slots = deep_blocks_per_sm(r.deep_threads) * sms;
        }
        if (t->deep_slots) r.deep_slots = t->deep_slots;
        if (t->small_blocks_per_sm) r.small_blocks_per_sm = t->small_blocks_per_sm;
        if (t->small_cap) r.small_cap = t->small_cap;
        if (t->pool_cap) r.pool_cap = t->pool_cap;
    }
    if (r.deep_threads != 128 && r.deep_threads != 256 && r.deep_threads != 512) return false;
    if (r.deep_slots < 1 || r.small_blocks_per_sm < 1 || r.small_blocks_per_sm > 32 ||
        r.small_cap < 64 || r.pool_cap < 32 || r.pool_cap > POOL_CAP_MAX)
        return false;
    *out = r;
    return true;
}

size_t multi_fixed_bytes(long long n, int sms, const Tuned &T)
{
    size_t off = align256(sizeof(Header));
    off = align256(off + sizeof(int) * (size_t)n);          // survivors
    off = align256(off + sizeof(int) * (size_t)n);          // pooled-solver hand-offs
    off = align256(off + sizeof(int) * (size_t)n);          // overflow
    off = align256(off + (size_t)n);                        // overflow levels
    off = align256(off + sizeof(int) * (size_t)n);          // deep list
    off = align256(off + sizeof(int) * (size_t)n);          // edge-edge overflow
    off = align256(off + (size_t)n);                        // its levels
    off = align256(off + sizeof(int) * (size_t)n);          // edge-edge deep list
    off = align256(off + sizeof(int) * (size_t)n);          // deferred (full-size) list
    off = align256(off + 3 * sizeof(double) * (size_t)n);  // kappa
    off = align256(off + sizeof(Box) * 3 * (size_t)T.pool_cap * POOL_SLOTS *
                             (size_t)(sms * POOL_BLOCKS_PER_SM));   // pooled-solver slots
    off = align256(off + sizeof(PoolMeta) * POOL_SLOTS *
                             (size_t)(sms * POOL_BLOCKS_PER_SM));   // their query records
    off = align256(off + sizeof(Box) * 2 * (size_t)T.small_cap * (size_t)(sms * T.small_blocks_per_sm));
    return off;
}

// One segmented batch, laid out in its workspace.  The deep tier's pages are
// the workspace's own, or (served batches) a pool shared with other batches,
// in which case the workspace holds only the full-size slots.
// A second stream per caller stream, for the second kind's launch of a
// segmented batch's deep stage: the two kinds' launches are independent, and
// run at once each fills the other's tail (the 20M-query step's deep stage
// took 24 ms against 33).  Fork and join
// go through events, so they also hold inside a CUDA graph capture.  The
// stream and events are created on a call made outside capture (creating
// them during capture is not attempted); without them the launches run one
// after the other on the caller's stream.  A process keeps at most 32.
struct SideStream {
    cudaStream_t caller, side;
    cudaEvent_t fork, join;
};
std::mutex g_side_mu;
SideStream g_side[32];
int g_nside = 0;

const SideStream *side_for(cudaStream_t caller)
{
    std::lock_guard<std::mutex> lock(g_side_mu);
    for (int i = 0; i < g_nside; ++i)
        if (g_side[i].caller == caller) return &g_side[i];
    if (g_nside == 32) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(caller, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return nullptr;
    SideStream x{caller, nullptr, nullptr, nullptr};
    if (cudaStreamCreateWithFlags(&x.side, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) != cudaSuccess) {
        if (x.fork) cudaEventDestroy(x.fork);
        cudaStreamDestroy(x.side);
        return nullptr;
    }
    g_side[g_nside] = x;
    return &g_side[g_nside++];
}

// Starts the second kind's launch: returns the stream to launch it on (the
// side stream after a fork from `st`, or `st` itself).
cudaStream_t fork_side(const SideStream *sd, cudaStream_t st)
{
    if (!sd || cudaEventRecord(sd->fork, st) != cudaSuccess ||
        cudaStreamWaitEvent(sd->side, sd->fork, 0) != cudaSuccess)
        return st;
    return sd->side;
}

// Joins the side stream back into `st` (after fork_side returned it).
bool join_side(const SideStream *sd, cudaStream_t st, cudaStream_t used)
{
    if (used == st) return true;
    return cudaEventRecord(sd->join, used) == cudaSuccess &&
           cudaStreamWaitEvent(st, sd->join, 0) == cudaSuccess;
}

struct MultiPlan {
    Params p;
    Tuned T;
    int sms;
    const ccd_segment *segs;
    int nseg;
    long long bound;
    char *ws;
    Box *pool_mem;
    PoolMeta *pool_meta;
    size_t off_small;
    int nb_small;
    DeepLayout D;
    PagePool pages;
};

ccd_status multi_plan(const double *verts, int64_t n, const ccd_segment *segs, int32_t nseg,
                      int64_t max_itr_bound, uint8_t *collides, double *toi, double *out_tol,
                      int64_t *checks, const ccd_tuning *tuning, void *workspace,
                      size_t ws_bytes, const PagePool *shared, MultiPlan *M)
{
    if (n < 0 || n >= 0x7fffffffLL || max_itr_bound <= 0 || nseg < 0) return CCD_ERR_ARG;
    if (n > 0 && (!verts || !segs || nseg < 1 || !collides || !toi || !out_tol)) return CCD_ERR_ARG;
    if (!workspace) return CCD_ERR_WORKSPACE;
    const int sms = device_sms();
    if (sms <= 0) return CCD_ERR_CUDA;
    MultiPlan m{};
    if (!resolve_tuning(tuning, sms, &m.T)) return CCD_ERR_ARG;
    const size_t fixed = multi_fixed_bytes(n, sms, m.T);
    if (shared) {
        const size_t slots = JUMBO_SLOTS * align256(sizeof(Box) * 2 * (size_t)deep_cap(max_itr_bound));
        if (ws_bytes < fixed + slots) return CCD_ERR_WORKSPACE;
        m.D.paged = true;
        m.D.nb_deep = m.T.deep_slots;
        m.D.nb_jumbo = JUMBO_SLOTS;
        m.D.cap_deep = deep_cap(max_itr_bound);
        m.D.off_slots = fixed;
        m.D.total = fixed + slots;
    } else if (!deep_layout(fixed, ws_bytes, max_itr_bound, m.T.deep_slots, &m.D) ||
               m.D.cap_deep < deep_cap(max_itr_bound)) {
        return CCD_ERR_WORKSPACE;
    }
    // the two kinds' deep launches share the pool at once
    if (m.D.paged && !shared) m.D.nb_deep = page_limited_blocks(m.D.nb_deep, m.D.npages, 2);
    char *ws = (char *)workspace;
    Params &p = m.p;
    p.verts = verts; p.n = n; p.err = nullptr; p.err_stride = 0;
    p.ms = 0.0; p.delta = 0.0; p.max_itr = 0;
    p.collides = collides; p.toi = toi; p.out_tol = out_tol; p.checks = (long long *)checks;
    p.hdr = (Header *)ws;
    size_t off = align256(sizeof(Header));
    p.surv = (int *)(ws + off); off = align256(off + sizeof(int) * (size_t)n);
    p.mid = (int *)(ws + off); off = align256(off + sizeof(int) * (size_t)n);
    p.over = (int *)(ws + off); off = align256(off + sizeof(int) * (size_t)n);
    p.over_level = (unsigned char *)(ws + off); off = align256(off + (size_t)n);
    p.deep_list = (int *)(ws + off); off = align256(off + sizeof(int) * (size_t)n);
    p.over_ee = (int *)(ws + off); off = align256(off + sizeof(int) * (size_t)n);
    p.over_level_ee = (unsigned char *)(ws + off); off = align256(off + (size_t)n);
    p.deep_list_ee = (int *)(ws + off); off = align256(off + sizeof(int) * (size_t)n);
    p.jumbo = (int *)(ws + off); off = align256(off + sizeof(int) * (size_t)n);
    p.kappa = (double *)(ws + off); off = align256(off + 3 * sizeof(double) * (size_t)n);
    m.pool_mem = (Box *)(ws + off);
    off = align256(off + sizeof(Box) * 3 * (size_t)m.T.pool_cap * POOL_SLOTS *
                             (size_t)(sms * POOL_BLOCKS_PER_SM));
    m.pool_meta = (PoolMeta *)(ws + off);
    off = align256(off + sizeof(PoolMeta) * POOL_SLOTS * (size_t)(sms * POOL_BLOCKS_PER_SM));
    m.off_small = off;
    m.nb_small = sms * m.T.small_blocks_per_sm;
    m.sms = sms;
    m.segs = segs;
    m.nseg = nseg;
    m.bound = max_itr_bound;
    m.ws = ws;
    m.pages = shared ? *shared : make_pool(ws, m.D, p.hdr);
    *M = m;
    return CCD_OK;
}

template <int DT>
ccd_status set_deep_attributes()
{
    const size_t tq_deep = sizeof(SharedUV<DT>);
    for (auto *k : {solve_kernel_seg<DT, true>, solve_kernel_seg<DT, false>,
                    solve_kernel_seg<DT, true, CCD_KIND_VF>, solve_kernel_seg<DT, true, CCD_KIND_EE>,
                    solve_kernel_seg<DT, false, CCD_KIND_VF>,
                    solve_kernel_seg<DT, false, CCD_KIND_EE>})
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tq_deep) !=
            cudaSuccess)
            return CCD_ERR_CUDA;
    return CCD_OK;
}

// Header reset, segment validation, level 0, the pooled and one-warp
// stages, and the deep list in schedule order.
ccd_status multi_front(const MultiPlan &M, bool init_pool, cudaStream_t st)
{
    const Params &p = M.p;
    if (cudaMemsetAsync(M.ws, 0, sizeof(Header), st) != cudaSuccess) return CCD_ERR_CUDA;
    if (p.n == 0) return CCD_OK;
    ccd_status r = M.T.deep_threads == 128   ? set_deep_attributes<128>()
                   : M.T.deep_threads == 256 ? set_deep_attributes<256>()
                                             : set_deep_attributes<512>();
    if (r != CCD_OK) return r;
    seg_validate_kernel<<<(M.nseg + 255) / 256, 256, 0, st>>>(M.segs, M.nseg, p.n, M.bound, p.hdr);
    stage_mark(0, st);
    if (init_pool && M.D.paged)
        pool_init_kernel<<<(M.D.nwords + 255) / 256, 256, 0, st>>>(M.pages.bits, M.D.nwords,
                                                                   (int)M.D.npages);
    root_kernel_seg<<<(unsigned)((p.n + ROOT_THREADS - 1) / ROOT_THREADS), ROOT_THREADS, 0, st>>>(
        p, M.segs, M.nseg);
    stage_mark(1, st);
    const size_t tq_small = sizeof(double) * 2 * SMALL_THREADS * TWidth<CCD_KIND_EE>::W;
    // pooled stage: one launch per kind over the survivor list, one after the
    // other (run at once they slowed each other: 817 against 790 ms for the
    // 20M-query step's pooled stage)
    pool_kernel<CCD_KIND_VF><<<pool_blocks(pool_kernel<CCD_KIND_VF>, M.sms), 32, 0, st>>>(
        p, M.pool_mem, M.pool_meta, M.T.pool_cap, p.surv, &p.hdr->survivors, &p.hdr->head_pool,
        M.segs, M.nseg);
    pool_kernel<CCD_KIND_EE><<<pool_blocks(pool_kernel<CCD_KIND_EE>, M.sms), 32, 0, st>>>(
        p, M.pool_mem, M.pool_meta, M.T.pool_cap, p.surv, &p.hdr->survivors, &p.hdr->head_pool_ee,
        M.segs, M.nseg);
    stage_mark(2, st);
    solve_kernel_seg<SMALL_THREADS, false><<<M.nb_small, SMALL_THREADS, tq_small, st>>>(
        p, M.segs, M.nseg, 0, (Box *)(M.ws + M.off_small), M.T.small_cap, PagePool{});
    order_by_level_kernel<<<1, 1024, 0, st>>>(p.over, p.over_level, &p.hdr->overflow, p.deep_list);
    order_by_level_kernel<<<1, 1024, 0, st>>>(p.over_ee, p.over_level_ee, &p.hdr->overflow_ee,
                                              p.deep_list_ee);
    stage_mark(3, st);
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}

// The deep stage (paged), one round of at most slice_ns (0: until the list
// is empty); or, for a contiguous layout, the whole deep stage.
template <int DT>
void multi_deep_launch(const MultiPlan &M, long long slice_ns, const volatile int *yield,
                       cudaStream_t st)
{
    const size_t tq_deep = sizeof(SharedUV<DT>);
    Box *slots = (Box *)(M.ws + M.D.off_slots);
    if (M.D.paged) {
        // the two kinds at once on the shared page pool
        const SideStream *sd = side_for(st);
        const cudaStream_t st2 = fork_side(sd, st);
        solve_kernel_seg<DT, true, CCD_KIND_EE><<<M.D.nb_deep, DT, tq_deep, st2>>>(
            M.p, M.segs, M.nseg, 1, nullptr, 0, M.pages, slice_ns, yield);
        solve_kernel_seg<DT, true, CCD_KIND_VF><<<M.D.nb_deep, DT, tq_deep, st>>>(
            M.p, M.segs, M.nseg, 1, nullptr, 0, M.pages, slice_ns, yield);
        join_side(sd, st, st2);
    } else {
        // contiguous slots are one set for both kinds: one after the other
        solve_kernel_seg<DT, false, CCD_KIND_VF><<<M.D.nb_deep, DT, tq_deep, st>>>(
            M.p, M.segs, M.nseg, 1, slots, M.D.cap_deep, PagePool{});
        solve_kernel_seg<DT, false, CCD_KIND_EE><<<M.D.nb_deep, DT, tq_deep, st>>>(
            M.p, M.segs, M.nseg, 1, slots, M.D.cap_deep, PagePool{});
    }
}

ccd_status multi_deep(const MultiPlan &M, long long slice_ns, const volatile int *yield,
                      cudaStream_t st)
{
    if (M.p.n == 0) return CCD_OK;
    if (slice_ns > 0 &&
        cudaMemsetAsync(&M.p.hdr->round_start, 0, sizeof(unsigned long long), st) != cudaSuccess)
        return CCD_ERR_CUDA;
    if (M.T.deep_threads == 128) multi_deep_launch<128>(M, slice_ns, yield, st);
    else if (M.T.deep_threads == 256) multi_deep_launch<256>(M, slice_ns, yield, st);
    else multi_deep_launch<512>(M, slice_ns, yield, st);
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}

// The queries the paged deep stage deferred, restarted in full-size slots.
ccd_status multi_jumbo(const MultiPlan &M, cudaStream_t st)
{
    if (M.p.n > 0 && M.D.paged) {
        Box *slots = (Box *)(M.ws + M.D.off_slots);
        if (M.T.deep_threads == 128)
            solve_kernel_seg<128, false><<<M.D.nb_jumbo, 128, sizeof(SharedUV<128>), st>>>(
                M.p, M.segs, M.nseg, 2, slots, M.D.cap_deep, PagePool{});
        else if (M.T.deep_threads == 256)
            solve_kernel_seg<256, false><<<M.D.nb_jumbo, 256, sizeof(SharedUV<256>), st>>>(
                M.p, M.segs, M.nseg, 2, slots, M.D.cap_deep, PagePool{});
        else
            solve_kernel_seg<512, false><<<M.D.nb_jumbo, 512, sizeof(SharedUV<512>), st>>>(
                M.p, M.segs, M.nseg, 2, slots, M.D.cap_deep, PagePool{});
    }
    stage_mark(4, st);
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}

ccd_status run_multi(const double *verts, int64_t n, const ccd_segment *segs, int32_t nseg,
                     int64_t max_itr_bound, uint8_t *collides, double *toi, double *out_tol,
                     int64_t *checks, const ccd_tuning *tuning, void *workspace, size_t ws_bytes,
                     void *stream)
{
    MultiPlan M;
    ccd_status r = multi_plan(verts, n, segs, nseg, max_itr_bound, collides, toi, out_tol, checks,
                              tuning, workspace, ws_bytes, nullptr, &M);
    if (r != CCD_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    if ((r = multi_front(M, true, st)) != CCD_OK) return r;
    if (n == 0) return CCD_OK;
    if ((r = multi_deep(M, 0, nullptr, st)) != CCD_OK) return r;
    return multi_jumbo(M, st);
}

}  // namespace

// ---- the served form's hooks (see internal.h) -------------------------------------

namespace ccd_internal {

namespace {
PagePool to_pages(const FrontierPool &f)
{
    PagePool p{};
    p.base = (Box *)f.pages;
    p.bits = f.bits;
    p.nwords = f.nwords;
    p.used = f.counters;
    p.peak = f.counters ? f.counters + 1 : nullptr;
    return p;
}

// A served batch's deep launches use the server's block size (see
// served_deep_threads) and share its pool with every other lane's: each
// takes its share of the pool's pages in blocks.
ccd_status plan(const ServedBatch &b, const FrontierPool &pool, MultiPlan *M)
{
    const PagePool pages = to_pages(pool);
    const int sms = device_sms();
    if (sms <= 0) return CCD_ERR_CUDA;
    const int dt = pool.deep_threads ? pool.deep_threads : SEG_DEEP_THREADS;
    const ccd_tuning t = {dt, page_limited_blocks(deep_blocks_per_sm(dt) * sms, pool.npages,
                                                  pool.sharers),
                          0, 0, 0};
    return multi_plan(b.verts, b.n, b.segs, b.nseg, b.max_itr_bound, b.collides, b.toi,
                      b.out_tol, b.checks, &t, b.workspace, b.ws_bytes, &pages, M);
}
}  // namespace

size_t page_bytes() { return PAGE_BYTES; }
size_t pool_bytes(long long npages) { return ::pool_bytes(npages); }

ccd_status pool_init(const FrontierPool &pool, cudaStream_t st)
{
    if (pool.npages < 1 || !pool.bits || !pool.pages) return CCD_ERR_ARG;
    pool_init_kernel<<<(pool.nwords + 255) / 256, 256, 0, st>>>(pool.bits, pool.nwords,
                                                                (int)pool.npages);
    if (pool.counters && cudaMemsetAsync(pool.counters, 0, 2 * sizeof(int), st) != cudaSuccess)
        return CCD_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}

size_t served_workspace_bytes(int64_t n, int64_t max_itr_bound)
{
    if (n < 0 || n >= 0x7fffffffLL || max_itr_bound <= 0) return 0;
    const int sms = device_sms();
    Tuned T;
    if (sms <= 0 || !resolve_tuning(nullptr, sms, &T)) return 0;   // deep shapes: no bytes
    return multi_fixed_bytes(n, sms, T) +
           JUMBO_SLOTS * align256(sizeof(Box) * 2 * (size_t)deep_cap(max_itr_bound));
}

size_t header_bytes() { return sizeof(Header); }

// The server's deep block size: 128 threads (six blocks per SM, the faster
// form for batches of expensive requests with many deep queries) when its
// pool leaves DEEP_MIN_PAGES pages to every such block of every lane and
// kind at once; 256 (three per SM) otherwise, so that a small arena's
// blocks still find pages.
int served_deep_threads(long long npages, int lanes)
{
    const int sms = device_sms();
    const long long need =
        DEEP_MIN_PAGES * 2LL * (lanes > 0 ? lanes : 1) * deep_blocks_per_sm(DEEP_THREADS) * (sms > 0 ? sms : 1);
    return npages >= need ? DEEP_THREADS : SEG_DEEP_THREADS;
}

ccd_status served_front(const ServedBatch &b, const FrontierPool &pool, cudaStream_t st)
{
    MultiPlan M;
    ccd_status r = plan(b, pool, &M);
    return r != CCD_OK ? r : multi_front(M, false, st);
}

ccd_status served_deep_round(const ServedBatch &b, const FrontierPool &pool, long long slice_ns,
                             const volatile int *yield, cudaStream_t st)
{
    MultiPlan M;
    ccd_status r = plan(b, pool, &M);
    return r != CCD_OK ? r : multi_deep(M, slice_ns, yield, st);
}

ccd_status served_finish(const ServedBatch &b, const FrontierPool &pool, cudaStream_t st)
{
    MultiPlan M;
    ccd_status r = plan(b, pool, &M);
    return r != CCD_OK ? r : multi_jumbo(M, st);
}

long long served_deep_left(const void *header)
{
    const Header *h = (const Header *)header;
    return (h->head_deep >= h->overflow ? 0 : (long long)(h->overflow - h->head_deep)) +
           (h->head_deep_ee >= h->overflow_ee ? 0 : (long long)(h->overflow_ee - h->head_deep_ee));
}

int served_status(const void *header) { return ((const Header *)header)->status; }

}  // namespace ccd_internal

extern "C" {

size_t ccd_multi_workspace_bytes(int64_t n, int64_t max_itr_bound, const ccd_tuning *tuning)
{
    if (n < 0 || n >= 0x7fffffffLL || max_itr_bound <= 0) return 0;
    const int sms = device_sms();
    if (sms <= 0) return 0;
    Tuned T;
    if (!resolve_tuning(tuning, sms, &T)) return 0;
    return multi_fixed_bytes(n, sms, T) + default_deep_bytes(max_itr_bound, T.deep_slots);
}

ccd_status ccd_multi_batch(const double *verts, int64_t n, const ccd_segment *segs, int32_t nseg,
                           int64_t max_itr_bound, uint8_t *collides, double *toi,
                           double *out_tol, int64_t *checks, const ccd_tuning *tuning,
                           void *workspace, size_t ws_bytes, void *stream)
{
    return run_multi(verts, n, segs, nseg, max_itr_bound, collides, toi, out_tol, checks, tuning,
                     workspace, ws_bytes, stream);
}

ccd_status ccd_group_reduce(const double *toi, const double *out_tol, int64_t n,
                            const ccd_segment *segs, int32_t nseg, int32_t ngroups,
                            double *alpha, double *tol, void *stream)
{
    if (n < 0 || n >= 0x7fffffffLL || ngroups < 1 || !alpha || !tol ||
        (n > 0 && (!toi || !out_tol || !segs || nseg < 1)))
        return CCD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    group_init_kernel<<<(ngroups + 255) / 256, 256, 0, st>>>(alpha, tol, ngroups);
    if (n > 0) {
        const int sms = device_sms();
        long long blocks = (n + 255) / 256;
        if (blocks > 8LL * sms) blocks = 8LL * sms;
        group_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(toi, out_tol, n, segs, nseg,
                                                             ngroups, alpha, tol);
    }
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}

ccd_status ccd_linf_distance(const double *verts, int64_t n, const ccd_segment *segs,
                             int32_t nseg, int32_t ngroups, double *dist, double *group_min,
                             void *stream)
{
    if (n < 0 || n >= 0x7fffffffLL || ngroups < 1 || !group_min ||
        (n > 0 && (!verts || !segs || nseg < 1)))
        return CCD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    linf_group_init_kernel<<<(ngroups + 255) / 256, 256, 0, st>>>(group_min, ngroups);
    if (n > 0) {
        const int sms = device_sms();
        if (sms <= 0) return CCD_ERR_CUDA;
        long long blocks = (n + 255) / 256;
        if (blocks > 8LL * sms) blocks = 8LL * sms;
        linf_distance_kernel<<<(unsigned)blocks, 256, 0, st>>>(verts, n, segs, nseg, ngroups,
                                                              dist, group_min);
    }
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}

// ---- Algorithm 4's CCD step (host driver over the device kernels) -------------

namespace {

constexpr size_t LS_OFF_SEGS = 0;      // 2 segments (160 B)
constexpr size_t LS_OFF_RED = 256;     // alpha, tol, d_i
constexpr size_t LS_OFF_OUT = 512;     // per-query outputs, then the batch workspace

size_t ls_out_bytes(long long n)
{
    return align256((size_t)n) + 2 * align256(sizeof(double) * (size_t)n);
}

double ls_cap(double x, double delta, int cap_max)
{
    if (cap_max) return x > delta ? x : delta;
    return x < delta ? x : delta;
}

}  // namespace

// MSCCD queries of a line search (ms = d <= delta) mostly bisect through many
// small-to-medium levels: the pooled solver keeps them up to 1024 boxes a level.
const ccd_tuning LS_TUNING = {0, 0, 0, 0, 1024};

size_t ccd_line_search_workspace_bytes(int64_t n, int64_t max_itr)
{
    const size_t m = ccd_multi_workspace_bytes(n, max_itr, &LS_TUNING);
    if (m == 0) return 0;
    return LS_OFF_OUT + ls_out_bytes(n) + m;
}

ccd_status ccd_line_search(const double *verts, int64_t n_vf, int64_t n_ee,
                           ccd_line_search_io *io, void *workspace, size_t ws_bytes, void *stream)
{
    if (!io || n_vf < 0 || n_ee < 0 || n_vf + n_ee >= 0x7fffffffLL) return CCD_ERR_ARG;
    const long long n = n_vf + n_ee;
    if (!(io->p > 0.0 && io->p < 1.0) || !(io->delta > 0.0) || !(io->rho >= 0.0) ||
        io->max_itr < 1 || io->max_passes < 1 || (n > 0 && !verts))
        return CCD_ERR_ARG;
    const size_t need = ccd_line_search_workspace_bytes(n, io->max_itr);
    if (need == 0) return CCD_ERR_CUDA;
    if (!workspace || ws_bytes < need) return CCD_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    ccd_segment *dsegs = (ccd_segment *)(ws + LS_OFF_SEGS);
    double *red = (double *)(ws + LS_OFF_RED);
    uint8_t *collides = (uint8_t *)(ws + LS_OFF_OUT);
    double *toi = (double *)(ws + LS_OFF_OUT + align256((size_t)n));
    double *out_tol = toi + align256(sizeof(double) * (size_t)n) / sizeof(double);
    char *mws = ws + LS_OFF_OUT + ls_out_bytes(n);
    const size_t mws_bytes = ws_bytes - (LS_OFF_OUT + ls_out_bytes(n));

    // two segments of one candidate set; ms > 0 selects Eq. msccd-error
    ccd_segment segs[2];
    for (int k = 0; k < 2; ++k) {
        segs[k].offset = k == 0 ? 0 : n_vf;
        segs[k].count = k == 0 ? n_vf : n_ee;
        segs[k].kind = k == 0 ? CCD_KIND_VF : CCD_KIND_EE;
        segs[k].group = 0;
        segs[k].err[0] = segs[k].err[1] = segs[k].err[2] = 0.0;
        segs[k].ms = 1.0;
        segs[k].delta = io->delta;
        segs[k].max_itr = io->max_itr;
        segs[k].t_max = 1.0;
    }
    const double inf = __builtin_inf();
    double d_i = inf, eps_i = 0.0;
    if (n > 0) {
        if (cudaMemcpyAsync(dsegs, segs, sizeof(segs), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return CCD_ERR_CUDA;
        ccd_status r = ccd_segments_err_from_bounds(verts, n, dsegs, 2, st);
        if (r != CCD_OK) return r;
        r = ccd_linf_distance(verts, n, dsegs, 2, 1, nullptr, red + 2, st);
        if (r != CCD_OK) return r;
        if (cudaMemcpyAsync(segs, dsegs, sizeof(segs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&d_i, red + 2, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return CCD_ERR_CUDA;
        for (int k = 0; k < 2; ++k)
            if (segs[k].count > 0)
                for (int c = 0; c < 3; ++c) eps_i = segs[k].err[c] > eps_i ? segs[k].err[c] : eps_i;
    }

    double p = io->p, alpha = 1.0, delta_cur = io->delta, delta_i = io->delta;
    double d = ls_cap(p * d_i, delta_cur, io->cap_max);
    bool validated = (d_i - d) > ((delta_cur + eps_i) + io->rho);
    int passes = 0;
    ccd_status result = CCD_OK;
    while (n > 0) {
        // find p: halve while the inequality fails and a smaller p could satisfy it
        while (!((d_i - d) > ((delta_cur + eps_i) + io->rho))) {
            const double lim = io->cap_max ? delta_cur : 0.0;
            if (!((d_i - lim) > ((delta_cur + eps_i) + io->rho)) || p == 0.0) break;
            p = p / 2.0;
            d = ls_cap(p * d_i, delta_cur, io->cap_max);
        }
        if (alpha == 0.0) break;   // no time interval left
        // one MSCCD pass on [0, alpha] (SolveMSCCD with ms = d)
        for (int k = 0; k < 2; ++k) {
            segs[k].ms = d;
            segs[k].delta = delta_cur;
            segs[k].t_max = alpha;
        }
        if (cudaMemcpyAsync(dsegs, segs, sizeof(segs), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return CCD_ERR_CUDA;
        ccd_status r = ccd_multi_batch(verts, n, dsegs, 2, io->max_itr, collides, toi, out_tol,
                                       nullptr, &LS_TUNING, mws, mws_bytes, stream);
        if (r != CCD_OK) return r;
        r = ccd_group_reduce(toi, out_tol, n, dsegs, 2, 1, red, red + 1, stream);
        if (r != CCD_OK) return r;
        double got[2];
        int32_t status = 0;
        if (cudaMemcpyAsync(got, red, sizeof(got), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&status, &((const Header *)mws)->status, sizeof(status),
                            cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return CCD_ERR_CUDA;
        if (status == CCD_ERR_ARG) return CCD_ERR_ARG;
        if (status != CCD_OK) result = (ccd_status)status;   // capacity: still conservative
        delta_i = delta_cur;
        alpha = got[0] < alpha ? got[0] : alpha;
        delta_i = got[1] > delta_i ? got[1] : delta_i;
        passes += 1;
        // validate after
        validated = (d_i - d) > ((delta_i + eps_i) + io->rho);
        if (validated || passes >= io->max_passes) break;
        delta_cur = delta_i;
    }
    io->alpha = alpha;
    io->p_out = p;
    io->d = d;
    io->d_i = d_i;
    io->eps_i = eps_i;
    io->delta_i = delta_i;
    io->passes = passes;
    io->validated = validated ? 1 : 0;
    return result;
}

ccd_status ccd_aos_to_soa(const double *aos, int64_t n, double *soa, int64_t ld, void *stream)
{
    if (n < 0 || ld < n || (n > 0 && (!aos || !soa))) return CCD_ERR_ARG;
    if (n == 0) return CCD_OK;
    aos_to_soa_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(aos, n, soa, ld);
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}

ccd_status ccd_segments_err_from_bounds(const double *verts, int64_t n, ccd_segment *segs,
                                        int32_t nseg, void *stream)
{
    if (n < 0 || n >= 0x7fffffffLL || nseg < 1 || !segs || (n > 0 && !verts)) return CCD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned sb = (unsigned)((nseg + 255) / 256);
    seg_err_init_kernel<<<sb, 256, 0, st>>>(segs, nseg);
    if (n > 0) {
        const int sms = device_sms();
        long long blocks = (n + 255) / 256;
        if (blocks > 8LL * sms) blocks = 8LL * sms;
        seg_err_reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(verts, n, segs, nseg);
    }
    seg_err_finish_kernel<<<sb, 256, 0, st>>>(segs, nseg);
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}

}  // extern "C"

// ---- vertex-face batch on a static scratch array (no allocation) -------------
//
// For callers that cannot allocate device memory at all: real-time loops
// that must not enter the driver's allocator, plugins running inside a host
// that owns every allocation, or processes under a fixed device-memory
// quota.  They get one entry point whose scratch is a file-scope device
// array that exists on every GPU that loads this library, until the process
// exits.  Its size bounds the batch: at most STATIC_MAX_N queries and a
// check limit of at most STATIC_MAX_ITR per call; the one-warp stage has
// slots for STATIC_SMALL_BLOCKS blocks and launches four per SM, at most
// that many.

namespace {

constexpr long long STATIC_MAX_N = 32768;
constexpr long long STATIC_MAX_ITR = 65536;
constexpr int STATIC_SMALL_BLOCKS = 608;
constexpr long long STATIC_SMALL_CAP = 256;
constexpr int STATIC_DEEP_SLOTS = 4;
constexpr long long STATIC_DEEP_CAP = 2 * STATIC_MAX_ITR + 64;

constexpr size_t st_al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t STATIC_OFF_SURV = st_al(sizeof(Header));
constexpr size_t STATIC_OFF_OVER = st_al(STATIC_OFF_SURV + sizeof(int) * STATIC_MAX_N);
constexpr size_t STATIC_OFF_KAPPA = st_al(STATIC_OFF_OVER + sizeof(int) * STATIC_MAX_N);
constexpr size_t STATIC_OFF_SMALL = st_al(STATIC_OFF_KAPPA + 3 * sizeof(double) * STATIC_MAX_N);
constexpr size_t STATIC_OFF_DEEP =
    st_al(STATIC_OFF_SMALL + sizeof(Box) * 2 * STATIC_SMALL_CAP * STATIC_SMALL_BLOCKS);
constexpr size_t STATIC_END = STATIC_OFF_DEEP + sizeof(Box) * 2 * STATIC_DEEP_CAP * STATIC_DEEP_SLOTS;

}  // namespace

// 40 MiB on every device that loads the library.
#define CCD_STATIC_SCRATCH_BYTES (40u << 20)
static __device__ __align__(256) unsigned char g_static_scratch[CCD_STATIC_SCRATCH_BYTES];
static_assert(STATIC_END <= CCD_STATIC_SCRATCH_BYTES, "static layout must fit the scratch array");

namespace {

constexpr int STATIC_MAX_DEVICES = 64;
std::mutex g_static_mu;
void *g_static_ptr[STATIC_MAX_DEVICES];

// Device address of the scratch array on the current device.  The array's
// host-side name is only a stand-in for the symbol; the device address comes
// from cudaGetSymbolAddress, once per device, with that device current.
char *static_scratch(ccd_status *why)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= STATIC_MAX_DEVICES) {
        *why = CCD_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            *why = CCD_ERR_CUDA;
            return nullptr;
        }
        g_static_ptr[dev] = p;
    }
    return (char *)g_static_ptr[dev];
}

}  // namespace

extern "C" ccd_status ccd_vf_batch_static(const double *verts, int64_t n, const double *err,
                                          int err_stride, double ms, double delta,
                                          int64_t max_itr, uint8_t *collides, double *toi,
                                          double *out_tol, int64_t *checks, void *stream)
{
    if (n < 0 || !(delta > 0.0) || max_itr <= 0 || !(ms >= 0.0) ||
        (err_stride != 0 && err_stride != 3))
        return CCD_ERR_ARG;
    if (n > 0 && (!verts || !err || !collides || !toi || !out_tol)) return CCD_ERR_ARG;
    if (n > STATIC_MAX_N || max_itr > STATIC_MAX_ITR) return CCD_ERR_WORKSPACE;
    ccd_status why = CCD_OK;
    char *ws = static_scratch(&why);
    if (!ws) return why;
    cudaStream_t st = (cudaStream_t)stream;
    // the counters at the front of the scratch must start at zero each call
    if (cudaMemsetAsync(ws, 0, sizeof(Header), st) != cudaSuccess) return CCD_ERR_CUDA;
    if (n == 0) return CCD_OK;

    Params p;
    p.verts = verts; p.n = n; p.err = err; p.err_stride = err_stride;
    p.ms = ms; p.delta = delta; p.max_itr = max_itr;
    p.collides = collides; p.toi = toi; p.out_tol = out_tol; p.checks = (long long *)checks;
    p.hdr = (Header *)ws;
    p.surv = (int *)(ws + STATIC_OFF_SURV);
    p.mid = nullptr;
    p.over = (int *)(ws + STATIC_OFF_OVER);
    p.over_level = nullptr;   // no deep-tier ordering in the static-scratch path
    p.deep_list = nullptr;
    p.over_ee = nullptr;
    p.over_level_ee = nullptr;
    p.deep_list_ee = nullptr;
    p.jumbo = nullptr;
    p.kappa = (double *)(ws + STATIC_OFF_KAPPA);
    Header *h = p.hdr;

    const long long blocks = (n + ROOT_THREADS - 1) / ROOT_THREADS;
    root_kernel<CCD_KIND_VF><<<(unsigned)blocks, ROOT_THREADS, 0, st>>>(p);
    const size_t tq_small = sizeof(double) * 2 * SMALL_THREADS * TWidth<CCD_KIND_VF>::W;
    const size_t tq_deep = sizeof(SharedUV<DEEP_THREADS>);
    if (cudaFuncSetAttribute(solve_kernel<CCD_KIND_VF, DEEP_THREADS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tq_deep) !=
        cudaSuccess)
        return CCD_ERR_CUDA;
    int small_blocks = 4 * device_sms();
    if (small_blocks < 1 || small_blocks > STATIC_SMALL_BLOCKS) small_blocks = STATIC_SMALL_BLOCKS;
    solve_kernel<CCD_KIND_VF, SMALL_THREADS><<<small_blocks, SMALL_THREADS, tq_small, st>>>(
        p, 0, (Box *)(ws + STATIC_OFF_SMALL), STATIC_SMALL_CAP, PagePool{}, p.surv, &h->survivors,
        &h->head_small, p.over, nullptr, &h->overflow);
    solve_kernel<CCD_KIND_VF, DEEP_THREADS><<<STATIC_DEEP_SLOTS, DEEP_THREADS, tq_deep, st>>>(
        p, 1, (Box *)(ws + STATIC_OFF_DEEP), STATIC_DEEP_CAP, PagePool{}, p.over, &h->overflow,
        &h->head_deep, nullptr, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ERR_CUDA;
}
