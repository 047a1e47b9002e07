/*
 * ccd.h -- C ABI of the GB300 (sm_103a) batched inclusion-based continuous
 * collision detection root finder.
 *
 * Method: Wang, Ferguson, Schneider, Jiang, Attene, Panozzo, "A Large Scale
 * Benchmark and an Inclusion-Based Algorithm for Continuous Collision
 * Detection", ACM TOG 40(5), 2021.  Every query solves Algorithm 2 (Sec. 4):
 * breadth-first bisection of the parameter box [0,1]^3 of F(t,u,v)
 * (Eq. F-vf, Eq. F-ee) with the box inclusion function B_F (Eq. box), the
 * conservative floating-point filter eps (Eq. ccd-error), the kappa-weighted
 * widest-dimension split (Eq. kappas), tolerance delta and the check limit
 * m_I; with minimum separation d > 0 the box is enlarged by d (Sec. 5.1).
 *
 * Conventions shared by every entry point:
 *  - All array pointers are DEVICE pointers owned by the caller; the library
 *    never allocates, frees or retains them.  Calls are asynchronous on
 *    `stream` (a cudaStream_t passed as void*; NULL = legacy default stream).
 *  - verts: structure of arrays, 24 planes of n doubles (plane stride n).
 *    Plane k holds coordinate k%3 of point (k/3)%4 at time k/12 (t0 for
 *    k < 12, t1 for k >= 12).  Vertex-face (VF) points are (p, v1, v2, v3);
 *    edge-edge (EE) points are (p1, p2, p3, p4) (Appendix A ordering).
 *  - Inputs must be finite.  n must be below 2^31.
 *  - Floating point is IEEE binary64, round to nearest, never contracted.
 *
 * Status codes are returned by value; errors found on the device are
 * recorded in the workspace and read with ccd_workspace_status().
 */
#ifndef CCD_GB300_H
#define CCD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CCD_OK = 0,
    CCD_ERR_ARG = -1,       /* invalid argument (checked on the host)          */
    CCD_ERR_WORKSPACE = -2, /* workspace too small for even one deep slot      */
    CCD_ERR_TIMEOUT = -3,   /* a bounded device wait gave up                   */
    CCD_ERR_CUDA = -4,      /* a CUDA launch or copy failed                    */
    CCD_ERR_CAPACITY = -5,  /* device: a frontier exceeded its slot; the query
                               was answered conservatively (see ccd_vf_batch)  */
    CCD_ERR_BUSY = -6,      /* server: no room for the request now; poll and
                               submit again (or the request is already running)*/
    CCD_ERR_CANCELLED = -7  /* server: the request was cancelled               */
} ccd_status;

#define CCD_KIND_VF 0
#define CCD_KIND_EE 1

/*
 * Workspace of ccd_vf_batch / ccd_ee_batch (n queries, check limit max_itr).
 * It holds per-query lists, the small-frontier solvers' slots and the deep
 * tier:
 *  - a pool of frontier pages (32,768 boxes of 24 bytes = 768 KB each)
 *    shared by the deep solver's blocks (six per SM): each level of a deep
 *    query takes pages for its children and frees the previous level's, so
 *    memory follows the frontiers actually reached;
 *  - two full-size slots (two arrays of 2 * max_itr + 64 boxes, which no
 *    level can outgrow: every box of a level is a child of a colliding box
 *    checked before the limit) for queries that found the pool empty; they
 *    restart there.
 * The pool's size therefore changes speed only, never results.
 * ccd_workspace_bytes gives a pool with pages for one level of
 * 2 * max_itr + 64 boxes (at least two pages) for three deep blocks per SM
 * (the six share it; levels rarely reach that size); ccd_workspace_bytes_pages
 * one of `pages` pages (>= 2).  A workspace too small for one full-size slot
 * and two pages is used as contiguous slots of fewer boxes, with the
 * capacity fallback described at ccd_vf_batch.  Both return 0 on bad
 * arguments or without a device.
 */
size_t ccd_workspace_bytes(int64_t n, int64_t max_itr);
size_t ccd_workspace_bytes_pages(int64_t n, int64_t max_itr, int64_t pages);

/* How a workspace of ws_bytes is laid out for n queries at max_itr. */
typedef struct {
    int32_t paged;        /* 1: page pool + full-size slots; 0: contiguous slots */
    int32_t deep_blocks;  /* deep-solver blocks (paged) or slots (contiguous)    */
    int32_t full_slots;   /* slots of slot_boxes boxes per level                 */
    int32_t pad;
    int64_t pages;        /* frontier pages in the pool (paged)                  */
    int64_t slot_boxes;   /* boxes per level of a slot                           */
    size_t fixed_bytes;   /* everything before the deep tier                     */
    size_t used_bytes;    /* bytes of the workspace the layout uses              */
} ccd_workspace_info;

/* CCD_ERR_WORKSPACE if ws_bytes cannot hold any layout. */
ccd_status ccd_workspace_layout(int64_t n, int64_t max_itr, size_t ws_bytes,
                                ccd_workspace_info *info);

/*
 * Batched vertex-face CCD (Algorithm 2 on F_vf, Eq. F-vf; prism-culled
 * splits, Sec. 4.2).
 *
 *  verts    [24][n] f64  query points (layout above).
 *  n        number of queries, 0 <= n < 2^31 (n = 0 is a no-op).
 *  err      eps per axis (Eq. ccd-error; with ms > 0 Eq. msccd-error):
 *           3 doubles shared by all queries when err_stride == 0, or
 *           [n][3] doubles when err_stride == 3.  ccd_err_from_bounds
 *           computes them.
 *  ms       minimum separation d >= 0 (L-infinity, Sec. 5.1); 0 = plain CCD.
 *  delta    tolerance delta > 0 on the co-domain width w(B).
 *  max_itr  check limit m_I > 0.
 *  collides [n] u8   1 if a (conservative) collision was found, else 0.
 *  toi      [n] f64  conservative time of impact: left end of the first
 *           colliding t-interval of the last level reached; +inf when
 *           collides == 0.
 *  out_tol  [n] f64  co-domain width w(B) of the box checked when the query
 *           returned (the reached tolerance); 0 when collides == 0.
 *  checks   [n] i64  number of box checks n of Algorithm 2; may be NULL.
 *  workspace, ws_bytes  device scratch (see ccd_workspace_bytes); it must
 *           not be used by another call that may overlap on the device.
 *
 * Results are deterministic and independent of the launch configuration
 * and of the workspace's pool size.  Only a workspace too small for a
 * full-size slot can fall short: a query whose frontier does not fit its
 * contiguous slot returns as at the check limit -- collides = 1, toi = left
 * end of the current level's first colliding t-interval -- and the workspace
 * status becomes CCD_ERR_CAPACITY.
 * Returns CCD_ERR_ARG for n < 0, n >= 2^31, delta <= 0 or NaN, max_itr <= 0,
 * ms < 0 or NaN, err_stride not in {0, 3}, or a NULL array with n > 0;
 * CCD_ERR_WORKSPACE if the workspace is NULL or too small; CCD_ERR_CUDA if a
 * launch fails.
 */
ccd_status ccd_vf_batch(const double *verts, int64_t n, const double *err,
                        int err_stride, double ms, double delta, int64_t max_itr,
                        uint8_t *collides, double *toi, double *out_tol,
                        int64_t *checks, void *workspace, size_t ws_bytes,
                        void *stream);

/*
 * Batched edge-edge CCD (Algorithm 2 on F_ee, Eq. F-ee; no culling since
 * the domain is the whole cube).  Arguments, outputs and errors exactly as
 * for ccd_vf_batch.
 */
ccd_status ccd_ee_batch(const double *verts, int64_t n, const double *err,
                        int err_stride, double ms, double delta, int64_t max_itr,
                        uint8_t *collides, double *toi, double *out_tol,
                        int64_t *checks, void *workspace, size_t ws_bytes,
                        void *stream);

/*
 * Floating-point filter eps (Eq. ccd-error, Eq. msccd-error):
 * eps_c = K * gamma_c^3 with gamma_c = max(max_i |x_i^c|, 1), computed as
 * K * ((gamma * gamma) * gamma), K = 30, 28, 34, 32 * 2^-52 for VF, EE,
 * VF with ms, EE with ms.  per_query == 0 takes the maximum over all points
 * of all n queries (scene-wide tolerance, Sec. 6) and writes 3 doubles;
 * per_query != 0 writes [n][3].  err_out is a device pointer.  The ms
 * constants assume d < gamma (Sec. 5.1).
 */
ccd_status ccd_err_from_bounds(int kind, const double *verts, int64_t n,
                               int ms_nonzero, int per_query, double *err_out,
                               void *stream);

/*
 * Device status recorded in the workspace by the last call that used it:
 * CCD_OK or CCD_ERR_CAPACITY; *fallbacks (may be NULL) receives how many
 * queries were answered by the capacity fallback.  Synchronizes `stream`.
 */
ccd_status ccd_workspace_status(const void *workspace, int32_t *status,
                                int32_t *fallbacks, void *stream);

/*
 * Counters of the last batch that used `workspace` (synchronizes `stream`);
 * the first min(count, CCD_NUM_COUNTERS) are written to `counters`:
 * [0] queries that survived the level-0 check, [1] queries moved to the deep
 * solver, [2] capacity fallbacks, [3] sum of check counts n of queries
 * finished by the small-frontier solver, [4] the same for the deep solver,
 * [5] box evaluations executed by the small-frontier solver (including work
 * of queries it handed on), [6] the same for the deep solver, [7] status,
 * [8] t-quantity evaluations (positions and edge vectors at one t, shared by
 * a run of boxes with equal t_L) by the small-frontier solver, [9] the same
 * for the deep solver, [10] shared partials computed by the deep solver (one
 * per t value and parameter value: u for VF, v for EE), [11] deep chunks
 * that exceeded the shared tables and were evaluated as sub-chunks of 128
 * boxes, [12] deep box evaluations that used the shared partials (all of
 * them), [13] queries the pooled solver handed to
 * the one-warp solver, [14] sum of check counts n of queries finished by
 * the pooled solver, [15] box evaluations executed by the pooled solver,
 * [16] and [17] the edge-edge parts of [9] and [10], [18] of [15], [19] of
 * [8] and [20] of [5]
 * (the vertex-face part is the difference), [21] deep queries that found
 * the page pool empty and restarted in a full-size slot, [22] the most
 * frontier pages held at once, [23] t-quantity evaluations of the pooled
 * solver (one per distinct t value of an iteration, shared by that
 * iteration's boxes), [24] their edge-edge part, [25] iterations of the
 * pooled solver's warps and [26] the sum over them of the most boxes one
 * query placed in the iteration, [27] shared partials computed by the
 * pooled solver (one per distinct t value and parameter value of an
 * iteration), [28] their edge-edge part, [29] pooled box evaluations that
 * used them (the rest evaluated their corners directly), [30] the
 * edge-edge part of [29], [31] the edge-edge part of [6] and [32] of [12].
 * The small-frontier solver of [3], [5], [8] is the one-warp solver.
 */
#define CCD_NUM_COUNTERS 33
ccd_status ccd_workspace_counters(const void *workspace, int64_t *counters, int32_t count,
                                  void *stream);

/*
 * Optional stage timing for benchmarks: with count == 5, every following
 * batch call records events[0] before the level-0 kernel, events[1] after
 * it, events[2] after the pooled solver, events[3] after the one-warp
 * solver and events[4] after the deep solver, on the call's stream
 * (ccd_multi_batch records events[0] after its segment validation).  The
 * events (cudaEvent_t, created by the caller) are not retained beyond the
 * next ccd_set_stage_events call; count == 0 switches recording off.  A call
 * captured into a CUDA graph while they are set records them at every
 * replay of that graph, so they must outlive the graph: replaying it after
 * destroying them is undefined (a crash on GB300).  Process-wide; not
 * thread-safe.
 */
ccd_status ccd_set_stage_events(void *const *events, int count);

/*
 * Multi-instance batches.  Queries of many simulation instances share one
 * call: the query array is split into segments, each with its own kind,
 * tolerances and check limit (Sec. 6 computes eps per scene, and a line
 * search calls CCD with its own delta, d and m_I per step).  A segment
 * covers queries [offset, offset + count) of verts; the segments of a call
 * must tile [0, n) in order (segment s + 1 starts where s ends).
 */
typedef struct {
    int64_t offset;   /* first query of the segment                          */
    int64_t count;    /* number of queries (>= 0)                            */
    int32_t kind;     /* CCD_KIND_VF or CCD_KIND_EE                          */
    int32_t group;    /* candidate set id >= 0, for ccd_group_reduce         */
    double err[3];    /* eps per axis for this segment (Eq. ccd-error)       */
    double ms;        /* minimum separation d >= 0 (Sec. 5.1)                */
    double delta;     /* tolerance delta > 0                                 */
    int64_t max_itr;  /* check limit m_I, 1 <= m_I <= the call's bound       */
    double t_max;     /* time interval [0, t_max], 0 < t_max <= 1: the
                         shortened interval of SolveMSCCD (Sec. 6); the
                         solver works in s in [0,1] with t = t_max * s
                         rounded once, and toi = t_max * s_L               */
} ccd_segment;        /* 80 bytes, 8-byte aligned */

/*
 * Launch shapes of the solver kernels.  They change speed only: results are
 * identical for every valid tuning.  A zero field takes the default.
 *  deep_threads         threads of a deep-solver block, 128, 256 or 512 (256)
 *  deep_slots           deep-solver blocks per kind (as many as fit at once:
 *                       six per SM of 128 threads, three of 256, one of 512)
 *  small_blocks_per_sm  one-warp solver blocks per SM, 1..32 (16)
 *  small_cap            boxes per one-warp solver frontier, >= 64 (256)
 *  pool_cap             boxes per level a query may reach in the pooled
 *                       solver before the one-warp solver takes it over,
 *                       32..4096 (64); the pooled slots take
 *                       72 * pool_cap bytes each, 32 slots per pooled
 *                       block and up to 24 blocks per SM
 */
typedef struct {
    int32_t deep_threads;
    int32_t deep_slots;
    int32_t small_blocks_per_sm;
    int32_t small_cap;
    int32_t pool_cap;
} ccd_tuning;

/* Workspace bytes for ccd_multi_batch (tuning may be NULL for defaults). */
size_t ccd_multi_workspace_bytes(int64_t n, int64_t max_itr_bound, const ccd_tuning *tuning);

/*
 * One batch over all segments (both kinds), with one launch per solver
 * stage.  segs: DEVICE array of nseg segments (read on the device, so a
 * captured CUDA graph can be replayed with new segment contents);
 * max_itr_bound: an upper bound on every segment's max_itr, used to size the
 * deep frontier slots.  Outputs as for ccd_vf_batch, per query.  The
 * segment table is checked on the device: a table that does not tile
 * [0, n), or has a bad kind, delta <= 0, ms < 0, max_itr < 1, max_itr >
 * max_itr_bound, t_max outside (0, 1] or group < 0, sets the workspace
 * status to CCD_ERR_ARG and no query is answered.  Host-side errors as for ccd_vf_batch, plus CCD_ERR_ARG for
 * nseg < 1 with n > 0, a NULL segs, or an invalid tuning.
 * The two kinds' deep launches run at once: the second on a
 * stream of the library's own (one per calling stream, created on the first
 * call from that stream made outside a CUDA graph capture), forked from and
 * joined back into `stream` with events, so the call stays ordered on
 * `stream`.  A first call captured before any uncaptured call from its
 * stream runs the two kinds one after the other.
 */
ccd_status ccd_multi_batch(const double *verts, int64_t n, const ccd_segment *segs, int32_t nseg,
                           int64_t max_itr_bound, uint8_t *collides, double *toi,
                           double *out_tol, int64_t *checks, const ccd_tuning *tuning,
                           void *workspace, size_t ws_bytes, void *stream);

/*
 * Writes each segment's err[] from the bounds of its own points (Eq.
 * ccd-error, or Eq. msccd-error when the segment's ms > 0; the constant
 * follows the segment's kind), as ccd_err_from_bounds does for one scene.
 * segs is a DEVICE array that this call updates in place.
 */
ccd_status ccd_segments_err_from_bounds(const double *verts, int64_t n, ccd_segment *segs,
                                        int32_t nseg, void *stream);

/*
 * Line-search reduction per candidate set (Algorithm 4): for every group g
 * of segments, alpha[g] = min toi and tol[g] = max out_tol over the group's
 * queries (+inf and 0 for a group without collisions), from the outputs of
 * a ccd_multi_batch over the same segment table.  The caller then takes
 * alpha <- min(alpha, alpha[g]) and delta_i <- max(delta, tol[g]).  Segments
 * whose group is >= ngroups are skipped.  All pointers are device pointers;
 * alpha and tol hold ngroups doubles.
 */
ccd_status ccd_group_reduce(const double *toi, const double *out_tol, int64_t n,
                            const ccd_segment *segs, int32_t nseg, int32_t ngroups,
                            double *alpha, double *tol, void *stream);

/*
 * L-infinity distance between the two primitives of each query at t = 0 (the
 * norm of minimum separation, Sec. 5.1): min over the domain (VF triangle
 * u, v >= 0, u + v <= 1; EE unit square) of max_c |F_c(0, u, v)|.  This is
 * Algorithm 4's distance d_i (Sec. 6, "Line Search") of a candidate.
 *
 * Fixed operation sequence (round to nearest, no contraction):
 *   A, B, C per axis, one subtraction each of t = 0 coordinates:
 *     VF: A = p - v1, B = v1 - v2, C = v1 - v3;  EE: A = p1 - p3,
 *     B = p2 - p1, C = p3 - p4;
 *   g(u, v) = max_c |(A_c + u B_c) + v C_c|;
 *   the result is the minimum of g over the linear program's candidate
 *   vertices that lie in the domain: the domain corners; on each domain edge
 *   (u, v) = (pu + tau du, pv + tau dv) with alpha_c = (A_c + pu B_c) +
 *   pv C_c and beta_c = du B_c + dv C_c, tau = -alpha_c / beta_c and tau =
 *   (s alpha_c2 - alpha_c1) / (beta_c1 - s beta_c2) for c1 < c2, s = +-1,
 *   where 0 <= tau <= 1; in the interior the solutions (u, v) = (b1 a22 -
 *   a12 b2, a11 b2 - b1 a21) / (a11 a22 - a12 a21) of f_c1 = f_c2 = 0 and of
 *   s1 f_1 = s2 f_2 = s3 f_3 for the sign patterns (+,+,+), (+,+,-),
 *   (+,-,+), (-,+,+).
 * The rounding of these few operations is the error rho_i that Algorithm 4
 * adds to its inequality.
 *
 * verts: SoA as for ccd_multi_batch, segs: DEVICE segment table (kind and
 * group of each query).  dist: n doubles or NULL; group_min: ngroups doubles,
 * the minimum over each group's queries (+inf for an empty group).  Queries
 * of segments with group >= ngroups only get dist.  Device pointers.
 */
ccd_status ccd_linf_distance(const double *verts, int64_t n, const ccd_segment *segs,
                             int32_t nseg, int32_t ngroups, double *dist, double *group_min,
                             void *stream);

/*
 * Algorithm 4's CCD step for one line search (Sec. 6): given the candidate
 * set C (n_vf vertex-face queries followed by n_ee edge-edge queries in one
 * SoA array, x1 = x0 + dx already applied), computes
 *   d_i     = min over C of the L-infinity distance at t = 0;
 *   eps_i   = max over kinds and axes of the scene's Eq. msccd-error;
 *   d       = min(p d_i, delta), or max(p d_i, delta) with cap_max = 1 (the
 *             printed formula; the text caps d at delta);
 *   find p:   while (d_i - d) > ((delta + eps_i) + rho) fails and a smaller p
 *             could satisfy it: p <- p / 2, d recomputed;
 *   a pass:   SolveMSCCD with ms = d, tolerance delta, check limit max_itr on
 *             the interval [0, alpha] for every candidate (all with the alpha
 *             of the pass's start); alpha <- min(alpha, min toi), delta_i <-
 *             max(delta, max out_tol);
 *   validate: done if (d_i - d) > ((delta_i + eps_i) + rho); otherwise
 *             delta <- delta_i and back to find p, for at most max_passes
 *             passes (or until alpha = 0).
 * The backtracking on the energy that follows in Algorithm 4 belongs to the
 * caller.  Inputs: p in (0, 1), delta > 0, rho >= 0 (the paper uses 1e-9),
 * max_itr >= 1, max_passes >= 1.  Outputs: alpha (the step bound in
 * [0, 1]), p_out (the validated p), d, d_i, eps_i, delta_i, passes and
 * validated (1 when the inequality holds at return).  Synchronizes `stream`
 * after each pass (the loop decides on the host).  verts is a device
 * pointer; io lives in host memory; workspace (device) is at least
 * ccd_line_search_workspace_bytes(n_vf + n_ee, max_itr).  Returns
 * CCD_ERR_CAPACITY when a pass fell back on a frontier (outputs stay
 * conservative), otherwise as for ccd_multi_batch.
 */
typedef struct {
    double p;            /* in  */
    double delta;        /* in  */
    double rho;          /* in  */
    int64_t max_itr;     /* in  */
    int32_t max_passes;  /* in  */
    int32_t cap_max;     /* in: 0 = min(p d_i, delta), 1 = max(p d_i, delta) */
    double alpha;        /* out */
    double p_out;        /* out */
    double d;            /* out */
    double d_i;          /* out */
    double eps_i;        /* out */
    double delta_i;      /* out */
    int32_t passes;      /* out */
    int32_t validated;   /* out */
} ccd_line_search_io;

size_t ccd_line_search_workspace_bytes(int64_t n, int64_t max_itr);
ccd_status ccd_line_search(const double *verts, int64_t n_vf, int64_t n_ee,
                           ccd_line_search_io *io, void *workspace, size_t ws_bytes,
                           void *stream);

/*
 * Active-set construction (Sec. 6, Algorithm 3) for a triangle mesh moving
 * linearly from x0 to x1.  Mesh arrays are DEVICE arrays: x0, x1 are nv x 3
 * doubles (vertex-major), faces nf x 3 and edges ne x 2 int32 vertex ids
 * (each edge once).  Three steps:
 *
 * ccd_scene_eps: eps of the scene (Sec. 6 computes it from the bounds of all
 *   the vertices of the simulation): gamma_c = max(1, max over every vertex
 *   at both times of |x_c|), eps[3 k + c] = K_k ((gamma_c gamma_c) gamma_c)
 *   with K of Eq. ccd-error for k = VF (0) and EE (1); eps is host memory.
 *   workspace: at least 256 bytes of device memory.  Synchronizes `stream`.
 *
 * ccd_broad_phase: the candidate set C (the paper names the broad phase
 *   only; this is its plain definition): every vertex-face pair (v, f), v not
 *   a vertex of f, and every edge-edge pair (a, b), a < b, without a shared
 *   vertex, whose swept boxes overlap.  A swept box is the per-axis min / max
 *   of the primitive's vertices at both times, minus / plus margin; boxes
 *   overlap when lo_1 <= hi_2 and lo_2 <= hi_1 on every axis.  With margin
 *   >= max eps / 2 no pair that the CCD filter could report is missing (boxes
 *   apart by more than eps on an axis keep |F_c| > eps there).  Output:
 *   vf_pairs (cap_vf x 2: v, f) and ee_pairs (cap_ee x 2: a, b), each sorted
 *   by (first, second); counts[0..1] (host) receive the numbers of pairs.
 *   If a count exceeds its capacity the call returns CCD_ERR_CAPACITY with
 *   the counts set and the lists undefined: call again with larger
 *   capacities.  Uniform-grid method: cells of a power-of-two edge >= 1.01
 *   times the largest swept box, CUB radix sorts.  Synchronizes `stream`.
 *
 * ccd_active_set: for every candidate, t <- CCD(x0 of c, x1 of c, delta,
 *   max_itr) (Algorithm 2, ms = 0, eps of the scene); C_A = the candidates
 *   with 0 <= t <= 1 (a reported collision), in candidate order (VF pairs,
 *   then EE pairs): out_kind[i] (CCD_KIND_VF / CCD_KIND_EE), out_pairs[2 i],
 *   out_pairs[2 i + 1] (the pair's ids) and out_toi[i]; each output holds
 *   n_vf + n_ee entries.  *n_active (host) receives |C_A|; eps_out (host,
 *   may be NULL) the 6 eps used.  Synchronizes `stream`.  Returns
 *   CCD_ERR_CAPACITY when a frontier fell back (answers stay conservative).
 */
ccd_status ccd_scene_eps(const double *x0, const double *x1, int64_t nv, double eps[6],
                         void *workspace, size_t ws_bytes, void *stream);
size_t ccd_broad_phase_workspace_bytes(int64_t nv, int64_t nf, int64_t ne, int64_t cap_vf,
                                       int64_t cap_ee);
ccd_status ccd_broad_phase(const double *x0, const double *x1, int64_t nv, const int32_t *faces,
                           int64_t nf, const int32_t *edges, int64_t ne, double margin,
                           int32_t *vf_pairs, int64_t cap_vf, int32_t *ee_pairs, int64_t cap_ee,
                           int64_t counts[2], void *workspace, size_t ws_bytes, void *stream);
size_t ccd_active_set_workspace_bytes(int64_t n_cand, int64_t max_itr);
ccd_status ccd_active_set(const double *x0, const double *x1, int64_t nv, const int32_t *faces,
                          const int32_t *edges, const int32_t *vf_pairs, int64_t n_vf,
                          const int32_t *ee_pairs, int64_t n_ee, double delta, int64_t max_itr,
                          int32_t *out_kind, int32_t *out_pairs, double *out_toi,
                          int64_t *n_active, double eps_out[6], void *workspace, size_t ws_bytes,
                          void *stream);

/*
 * Layout helper: copies n queries from an array of structures aos[n][24]
 * (query-major, the same 24-value order) into columns [0, n) of a structure
 * of arrays with plane stride ld >= n: soa[k * ld + i] = aos[i * 24 + k].
 * Device pointers; soa may point into a larger batch array (column offset).
 */
ccd_status ccd_aos_to_soa(const double *aos, int64_t n, double *soa, int64_t ld, void *stream);

/*
 * Vertex-face batch that allocates nothing (the paper has no counterpart;
 * this is a deployment variant of ccd_vf_batch).
 *
 * For callers that cannot allocate device memory: real-time loops that must
 * not enter the allocator, plugins inside a host application that owns every
 * allocation, processes under a fixed device-memory quota.  Instead of a
 * caller workspace it uses a 40 MiB file-scope device array that every GPU
 * loading this library holds until the process exits.  Inputs and outputs
 * are as for ccd_vf_batch and still come from the caller; results are
 * identical to ccd_vf_batch's for the same arguments.
 *
 * Limits: n <= 32768 queries and max_itr <= 65536 per call; larger requests
 * return CCD_ERR_WORKSPACE without doing any work.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture.
 * The array keeps the last call's contents and every call shares it: the
 * counters it needs zeroed are cleared on the stream at the start of each
 * call, and calls that may overlap on the GPU (different streams, or
 * concurrent host threads) race with each other and must be serialized by
 * the caller.  No cudaMalloc, cudaFree or other allocating routine is called.
 */
ccd_status ccd_vf_batch_static(const double *verts, int64_t n, const double *err,
                               int err_stride, double ms, double delta, int64_t max_itr,
                               uint8_t *collides, double *toi, double *out_tol,
                               int64_t *checks, void *stream);

/*
 * The served form: a request server with continuous batching.
 *
 * Clients submit requests -- a set of queries of one kind with their own
 * delta, ms and m_I (a line search calls CCD with its own d, delta and m_I
 * every step, Algorithm 4) -- whenever they have them, and poll for the ones
 * that finished.  The server owns one device arena of budget_bytes, split
 * into:
 *  - a device-resident request queue: an inbox ring of query records (the
 *    request's 24 doubles per query are copied there on submission) and a
 *    ring of request descriptors;
 *  - per lane (a CUDA stream) the region of one batch;
 *  - a pool of deep-frontier pages shared by every lane's deep stage.
 * Whenever a lane is free, poll() and submit() give it the oldest run of
 * waiting requests of one cost class, up to max_batch queries and
 * max_segments requests.  Requests with ms > delta subdivide whole |F| <= ms
 * regions (about 10^6 checks per colliding query at the paper's m_I) and are
 * "expensive": they run only on the last lane, at the lower stream priority,
 * one batch (of at most 65,536 queries) at a time in arrival order; the
 * other lanes, at the higher priority, take only cheap requests.  On the
 * lane's stream the batch's segment table is gathered from the descriptors
 * and its records turned into planes, on the device; eps comes from each
 * request's own bounds (Eq. ccd-error / msccd-error over its points, Sec.
 * 6), and the solver stages of ccd_multi_batch run.  The deep stage runs in
 * rounds: when a cheap batch starts while an expensive one is in its deep
 * stage, the latter's blocks are asked (a flag in mapped host memory) to take
 * no new query, which lets the cheap batch's kernels onto the SMs, and
 * poll() starts the next round; with deep_slice_us > 0 rounds also end after
 * that long.  No kernel waits for anything.  Every request's outputs equal
 * those of ccd_vf_batch / ccd_ee_batch on its queries alone with eps from
 * its own bounds.
 *
 * Requests whose queries do not fit the inbox or the descriptor ring right
 * now are refused with CCD_ERR_BUSY (submit again after a poll); requests
 * larger than max_batch, or with max_itr above max_itr_bound, can never run
 * and are refused with CCD_ERR_ARG.  A waiting request can be cancelled.
 * One host thread drives a server; it uses the device current at begin.
 * poll() advances the batches (the next deep round, result copies): call it
 * often while requests are in flight.
 */
typedef struct ccd_server ccd_server;

typedef struct {
    size_t budget_bytes;     /* device bytes of the arena (default 40 GiB)      */
    int32_t lanes;           /* batches in flight, 1..16 (default 4)            */
    int32_t max_requests;    /* requests holding inbox space (default 4096)     */
    int64_t max_batch;       /* queries per batch and per request (2^20)        */
    int64_t inbox_queries;   /* inbox capacity in queries (4 * max_batch)       */
    int32_t max_segments;    /* requests per batch (default 1024)               */
    int32_t pad;
    int64_t max_itr_bound;   /* largest m_I a request may ask for (10^6)        */
    int64_t deep_slice_us;   /* deep rounds also end after this long (0: no)    */
} ccd_server_config;         /* zero fields take the defaults */

typedef struct {
    int32_t kind;            /* CCD_KIND_VF or CCD_KIND_EE                       */
    int32_t pad;
    int64_t n;               /* queries, 0 <= n <= max_batch                     */
    const double *verts;     /* HOST, n x 24 (query-major, the 24-value order of
                                the SoA planes); copied during the call         */
    double ms, delta;        /* minimum separation d >= 0, tolerance delta > 0   */
    int64_t max_itr;         /* check limit, 1 <= m_I <= max_itr_bound            */
    uint8_t *collides;       /* HOST outputs, n each, written by the poll that  */
    double *toi;             /* reports the request                              */
    double *out_tol;
    int64_t *checks;         /* HOST, may be NULL                                */
} ccd_request;

typedef struct {
    int64_t submitted, completed, cancelled, busy_rejections;
    int64_t batches, deep_rounds;
    int64_t yields;              /* deep rounds asked to end for a cheap batch  */
    int64_t inbox_peak_queries;  /* the most inbox records held at once         */
    int64_t pages;               /* frontier pages in the shared pool           */
    int32_t pages_peak;          /* the most pages held at once                 */
    int32_t lanes_busy_peak;     /* the most lanes busy at once                 */
    size_t arena_bytes;          /* device bytes the server holds               */
} ccd_server_stats;

/* Creates a server (config may be NULL: all defaults).  CCD_ERR_WORKSPACE
 * when budget_bytes cannot hold the inbox, the lanes and two pages, or the
 * arena cannot be allocated. */
ccd_status ccd_batch_begin(const ccd_server_config *config, ccd_server **server);
/* Queues a request; *ticket identifies it in poll and cancel. */
ccd_status ccd_batch_submit(ccd_server *server, const ccd_request *request, int64_t *ticket);
/* Advances the batches in flight and reports up to cap finished requests
 * (tickets in done[], their status -- CCD_OK, CCD_ERR_CANCELLED or an error
 * -- in status[] if not NULL; *ndone of them).  With wait_us > 0 it waits,
 * bounded by wait_us, until at least one is reported. */
ccd_status ccd_batch_poll(ccd_server *server, int64_t *done, int32_t *status, int32_t cap,
                          int32_t *ndone, int32_t wait_us);
/* Cancels a waiting request (reported by a later poll as CCD_ERR_CANCELLED);
 * CCD_ERR_BUSY if it already runs (its results will come), CCD_ERR_ARG if the
 * ticket is unknown or reported. */
ccd_status ccd_batch_cancel(ccd_server *server, int64_t ticket);
ccd_status ccd_batch_stats(ccd_server *server, ccd_server_stats *stats);
/* Waits for the device, then frees everything the server holds. */
ccd_status ccd_batch_end(ccd_server *server);

/* Static description of a status code. */
const char *ccd_status_str(int status);

/*
 * FP64 pipe throughput probe used for the roofline denominator: runs
 * `blocks` x 256 threads of independent fma.rn.f64 chains for `iters`
 * iterations and writes the elapsed device milliseconds to *ms_out.
 * Synchronizes `stream`.  The number of FP64 operations issued is
 * blocks * 256 * iters * 8.
 */
ccd_status ccd_fp64_peak_probe(int blocks, int iters, float *ms_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CCD_GB300_H */
