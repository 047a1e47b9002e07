/*
 * ccd_oracle.c -- plain, slow, single-query CPU oracle for the inclusion-based
 * CCD root finder of Wang et al., "A Large Scale Benchmark and an
 * Inclusion-Based Algorithm for Continuous Collision Detection" (Sec. 4,
 * Algorithm 2; minimum separation: Sec. 5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU library never
 * links, includes or calls it, and it shares no code with the GPU library.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 * (no FMA contraction: every + - * below is one IEEE double operation,
 * rounded to nearest, in the order written).
 *
 * Query layout: 24 doubles, index = time*12 + point*3 + coord, i.e. the four
 * points at t0 followed by the four points at t1 (Appendix A ordering).
 * Vertex-face (VF): points (p, v1, v2, v3).  Edge-edge (EE): (p1, p2, p3, p4).
 *
 * Readings of the paper taken here (each listed in the design notes):
 *  - Box order: Q is ordered by (level, left end of I_t); ties keep insertion
 *    order (a stable sort), children inserted left then right.
 *  - A colliding box that meets the termination test but is not the first
 *    colliding box of its level is split like a too-large box (the literal
 *    Algorithm 2 drops it; flag ORACLE_LITERAL_DROP restores that).
 *  - The returned tolerance is the co-domain width w(B) of the box checked
 *    when the algorithm returns; no collision returns (inf, 0).
 *  - w(B) and the box-inside test use the un-enlarged width / enlarged box.
 *  - A split whose dimension already has width 2^-53 is not made: the query
 *    returns as at the check limit (keeps every endpoint an exact double).
 *  - F is evaluated with the fixed expression in corner_F below.
 *  - SolveMSCCD's shortened time interval [0, t_max] (Sec. 6, line search)
 *    is solved in s in [0,1]^3 with t = t_max * s rounded once: interval
 *    endpoints stay exact dyadics in s, and kappa_t is taken over the
 *    corners t = 0 and t = t_max.  t_max = 1 is the plain solver.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_LITERAL_DROP 1
#define ORACLE_VF 0

/* Sec. 3, "Multivariate CCD Formulation": linear trajectory
 * p(t) = (1-t) p^0 + t p^1, evaluated as p^0 + (p^1 - p^0) t with one
 * rounding for the product and sum: fma(p^1 - p^0, t, p^0). */
static double traj(const double *q, int point, int c, double t)
{
    double x0 = q[point * 3 + c];
    double x1 = q[12 + point * 3 + c];
    double d = x1 - x0;
    return fma(d, t, x0);
}

/* Eq. (F-vf) and Eq. (F-ee), written in a fixed operation order (fma is
 * the correctly rounded fused multiply-add of C99):
 *   VF: q = p - v1, e1 = v2 - v1, e2 = v3 - v1;
 *       F = fma(-v, e2, fma(-u, e1, q))   (= p - ((1-u-v) v1 + u v2 + v v3))
 *   EE: d1 = p2 - p1, d2 = p4 - p3;
 *       F = fma(u, d1, p1 - fma(v, d2, p3))
 *                                  (= ((1-u) p1 + u p2) - ((1-v) p3 + v p4))
 * All positions are taken at time t first. */
void oracle_corner(int kind, const double *q, double t, double u, double v,
                   double F[3])
{
    for (int c = 0; c < 3; ++c) {
        double a = traj(q, 0, c, t);
        double b = traj(q, 1, c, t);
        double e = traj(q, 2, c, t);
        double f = traj(q, 3, c, t);
        if (kind == 0) {
            double qq = a - b;   /* p - v1  */
            double e1 = e - b;   /* v2 - v1 */
            double e2 = f - b;   /* v3 - v1 */
            F[c] = fma(-v, e2, fma(-u, e1, qq));
        } else {
            double d1 = b - a;   /* p2 - p1 */
            double d2 = f - e;   /* p4 - p3 */
            F[c] = fma(u, d1, a - fma(v, d2, e));
        }
    }
}

/* Eq. (box): B_F(I) is the axis-aligned box of F at the 8 corners of I;
 * I[0..1] are s-values, the corner times are t_max * s. */
void oracle_box_t(int kind, const double *q, const double I[6], double t_max,
                  double m[3], double M[3])
{
    int first = 1;
    for (int it = 0; it < 2; ++it)
        for (int iu = 0; iu < 2; ++iu)
            for (int iv = 0; iv < 2; ++iv) {
                double F[3];
                oracle_corner(kind, q, t_max * I[it], I[2 + iu], I[4 + iv], F);
                for (int c = 0; c < 3; ++c) {
                    if (first || F[c] < m[c]) m[c] = F[c];
                    if (first || F[c] > M[c]) M[c] = F[c];
                }
                first = 0;
            }
}

void oracle_box(int kind, const double *q, const double I[6], double m[3],
                double M[3])
{
    oracle_box_t(kind, q, I, 1.0, m, M);
}

/* Eq. (kappas): kappa_t = 3 max_{u,v in {0,1}} ||F(0,u,v) - F(t_max,u,v)||_inf,
 * and likewise along u and v, over the corners of the domain
 * [0,t_max] x [0,1]^2 (t_max = 1: the paper's [0,1]^3). */
void oracle_kappa_t(int kind, const double *q, double t_max, double kappa[3])
{
    double F[2][2][2][3];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c)
                oracle_corner(kind, q, t_max * (double)a, (double)b, (double)c, F[a][b][c]);
    double kt = 0.0, ku = 0.0, kv = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int c = 0; c < 3; ++c) {
                double dt = fabs(F[0][i][j][c] - F[1][i][j][c]);
                double du = fabs(F[i][0][j][c] - F[i][1][j][c]);
                double dv = fabs(F[i][j][0][c] - F[i][j][1][c]);
                if (dt > kt) kt = dt;
                if (du > ku) ku = du;
                if (dv > kv) kv = dv;
            }
    kappa[0] = 3.0 * kt;
    kappa[1] = 3.0 * ku;
    kappa[2] = 3.0 * kv;
}

void oracle_kappa(int kind, const double *q, double kappa[3])
{
    oracle_kappa_t(kind, q, 1.0, kappa);
}

/* Eq. (ccd-error) and Eq. (msccd-error): eps^c = K gamma_c^3 with
 * gamma_c = max(max_i |x_i^c|, 1).  The four constants are the paper's. */
static const double K_VF = 6.661338147750939e-15;
static const double K_EE = 6.217248937900877e-15;
static const double K_VF_MS = 7.549516567451064e-15;
static const double K_EE_MS = 7.105427357601002e-15;

double oracle_filter_constant(int kind, int ms_nonzero)
{
    if (kind == 0) return ms_nonzero ? K_VF_MS : K_VF;
    return ms_nonzero ? K_EE_MS : K_EE;
}

/* Sec. 6: the tolerances may be taken over a whole scene.  per_query != 0
 * gives one eps triple per query (n x 3), else one triple over all points. */
void oracle_err_from_bounds(int kind, const double *verts, long long n,
                            int ms_nonzero, int per_query, double *err_out)
{
    double K = oracle_filter_constant(kind, ms_nonzero);
    double g[3] = {1.0, 1.0, 1.0};
    for (long long i = 0; i < n; ++i) {
        const double *q = verts + 24 * i;
        if (per_query) g[0] = g[1] = g[2] = 1.0;
        for (int k = 0; k < 8; ++k)
            for (int c = 0; c < 3; ++c) {
                double a = fabs(q[k * 3 + c]);
                if (a > g[c]) g[c] = a;
            }
        if (per_query)
            for (int c = 0; c < 3; ++c)
                err_out[3 * i + c] = K * ((g[c] * g[c]) * g[c]);
    }
    if (!per_query)
        for (int c = 0; c < 3; ++c)
            err_out[c] = K * ((g[c] * g[c]) * g[c]);
}

/* ---- the priority queue Q of Algorithm 2 -------------------------------- */

typedef struct {
    int level;
    unsigned long long seq; /* insertion counter: stable order among ties */
    double I[6];            /* tL, tR, uL, uR, vL, vR */
} entry;

typedef struct {
    entry *a;
    long long size, cap;
    unsigned long long next_seq;
} heap;

/* order(): level first, then the left end of I_t, then insertion order. */
static int before(const entry *x, const entry *y)
{
    if (x->level != y->level) return x->level < y->level;
    if (x->I[0] != y->I[0]) return x->I[0] < y->I[0];
    return x->seq < y->seq;
}

static int heap_push(heap *h, int level, const double I[6])
{
    if (h->size == h->cap) {
        long long nc = h->cap ? 2 * h->cap : 64;
        entry *na = (entry *)realloc(h->a, (size_t)nc * sizeof(entry));
        if (!na) return -1;
        h->a = na;
        h->cap = nc;
    }
    entry e;
    e.level = level;
    e.seq = h->next_seq++;
    memcpy(e.I, I, sizeof(e.I));
    long long i = h->size++;
    while (i > 0) {
        long long p = (i - 1) / 2;
        if (!before(&e, &h->a[p])) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i] = e;
    return 0;
}

static entry heap_pop(heap *h)
{
    entry top = h->a[0];
    entry last = h->a[--h->size];
    long long i = 0;
    for (;;) {
        long long l = 2 * i + 1, r = l + 1, s = i;
        const entry *best = &last;
        if (l < h->size && before(&h->a[l], best)) { s = l; best = &h->a[l]; }
        if (r < h->size && before(&h->a[r], best)) { s = r; best = &h->a[r]; }
        if (s == i) break;
        h->a[i] = h->a[s];
        i = s;
    }
    if (h->size > 0) h->a[i] = last;
    return top;
}

/* ---- Algorithm 2 (with the minimum-separation change of Sec. 5.1) -------- */

/* Returns 1 (collision) or 0; -1 if memory for Q could not be obtained.
 * toi: left end of the recorded first colliding t-interval, or +inf.
 * out_tol: w(B) of the box checked at return, or 0.  checks: n. */
int oracle_ccd_t(int kind, const double *q, const double err[3], double ms,
                 double delta, long long max_itr, double t_max, int flags,
                 double *toi, double *out_tol, long long *checks)
{
    double kappa[3];
    oracle_kappa_t(kind, q, t_max, kappa);

    heap Q = {0};
    const double root[6] = {0.0, 1.0, 0.0, 1.0, 0.0, 1.0};
    if (heap_push(&Q, 0, root)) return -1;

    long long n = 0;
    int lp = -1;
    double If_left = 0.0;
    int result = 0;
    double r_toi = INFINITY, r_tol = 0.0;

    while (Q.size > 0) {
        entry e = heap_pop(&Q);
        const double *I = e.I;
        double m[3], M[3];
        oracle_box_t(kind, q, I, t_max, m, M);
        n += 1;

        /* B intersects C_eps: every axis interval, moved out by ms, meets
         * [-eps, eps]. */
        int hit = 1;
        for (int c = 0; c < 3; ++c)
            if (!((m[c] - ms) <= err[c] && (M[c] + ms) >= -err[c])) hit = 0;
        if (!hit) continue;

        int first = (e.level != lp);
        if (first) If_left = I[0];

        double wB = 0.0;
        for (int c = 0; c < 3; ++c) {
            double w = M[c] - m[c];
            if (w > wB) wB = w;
        }

        if (n >= max_itr) {
            result = 1; r_toi = If_left; r_tol = wB;
            break;
        }

        int inside = 1;
        for (int c = 0; c < 3; ++c)
            if (!((m[c] - ms) >= -err[c] && (M[c] + ms) <= err[c])) inside = 0;

        if (wB < delta || inside) {
            if (first) {
                result = 1; r_toi = If_left; r_tol = wB;
                break;
            }
            if (flags & ORACLE_LITERAL_DROP) {
                lp = e.level;
                continue;
            }
        }

        /* split(): c_d = w(I_d) kappa_d, widest estimated co-domain extent,
         * ties resolved t, then u, then v. */
        double ct = (I[1] - I[0]) * kappa[0];
        double cu = (I[3] - I[2]) * kappa[1];
        double cv = (I[5] - I[4]) * kappa[2];
        double cmax = ct;
        if (cu > cmax) cmax = cu;
        if (cv > cmax) cmax = cv;
        int dim = (ct == cmax) ? 0 : (cu == cmax) ? 1 : 2;

        double L = I[2 * dim], R = I[2 * dim + 1];
        if (R - L <= 0x1p-53) { /* depth guard */
            result = 1; r_toi = If_left; r_tol = wB;
            break;
        }
        double mid = (L + R) / 2.0;
        double I1[6], I2[6];
        memcpy(I1, I, sizeof(I1));
        memcpy(I2, I, sizeof(I2));
        I1[2 * dim + 1] = mid;
        I2[2 * dim] = mid;

        /* VF: keep a child only if it meets the prism u, v >= 0, u + v <= 1,
         * i.e. uL + vL <= 1 (tested as uL <= 1 - vL, exact for these
         * dyadic endpoints). */
        int keep1 = 1, keep2 = 1;
        if (kind == 0) {
            keep1 = I1[2] <= 1.0 - I1[4];
            keep2 = I2[2] <= 1.0 - I2[4];
        }
        if (keep1 && heap_push(&Q, e.level + 1, I1)) { result = -1; break; }
        if (keep2 && heap_push(&Q, e.level + 1, I2)) { result = -1; break; }
        lp = e.level;
    }
    free(Q.a);
    if (result == 1) r_toi = t_max * r_toi;   /* s -> t */
    if (toi) *toi = r_toi;
    if (out_tol) *out_tol = r_tol;
    if (checks) *checks = n;
    return result;
}

int oracle_ccd(int kind, const double *q, const double err[3], double ms,
               double delta, long long max_itr, int flags, double *toi,
               double *out_tol, long long *checks)
{
    return oracle_ccd_t(kind, q, err, ms, delta, max_itr, 1.0, flags, toi, out_tol, checks);
}

/* Batch driver: one oracle_ccd per query (queries are independent; OpenMP
 * only spreads whole queries over host threads). verts: n x 24 doubles;
 * err: 3 doubles (err_stride 0) or n x 3 (err_stride 3).  Returns the number
 * of queries whose Q could not be allocated (their result is left as a
 * conservative collision at t = 0). */
long long oracle_ccd_batch_t(int kind, const double *verts, long long n,
                             const double *err, int err_stride, double ms,
                             double delta, long long max_itr, double t_max, int flags,
                             unsigned char *collides, double *toi,
                             double *out_tol, long long *checks, int nthreads)
{
    long long failures = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads) reduction(+ : failures)
    for (long long i = 0; i < n; ++i) {
        double t, w;
        long long c;
        int r = oracle_ccd_t(kind, verts + 24 * i, err + (long long)err_stride * i,
                             ms, delta, max_itr, t_max, flags, &t, &w, &c);
        if (r < 0) {
            failures += 1;
            r = 1; t = 0.0; w = INFINITY;
        }
        collides[i] = (unsigned char)r;
        toi[i] = t;
        out_tol[i] = w;
        if (checks) checks[i] = c;
    }
    return failures;
}

long long oracle_ccd_batch(int kind, const double *verts, long long n,
                           const double *err, int err_stride, double ms,
                           double delta, long long max_itr, int flags,
                           unsigned char *collides, double *toi,
                           double *out_tol, long long *checks, int nthreads)
{
    return oracle_ccd_batch_t(kind, verts, n, err, err_stride, ms, delta, max_itr, 1.0,
                              flags, collides, toi, out_tol, checks, nthreads);
}

/* ---- L-infinity distance at t = 0 (Sec. 5.1 norm; Algorithm 4's d_i) -------
 *
 * f(u,v) = F(0,u,v) = A + u B + v C with, per axis c, one rounded
 * subtraction of t = 0 coordinates:
 *   VF: A = p - v1, B = v1 - v2, C = v1 - v3   (F = (q - u e1) - v e2)
 *   EE: A = p1 - p3, B = p2 - p1, C = p3 - p4  (F = (p1 + u d1) - (p3 + v d2))
 * The distance is min over the domain (VF: u, v >= 0, u + v <= 1; EE:
 * [0,1]^2) of g(u,v) = max_c |(A_c + u B_c) + v C_c|.  That is a linear
 * program in (u, v, s) whose minimum lies at a vertex of its feasible set,
 * and every vertex is one of:
 *   - a corner of the domain;
 *   - a point of a domain edge where two of the six lines +-f_c cross
 *     (f_c = 0, or f_c1 = +-f_c2);
 *   - an interior point where f_c1 = f_c2 = 0, or s1 f_1 = s2 f_2 = s3 f_3
 *     for a sign pattern s (four patterns up to a global sign).
 * g is evaluated at each such candidate that lies in the domain and the
 * minimum is returned.  Candidate points carry rounding, so the result is
 * the distance up to the rounding of these few operations. */
static double linf_g(const double A[3], const double B[3], const double C[3], double u, double v)
{
    double g = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double f = fabs((A[c] + u * B[c]) + v * C[c]);
        if (f > g) g = f;
    }
    return g;
}

static int in_domain(int kind, double u, double v)
{
    if (!(u >= 0.0 && v >= 0.0)) return 0;
    if (kind == ORACLE_VF) return u + v <= 1.0;
    return u <= 1.0 && v <= 1.0;
}

double oracle_linf_distance(int kind, const double *q)
{
    double A[3], B[3], C[3];
    for (int c = 0; c < 3; ++c) {
        const double x0 = q[c], x1 = q[3 + c], x2 = q[6 + c], x3 = q[9 + c];
        if (kind == ORACLE_VF) {
            A[c] = x0 - x1; B[c] = x1 - x2; C[c] = x1 - x3;
        } else {
            A[c] = x0 - x2; B[c] = x1 - x0; C[c] = x2 - x3;
        }
    }
    double best = INFINITY, g;
    /* domain corners */
    const double cu[4] = {0.0, 1.0, 0.0, 1.0}, cv[4] = {0.0, 0.0, 1.0, 1.0};
    const int ncorner = kind == ORACLE_VF ? 3 : 4;
    for (int i = 0; i < ncorner; ++i) {
        g = linf_g(A, B, C, cu[i], cv[i]);
        if (g < best) best = g;
    }
    /* domain edges (u, v) = P + tau D, tau in [0, 1]:
     * VF: v = 0, u = 0, u + v = 1;  EE: v = 0, u = 0, u = 1, v = 1 */
    const double vf_P[3][2] = {{0, 0}, {0, 0}, {1, 0}}, vf_D[3][2] = {{1, 0}, {0, 1}, {-1, 1}};
    const double ee_P[4][2] = {{0, 0}, {0, 0}, {1, 0}, {0, 1}};
    const double ee_D[4][2] = {{1, 0}, {0, 1}, {0, 1}, {1, 0}};
    const int nedge = kind == ORACLE_VF ? 3 : 4;
    for (int e = 0; e < nedge; ++e) {
        const double pu = kind == ORACLE_VF ? vf_P[e][0] : ee_P[e][0];
        const double pv = kind == ORACLE_VF ? vf_P[e][1] : ee_P[e][1];
        const double du = kind == ORACLE_VF ? vf_D[e][0] : ee_D[e][0];
        const double dv = kind == ORACLE_VF ? vf_D[e][1] : ee_D[e][1];
        double al[3], be[3];
        for (int c = 0; c < 3; ++c) {
            al[c] = (A[c] + pu * B[c]) + pv * C[c];
            be[c] = du * B[c] + dv * C[c];
        }
        double tau[9];
        int nt = 0;
        for (int c = 0; c < 3; ++c)
            if (be[c] != 0.0) tau[nt++] = -al[c] / be[c];
        for (int c1 = 0; c1 < 3; ++c1)
            for (int c2 = c1 + 1; c2 < 3; ++c2)
                for (int s = 0; s < 2; ++s) {
                    const double sg = s ? -1.0 : 1.0;
                    const double den = be[c1] - sg * be[c2];
                    if (den != 0.0) tau[nt++] = (sg * al[c2] - al[c1]) / den;
                }
        for (int i = 0; i < nt; ++i) {
            const double t = tau[i];
            if (!(t >= 0.0 && t <= 1.0)) continue;
            g = linf_g(A, B, C, pu + t * du, pv + t * dv);
            if (g < best) best = g;
        }
    }
    /* interior: two axes zero */
    for (int c1 = 0; c1 < 3; ++c1)
        for (int c2 = c1 + 1; c2 < 3; ++c2) {
            const double det = B[c1] * C[c2] - C[c1] * B[c2];
            if (det == 0.0) continue;
            const double u = (C[c1] * A[c2] - A[c1] * C[c2]) / det;
            const double v = (A[c1] * B[c2] - B[c1] * A[c2]) / det;
            if (!in_domain(kind, u, v)) continue;
            g = linf_g(A, B, C, u, v);
            if (g < best) best = g;
        }
    /* interior: s1 f_1 = s2 f_2 = s3 f_3 */
    const double sgn[4][3] = {{1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {-1, 1, 1}};
    for (int k = 0; k < 4; ++k) {
        const double s1 = sgn[k][0], s2 = sgn[k][1], s3 = sgn[k][2];
        const double a11 = s1 * B[0] - s2 * B[1], a12 = s1 * C[0] - s2 * C[1];
        const double b1 = s2 * A[1] - s1 * A[0];
        const double a21 = s2 * B[1] - s3 * B[2], a22 = s2 * C[1] - s3 * C[2];
        const double b2 = s3 * A[2] - s2 * A[1];
        const double det = a11 * a22 - a12 * a21;
        if (det == 0.0) continue;
        const double u = (b1 * a22 - a12 * b2) / det;
        const double v = (a11 * b2 - b1 * a21) / det;
        if (!in_domain(kind, u, v)) continue;
        g = linf_g(A, B, C, u, v);
        if (g < best) best = g;
    }
    return best;
}

void oracle_linf_distance_batch(int kind, const double *verts, long long n, double *out,
                                int nthreads)
{
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (long long i = 0; i < n; ++i) out[i] = oracle_linf_distance(kind, verts + 24 * i);
}
