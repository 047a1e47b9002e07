"""The identity behind the solvers' two-fma corner range.

On one axis at one t the four corners of a box are fma(x, g, p) for x in
{x_lo, x_hi} (x_lo < x_hi, both of one sign: -v for VF, u for EE) and p in
{p0, p1} (the two shared partials).  The solvers take the minimum as
fma(x_min, g, min p) and the maximum as fma(x_max, g, max p), with x_min the
end that makes x g smallest (x_lo when g's sign bit is clear), instead of
evaluating all four corners.  This holds because rounding is monotone and
x g + p is monotone in each argument; it must also give the same signed zero
as the four-corner minimum / maximum in the solvers' key order (-0 before
+0).

The check runs in C with libm's correctly rounded fma() on random values,
values with wide exponent ranges, and edge values (signed zeros, subnormals,
exact cancellations), with the same key order as the solvers.  It restates
the selection rule independently of the CUDA source.
"""
import os
import subprocess
import tempfile

SRC = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

static int64_t key(double x) {            /* signed order = numeric order, -0 < +0 */
    int64_t b; memcpy(&b, &x, 8);
    return b ^ ((b >> 63) & INT64_MAX);
}
static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t rnd(void) { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; }
static double unit(void) { return (double)(rnd() >> 11) * 0x1p-53; }
static double dyad(int k) { return ldexp((double)(rnd() % ((1ull << k) + 1)), -k); }

static const double edge[] = {0.0, -0.0, 0x1p-1074, -0x1p-1074, 0x1p-1022, -0x1p-1022,
                              1.0, -1.0, 0.5, -0.5, 3.0, -3.0, 0x1p-60, -0x1p-60};

static double pick(int mode) {
    switch (mode) {
    case 0: return unit() * 2.0 - 1.0;
    case 1: return ldexp(unit() * 2.0 - 1.0, (int)(rnd() % 120) - 60);
    default: return edge[rnd() % (sizeof edge / sizeof edge[0])];
    }
}

/* returns the number of mismatches over n cases */
static long check(long n, int ee) {
    long bad = 0;
    for (long i = 0; i < n; ++i) {
        int k = 1 + (int)(rnd() % 40);
        double a = dyad(k), b = dyad(k);
        if (a == b) b = a + ldexp(1.0, -k);
        double lo = a < b ? a : b, hi = a < b ? b : a;          /* parameter interval */
        double x_lo = ee ? lo : -hi, x_hi = ee ? hi : -lo;      /* EE: u; VF: -v */
        int mode = (int)(rnd() % 3);
        double g = pick(mode), p0 = pick(mode), p1 = pick(mode);
        if (rnd() % 8 == 0) p1 = p0;                            /* equal partials */
        if (rnd() % 8 == 0) p1 = -fma(x_lo, g, 0.0);            /* exact cancellation */
        if (rnd() % 16 == 0) g = (rnd() & 1) ? 0.0 : -0.0;
        double f[4] = {fma(x_lo, g, p0), fma(x_hi, g, p0), fma(x_lo, g, p1), fma(x_hi, g, p1)};
        int64_t kmin = key(f[0]), kmax = kmin;
        for (int j = 1; j < 4; ++j) {
            int64_t kj = key(f[j]);
            if (kj < kmin) kmin = kj;
            if (kj > kmax) kmax = kj;
        }
        int sw = key(p1) < key(p0);
        double pmin = sw ? p1 : p0, pmax = sw ? p0 : p1;
        int neg = signbit(g) != 0;
        int64_t rmin = key(fma(neg ? x_hi : x_lo, g, pmin));
        int64_t rmax = key(fma(neg ? x_lo : x_hi, g, pmax));
        if (rmin != kmin || rmax != kmax) {
            if (bad < 5)
                printf("mismatch ee=%d x=[%a,%a] g=%a p=[%a,%a]\n", ee, x_lo, x_hi, g, p0, p1);
            ++bad;
        }
    }
    return bad;
}

int main(void) {
    long bad = check(2000000, 0) + check(2000000, 1);
    printf("%ld\n", bad);
    return bad != 0;
}
"""


def test_two_fma_corner_range_equals_four_corner_range():
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "cr.c")
        exe = os.path.join(tmp, "cr")
        with open(src, "w") as f:
            f.write(SRC)
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-o", exe, src, "-lm"], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout
    assert r.stdout.strip().splitlines()[-1] == "0"
