"""The oracle's pins are not circular: each plausible mistake planted in a
copy of the oracle makes the pin suite fail.

Every mutant below is a one-spot edit (a dropped term, a wrong sign or
index, a swapped comparison or constant, a wrong tie order ...) of
``oracle/ccd_oracle.c`` or of one of the oracle's Python modules (the active
set of Algorithm 3, the line-search step of Algorithm 4).  A C mutant is
built into its own library and the CPU pin files run against it
(``CCD_ORACLE_LIB``); a Python mutant goes into a copy of the ``oracle``
package in a scratch directory, with copies of the pin files, and the pins
run there.  A mutant that passes them all would be a mistake the pins cannot
see.  An unmodified copy handled the same way must pass, which checks each
harness itself.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile


import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ccd_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_linesearch.py",
        "tests/test_oracle_activeset.py"]

MUTANTS = [
    ("VF corner drops the v e2 term",
     [("F[c] = fma(-v, e2, fma(-u, e1, qq));", "F[c] = fma(-u, e1, qq);")]),
    ("EE corner adds instead of subtracting",
     [("F[c] = fma(u, d1, a - fma(v, d2, e));", "F[c] = fma(u, d1, a + fma(v, d2, e));")]),
    ("VF e2 taken from the wrong vertex",
     [("double e2 = f - b;   /* v3 - v1 */", "double e2 = e - b;   /* v3 - v1 */")]),
    ("trajectory reversed in time",
     [("return fma(d, t, x0);", "return fma(d, 1.0 - t, x0);")]),
    ("box minimum keeps the maximum",
     [("if (first || F[c] < m[c]) m[c] = F[c];", "if (first || F[c] > m[c]) m[c] = F[c];")]),
    ("filter comparisons made strict",
     [("if (!((m[c] - ms) <= err[c] && (M[c] + ms) >= -err[c])) hit = 0;",
       "if (!((m[c] - ms) < err[c] && (M[c] + ms) > -err[c])) hit = 0;")]),
    ("minimum separation moves the box inward",
     [("if (!((m[c] - ms) <= err[c] && (M[c] + ms) >= -err[c])) hit = 0;",
       "if (!((m[c] + ms) <= err[c] && (M[c] - ms) >= -err[c])) hit = 0;")]),
    ("split ties resolved v, then u, then t",
     [("int dim = (ct == cmax) ? 0 : (cu == cmax) ? 1 : 2;",
       "int dim = (cv == cmax) ? 2 : (cu == cmax) ? 1 : 0;")]),
    ("prism cull strict",
     [("keep1 = I1[2] <= 1.0 - I1[4];", "keep1 = I1[2] < 1.0 - I1[4];"),
      ("keep2 = I2[2] <= 1.0 - I2[4];", "keep2 = I2[2] < 1.0 - I2[4];")]),
    ("check limit off by one", [("if (n >= max_itr) {", "if (n > max_itr) {")]),
    ("VF filter constant replaced by EE's",
     [("static const double K_VF = 6.661338147750939e-15;",
       "static const double K_VF = 6.217248937900877e-15;")]),
    ("time of impact from the right end", [("if (first) If_left = I[0];", "if (first) If_left = I[1];")]),
    ("only colliding boxes counted",
     [("        n += 1;\n", ""), ("        if (!hit) continue;\n", "        if (!hit) continue;\n        n += 1;\n")]),
    ("every terminating box returns", [("int first = (e.level != lp);", "int first = 1;")]),
    ("queue ordered by descending t",
     [("if (x->I[0] != y->I[0]) return x->I[0] < y->I[0];",
       "if (x->I[0] != y->I[0]) return x->I[0] > y->I[0];")]),
    ("shortened interval not scaled back to t",
     [("if (result == 1) r_toi = t_max * r_toi;", "if (result == 1) r_toi = r_toi;")]),
    ("distance skips the hypotenuse edge",
     [("const int nedge = kind == ORACLE_VF ? 3 : 4;", "const int nedge = kind == ORACLE_VF ? 2 : 4;")]),
    # (Flipping the sign of the distance's edge zero crossings is not in the
    # list: those candidates are implied by the pair crossings f_c1 = +-f_c2,
    # which meet at every point where all three f_c vanish, so that mutant
    # computes the same distance.)
    ("distance interior determinant with the wrong sign",
     [("const double det = a11 * a22 - a12 * a21;", "const double det = a11 * a22 + a12 * a21;")]),
    ("scene bound without the floor of 1",
     [("double g[3] = {1.0, 1.0, 1.0};", "double g[3] = {0.0, 0.0, 0.0};")]),
    ("kappa_u without its factor 3", [("kappa[1] = 3.0 * ku;", "kappa[1] = ku;")]),
    ("kappa_u measured along t",
     [("double du = fabs(F[i][0][j][c] - F[i][1][j][c]);",
       "double du = fabs(F[0][i][j][c] - F[1][i][j][c]);")]),
    ("per-query bound carried over from the previous query",
     [("        if (per_query) g[0] = g[1] = g[2] = 1.0;\n", "")]),
    ("termination ignores B inside C_eps",
     [("if (wB < delta || inside) {", "if (wB < delta) {")]),
    ("inside test on the un-enlarged box",
     [("if (!((m[c] - ms) >= -err[c] && (M[c] + ms) <= err[c])) inside = 0;",
       "if (!(m[c] >= -err[c] && M[c] <= err[c])) inside = 0;")]),
    ("inside test moves the box inward",
     [("if (!((m[c] - ms) >= -err[c] && (M[c] + ms) <= err[c])) inside = 0;",
       "if (!((m[c] + ms) >= -err[c] && (M[c] - ms) <= err[c])) inside = 0;")]),
    ("reached tolerance from the enlarged box",
     [("double w = M[c] - m[c];", "double w = (M[c] + ms) - (m[c] - ms);")]),
    ("depth guard removed", [("if (R - L <= 0x1p-53) { /* depth guard */", "if (0) {")]),
    ("scene eps with the bound squared",
     [("            err_out[c] = K * ((g[c] * g[c]) * g[c]);",
       "            err_out[c] = K * (g[c] * g[c]);")]),
]


def _build(tmp, name, subs):
    text = open(SRC).read()
    for old, new in subs:
        assert text.count(old) == 1, f"{name}: mutation site not unique: {old!r}"
        text = text.replace(old, new)
    src = os.path.join(tmp, f"{abs(hash(name))}.c")
    lib = src[:-2] + ".so"
    open(src, "w").write(text)
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", lib, src, "-lm"], check=True)
    return lib


def _run_pins(lib):
    env = dict(os.environ, CCD_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", *PINS], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    return r.returncode


# (module under oracle/, name, substitutions)
PY_MUTANTS = [
    ("activeset.py", "swept boxes overlap only strictly",
     [("return np.all((lo_a <= hi_b) & (lo_b <= hi_a), axis=-1)",
       "return np.all((lo_a < hi_b) & (lo_b < hi_a), axis=-1)")]),
    ("activeset.py", "a face's own vertices kept as candidates",
     [("        hit[faces[f]] = False\n", "")]),
    ("activeset.py", "margin added on one side only",
     [("return pts.min(axis=1) - r, pts.max(axis=1) + r", "return pts.min(axis=1), pts.max(axis=1) + r")]),
    ("activeset.py", "scene eps from the start positions only",
     [("g = np.maximum(1.0, np.abs(np.concatenate([x0, x1])).max(axis=0))",
       "g = np.maximum(1.0, np.abs(x0).max(axis=0))")]),
    ("linesearch.py", "d_i as the largest distance",
     [("d_i = min(d_i, float(linf_distance_batch(k, q, nthreads).min()))",
       "d_i = min(d_i, float(linf_distance_batch(k, q, nthreads).max()))")]),
    ("linesearch.py", "delta_i from the smallest tolerance",
     [("delta_i = max(delta_i, float(tol.max()))", "delta_i = max(delta_i, float(tol.min()))")]),
    ("linesearch.py", "alpha from the latest time of impact",
     [("alpha = min(alpha, float(toi.min()))",
       "alpha = min(alpha, float(np.where(np.isfinite(toi), toi, 0.0).max()))")]),
    ("linesearch.py", "cap min and max swapped",
     [('return min(x, delta) if cap == "min" else max(x, delta)',
       'return max(x, delta) if cap == "min" else min(x, delta)')]),
]
PY_PINS = ["tests/test_oracle_linesearch.py", "tests/test_oracle_activeset.py"]


def _py_tree(tmp, idx, module, subs):
    """A scratch copy of what the Python-side pins import, with one module of
    the oracle package mutated."""
    d = os.path.join(tmp, f"py{idx}")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    os.makedirs(os.path.join(d, "paper_2009_13349_gb300"))
    for f in ("__init__.py", "workloads.py"):
        shutil.copy(os.path.join(ROOT, "paper_2009_13349_gb300", f),
                    os.path.join(d, "paper_2009_13349_gb300", f))
    os.makedirs(os.path.join(d, "tests"))
    for f in ["tests/conftest.py", *PY_PINS]:
        shutil.copy(os.path.join(ROOT, f), os.path.join(d, f))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    if module:
        path = os.path.join(d, "oracle", module)
        text = open(path).read()
        for old, new in subs:
            assert text.count(old) == 1, f"{module}: mutation site not unique: {old!r}"
            text = text.replace(old, new)
        open(path, "w").write(text)
    return d


def _run_py_pins(args):
    d, lib = args
    env = dict(os.environ, CCD_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    env.pop("PYTHONPATH", None)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu", *PY_PINS], cwd=d, env=env, capture_output=True,
                       text=True, timeout=600)
    return r.returncode


def test_pins_kill_every_python_mutant():
    with tempfile.TemporaryDirectory() as tmp:
        lib = _build(tmp, "unmodified", [])
        jobs = [(None, "unmodified", [])] + PY_MUTANTS
        dirs = [_py_tree(tmp, i, m, subs) for i, (m, _, subs) in enumerate(jobs)]
        workers = max(1, min(len(jobs), (os.cpu_count() or 2)))
        with cf.ThreadPoolExecutor(workers) as ex:
            codes = list(ex.map(_run_py_pins, [(d, lib) for d in dirs]))
    assert codes[0] == 0, "the unmodified oracle copy must pass its pins"
    survivors = [name for (_, name, _), c in zip(jobs[1:], codes[1:]) if c == 0]
    assert not survivors, f"mutants not caught by any pin: {survivors}"


def test_pins_kill_every_mutant():
    with tempfile.TemporaryDirectory() as tmp:
        jobs = [("unmodified", [])] + MUTANTS
        libs = [_build(tmp, name, subs) for name, subs in jobs]
        workers = max(1, min(len(jobs), (os.cpu_count() or 2)))
        with cf.ThreadPoolExecutor(workers) as ex:
            codes = list(ex.map(_run_pins, libs))
    assert codes[0] == 0, "the unmodified oracle must pass its pins"
    survivors = [name for (name, _), c in zip(jobs[1:], codes[1:]) if c == 0]
    assert not survivors, f"mutants not caught by any pin: {survivors}"
