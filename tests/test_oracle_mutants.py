"""The oracle's pins catch plausible mistakes: each case plants one bug in a
copy of the oracle's C source (on the CPU), builds it, and runs the pin suite
(tests/test_oracle.py) against the copy, which must fail. A dropped term, a
wrong sign, index or rounding direction, a transposed operand each break at
least one pin."""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ivb_oracle.c")

# (name, exact text in the oracle, replacement)
MUTANTS = [
    ("mvf drops the last dimension",
     "        for (int i = 0; i < n; ++i) {\n            iv dx = {sub_dn(w->X[i].lo, w->c[i]), sub_up(w->X[i].hi, w->c[i])};",
     "        for (int i = 0; i < n - 1; ++i) {\n            iv dx = {sub_dn(w->X[i].lo, w->c[i]), sub_up(w->X[i].hi, w->c[i])};"),
    ("addition rounds its lower end upward",
     "static iv iv_add(iv x, iv y) { iv r = {add_dn(x.lo, y.lo), add_up(x.hi, y.hi)}; return r; }",
     "static iv iv_add(iv x, iv y) { iv r = {add_up(x.lo, y.lo), add_up(x.hi, y.hi)}; return r; }"),
    ("subtraction pairs the wrong endpoints",
     "static iv iv_sub(iv x, iv y) { iv r = {sub_dn(x.lo, y.hi), sub_up(x.hi, y.lo)}; return r; }",
     "static iv iv_sub(iv x, iv y) { iv r = {sub_dn(x.lo, y.lo), sub_up(x.hi, y.hi)}; return r; }"),
    ("adjoint of a difference adds instead of subtracting",
     "case OP_SUB: A[a] = iv_add(A[a], w); A[b] = iv_sub(A[b], w); break;",
     "case OP_SUB: A[a] = iv_add(A[a], w); A[b] = iv_add(A[b], w); break;"),
    ("adjoint of a product uses the wrong operand",
     "            A[a] = iv_fma(w, V[b], A[a]);",
     "            A[a] = iv_fma(w, V[a], A[a]);"),
    ("tangent of a product drops a term",
     "for (int d = 0; d < n; ++d) Dt[d] = iv_fma(V[a], Db[d], iv_mul(Da[d], V[b]));",
     "for (int d = 0; d < n; ++d) Dt[d] = iv_mul(Da[d], V[b]);"),
    ("tangent of a quotient transposes an operand",
     "for (int d = 0; d < n; ++d) Dt[d] = iv_mul(iv_fma(iv_neg(V[t]), Db[d], Da[d]), R);",
     "for (int d = 0; d < n; ++d) Dt[d] = iv_mul(iv_fma(iv_neg(V[t]), Da[d], Da[d]), R);"),
    ("fused accumulation rounds its lower end upward",
     "static double fprod_dn(double x, double y, double z) { return (x == 0.0 || y == 0.0) ? add_dn(z, 0.0) : fma_dn(x, y, z); }",
     "static double fprod_dn(double x, double y, double z) { return (x == 0.0 || y == 0.0) ? add_dn(z, 0.0) : fma_up(x, y, z); }"),
    ("fused accumulation drops an endpoint product",
     "    r.lo = minnn(minnn(fprod_dn(x.lo, y.lo, acc.lo), fprod_dn(x.lo, y.hi, acc.lo)),",
     "    r.lo = minnn(minnn(fprod_dn(x.lo, y.lo, acc.lo), fprod_dn(x.lo, y.lo, acc.lo)),"),
    ("adjoint of a quotient keeps the sign of its second operand",
     "            A[b] = iv_fma(iv_neg(iv_mul(w, V[t])), R, A[b]);",
     "            A[b] = iv_fma(iv_mul(w, V[t]), R, A[b]);"),
    ("square drops the factor two in its derivative",
     "            R = iv_twice(V[a]);\n            for (int d = 0; d < n; ++d) Dt[d] = iv_mul(R, Da[d]);",
     "            R = V[a];\n            for (int d = 0; d < n; ++d) Dt[d] = iv_mul(R, Da[d]);"),
    ("decode makes the last dimension fastest",
     "    for (int i = 0; i < n; ++i) {\n        const int64_t N = splits[i];",
     "    for (int ii = 0, i = n - 1; ii < n; ++ii, --i) {\n        const int64_t N = splits[i];"),
    ("parity bracket of exp widens one step too few",
     "r = q_to_dn(q - q * Q_EPS); if (tight > 1) r = step_dn(r, tight - 1); }",
     "r = q_to_dn(q - q * Q_EPS); if (tight > 1) r = step_dn(r, tight - 2); }"),
    ("parity bracket of log moves its upper end inward",
     "        return tight > 1 ? step_up(r, tight - 1) : r;\n    }\n    return step_up(log(x), 2);",
     "        return tight > 1 ? step_dn(r, tight - 1) : r;\n    }\n    return step_up(log(x), 2);"),
    ("subdomain endpoint off by one",
     "    double e = lo + (double)j * h;",
     "    double e = lo + (double)(j + 1) * h;"),
    ("centre taken at the lower end",
     "        c[i] = (X[i].lo + X[i].hi) * 0.5;",
     "        c[i] = X[i].lo;"),
    ("refinement takes the maximum of the lower ends",
     "                        if (F[q].lo < lmin[q]) lmin[q] = F[q].lo;",
     "                        if (F[q].lo > lmin[q] || lmin[q] == INFINITY) lmin[q] = F[q].lo;"),
    ("inequality feasibility tests the upper end",
     "            if (out_kind[q] == KIND_INEQ && minlo[q] > 0.0) inf = 1;",
     "            if (out_kind[q] == KIND_INEQ && maxhi[q] > 0.0) inf = 1;"),
    ("tight exp widens its lower end the wrong way",
     "    if (tight) { qreal q = Q_EXP((qreal)x); r = q_to_dn(q - q * Q_EPS); if (tight > 1)",
     "    if (tight) { qreal q = Q_EXP((qreal)x); r = q_to_up(q + q * Q_EPS); if (tight > 1)"),
    ("square root rounds its lower end upward",
     "static double sqrt_dn(double x) {\n    volatile double vx = x, r;\n    fesetround(FE_DOWNWARD);",
     "static double sqrt_dn(double x) {\n    volatile double vx = x, r;\n    fesetround(FE_UPWARD);"),
    ("products lose the 0 * inf = 0 rule",
     "static double prod_dn(double x, double y) { return (x == 0.0 || y == 0.0) ? 0.0 : mul_dn(x, y); }",
     "static double prod_dn(double x, double y) { return mul_dn(x, y); }"),
    ("square of a straddling interval keeps a positive lower end",
     "    else { r.lo = 0.0; r.hi = max2(prod_up(x.lo, x.lo), prod_up(x.hi, x.hi)); }",
     "    else { r.lo = min2(prod_dn(x.lo, x.lo), prod_dn(x.hi, x.hi)); r.hi = max2(prod_up(x.lo, x.lo), prod_up(x.hi, x.hi)); }"),
    ("propagation projects a difference onto its subtrahend with the wrong sign",
     "case OP_SUB: ok = meet_iv(&V[a], iv_add(z, V[b])) && meet_iv(&V[b], iv_sub(V[a], z)); break;",
     "case OP_SUB: ok = meet_iv(&V[a], iv_add(z, V[b])) && meet_iv(&V[b], iv_sub(z, V[a])); break;"),
    ("propagation of a square keeps only the nonnegative root",
     "else { r.lo = -r_hi; r.hi = r_hi; }",
     "else { r.lo = r_lo; r.hi = r_hi; }"),
    ("propagation cuts the objective at the wrong side",
     "else if (ub < INFINITY) { iv f = {-INFINITY, ub}; ok = meet_iv(z, f); }",
     "else if (ub < INFINITY) { iv f = {ub, INFINITY}; ok = meet_iv(z, f); }"),
    ("propagation of a product multiplies instead of dividing",
     "if (!straddles0(V[b])) ok = meet_iv(&V[a], iv_div(z, V[b]));",
     "if (!straddles0(V[b])) ok = meet_iv(&V[a], iv_mul(z, V[b]));"),
    ("propagation through a square root forgets to square",
     "iv r = {z.lo > 0.0 ? prod_dn(z.lo, z.lo) : -INFINITY, prod_up(z.hi, z.hi)};",
     "iv r = {z.lo > 0.0 ? z.lo : -INFINITY, z.hi};"),
    ("propagation through exp applies exp instead of log",
     "iv r = {z.lo > 0.0 ? log_dn(z.lo, tight) : -INFINITY, log_up(z.hi, tight)};",
     "iv r = {exp_dn(z.lo, tight), exp_up(z.hi, tight)};"),
    ("adaptive partitioning grows the narrowest dimension",
     "                double v = rw[i] / out[i];\n                if (v > bestv) { bestv = v; best = i; }",
     "                double v = 1.0 / (rw[i] / out[i] + 1e-300);\n                if (v > bestv) { bestv = v; best = i; }"),
]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(source, name, old, new):
    assert source.count(old) == 1, f"mutation site not found once: {name}"
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "mutant.c")
        with open(src, "w") as fh:
            fh.write(source.replace(old, new))
        so = oracle.compile_source(src, os.path.join(tmp, "libmutant.so"))
        env = dict(os.environ, IVB_ORACLE_SO=so, OMP_NUM_THREADS="4")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"no pin failed with the planted mistake: {name}"
