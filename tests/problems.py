"""Hand-written test problems (tapes with known closed-form answers) and an
independent high-precision point evaluator (mpmath) for pinning the oracle."""
from __future__ import annotations

import math

import numpy as np

from paper_2507_20769_gb300.workloads import (KIND_EQ, KIND_INEQ, KIND_OBJ, OP_ADD, OP_CONST, OP_DIV,
                                              OP_EXP, OP_LOG, OP_MUL, OP_NEG, OP_SQR, OP_SQRT, OP_SUB,
                                              OP_VAR, Tape)


class Builder:
    """tiny tape builder for hand-written expressions"""

    def __init__(self, n_vars: int):
        self.n = n_vars
        self.rows = [(OP_VAR, i, 0, 0.0) for i in range(n_vars)]
        self.outs = []

    def _add(self, op, a=0, b=0, c=0.0):
        self.rows.append((op, a, b, float(c)))
        return len(self.rows) - 1

    def x(self, i):
        return i

    def const(self, v):
        return self._add(OP_CONST, c=v)

    def add(self, a, b): return self._add(OP_ADD, a, b)
    def sub(self, a, b): return self._add(OP_SUB, a, b)
    def mul(self, a, b): return self._add(OP_MUL, a, b)
    def div(self, a, b): return self._add(OP_DIV, a, b)
    def sqr(self, a): return self._add(OP_SQR, a)
    def sqrt(self, a): return self._add(OP_SQRT, a)
    def exp(self, a): return self._add(OP_EXP, a)
    def log(self, a): return self._add(OP_LOG, a)
    def neg(self, a): return self._add(OP_NEG, a)

    def output(self, t, kind=KIND_OBJ):
        self.outs.append((t, kind))

    def tape(self, box, name=""):
        r = self.rows
        return Tape(n_vars=self.n,
                    op=np.array([x[0] for x in r], np.uint8), a=np.array([x[1] for x in r], np.int32),
                    b=np.array([x[2] for x in r], np.int32), c=np.array([x[3] for x in r], np.float64),
                    out_idx=np.array([o[0] for o in self.outs], np.int32),
                    out_kind=np.array([o[1] for o in self.outs], np.uint8),
                    root_box=np.asarray(box, np.float64).reshape(self.n, 2), name=name)


def cubic_fig5():
    """f(x) = 3x^3 + x^2 - 5x - 1 (Fig. 5)"""
    B = Builder(1)
    x = B.x(0)
    xx = B.mul(x, x)
    xxx = B.mul(xx, x)
    t = B.mul(B.const(3.0), xxx)
    t = B.add(t, B.sqr(x))
    t = B.sub(t, B.mul(B.const(5.0), x))
    t = B.sub(t, B.const(1.0))
    B.output(t)
    return B.tape([[-1.0, 2.0]], "cubic")


def cubic_range(lo, hi):
    """exact range of 3x^3 + x^2 - 5x - 1 on [lo, hi] (critical points of 9x^2+2x-5)"""
    f = lambda v: 3 * v ** 3 + v ** 2 - 5 * v - 1
    pts = [lo, hi] + [r for r in ((-1 + math.sqrt(46)) / 9, (-1 - math.sqrt(46)) / 9) if lo < r < hi]
    vals = [f(v) for v in pts]
    return min(vals), max(vals)


def shifted_squares(n, a, box):
    """sum_i (x_i - a_i)^2, minimum 0 at a"""
    B = Builder(n)
    acc = None
    for i in range(n):
        t = B.sqr(B.sub(B.x(i), B.const(a[i])))
        acc = t if acc is None else B.add(acc, t)
    B.output(acc)
    return B.tape(box, "shifted squares")


def separable_quartic(n, box):
    """sum_i (x_i^4 - 3 x_i^2 + x_i); per-dimension minimum at a root of 4x^3 - 6x + 1"""
    B = Builder(n)
    acc = None
    for i in range(n):
        x = B.x(i)
        s = B.sqr(x)
        t = B.add(B.sub(B.sqr(s), B.mul(B.const(3.0), s)), x)
        acc = t if acc is None else B.add(acc, t)
    B.output(acc)
    return B.tape(box, "separable quartic")


def quartic_min_1d(lo, hi):
    f = lambda v: v ** 4 - 3 * v ** 2 + v
    roots = [r.real for r in np.roots([4.0, 0.0, -6.0, 1.0]) if abs(r.imag) < 1e-12 and lo <= r.real <= hi]
    return min(f(v) for v in [lo, hi] + roots)


def peaks():
    """Peaks function of Section 4.1 on [-3,3]^2"""
    B = Builder(2)
    x1, x2 = B.x(0), B.x(1)
    one = B.const(1.0)
    # 3 (1 - x1)^2 exp(-x1^2 - (x2+1)^2)
    t1 = B.mul(B.const(3.0), B.sqr(B.sub(one, x1)))
    e1 = B.exp(B.sub(B.neg(B.sqr(x1)), B.sqr(B.add(x2, one))))
    term1 = B.mul(t1, e1)
    # 10 (x1/5 - x1^3 - x2^5) exp(-x1^2 - x2^2)
    x1c = B.mul(x1, B.sqr(x1))
    x2q = B.sqr(B.sqr(x2))
    x2f = B.mul(x2, x2q)
    inner = B.sub(B.sub(B.div(x1, B.const(5.0)), x1c), x2f)
    e2 = B.exp(B.sub(B.neg(B.sqr(x1)), B.sqr(x2)))
    term2 = B.mul(B.mul(B.const(10.0), inner), e2)
    # exp(-(x1+1)^2 - x2^2) / 3
    e3 = B.exp(B.sub(B.neg(B.sqr(B.add(x1, one))), B.sqr(x2)))
    term3 = B.div(e3, B.const(3.0))
    B.output(B.sub(B.sub(term1, term2), term3))
    return B.tape([[-3.0, 3.0], [-3.0, 3.0]], "peaks")


def peaks_np(x1, x2):
    return (3 * (1 - x1) ** 2 * np.exp(-x1 ** 2 - (x2 + 1) ** 2)
            - 10 * (x1 / 5 - x1 ** 3 - x2 ** 5) * np.exp(-x1 ** 2 - x2 ** 2)
            - np.exp(-(x1 + 1) ** 2 - x2 ** 2) / 3)


def constrained_toy(kind_g="feasible"):
    """min x0 + x1 on [-2,2]^2 with one constraint:
       feasible   : g = x0^2 + x1^2 - 1 <= 0
       infeasible : g = x0^2 + 1 <= 0 (never satisfied)
       eq_out     : h = x0 - 5 = 0 (no solution in the box)
       eq_in      : h = x0 - x1 = 0"""
    B = Builder(2)
    f = B.add(B.x(0), B.x(1))
    B.output(f, KIND_OBJ)
    if kind_g == "feasible":
        B.output(B.sub(B.add(B.sqr(B.x(0)), B.sqr(B.x(1))), B.const(1.0)), KIND_INEQ)
    elif kind_g == "infeasible":
        B.output(B.add(B.sqr(B.x(0)), B.const(1.0)), KIND_INEQ)
    elif kind_g == "eq_out":
        B.output(B.sub(B.x(0), B.const(5.0)), KIND_EQ)
    elif kind_g == "eq_in":
        B.output(B.sub(B.x(0), B.x(1)), KIND_EQ)
    return B.tape([[-2.0, 2.0], [-2.0, 2.0]], "constrained " + kind_g)


# ------------------------------------------------ independent evaluation

def mp_eval(tape, x, dps=60, grad=False):
    """Point values (and forward-mode gradients) of every output at x in mpmath
    with `dps` digits: an evaluation that shares nothing with the oracle."""
    import mpmath
    with mpmath.workdps(dps):
        n = tape.n_vars
        v, d = [], []
        xs = [mpmath.mpf(float(xi)) for xi in x]
        for t in range(tape.n_ops):
            op, a, b, c = int(tape.op[t]), int(tape.a[t]), int(tape.b[t]), float(tape.c[t])
            if op == OP_VAR:
                val, der = xs[a], [mpmath.mpf(1) if i == a else mpmath.mpf(0) for i in range(n)]
            elif op == OP_CONST:
                val, der = mpmath.mpf(c), [mpmath.mpf(0)] * n
            elif op == OP_ADD:
                val, der = v[a] + v[b], [p + q for p, q in zip(d[a], d[b])]
            elif op == OP_SUB:
                val, der = v[a] - v[b], [p - q for p, q in zip(d[a], d[b])]
            elif op == OP_MUL:
                val, der = v[a] * v[b], [p * v[b] + v[a] * q for p, q in zip(d[a], d[b])]
            elif op == OP_DIV:
                val = v[a] / v[b]
                der = [(p - val * q) / v[b] for p, q in zip(d[a], d[b])]
            elif op == OP_SQR:
                val, der = v[a] ** 2, [2 * v[a] * p for p in d[a]]
            elif op == OP_SQRT:
                val = mpmath.sqrt(v[a])
                der = [p / (2 * val) for p in d[a]]
            elif op == OP_EXP:
                val = mpmath.exp(v[a])
                der = [val * p for p in d[a]]
            elif op == OP_LOG:
                val, der = mpmath.log(v[a]), [p / v[a] for p in d[a]]
            elif op == OP_NEG:
                val, der = -v[a], [-p for p in d[a]]
            else:
                raise ValueError(op)
            v.append(val)
            d.append(der)
        f = [v[int(o)] for o in tape.out_idx]
        if grad:
            return f, [d[int(o)] for o in tape.out_idx]
        return f


def np_eval(tape, X):
    """vectorised float64 point values of every output at points X [m][n]"""
    X = np.asarray(X, dtype=np.float64)
    v = []
    with np.errstate(all="ignore"):
        for t in range(tape.n_ops):
            op, a, b, c = int(tape.op[t]), int(tape.a[t]), int(tape.b[t]), float(tape.c[t])
            if op == OP_VAR: r = X[:, a]
            elif op == OP_CONST: r = np.full(X.shape[0], c)
            elif op == OP_ADD: r = v[a] + v[b]
            elif op == OP_SUB: r = v[a] - v[b]
            elif op == OP_MUL: r = v[a] * v[b]
            elif op == OP_DIV: r = v[a] / v[b]
            elif op == OP_SQR: r = v[a] * v[a]
            elif op == OP_SQRT: r = np.sqrt(v[a])
            elif op == OP_EXP: r = np.exp(v[a])
            elif op == OP_LOG: r = np.log(v[a])
            elif op == OP_NEG: r = -v[a]
            v.append(r)
    return np.stack([v[int(o)] for o in tape.out_idx], axis=1)


def rational_tape_for_shards():
    """seeded rational problem with constraints (n=3, objective + 2
    inequalities of 50 entries) for the multi-rank host-path test"""
    from paper_2507_20769_gb300 import workloads as W
    return W.random_problem(3, 50, 2, W.OPS_RATIONAL, [[-3, 2]] * 3, 313, "rational shards")


def shard_boxes(t, n_nodes=11):
    """a bisection frontier of the root box, one shard item per node"""
    from paper_2507_20769_gb300 import workloads as W
    return W.bisection_frontier(t.root_box, n_nodes, seed=8)
