"""CPU oracle for interval Mean Value Form subdomain bounding (plain C, fesetround).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package. The CUDA library never
loads it, and it shares no code with the CUDA library.

`build()` compiles ivb_oracle.c with gcc; `lib()` loads it (building on first
use). The wrappers take a tape object with attributes n_vars, op, a, b, c,
out_idx, out_kind (numpy arrays) and return numpy arrays.

`tight` selects the exp/log enclosures: True / 1 binary128 evaluation rounded
outward (within one ulp of the true value), False / 0 the libm result widened
by two ulps (timing), an integer k > 1 the tight enclosure moved k - 1 further
steps outward on each side (the outer end of a parity bracket).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ivb_oracle.c")
_SO = os.path.join(_HERE, "libivb_oracle.so")
# tests that plant a mistake in a copy of the oracle point this at the copy's build
_SO_OVERRIDE = os.environ.get("IVB_ORACLE_SO")

GRAD = {"forward": 0, "adjoint": 1}
FORM = {"mvf": 0, "nie": 1, "mvf_nie": 2}
STRATEGY = {"uniform": 0, "largest": 1, "adaptive": 2}

_lib = None


def compile_source(src: str, out: str) -> str:
    """gcc with the oracle's strict IEEE flags"""
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-frounding-math", "-fno-fast-math", "-ffp-contract=off", "-fno-math-errno",
           "-fsignaling-nans", "-Wall", "-Wno-unknown-pragmas", src, "-o", out, "-lm"]
    if platform.machine() in ("x86_64", "AMD64", "i686"):
        cmd.append("-lquadmath")
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libivb_oracle.so (strict IEEE flags)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    compile_source(_SRC, _SO + ".tmp")
    os.replace(_SO + ".tmp", _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if _SO_OVERRIDE:
            L = ctypes.CDLL(_SO_OVERRIDE)
        else:
            build()
            L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        I, I64, D = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.orc_decode.argtypes = [I, P, P, I64, P, P]
        L.orc_value_sweep.argtypes = [I, I, P, P, P, P, P, I, P]
        L.orc_gradient.argtypes = [I, I, I, P, P, P, P, P, P, I, I, P]
        L.orc_enclose.argtypes = [I, I, I, P, P, P, P, P, P, P, I64, I64, I, I, I, P, P, P]
        L.orc_bound_nodes.argtypes = [I, I, I, P, P, P, P, P, P, I, P, P, I, I, I, I, P, P, P, P, P]
        L.orc_point_grad.argtypes = [I, I, I, P, P, P, P, P, P, P, P]
        L.orc_point_value_q.argtypes = [I, I, I, P, P, P, P, P, P, P, P]
        L.orc_central_diff_q.argtypes = [I, I, I, P, P, P, P, P, P, P, P]
        L.orc_exp_enclose.argtypes = [I64, P, I, P, P]
        L.orc_log_enclose.argtypes = [I64, P, I, P, P]
        L.orc_iv_op.argtypes = [I, I64, P, P, I, P]
        L.orc_pick_splits.argtypes = [I, P, P, I64, I, P]
        L.orc_bnb.argtypes = [I, I, I, P, P, P, P, P, P, P, P, I64, I, I, I, I, D, D, I64, D, I, I, P]
        L.orc_propagate.argtypes = [I, I, I, P, P, P, P, P, P, I64, P, D, I, I, P]
        L.orc_set_threads.argtypes = [I]
        L.orc_max_threads.restype = I
        _lib = L
    return _lib


def _p(x):
    return None if x is None else x.ctypes.data_as(ctypes.c_void_p)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def _tape_args(t):
    return (_i32(t.a), _i32(t.b), _f64(t.c), np.ascontiguousarray(t.op, dtype=np.uint8),
            _i32(t.out_idx), np.ascontiguousarray(t.out_kind, dtype=np.uint8))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def decode(box, splits, k: int):
    box, splits = _f64(box), _i32(splits)
    n = splits.shape[0]
    X, c = np.empty((n, 2)), np.empty(n)
    lib().orc_decode(n, _p(box), _p(splits), int(k), _p(X), _p(c))
    return X, c


def value_sweep(t, X, tight: bool = True):
    a, b, c, op, _, _ = _tape_args(t)
    X = _f64(X)
    V = np.empty((t.n_ops, 2))
    rc = lib().orc_value_sweep(t.n_vars, t.n_ops, _p(op), _p(a), _p(b), _p(c), _p(X), int(tight), _p(V))
    assert rc == 0
    return V


def gradient(t, X, grad_mode: str = "adjoint", tight: bool = True):
    a, b, c, op, oi, _ = _tape_args(t)
    X = _f64(X)
    G = np.empty((t.n_out, t.n_vars, 2))
    rc = lib().orc_gradient(t.n_vars, t.n_ops, t.n_out, _p(op), _p(a), _p(b), _p(c), _p(oi), _p(X),
                            GRAD[grad_mode], int(tight), _p(G))
    assert rc == 0
    return G


def enclose(t, box, splits, first: int = 0, count: int | None = None, grad_mode: str = "adjoint",
            form: str = "mvf", tight: bool = True, want_fc: bool = False, want_g: bool = False):
    """per-subdomain enclosures F [count][n_out][2] (+ Fc, G)"""
    a, b, c, op, oi, _ = _tape_args(t)
    box, splits = _f64(box), _i32(splits)
    if count is None:
        count = int(np.prod(splits.astype(np.int64))) - first
    F = np.empty((count, t.n_out, 2))
    Fc = np.empty((count, t.n_out, 2)) if want_fc else None
    G = np.empty((count, t.n_out, t.n_vars, 2)) if want_g else None
    rc = lib().orc_enclose(t.n_vars, t.n_ops, t.n_out, _p(op), _p(a), _p(b), _p(c), _p(oi), _p(box),
                           _p(splits), int(first), int(count), GRAD[grad_mode], FORM[form], int(tight),
                           _p(F), _p(Fc), _p(G))
    assert rc == 0
    return F, Fc, G


def bound_nodes(t, boxes, splits, grad_mode: str = "adjoint", form: str = "mvf", tight: bool = True,
                filter: bool = False):
    """Steps 1-3 for a batch of nodes: dict of lb, infeasible, ub, minlo, maxhi"""
    a, b, c, op, oi, ok = _tape_args(t)
    boxes = _f64(boxes).reshape(-1, t.n_vars, 2)
    nn = boxes.shape[0]
    splits = _i32(np.broadcast_to(np.asarray(splits, dtype=np.int32).reshape(-1, t.n_vars), (nn, t.n_vars)))
    lb, ub = np.empty(nn), np.empty(nn)
    inf = np.empty(nn, dtype=np.uint8)
    minlo, maxhi = np.empty((nn, t.n_out)), np.empty((nn, t.n_out))
    rc = lib().orc_bound_nodes(t.n_vars, t.n_ops, t.n_out, _p(op), _p(a), _p(b), _p(c), _p(oi), _p(ok), nn,
                               _p(boxes), _p(splits), GRAD[grad_mode], FORM[form], int(tight), int(filter),
                               _p(lb), _p(inf), _p(ub), _p(minlo), _p(maxhi))
    assert rc == 0
    return {"lb": lb, "infeasible": inf.astype(bool), "ub": ub, "minlo": minlo, "maxhi": maxhi}


def point_grad(t, x):
    a, b, c, op, oi, _ = _tape_args(t)
    x = _f64(x)
    f, g = np.empty(t.n_out), np.empty((t.n_out, t.n_vars))
    rc = lib().orc_point_grad(t.n_vars, t.n_ops, t.n_out, _p(op), _p(a), _p(b), _p(c), _p(oi), _p(x), _p(f), _p(g))
    assert rc == 0
    return f, g


def point_value_q(t, x, dx=None):
    a, b, c, op, oi, _ = _tape_args(t)
    x = _f64(x)
    dx = None if dx is None else _f64(dx)
    f = np.empty(t.n_out)
    rc = lib().orc_point_value_q(t.n_vars, t.n_ops, t.n_out, _p(op), _p(a), _p(b), _p(c), _p(oi), _p(x),
                                 _p(dx), _p(f))
    assert rc == 0
    return f


def central_diff_q(t, x, h):
    a, b, c, op, oi, _ = _tape_args(t)
    x, h = _f64(x), _f64(h)
    g = np.empty((t.n_out, t.n_vars))
    rc = lib().orc_central_diff_q(t.n_vars, t.n_ops, t.n_out, _p(op), _p(a), _p(b), _p(c), _p(oi), _p(x),
                                  _p(h), _p(g))
    assert rc == 0
    return g


def exp_enclose(x, tight: bool = True):
    x = _f64(x).ravel()
    lo, hi = np.empty_like(x), np.empty_like(x)
    lib().orc_exp_enclose(x.size, _p(x), int(tight), _p(lo), _p(hi))
    return lo, hi


def log_enclose(x, tight: bool = True):
    x = _f64(x).ravel()
    lo, hi = np.empty_like(x), np.empty_like(x)
    lib().orc_log_enclose(x.size, _p(x), int(tight), _p(lo), _p(hi))
    return lo, hi


def iv_op(opcode: int, x, y=None, tight: bool = True):
    """one interval op on arrays of intervals [..., 2]"""
    x = _f64(x).reshape(-1, 2)
    y = None if y is None else _f64(np.broadcast_to(np.asarray(y, dtype=np.float64).reshape(-1, 2), x.shape))
    r = np.empty_like(x)
    lib().orc_iv_op(int(opcode), x.shape[0], _p(x), _p(y), int(tight), _p(r))
    return r


def iv_fma(x, y, acc):
    """acc + x*y with one directed rounding per end, on arrays of intervals [..., 2]"""
    x = _f64(x).reshape(-1, 2)
    y = _f64(np.broadcast_to(np.asarray(y, dtype=np.float64).reshape(-1, 2), x.shape))
    r = _f64(np.broadcast_to(np.asarray(acc, dtype=np.float64).reshape(-1, 2), x.shape)).copy()
    lib().orc_iv_op(105, x.shape[0], _p(x), _p(y), 1, _p(r))
    return r


def pick_splits(box, target: int, strategy: str = "adaptive", ref=None):
    box = _f64(box).reshape(-1, 2)
    n = box.shape[0]
    ref = None if ref is None else _f64(ref)
    out = np.empty(n, dtype=np.int32)
    rc = lib().orc_pick_splits(n, _p(box), _p(ref), int(target), STRATEGY[strategy], _p(out))
    assert rc == 0
    return out


def bnb(t, root=None, splits=None, target: int = 0, strategy: str = "adaptive", grad_mode: str = "adjoint",
        form: str = "mvf", tight: bool = False, eps_abs: float = 0.0, eps_rel: float = 1e-3,
        max_nodes: int = 0, time_limit: float = 0.0, corner_ub: bool = True, propagate: int = 0):
    """best-first B&B with the oracle as lower-bounding solver; propagate > 0:
    tighten every box by that many rounds of constraint propagation first"""
    a, b, c, op, oi, ok = _tape_args(t)
    root = _f64(t.root_box if root is None else root)
    sp = _i32(splits if splits is not None else np.ones(t.n_vars, np.int32))
    stats = np.empty(8)
    rc = lib().orc_bnb(t.n_vars, t.n_ops, t.n_out, _p(op), _p(a), _p(b), _p(c), _p(oi), _p(ok), _p(root), _p(sp),
                       int(target), STRATEGY[strategy], GRAD[grad_mode], FORM[form], int(tight), float(eps_abs),
                       float(eps_rel), int(max_nodes), float(time_limit), int(corner_ub), int(propagate), _p(stats))
    assert rc == 0
    return {"lb": stats[0], "ub": stats[1], "iterations": int(stats[2]), "nodes": int(stats[3]),
            "subdomains": int(stats[4]), "seconds": stats[5], "converged": bool(stats[6]),
            "open": int(stats[7])}


def propagate(t, boxes, ub: float = float("inf"), passes: int = 4, tight: bool = True):
    """forward-backward bound tightening of boxes [..., n, 2] against the
    tape's constraints and f <= ub: (tightened boxes, infeasible flags)"""
    a, b, c, op, oi, ok = _tape_args(t)
    bx = np.array(_f64(boxes).reshape(-1, t.n_vars, 2))
    inf = np.empty(bx.shape[0], dtype=np.uint8)
    rc = lib().orc_propagate(t.n_vars, t.n_ops, t.n_out, _p(op), _p(a), _p(b), _p(c), _p(oi), _p(ok),
                             bx.shape[0], _p(bx), float(ub), int(passes), int(tight), _p(inf))
    assert rc == 0
    return bx, inf.astype(bool)
