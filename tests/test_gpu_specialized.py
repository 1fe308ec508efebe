"""GPU parity of the tape-specialised bounding kernel (option specialize=1:
the tape's programs written out as straight-line CUDA and compiled with NVRTC
at problem creation).

It evaluates the same interval primitives on the same operands in the same
accumulation order as the tape interpreter, so every result must equal the
interpreter's bit for bit, and on rational tapes the oracle's bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import problems as P
from paper_2507_20769_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_20769_gb300 import build as B  # noqa: E402

B.build()
from paper_2507_20769_gb300 import ivb  # noqa: E402

KEYS = ("lb", "ub", "minlo", "maxhi", "infeasible")


def rational_problem(n=3, K=60, n_ineq=2, seed=777):
    return W.random_problem(n, K, n_ineq, W.OPS_RATIONAL, [[-3, 2]] * n, seed, "rational")


def ragged_batch(t, n_nodes, seed, max_split=6):
    rng = np.random.default_rng(seed)
    boxes = W.bisection_frontier(t.root_box, n_nodes, seed=seed)
    splits = rng.integers(1, max_split + 1, (n_nodes, t.n_vars)).astype(np.int32)
    splits[0] = 1                          # S = 1
    boxes[1, 0, 1] = boxes[1, 0, 0]        # degenerate dimension
    return boxes, splits


def same_bits(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8))


def bound_both(t, boxes, splits, spec_mode=1, **opts):
    """results of the interpreter and of the specialised kernel (spec_mode 1:
    per-output sweeps and long primitives out of line, or 2: fully inlined),
    same options"""
    out = []
    for spec in (0, spec_mode):
        with ivb.Problem(t, specialize=spec, **opts) as p:
            if spec:
                assert p.get_specialization()["active"]
            out.append(p.bound_nodes_ex(boxes, splits, want_hull=True))
    return out


@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
@pytest.mark.parametrize("path", ["graph", "nograph", "plain"])
@pytest.mark.parametrize("emulate,spec_mode", [(0, 1), (15, 1), (0, 2)])
def test_specialized_bit_exact_rational_vs_oracle(grad_mode, path, emulate, spec_mode):
    """ragged batch (S from 1 to 216 per node, tiles crossing nodes), every
    launch path, endpoint operations on the FP64 pipe (0) or all emulated on
    the integer pipes (15): lb, infeasibility, centre upper bound and each
    output's hull equal the oracle's bit for bit"""
    t = rational_problem()
    boxes, splits = ragged_batch(t, 37, seed=11)
    opts = dict(grad_mode=grad_mode, use_graph=int(path == "graph"), batched=int(path != "plain"),
                specialize=spec_mode, emulate=emulate)
    with ivb.Problem(t, **opts) as p:
        assert p.get_specialization()["active"]
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
        r2 = p.bound_nodes_ex(boxes, splits, want_hull=True)
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode=grad_mode, tight=True)
    for rr in (r, r2):
        for k in ("lb", "ub", "minlo", "maxhi"):
            assert np.array_equal(rr[k], ref[k]), k
        assert np.array_equal(rr["infeasible"].astype(bool), ref["infeasible"])


@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
@pytest.mark.parametrize("form", ["mvf", "nie", "mvf_nie"])
@pytest.mark.parametrize("emulate", [-1, 0, 5, 10, 15])
def test_specialized_identical_to_interpreter_exp_log(grad_mode, form, emulate):
    """configuration 1 (exp/log tape), any emulation policy, compact or not:
    all results bit-identical to the interpreter"""
    t = W.config_tape(1)
    boxes, splits = ragged_batch(t, 23, seed=5, max_split=40)
    a, b = bound_both(t, boxes, splits, spec_mode=1 + (emulate == 5), grad_mode=grad_mode, form=form,
                      emulate=emulate)
    for k in KEYS:
        assert same_bits(a[k], b[k]), k


@pytest.mark.parametrize("kind", ["feasible", "infeasible", "eq_out", "eq_in"])
@pytest.mark.parametrize("filt", [0, 1])
def test_specialized_feasibility_filter_and_ub_match_oracle(kind, filt):
    t = P.constrained_toy(kind)
    boxes = W.bisection_frontier(t.root_box, 9, seed=2)
    splits = np.array([[6, 5]] * 9, np.int32)
    with ivb.Problem(t, filter=filt, specialize=1) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
    ref = oracle.bound_nodes(t, boxes, splits, filter=bool(filt))
    assert np.array_equal(r["lb"], ref["lb"])
    assert np.array_equal(r["infeasible"].astype(bool), ref["infeasible"])
    assert np.array_equal(r["ub"], ref["ub"])


def variable_and_constant_outputs():
    """objective that is a variable entry itself, an inequality that is a
    constant entry, and an equality sharing the objective's variable: the
    generator's special cases (gradient e_i, no adjoint slot, a product of an
    entry with itself, a negation)"""
    Bd = P.Builder(2)
    x0, x1 = Bd.x(0), Bd.x(1)
    Bd.output(x0, P.KIND_OBJ)
    Bd.output(Bd.const(-0.5), P.KIND_INEQ)
    Bd.output(Bd.sub(Bd.mul(x0, x0), Bd.neg(x1)), P.KIND_EQ)
    return Bd.tape([[-1.0, 2.0], [-1.5, 1.0]], "variable and constant outputs")


@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
@pytest.mark.parametrize("spec_mode", [1, 2])
def test_specialized_variable_and_constant_outputs(grad_mode, spec_mode):
    t = variable_and_constant_outputs()
    boxes, splits = ragged_batch(t, 11, seed=4)
    a, b = bound_both(t, boxes, splits, spec_mode=spec_mode, grad_mode=grad_mode)
    for k in KEYS:
        assert same_bits(a[k], b[k]), k
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode=grad_mode, tight=True)
    for k in ("lb", "ub", "minlo", "maxhi"):
        assert np.array_equal(b[k], ref[k]), k


@pytest.mark.parametrize("emulate,spec_mode", [(-1, 1), (15, 1), (-1, 2)])
def test_specialized_full_size_config2_identical_to_interpreter(emulate, spec_mode):
    """configuration 2 at full size (16 nodes x 16^4 subdomains, autotuned,
    CUDA graph): bit-identical to the interpreter"""
    wl = W.config_workload(2)
    t = wl.tape
    boxes = W.bisection_frontier(t.root_box, 16, seed=20)
    splits = np.tile(wl.splits, (16, 1)).astype(np.int32)
    a, b = bound_both(t, boxes, splits, spec_mode=spec_mode, emulate=emulate)
    for k in KEYS:
        assert same_bits(a[k], b[k]), k


def test_specialize_auto_info_and_empty_batch():
    """specialize=-1 compiles a small tape as one program; a large one
    (configuration 4, above the size limit) gets the segmented kernel in
    adjoint mode and the interpreter in forward mode; an empty batch is a
    no-op"""
    with ivb.Problem(W.config_tape(1), specialize=-1) as p:
        info = p.get_specialization()
        assert info["active"] and 0 < info["registers"] <= 128 and info["compile_seconds"] > 0
        assert p.get_segmentation()["chunks"] == 0
        r = p.bound_nodes_ex(np.zeros((0, 2, 2)), np.zeros((0, 2), np.int32))
        assert r["lb"].shape == (0,)
    with ivb.Problem(W.config_tape(4), specialize=-1, grad_mode="forward") as p:
        assert not p.get_specialization()["active"]
    with ivb.Problem(W.config_tape(4), specialize=-1, grad_mode="adjoint") as p:
        assert p.get_specialization()["active"] and p.get_segmentation()["chunks"] > 1
    with ivb.Problem(W.config_tape(1)) as p:
        assert not p.get_specialization()["active"]


def shared_dag(n, n_ops, n_ineq, n_eq, ops, seed):
    """random DAG whose outputs share subexpressions: every operand is any
    earlier entry, so the outputs' cones overlap; some outputs are plain
    variable or constant entries"""
    rng = np.random.default_rng(seed)
    Bd = P.Builder(n)
    ids = list(range(n))
    for _ in range(max(2, n // 4)):
        ids.append(Bd.const(float(rng.uniform(-2, 2))))
    names = {W.OP_ADD: Bd.add, W.OP_SUB: Bd.sub, W.OP_MUL: Bd.mul, W.OP_DIV: Bd.div, W.OP_SQR: Bd.sqr,
             W.OP_SQRT: Bd.sqrt, W.OP_EXP: Bd.exp, W.OP_LOG: Bd.log, W.OP_NEG: Bd.neg}
    for _ in range(n_ops):
        op = int(rng.choice(ops))
        a = ids[int(rng.integers(len(ids)))]
        b = ids[int(rng.integers(len(ids)))]
        if op in (W.OP_DIV,):      # keep divisors away from 0: b^2 + 1
            b = Bd.add(Bd.sqr(b), Bd.const(1.0))
        if op in (W.OP_SQRT, W.OP_LOG):
            a = Bd.add(Bd.sqr(a), Bd.const(0.5))
        if op == W.OP_EXP:
            a = Bd.mul(Bd.const(0.01), a)
        ids.append(names[op](a, b) if op in (W.OP_ADD, W.OP_SUB, W.OP_MUL, W.OP_DIV) else names[op](a))
    interior = ids[n:]
    Bd.output(interior[-1], P.KIND_OBJ)
    for q in range(n_ineq):
        pick = interior[int(rng.integers(len(interior)))]
        Bd.output(Bd.sub(pick, Bd.const(float(rng.uniform(0, 3)))), P.KIND_INEQ)
    for q in range(n_eq):
        Bd.output(Bd.sub(ids[q % n], ids[(q + 1) % n]), P.KIND_EQ)
    Bd.output(0, P.KIND_INEQ)                   # a variable entry as an output
    Bd.output(Bd.const(-1.0), P.KIND_INEQ)      # a constant entry as an output
    return Bd.tape([[-1.5, 1.0]] * n, f"shared dag {seed}")


RATIONAL = [W.OP_ADD, W.OP_SUB, W.OP_MUL, W.OP_DIV, W.OP_SQR, W.OP_NEG]
ALL = RATIONAL + [W.OP_SQRT, W.OP_EXP, W.OP_LOG]


@pytest.mark.parametrize("n,ops_kind,seed", [(1, "rational", 1), (3, "rational", 2), (5, "all", 3),
                                              (8, "all", 4), (32, "rational", 5)])
@pytest.mark.parametrize("grad_mode", ["adjoint", "forward"])
def test_specialized_shared_subexpressions(n, ops_kind, seed, grad_mode):
    """overlapping output cones, variable and constant outputs, equalities,
    one to 32 variables: bit-identical to the interpreter, and to the oracle
    on rational tapes"""
    t = shared_dag(n, 30 if n < 32 else 20, 2, 1 if n > 1 else 0, RATIONAL if ops_kind == "rational" else ALL, seed)
    nn = 9
    boxes = W.bisection_frontier(t.root_box, nn, seed=seed)
    splits = np.ones((nn, n), np.int32)
    splits[:, : min(n, 3)] = 3
    a, b = bound_both(t, boxes, splits, grad_mode=grad_mode)
    for k in KEYS:
        assert same_bits(a[k], b[k]), k
    if ops_kind == "rational":
        ref = oracle.bound_nodes(t, boxes, splits, grad_mode=grad_mode, tight=True)
        for k in ("lb", "ub", "minlo", "maxhi"):
            assert np.array_equal(b[k], ref[k]), k


@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
@pytest.mark.parametrize("spec", [0, 1])
def test_nie_form_skips_gradients_and_matches_oracle(grad_mode, spec):
    """with the natural interval extension alone the reduce kernels skip the
    gradient sweeps; the bounds equal the oracle's NIE bounds bit for bit and
    the reported work drops"""
    t = rational_problem()
    boxes, splits = ragged_batch(t, 29, seed=8)
    with ivb.Problem(t, grad_mode=grad_mode, form="nie", specialize=spec) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
        nie_work = sum(p.op_counts().values())
    with ivb.Problem(t, grad_mode=grad_mode, form="mvf") as p:
        mvf_work = sum(p.op_counts().values())
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode=grad_mode, form="nie", tight=True)
    for k in ("lb", "ub", "minlo", "maxhi"):
        assert np.array_equal(r[k], ref[k]), k
    assert np.array_equal(r["infeasible"].astype(bool), ref["infeasible"])
    assert nie_work < 0.75 * mvf_work
