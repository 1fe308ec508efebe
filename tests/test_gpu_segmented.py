"""GPU parity of the segmented tape-specialised kernel (option specialize=3):
the per-subdomain program cut into chunk functions, values that cross chunks
kept in a per-thread state area, the reverse chunks recomputing their
segment's forward values from checkpoints (option recompute: 0 none, 1 cheap
operations, 2 all).

A recomputed value is the same interval primitive on the same operands as the
stored one, and the adjoint accumulations and the Mean Value Form sum keep
their order, so every result must equal the tape interpreter's bit for bit,
and the oracle's bit for bit on rational tapes. Small chunk budgets cut even
short tapes into many chunks, so the state area, the slot reuse and the
recomputation across chunk boundaries are exercised at every size."""
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

from test_gpu_specialized import KEYS, ragged_batch, rational_problem, same_bits, shared_dag  # noqa: E402
from test_gpu_specialized import ALL, RATIONAL, variable_and_constant_outputs  # noqa: E402


def bound_seg_and_interp(t, boxes, splits, seg_opts, **opts):
    out = []
    for spec in (0, 3):
        extra = seg_opts if spec == 3 else {}
        with ivb.Problem(t, grad_mode="adjoint", specialize=spec, **opts, **extra) as p:
            if spec == 3:
                info = p.get_segmentation()
                assert p.get_specialization()["active"] and info["chunks"] >= 1 and info["state_units"] >= 2
            out.append(p.bound_nodes_ex(boxes, splits, want_hull=True))
    return out


@pytest.mark.parametrize("path", ["graph", "nograph", "plain"])
@pytest.mark.parametrize("recompute", [0, 1, 2])
@pytest.mark.parametrize("chunk", [6, 40, 0])
def test_segmented_bit_exact_rational_vs_oracle(path, recompute, chunk):
    """ragged batch (S from 1 to 216 per node, tiles crossing nodes), every
    launch path, every recomputation policy, chunks of a few operations up to
    the default budget: lb, infeasibility, centre upper bound and every
    output's hull equal the oracle's bit for bit"""
    t = rational_problem()
    boxes, splits = ragged_batch(t, 37, seed=11)
    opts = dict(grad_mode="adjoint", use_graph=int(path == "graph"), batched=int(path != "plain"),
                specialize=3, recompute=recompute, seg_chunk=chunk)
    with ivb.Problem(t, **opts) as p:
        seg = p.get_segmentation()
        assert seg["recompute"] == recompute
        if chunk == 6:
            assert seg["chunks"] > 20
        if recompute == 0:
            assert seg["recomputed"] == 0
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
        r2 = p.bound_nodes_ex(boxes, splits, want_hull=True)
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode="adjoint", tight=True)
    for rr in (r, r2):
        for k in ("lb", "ub", "minlo", "maxhi"):
            assert np.array_equal(rr[k], ref[k]), k
        assert np.array_equal(rr["infeasible"].astype(bool), ref["infeasible"])


@pytest.mark.parametrize("config", [1, 2])
@pytest.mark.parametrize("form", ["mvf", "nie", "mvf_nie"])
@pytest.mark.parametrize("recompute,chunk", [(0, 24), (1, 24), (2, 24), (1, 0)])
def test_segmented_identical_to_interpreter_exp_log(config, form, recompute, chunk):
    """configurations 1 and 2 (exp/log tapes), every form and policy: all
    results bit-identical to the interpreter"""
    t = W.config_tape(config)
    boxes, splits = ragged_batch(t, 23, seed=5, max_split=40 if t.n_vars == 2 else 6)
    a, b = bound_seg_and_interp(t, boxes, splits, dict(recompute=recompute, seg_chunk=chunk), form=form)
    for k in KEYS:
        assert same_bits(a[k], b[k]), k


@pytest.mark.parametrize("n,ops_kind,seed", [(1, "rational", 1), (3, "rational", 2), (5, "all", 3),
                                              (8, "all", 4), (32, "rational", 5)])
@pytest.mark.parametrize("recompute", [1, 2])
def test_segmented_shared_subexpressions(n, ops_kind, seed, recompute):
    """overlapping output cones, variable and constant outputs, equalities,
    one to 32 variables, small chunks: bit-identical to the interpreter, and
    to the oracle on rational tapes"""
    t = shared_dag(n, 30 if n < 32 else 20, 2, 1 if n > 1 else 0, RATIONAL if ops_kind == "rational" else ALL, seed)
    nn = 9
    boxes = W.bisection_frontier(t.root_box, nn, seed=seed)
    splits = np.ones((nn, n), np.int32)
    splits[:, : min(n, 3)] = 3
    a, b = bound_seg_and_interp(t, boxes, splits, dict(recompute=recompute, seg_chunk=12))
    for k in KEYS:
        assert same_bits(a[k], b[k]), k
    if ops_kind == "rational":
        ref = oracle.bound_nodes(t, boxes, splits, grad_mode="adjoint", tight=True)
        for k in ("lb", "ub", "minlo", "maxhi"):
            assert np.array_equal(b[k], ref[k]), k


def test_segmented_variable_and_constant_outputs():
    t = variable_and_constant_outputs()
    boxes, splits = ragged_batch(t, 11, seed=4)
    a, b = bound_seg_and_interp(t, boxes, splits, dict(recompute=1, seg_chunk=4))
    for k in KEYS:
        assert same_bits(a[k], b[k]), k
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode="adjoint", tight=True)
    for k in ("lb", "ub", "minlo", "maxhi"):
        assert np.array_equal(b[k], ref[k]), k


@pytest.mark.parametrize("kind", ["feasible", "infeasible", "eq_out", "eq_in"])
@pytest.mark.parametrize("filt", [0, 1])
def test_segmented_feasibility_filter_and_ub_match_oracle(kind, filt):
    t = P.constrained_toy(kind)
    boxes = W.bisection_frontier(t.root_box, 9, seed=2)
    splits = np.array([[6, 5]] * 9, np.int32)
    with ivb.Problem(t, filter=filt, specialize=3, seg_chunk=8) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
    ref = oracle.bound_nodes(t, boxes, splits, filter=bool(filt))
    assert np.array_equal(r["lb"], ref["lb"])
    assert np.array_equal(r["infeasible"].astype(bool), ref["infeasible"])
    assert np.array_equal(r["ub"], ref["ub"])


def test_segmented_rejects_forward_mode_and_bad_options():
    t = rational_problem()
    for bad in (dict(specialize=3, grad_mode="forward"), dict(specialize=3, recompute=3),
                dict(specialize=3, seg_regs=32), dict(specialize=4)):
        with pytest.raises(ivb.IvbError) as e:
            ivb.Problem(t, **bad)
        assert e.value.status == ivb.IVB_EINVAL


def test_segmented_full_scale_config5_identical_to_interpreter():
    """configuration 5 at full scale: 64 nodes x 2^18 = 2^24 subdomains of the
    n=8 problem with 11 outputs of 1000-entry tapes, one batched launch,
    autotuned: node hulls, lb, ub and flags bit-identical to the interpreter;
    specialize=-1 picks the segmented kernel for these tapes"""
    t = W.config_tape(5)
    boxes = W.bisection_frontier(t.root_box, 64, seed=2026)
    splits = np.array([W.full_scale_splits(b, t.root_box) for b in boxes], np.int32)
    assert int(np.prod(splits.astype(np.int64), axis=1).sum()) == 1 << 24
    res = []
    for spec in (0, -1):
        with ivb.Problem(t, grad_mode="adjoint", specialize=spec, max_nodes=64) as p:
            if spec == -1:
                assert p.get_segmentation()["chunks"] > 50
            res.append(p.bound_nodes_ex(boxes, splits, want_hull=True))
    for k in KEYS:
        assert same_bits(res[0][k], res[1][k]), k
