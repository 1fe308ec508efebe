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
                dict(specialize=3, seg_regs=32), dict(specialize=4), dict(specialize=3, seg_outline=3)):
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
            # with the library's choice the autotuner keeps whichever kernel timed faster
            assert p.get_tuning()["kernel"] in ((0,) if spec == 0 else (0, 2))
    for k in KEYS:
        assert same_bits(res[0][k], res[1][k]), k


# ------------------------------------------- the autotuner's launch knobs

@pytest.mark.parametrize("tpsub", [1, 2, 4])
@pytest.mark.parametrize("path", ["graph", "plain"])
def test_threads_per_subdomain_bit_exact_rational(tpsub, path):
    """1, 2 or 4 threads share each subdomain (output groups in different
    warps, flags combined in shared memory): the ragged batch's lb, ub,
    flags and hulls equal the oracle's bit for bit"""
    t = rational_problem(n=3, K=50, n_ineq=3)
    boxes, splits = ragged_batch(t, 37, seed=13)
    opts = dict(grad_mode="adjoint", specialize=3, seg_chunk=24, threads_per_subdomain=tpsub,
                use_graph=int(path == "graph"), batched=int(path != "plain"))
    with ivb.Problem(t, **opts) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
        assert p.get_tuning()["threads_per_subdomain"] == tpsub
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode="adjoint", tight=True)
    for k in ("lb", "ub", "minlo", "maxhi"):
        assert np.array_equal(r[k], ref[k]), k
    assert np.array_equal(r["infeasible"].astype(bool), ref["infeasible"])


@pytest.mark.parametrize("kind", ["feasible", "infeasible", "eq_in"])
def test_threads_per_subdomain_filter_and_ub(kind):
    """the tests that need every output of a subdomain (filtered objective,
    certified-feasible centre) across two output groups"""
    t = P.constrained_toy(kind)
    boxes = W.bisection_frontier(t.root_box, 9, seed=2)
    splits = np.array([[6, 5]] * 9, np.int32)
    with ivb.Problem(t, filter=1, specialize=3, threads_per_subdomain=2) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
        assert p.get_tuning()["threads_per_subdomain"] == 2
    ref = oracle.bound_nodes(t, boxes, splits, filter=True)
    for k in ("lb", "ub", "minlo", "maxhi"):
        assert np.array_equal(r[k], ref[k]), k
    assert np.array_equal(r["infeasible"].astype(bool), ref["infeasible"])


def test_every_launch_candidate_gives_identical_bounds():
    """threads per subdomain x block size x subdomains per grab x chunk
    synchronisation, fixed by options (no timing): every combination the
    autotuner can pick gives the interpreter's bits on configuration 2
    (exp/log tape)"""
    t = W.config_tape(2)
    boxes, splits = ragged_batch(t, 23, seed=5)
    with ivb.Problem(t, grad_mode="adjoint", specialize=0) as p:
        ref = p.bound_nodes_ex(boxes, splits, want_hull=True)
    seen = set()
    for sync in (0, 1):
        for tpsub in (1, 2, 4):
            for block, mult in ((64, 1), (128, 4), (256, 16)):
                if block < 32 * tpsub:
                    continue
                per = block // tpsub
                with ivb.Problem(t, grad_mode="adjoint", specialize=3, threads_per_subdomain=tpsub,
                                 block_threads=block, blocks_per_sm=2, tile=mult * per, seg_sync=sync) as p:
                    r = p.bound_nodes_ex(boxes, splits, want_hull=True)
                    tun = p.get_tuning()
                assert (tun["threads_per_subdomain"], tun["block_threads"], tun["tile"], tun["chunk_sync"]) == \
                    (tpsub, block, mult * per, sync)
                seen.add((sync, tpsub, block, mult))
                for k in KEYS:
                    assert same_bits(ref[k], r[k]), (sync, tpsub, block, mult, k)
    assert len(seen) == 16


def test_autotuner_full_size_choice_reported_and_identical():
    """configuration 2 at full size (16 nodes x 16^4): the autotuner times
    threads per subdomain, block size, blocks per SM and grab size, reports
    its choice, and the bounds equal the interpreter's"""
    wl = W.config_workload(2)
    t = wl.tape
    boxes = W.bisection_frontier(t.root_box, 16, seed=20)
    splits = np.tile(wl.splits, (16, 1)).astype(np.int32)
    out = []
    for spec in (0, 3):
        with ivb.Problem(t, grad_mode="adjoint", specialize=spec) as p:
            out.append(p.bound_nodes_ex(boxes, splits, want_hull=True))
            tun = p.get_tuning()
        if spec == 3:
            assert tun["kernel"] == 2    # an explicit segmented kernel is never replaced
            assert tun["candidates"] > 10 and tun["threads_per_subdomain"] in (1, 2, 4)
            assert tun["tile"] % tun["subdomains_per_pass"] == 0
            assert tun["subdomains_per_pass"] * tun["threads_per_subdomain"] == tun["block_threads"]
            assert 0 < tun["best_ms"] <= tun["worst_ms"]
    for k in KEYS:
        assert same_bits(out[0][k], out[1][k]), k


def test_bnb_split_target_picked_from_the_launch():
    """B&B with the split picker and target 0: each iteration's target is
    the smallest power of two >= 2^8 (at most 2^20) that makes its children
    cover four waves of the launch; an explicit target is used as given"""
    t = rational_problem(n=2, K=40, n_ineq=1, seed=99)
    with ivb.Problem(t, grad_mode="adjoint", specialize=3) as p:
        r = p.bnb_solve(t.root_box, target=0, strategy="adaptive", batch=4, eps_rel=1e-4, max_nodes=64)
        tun = p.get_tuning()
        r2 = p.bnb_solve(t.root_box, target=1000, strategy="adaptive", batch=4, eps_rel=1e-4, max_nodes=64)
    tgt = r["split_target"]
    assert 256 <= tgt <= 1 << 20 and tgt & (tgt - 1) == 0
    wave = torch.cuda.get_device_properties(0).multi_processor_count * tun["blocks_per_sm"] * tun["subdomains_per_pass"]
    assert tgt == 1 << 20 or tgt * 8 >= 4 * wave
    assert r2["split_target"] == 1000
    assert r["lb"] <= r["ub"] and r2["lb"] <= r2["ub"]


# ------------------------------------ two subdomains per thread (seg_ilp = 2)

@pytest.mark.parametrize("path", ["graph", "plain"])
@pytest.mark.parametrize("tpsub", [1, 2])
@pytest.mark.parametrize("recompute", [0, 1])
def test_two_subdomains_per_thread_bit_exact_rational(path, tpsub, recompute):
    """every statement run on two subdomains at once (the second copy repeats
    the first where the index range ends): the ragged batch's results equal
    the oracle's bit for bit"""
    t = rational_problem(n=3, K=50, n_ineq=3)
    boxes, splits = ragged_batch(t, 37, seed=17)
    opts = dict(grad_mode="adjoint", specialize=3, seg_ilp=2, threads_per_subdomain=tpsub, recompute=recompute,
                seg_chunk=24, use_graph=int(path == "graph"), batched=int(path != "plain"))
    with ivb.Problem(t, **opts) as p:
        assert p.get_segmentation()["ilp"] == 2
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
        tun = p.get_tuning()
        assert tun["subdomains_per_pass"] == 2 * tun["block_threads"] // tun["threads_per_subdomain"]
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode="adjoint", tight=True)
    for k in ("lb", "ub", "minlo", "maxhi"):
        assert np.array_equal(r[k], ref[k]), k
    assert np.array_equal(r["infeasible"].astype(bool), ref["infeasible"])


@pytest.mark.parametrize("form", ["mvf", "mvf_nie"])
@pytest.mark.parametrize("sync", [0, 1])
def test_two_subdomains_per_thread_identical_to_interpreter(form, sync):
    """configuration 2 (exp/log tape), both chunk synchronisation variants"""
    t = W.config_tape(2)
    boxes, splits = ragged_batch(t, 23, seed=5)
    a, b = bound_seg_and_interp(t, boxes, splits, dict(seg_ilp=2, seg_sync=sync), form=form)
    for k in KEYS:
        assert same_bits(a[k], b[k]), k


@pytest.mark.parametrize("emulate", [3, 12, 15])
def test_paired_form_with_emulated_second_copy_bit_exact(emulate):
    """two subdomains per thread in the paired form, the second copy's
    products and sums on the integer-pipe emulation: the oracle's bits on a
    rational tape, the interpreter's on configuration 2 (exp/log)"""
    t = rational_problem(n=3, K=50, n_ineq=3)
    boxes, splits = ragged_batch(t, 31, seed=23)
    with ivb.Problem(t, specialize=3, seg_ilp=2, emulate=emulate, seg_chunk=24) as p:
        assert p.get_segmentation()["ilp"] == 2
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode="adjoint", tight=True)
    for k in ("lb", "ub", "minlo", "maxhi"):
        assert np.array_equal(r[k], ref[k]), k
    assert np.array_equal(r["infeasible"].astype(bool), ref["infeasible"])
    t2 = W.config_tape(2)
    boxes, splits = ragged_batch(t2, 19, seed=8)
    a, b = bound_seg_and_interp(t2, boxes, splits, dict(seg_ilp=2, emulate=emulate))
    for k in KEYS:
        assert same_bits(a[k], b[k]), k


def test_products_only_out_of_line_bit_exact():
    """seg_outline = 2 (x, sqr and the fused accumulation called out of line,
    + and - inline): the oracle's bits on a rational tape, the interpreter's
    on configuration 2"""
    t = rational_problem(n=3, K=50, n_ineq=3)
    boxes, splits = ragged_batch(t, 27, seed=29)
    with ivb.Problem(t, specialize=3, seg_outline=2, seg_chunk=24) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode="adjoint", tight=True)
    for k in ("lb", "ub", "minlo", "maxhi"):
        assert np.array_equal(r[k], ref[k]), k
    t2 = W.config_tape(2)
    boxes, splits = ragged_batch(t2, 15, seed=10)
    a, b = bound_seg_and_interp(t2, boxes, splits, dict(seg_outline=2))
    for k in KEYS:
        assert same_bits(a[k], b[k]), k


def test_two_subdomains_inlined_interleaved_bit_exact():
    """seg_ilp = 2 with the short operations inlined (every statement written
    twice, interleaved, instead of the paired calls): the interpreter's bits
    on configuration 2"""
    t2 = W.config_tape(2)
    boxes, splits = ragged_batch(t2, 21, seed=9)
    a, b = bound_seg_and_interp(t2, boxes, splits, dict(seg_ilp=2, seg_outline=0))
    for k in KEYS:
        assert same_bits(a[k], b[k]), k


@pytest.mark.parametrize("recompute", [0, 1])
@pytest.mark.parametrize("tpsub", [1, 2])
def test_inlined_short_operations_bit_exact(recompute, tpsub):
    """seg_outline = 0 (+ - * sqr and the fused accumulation inlined instead
    of called out of line, the default): the oracle's bits on a rational
    tape, the interpreter's on configuration 2"""
    t = rational_problem(n=3, K=50, n_ineq=3)
    boxes, splits = ragged_batch(t, 29, seed=19)
    with ivb.Problem(t, specialize=3, seg_outline=0, recompute=recompute, threads_per_subdomain=tpsub,
                     seg_chunk=40) as p:
        r = p.bound_nodes_ex(boxes, splits, want_hull=True)
    ref = oracle.bound_nodes(t, boxes, splits, grad_mode="adjoint", tight=True)
    for k in ("lb", "ub", "minlo", "maxhi"):
        assert np.array_equal(r[k], ref[k]), k
    t2 = W.config_tape(2)
    boxes, splits = ragged_batch(t2, 17, seed=6)
    a, b = bound_seg_and_interp(t2, boxes, splits, dict(seg_outline=0, recompute=recompute,
                                                        threads_per_subdomain=tpsub))
    for k in KEYS:
        assert same_bits(a[k], b[k]), k


def test_library_choice_times_the_interpreter_beside_the_specialised_kernel():
    """specialize = -1 on a large adjoint tape: the autotuner times the
    interpreter's launch shapes beside the segmented kernel's and keeps the
    faster; either way the bounds are the interpreter's bits, on the graph
    and on later calls"""
    t = W.config_tape(4)
    boxes = W.bisection_frontier(t.root_box, 4, seed=3)
    splits = np.tile(W.config_workload(4).splits, (4, 1)).astype(np.int32)
    with ivb.Problem(t, grad_mode="adjoint", specialize=0) as p:
        ref = p.bound_nodes_ex(boxes, splits, want_hull=True)
    with ivb.Problem(t, grad_mode="adjoint", specialize=-1) as p:
        assert p.get_specialization()["active"]
        r1 = p.bound_nodes_ex(boxes, splits, want_hull=True)
        tun = p.get_tuning()
        r2 = p.bound_nodes_ex(boxes, splits, want_hull=True)
    assert tun["kernel"] in (0, 2) and tun["candidates"] > 20
    for r in (r1, r2):
        for k in KEYS:
            assert same_bits(ref[k], r[k]), k
