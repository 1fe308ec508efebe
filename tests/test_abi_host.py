"""CPU-only checks of the C-ABI library: it loads, exports every entry point
that include/ivb.h declares, and its host-side logic (tape validation, split
pickers) behaves as specified. No kernel is launched."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import problems as P
from paper_2507_20769_gb300 import build as B
from paper_2507_20769_gb300 import ivb
from paper_2507_20769_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ivb.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ivb.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ivb_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_struct_sizes_match_header(lib):
    assert W.IVB_OP_DTYPE.itemsize == 24
    assert ctypes.sizeof(ivb.ivb_options) == 20 * 4
    assert ctypes.sizeof(ivb.ivb_tuning) == 11 * 4
    o = ivb.ivb_options_default()
    assert (o.grad_mode, o.form, o.batched, o.use_graph, o.max_nodes, o.specialize, o.emulate) == (1, 0, 1, 1, 4096, 0, -1)
    assert (o.recompute, o.seg_chunk, o.seg_regs, o.threads_per_subdomain, o.seg_sync, o.seg_ilp,
            o.seg_outline) == (-1, 0, 0, 0, -1, 0, -1)


def _raw_create(tape_like):
    recs, oi, ok, n = tape_like
    t = ivb.ivb_tape(n, recs.shape[0], oi.shape[0], recs.ctypes.data, oi.ctypes.data, ok.ctypes.data)
    h = ctypes.c_void_p()
    st = ivb.lib().ivb_create_problem(ctypes.byref(t), None, ctypes.byref(h))
    return st, ivb.lib().ivb_last_error(None).decode()


def _tape_arrays(t):
    return (t.records(), np.ascontiguousarray(t.out_idx, np.int32), np.ascontiguousarray(t.out_kind, np.uint8),
            t.n_vars)


@pytest.mark.parametrize("breakage,fragment", [
    ("forward_ref", "earlier entry"),
    ("bad_op", "unknown opcode"),
    ("var_range", "VAR index"),
    ("nan_const", "not finite"),
    ("two_obj", "exactly one objective"),
    ("out_range", "output index"),
])
def test_invalid_tapes_rejected_before_any_device_work(lib, breakage, fragment):
    t = P.constrained_toy("feasible")
    recs, oi, ok, n = _tape_arrays(t)
    recs = recs.copy(); oi = oi.copy(); ok = ok.copy()
    if breakage == "forward_ref":
        recs["a"][5] = 7
    elif breakage == "bad_op":
        recs["op"][3] = 42
    elif breakage == "var_range":
        recs["a"][1] = 5
    elif breakage == "nan_const":
        i = int(np.nonzero(recs["op"] == W.OP_CONST)[0][0])
        recs["c"][i] = np.nan
    elif breakage == "two_obj":
        ok[1] = W.KIND_OBJ
    elif breakage == "out_range":
        oi[0] = recs.shape[0]
    st, msg = _raw_create((recs, oi, ok, n))
    assert st == ivb.IVB_ETAPE and fragment in msg


def test_pick_splits_matches_oracle_and_worked_examples(lib):
    assert ivb.ivb_pick_splits([[0, 1]] * 5, 2560, "adaptive").tolist() == [5, 5, 5, 5, 4]
    assert ivb.ivb_pick_splits([[0, 1]] * 5, 2560, "uniform").tolist() == [4] * 5
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = int(rng.integers(1, 7))
        lo = rng.uniform(-5, 5, n)
        box = np.stack([lo, lo + 10.0 ** rng.uniform(-3, 1, n)], 1)
        ref = 10.0 ** rng.uniform(-1, 1, n)
        target = int(2 ** rng.integers(0, 21))
        for s in ("uniform", "largest", "adaptive"):
            a = ivb.ivb_pick_splits(box, target, s, ref)
            b = oracle.pick_splits(box, target, s, ref)
            assert a.tolist() == b.tolist()
            assert int(np.prod(a.astype(np.int64))) <= target


def test_pick_splits_rejects_bad_arguments(lib):
    with pytest.raises(ivb.IvbError):
        ivb.ivb_pick_splits([[0, 1]], 0, "uniform")
