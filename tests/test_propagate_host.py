"""Constraint propagation on the host (ivb_propagate, part of the CUDA
library's B&B, no GPU needed) against the oracle's independent
implementation: bit for bit on rational tapes (both round every endpoint
operation correctly), containment of the oracle's tight result on tapes with
exp and log (the library widens the C library's exp/log by two ulps)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import problems as P
from paper_2507_20769_gb300 import build as B
from paper_2507_20769_gb300 import workloads as W


@pytest.fixture(scope="module")
def ivb():
    B.build()
    from paper_2507_20769_gb300 import ivb as m
    return m


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("ub", [np.inf, "median"])
def test_propagation_bit_exact_rational(ivb, seed, ub):
    t = W.random_problem(3 + seed % 3, 60, 2, W.OPS_RATIONAL, [[-3, 2]] * (3 + seed % 3), 500 + seed, "rational")
    boxes = W.bisection_frontier(t.root_box, 150, seed=seed)
    if ub == "median":
        c = 0.5 * (boxes[:, :, 0] + boxes[:, :, 1])
        ub = float(np.median(P.np_eval(t, c)[:, 0]))
    bo, io = oracle.propagate(t, boxes, ub=ub, passes=4)
    bh, ih = ivb.ivb_propagate(t, boxes, ub=ub, passes=4)
    assert np.array_equal(io, ih)
    assert np.array_equal(bo[~io], bh[~ih])
    if np.isfinite(ub):   # the objective cut always removes something
        assert io.sum() + (bo != boxes).any(axis=(1, 2)).sum() > 0


@pytest.mark.parametrize("config", [1, 2, 3])
def test_propagation_contains_oracle_with_exp_log(ivb, config):
    t = W.config_tape(config)
    boxes = W.bisection_frontier(t.root_box, 60, seed=config)
    bo, io = oracle.propagate(t, boxes, passes=3, tight=True)
    bh, ih = ivb.ivb_propagate(t, boxes, passes=3)
    # the library's result is never tighter than the tight oracle's
    assert not np.any(ih & ~io)
    keep = ~ih
    assert np.all(bh[keep, :, 0] <= bo[keep, :, 0]) and np.all(bh[keep, :, 1] >= bo[keep, :, 1])
    # and never wider than the input
    assert np.all(bh[:, :, 0] >= boxes[:, :, 0]) and np.all(bh[:, :, 1] <= boxes[:, :, 1])


def test_propagation_rejects_bad_input(ivb):
    t = P.constrained_toy("feasible")
    bad = P.constrained_toy("feasible")
    bad.a = np.array(bad.a)
    bad.a[3] = 50
    with pytest.raises(ivb.IvbError) as e:
        ivb.ivb_propagate(bad, t.root_box)
    assert e.value.status == ivb.IVB_ETAPE
    out, inf = ivb.ivb_propagate(t, np.zeros((0, 2, 2)))
    assert out.shape == (0, 2, 2) and inf.shape == (0,)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
def test_host_gradient_bit_exact_rational(ivb, seed, grad_mode):
    """the host gradient behind the B&B's descent corner (ivb_host_gradient)
    equals the oracle's gradient enclosure over the same box bit for bit on
    rational tapes, fused accumulation included, for every output"""
    n = 3 + seed % 3
    t = W.random_problem(n, 60, 2, W.OPS_RATIONAL, [[-3, 2]] * n, 700 + seed, "rational")
    boxes = W.bisection_frontier(t.root_box, 40, seed=seed)
    ones = np.ones(n, np.int32)
    for box in boxes:
        _, _, Go = oracle.enclose(t, box, ones, grad_mode=grad_mode, want_g=True)
        for o in range(t.n_out):
            Gh = ivb.ivb_host_gradient(t, box, o, grad_mode)
            assert np.array_equal(Gh, Go[0, o]), (o, Gh, Go[0, o])


@pytest.mark.parametrize("config", [1, 2])
def test_host_gradient_contains_oracle_with_exp_log(ivb, config):
    """with exp and log the host widens the C library's values by two ulps, so
    its gradient enclosures contain the oracle's tight ones"""
    t = W.config_tape(config)
    boxes = W.bisection_frontier(t.root_box, 24, seed=config)
    ones = np.ones(t.n_vars, np.int32)
    for grad_mode in ("forward", "adjoint"):
        for box in boxes:
            _, _, Go = oracle.enclose(t, box, ones, grad_mode=grad_mode, want_g=True)
            for o in range(t.n_out):
                Gh = ivb.ivb_host_gradient(t, box, o, grad_mode)
                assert np.all(Gh[:, 0] <= Go[0, o, :, 0]) and np.all(Gh[:, 1] >= Go[0, o, :, 1])


def test_host_gradient_rejects_bad_arguments(ivb):
    t = W.config_tape(1)
    with pytest.raises(ivb.IvbError):
        ivb.ivb_host_gradient(t, t.root_box, t.n_out, "adjoint")
