"""The branch and bound around the GPU bounding path (ivb_bnb_solve) with
the host-side additions: constraint propagation of every child, and the
host overlapping the GPU (the next batch enqueued before the batch in flight
is absorbed). One batch at a time, the B&B with propagation follows the
oracle's B&B with propagation node for node on rational tapes; overlapped
runs search in a lagged order and must reach the gap with bounds that
bracket the same minimum."""
from __future__ import annotations

import math

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


def rational_problem(n=2, K=40, n_ineq=1, seed=99):
    return W.random_problem(n, K, n_ineq, W.OPS_RATIONAL, [[-3, 2]] * n, seed, "rational")


@pytest.mark.parametrize("seed,propagate", [(99, 0), (99, 3), (17, 2), (23, 4)])
def test_bnb_follows_oracle_trajectory_with_propagation(seed, propagate):
    """bit-exact bounds and bit-exact propagation give the same search: same
    bounded-node count and final bounds"""
    t = rational_problem(seed=seed)
    sp = np.array([6, 6], np.int32)
    ref = oracle.bnb(t, splits=sp, eps_abs=0.0, eps_rel=1e-4, grad_mode="adjoint", tight=True, max_nodes=400,
                     propagate=propagate)
    with ivb.Problem(t, grad_mode="adjoint", batched=0) as p:
        r = p.bnb_solve(t.root_box, splits=sp, batch=1, eps_abs=0.0, eps_rel=1e-4, max_nodes=400,
                        propagate=propagate)
    assert (r["nodes"], r["lb"], r["ub"], r["converged"]) == (ref["nodes"], ref["lb"], ref["ub"], ref["converged"])


@pytest.mark.parametrize("overlap,propagate", [(1, 0), (1, 3), (0, 3)])
def test_bnb_host_additions_bracket_the_minimum(overlap, propagate):
    """configuration 1 to absolute gap 1e-4 and the unit-disc problem
    (minimum -sqrt 2) to 1e-6, batched, with and without the additions"""
    wl = W.config_workload(1)
    t = wl.tape
    ref = oracle.bnb(t, splits=wl.splits, eps_abs=wl.gap_abs, eps_rel=0.0, grad_mode="adjoint", tight=True,
                     max_nodes=100000)
    with ivb.Problem(t, grad_mode="adjoint", batched=1) as p:
        r = p.bnb_solve(t.root_box, splits=wl.splits, batch=8, eps_abs=wl.gap_abs, eps_rel=0.0, max_nodes=100000,
                        overlap=overlap, propagate=propagate)
    assert r["converged"] and r["ub"] - r["lb"] <= wl.gap_abs
    assert r["lb"] <= ref["ub"] and ref["lb"] <= r["ub"]
    t = P.constrained_toy("feasible")
    with ivb.Problem(t, grad_mode="adjoint", batched=1) as p:
        r = p.bnb_solve(t.root_box, splits=[6, 6], batch=4, eps_abs=1e-6, eps_rel=0.0, max_nodes=100000,
                        overlap=overlap, propagate=propagate)
    assert r["converged"] and r["lb"] - 1e-12 <= -math.sqrt(2.0) <= r["ub"] + 1e-12


def test_bnb_infeasible_problem_and_stream():
    """a problem without feasible points ends at once with lb = ub = +inf;
    a caller's stream is honoured"""
    t = P.constrained_toy("infeasible")
    s = torch.cuda.Stream()
    with ivb.Problem(t) as p:
        r = p.bnb_solve(t.root_box, splits=[4, 4], batch=2, eps_abs=1e-6, eps_rel=0.0, propagate=2, overlap=1,
                        stream=s.cuda_stream)
        assert r["converged"] and r["lb"] == math.inf and r["ub"] == math.inf and r["nodes"] == 0
        r = p.bnb_solve(t.root_box, splits=[4, 4], batch=2, eps_abs=1e-6, eps_rel=0.0, overlap=1)
        assert r["converged"] and r["ub"] == math.inf


def test_bnb_config2_overlap_propagation_specialised():
    """configuration 2 to relative gap 1e-3 with everything on: brackets the
    plain synchronous run's minimum"""
    wl = W.config_workload(2)
    t = wl.tape
    with ivb.Problem(t, grad_mode="adjoint", batched=1) as p:
        a = p.bnb_solve(t.root_box, splits=wl.splits, batch=32, eps_abs=0.0, eps_rel=wl.gap_rel, time_limit=60)
    with ivb.Problem(t, grad_mode="adjoint", batched=1, specialize=1) as p:
        b = p.bnb_solve(t.root_box, splits=wl.splits, batch=32, eps_abs=0.0, eps_rel=wl.gap_rel, time_limit=60,
                        propagate=3, overlap=1)
    assert a["converged"] and b["converged"]
    assert b["lb"] <= a["ub"] and a["lb"] <= b["ub"]
    assert b["ub"] - b["lb"] <= wl.gap_rel * abs(b["ub"]) * (1 + 1e-12)


@pytest.mark.parametrize("grad_mode", ["forward", "adjoint"])
def test_bnb_plain_path_with_host_additions(grad_mode):
    """one launch per node (batched = 0) with propagation and overlap:
    converges on the unit-disc problem and brackets -sqrt 2"""
    t = P.constrained_toy("feasible")
    with ivb.Problem(t, grad_mode=grad_mode, batched=0) as p:
        r = p.bnb_solve(t.root_box, splits=[6, 6], batch=3, eps_abs=1e-6, eps_rel=0.0, max_nodes=100000,
                        overlap=1, propagate=2)
    assert r["converged"] and r["lb"] - 1e-12 <= -math.sqrt(2.0) <= r["ub"] + 1e-12


def test_bnb_rejects_bad_arguments():
    t = P.constrained_toy("feasible")
    with ivb.Problem(t, max_nodes=8) as p:
        with pytest.raises(ivb.IvbError) as e:
            p.bnb_solve(t.root_box, splits=[6, 6], batch=16)      # 2 * batch > max_nodes
        assert e.value.status == ivb.IVB_EINVAL and "max_nodes" in str(e.value)
        with pytest.raises(ivb.IvbError):
            p.bnb_solve(t.root_box, splits=[6, 6], batch=2, propagate=-1)
