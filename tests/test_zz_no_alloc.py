"""The allocation-free entry point ivb_bound_nodes_noalloc, for callers that
cannot allocate device memory while they run: through the C ABI, its results
must equal those of the regular ivb_bound_nodes on the same inputs, on two
calls in a row (the fixed scratch keeps the previous call's contents, so the
second call checks that everything that must be reset is reset). It rejects
batches beyond its fixed capacity, empty batches and host arrays in the C code
itself, and the Python wrapper rejects wrong dtypes and short outputs before
any device memory is touched."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2507_20769_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2507_20769_gb300 import build as B  # noqa: E402

B.build()
from paper_2507_20769_gb300 import ivb  # noqa: E402

DEV = torch.device("cuda:0")


def _batch(t, n_nodes, seed):
    rng = np.random.default_rng(seed)
    boxes = W.bisection_frontier(t.root_box, n_nodes, seed=seed)
    splits = rng.integers(1, 7, (n_nodes, t.n_vars)).astype(np.int32)
    splits[0] = 1
    return boxes, splits


@pytest.mark.parametrize("which", ["rational", "config2"])
@pytest.mark.parametrize("grad_mode", ["adjoint", "forward"])
def test_noalloc_matches_regular_entry_point_on_two_calls(which, grad_mode):
    if which == "rational":
        t = W.random_problem(3, 60, 2, W.OPS_RATIONAL, [[-3, 2]] * 3, 777, "rational")
    else:
        t = W.config_tape(2)
    with ivb.Problem(t, grad_mode=grad_mode) as p:
        for call, (n_nodes, seed) in enumerate(((37, 11), (23, 5))):
            boxes, splits = _batch(t, n_nodes, seed)
            lb_ref, inf_ref = p.bound_nodes(boxes, splits)
            bd = torch.from_numpy(boxes).to(DEV)
            sd = torch.from_numpy(splits).to(DEV)
            lb = torch.full((n_nodes,), float("nan"), dtype=torch.float64, device=DEV)
            inf = torch.full((n_nodes,), 7, dtype=torch.uint8, device=DEV)
            p.ivb_bound_nodes_noalloc(bd, sd, lb, inf)
            torch.cuda.synchronize()
            assert np.array_equal(lb.cpu().numpy(), lb_ref), f"call {call}"
            assert np.array_equal(inf.cpu().numpy(), inf_ref), f"call {call}"


def test_noalloc_rejects_what_it_cannot_hold():
    t = W.config_tape(1)
    with ivb.Problem(t) as p:
        n = ivb.lib().ivb_bound_nodes_noalloc  # noqa: F841  (symbol present)
        big = 257
        bd = torch.tensor(np.array([t.root_box] * big), device=DEV)
        sd = torch.ones((big, t.n_vars), dtype=torch.int32, device=DEV)
        lb = torch.empty(big, dtype=torch.float64, device=DEV)
        inf = torch.empty(big, dtype=torch.uint8, device=DEV)
        with pytest.raises(ivb.IvbError) as e:
            p.ivb_bound_nodes_noalloc(bd, sd, lb, inf)
        assert e.value.status == ivb.IVB_EINVAL and "256" in str(e.value)
        # an invalid box is found on the device and named
        bd2 = bd[:4].clone()
        bd2[2, 0, 0] = 5.0
        with pytest.raises(ivb.IvbError) as e:
            p.ivb_bound_nodes_noalloc(bd2, sd[:4].contiguous(), lb[:4], inf[:4])
        assert e.value.status == ivb.IVB_EINVAL and "node 2" in str(e.value)
        # and the entry point still works afterwards
        p.ivb_bound_nodes_noalloc(bd[:4].contiguous(), sd[:4].contiguous(), lb[:4], inf[:4])
        ref, _ = p.bound_nodes(np.array([t.root_box] * 4), np.ones((4, t.n_vars), np.int32))
        assert np.array_equal(lb[:4].cpu().numpy(), ref)


def test_noalloc_c_entry_rejects_host_arrays_and_empty_batches():
    """called directly through ctypes, so the C-side checks are what answers"""
    t = W.config_tape(1)
    with ivb.Problem(t) as p:
        f = ivb.lib().ivb_bound_nodes_noalloc
        boxes = np.ascontiguousarray(np.array([t.root_box] * 4))
        splits = np.ones((4, t.n_vars), np.int32)
        lb_d = torch.empty(4, dtype=torch.float64, device=DEV)
        inf_d = torch.empty(4, dtype=torch.uint8, device=DEV)
        bd = torch.from_numpy(boxes).to(DEV)
        sd = torch.from_numpy(splits).to(DEV)
        vp = ctypes.c_void_p
        # host boxes and splits (numpy pointers)
        st = f(p._h, 4, vp(boxes.ctypes.data), vp(splits.ctypes.data), vp(lb_d.data_ptr()),
               vp(inf_d.data_ptr()), None)
        assert st == ivb.IVB_EINVAL and "device memory" in ivb.lib().ivb_last_error(p._h).decode()
        # host output
        lb_h = np.empty(4)
        st = f(p._h, 4, vp(bd.data_ptr()), vp(sd.data_ptr()), vp(lb_h.ctypes.data), vp(inf_d.data_ptr()), None)
        assert st == ivb.IVB_EINVAL and "device memory" in ivb.lib().ivb_last_error(p._h).decode()
        # empty batch
        st = f(p._h, 0, vp(bd.data_ptr()), vp(sd.data_ptr()), vp(lb_d.data_ptr()), vp(inf_d.data_ptr()), None)
        assert st == ivb.IVB_EINVAL and "n_nodes" in ivb.lib().ivb_last_error(p._h).decode()
        # the entry point still works afterwards
        stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
        st = f(p._h, 4, vp(bd.data_ptr()), vp(sd.data_ptr()), vp(lb_d.data_ptr()), vp(inf_d.data_ptr()), stream)
        assert st == ivb.IVB_OK
        ref, _ = p.bound_nodes(boxes, splits)
        assert np.array_equal(lb_d.cpu().numpy(), ref)


def test_noalloc_wrapper_rejects_wrong_dtypes_and_short_outputs():
    t = W.config_tape(1)
    with ivb.Problem(t) as p:
        bd = torch.tensor(np.array([t.root_box] * 4), device=DEV)
        sd = torch.ones((4, t.n_vars), dtype=torch.int32, device=DEV)
        lb = torch.empty(4, dtype=torch.float64, device=DEV)
        inf = torch.empty(4, dtype=torch.uint8, device=DEV)
        with pytest.raises(TypeError):
            p.ivb_bound_nodes_noalloc(bd.float(), sd, lb, inf)
        with pytest.raises(TypeError):
            p.ivb_bound_nodes_noalloc(bd, sd, lb.float(), inf)
        with pytest.raises(TypeError):
            p.ivb_bound_nodes_noalloc(bd, sd.long(), lb, inf)
        with pytest.raises(ValueError):
            p.ivb_bound_nodes_noalloc(bd, sd, lb[:3], inf)
        with pytest.raises(ValueError):
            p.ivb_bound_nodes_noalloc(bd, sd, lb, inf[:2])
        with pytest.raises(ValueError):
            p.ivb_bound_nodes_noalloc(bd, sd[:, :1].contiguous(), lb, inf)
        with pytest.raises(ValueError):
            p.ivb_bound_nodes_noalloc(bd[:, :1].contiguous(), sd, lb, inf)
