"""The tape-specialised kernels compile (NVRTC for sm_103a, on the CPU: no
GPU is needed to generate and compile them) for tapes that use every
operation, in both gradient modes, within the 128-register budget of their
launch bounds; invalid tapes are rejected before any code is generated."""
from __future__ import annotations

import numpy as np
import pytest

import problems as P
from paper_2507_20769_gb300 import build as B
from paper_2507_20769_gb300 import workloads as W


@pytest.fixture(scope="module")
def ivb():
    B.build()
    from paper_2507_20769_gb300 import ivb as m
    return m


def every_op_tape():
    """all eleven opcodes, outputs that are a variable and a constant entry"""
    Bd = P.Builder(3)
    x0, x1, x2 = Bd.x(0), Bd.x(1), Bd.x(2)
    a = Bd.add(Bd.mul(x0, x1), Bd.div(x2, Bd.add(Bd.sqr(x1), Bd.const(1.5))))
    b = Bd.sub(Bd.exp(Bd.mul(Bd.const(0.25), x0)), Bd.log(Bd.add(Bd.sqr(x2), Bd.const(2.0))))
    c = Bd.sqrt(Bd.add(Bd.sqr(a), Bd.const(0.5)))
    Bd.output(Bd.add(Bd.neg(b), c), P.KIND_OBJ)
    Bd.output(Bd.sub(a, Bd.const(1.0)), P.KIND_INEQ)
    Bd.output(x1, P.KIND_EQ)
    Bd.output(Bd.const(-1.0), P.KIND_INEQ)
    return Bd.tape([[-1.0, 1.0]] * 3, "every op")


@pytest.mark.parametrize("grad_mode", ["adjoint", "forward"])
@pytest.mark.parametrize("which", ["every_op", "config1"])
@pytest.mark.parametrize("compact", [False, True])
def test_specialized_kernel_compiles(ivb, which, grad_mode, compact):
    t = every_op_tape() if which == "every_op" else W.config_tape(1)
    r = ivb.ivb_specialize_compile(t, grad_mode, compact)
    assert 0 < r["registers"] <= 128
    assert r["spill_bytes"] >= 0 and r["seconds"] > 0


def test_specialize_compile_rejects_invalid_tape(ivb):
    t = every_op_tape()
    t.a = np.array(t.a)
    t.a[3] = 40          # the first product refers to a later entry
    with pytest.raises(ivb.IvbError) as e:
        ivb.ivb_specialize_compile(t, "adjoint")
    assert e.value.status == ivb.IVB_ETAPE


@pytest.mark.parametrize("variant", [3, 4])
@pytest.mark.parametrize("which", ["every_op", "config2"])
def test_segmented_kernel_compiles(ivb, which, variant):
    """the segmented kernel (specialize = 3; variant 4: two subdomains per
    thread in the paired dual-pipe form): chunk functions compiled in
    parallel as relocatable programs and linked, within the register budget"""
    t = every_op_tape() if which == "every_op" else W.config_tape(2)
    r = ivb.ivb_specialize_compile(t, "adjoint", variant=variant)
    assert 0 < r["registers"] <= 128
    assert r["spill_bytes"] >= 0 and r["seconds"] > 0
    with pytest.raises(ivb.IvbError) as e:
        ivb.ivb_specialize_compile(t, "forward", variant=variant)
    assert e.value.status == ivb.IVB_EINVAL
