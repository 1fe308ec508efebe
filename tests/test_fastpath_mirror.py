"""Host model of the kernels' directed-primitive fast paths (tests/mirror/
fastpath_mirror.c), compiled with gcc and run on the CPU: the integer-pipe
remainder signs and seed residuals of reciprocal, division and square root
give the correctly rounded directed results (fesetround) on every operand,
exact quotients and squares included; exp's and log's error before the final
rounding stays inside what the two-step outward widening covers (0.75 ulp
where the rounded result is a power of two, 1.5 ulp elsewhere) and no widened
result misses the binary128 value. The GPU tests check the device code itself
against the oracle; this checks the error analysis it rests on."""
from __future__ import annotations

import os
import platform
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mirror", "fastpath_mirror.c")


@pytest.fixture(scope="module")
def mirror(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    exe = str(tmp_path_factory.mktemp("mirror") / "fastpath_mirror")
    cmd = ["gcc", "-O2", "-std=gnu11", "-frounding-math", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wno-unknown-pragmas", SRC, "-o", exe, "-lm"]
    if platform.machine() in ("x86_64", "AMD64", "i686"):
        cmd.insert(-1, "-lquadmath")
    subprocess.run(cmd, check=True)

    def run(mode: str, n: int) -> dict:
        out = subprocess.run([exe, mode, str(n)], check=True, capture_output=True, text=True).stdout
        return {k: float(v) for k, v in (kv.split("=") for kv in out.split())}
    return run


@pytest.mark.parametrize("mode", ["rcp", "div", "sqrt"])
def test_integer_remainders_give_correctly_rounded_results(mirror, mode):
    r = mirror(mode, 1_000_000)
    assert r["fast"] > 700_000
    assert r["wrong"] == 0 and r["sign_bad"] == 0 and r["shift_bad"] == 0
    if mode != "rcp":
        assert r["exact"] > 10_000            # zero remainders were exercised


@pytest.mark.parametrize("mode,bound", [("exp", 0.3), ("log", 1.0)])
def test_exp_log_error_inside_the_widening(mirror, mode, bound):
    r = mirror(mode, 400_000)
    assert r["inputs"] > 390_000
    assert r["missed"] == 0
    assert r["worst_ulp"] < bound < 1.5
    assert r["worst_ulp_pow2"] < 0.75
