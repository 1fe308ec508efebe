import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built ivb library")


# largest distance (in representable steps) between a GPU enclosure end and the
# oracle's tight end, per parity check with exp/log (filled by the GPU tests)
ULP_LOG: dict = {}


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    if ULP_LOG:
        terminalreporter.section("exp/log parity: largest end distance from the oracle's tight enclosure (steps)")
        for k in sorted(ULP_LOG):
            terminalreporter.write_line(f"{k}: {ULP_LOG[k]}")
