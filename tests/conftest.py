import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test (still part of the default run)")


# Observed worst per-component error of the FP32 pair sums, in units of
# 2^-24 B (B = the oracle's magnitude sum), per mixed-precision mobility test;
# printed at the end of the run beside the bound the tests assert.
MIXED_MAX_C = {}


def pytest_terminal_summary(terminalreporter):
    if MIXED_MAX_C:
        terminalreporter.write_line("observed max c of the FP32 pair sums (bound 144):")
        for name, c in sorted(MIXED_MAX_C.items()):
            terminalreporter.write_line("  %-70s %.2f" % (name, c))
