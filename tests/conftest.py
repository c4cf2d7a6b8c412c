import functools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def read_golden(name):
    """key = value lines of tests/golden/<name>; '#' starts a comment."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = line.split("=", 1)
            out[k.strip()] = v.strip()
    return out


@functools.lru_cache(maxsize=1)
def c3_walk():
    """The 1 Mbp confined self-avoiding walk of the throughput benchmark,
    built once per test session (about a minute of host time)."""
    from paper_1608_03722_gb300 import inputs as I
    return I.c3_walk()
