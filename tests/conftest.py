import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (runs the CUDA library through its C ABI)")
    config.addinivalue_line(
        "markers", "slow: larger CPU cases (still minutes at most)")


@pytest.fixture(scope="session")
def many_criteria_full():
    """The 64 bitmaps over 2^26 rows of the many-criteria workload (drawn
    once per session, in a spawned process pool)."""
    import synth
    words, _ = synth.many_criteria(0, synth.MANY_N, synth.MANY_R, workers=8)
    return words, synth.MANY_R
