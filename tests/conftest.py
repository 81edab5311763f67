import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def tiny():
    import synth
    return synth.config_tiny()


@pytest.fixture(scope="session", autouse=True)
def _built():
    """Compile the CUDA library, the oracle and the input generator if stale."""
    from paper_2608_06853_b300 import build as b
    import oracle
    import synth
    b.build()
    oracle.build()
    synth.build()
    synth.build_gpu()
