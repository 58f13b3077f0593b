import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libdupin.so")
    config.addinivalue_line("markers", "slow: large inputs (minutes on the CPU)")


@pytest.fixture(scope="session", autouse=True)
def _built_host_libs():
    """Compile the input generator and the oracle (plain gcc, seconds)."""
    from paper_2504_09311_gb300 import synth
    import oracle

    synth.build()
    oracle.build()
    yield
