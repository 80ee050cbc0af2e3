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
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session", autouse=True)
def _cpu_libs():
    """Build the CPU-side libraries (oracle, generator host part) once."""
    import lobgen
    import oracle
    lobgen.build(cuda=False)
    oracle.build()
    yield
