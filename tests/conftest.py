import os
import sys

# single-threaded BLAS: the oracle issues many tiny products where thread start-up dominates
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import pytest  # noqa: E402


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libhmsolve.so")
    config.addinivalue_line("markers", "slow: large problem sizes")


@pytest.fixture(scope="session")
def sphere480():
    import efie_problem as ep
    return ep.build("sphere480")


@pytest.fixture(scope="session")
def sphere1920():
    import efie_problem as ep
    return ep.build("sphere1920")


@pytest.fixture(scope="session")
def sphere7680():
    import efie_problem as ep
    return ep.build("sphere7680")


@pytest.fixture(scope="session")
def sphere30720():
    import efie_problem as ep
    return ep.build("sphere30720")
