import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def target():
    """One libsx target on cuda:0 with its own stream, shared by the GPU tests."""
    import paper_2206_06302_b300 as sx
    t = sx.sx_target_create(0)
    yield t
    sx.sx_target_destroy(t)


@pytest.fixture(scope="session")
def executor(target):
    import paper_2206_06302_b300 as sx
    e = sx.sx_executor_create(target, sx.SX_PAR)
    yield e
    sx.sx_executor_destroy(e)
