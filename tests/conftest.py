import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_addoption(parser):
    parser.addoption("--eig-fp32", action="store_true", default=False,
                     help="run the GPU tests with complex64 eigenproblems solved in float32 (NNE_OPT_EIG_FP64 = 0)")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libnne.so")


@pytest.fixture(autouse=True, scope="session")
def _eig_precision(request):
    if not request.config.getoption("--eig-fp32"):
        yield
        return
    from paper_2501_13237_gb300 import nne
    nne.set_option(nne.OPT_EIG_FP64, 0)
    yield
    nne.set_option(nne.OPT_EIG_FP64, 1)
