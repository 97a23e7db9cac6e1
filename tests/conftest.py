import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def oracle_default():
    from oracle import vdw
    return vdw.Oracle(vdw.Params())


@pytest.fixture(scope="session")
def oracle_linear():
    from oracle import vdw
    p = vdw.Params(interp="linear")
    phik, _ = vdw.kernel_table(vdw.Params())
    return vdw.Oracle(p, phik=phik)
