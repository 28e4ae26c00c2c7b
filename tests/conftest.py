import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def slab_oracle():
    import oracle
    from paper_2209_15445_gb300 import workloads as w
    return oracle.Oracle(w.slab_calorimeter())


@pytest.fixture(scope="session")
def barrel_oracle():
    import oracle
    from paper_2209_15445_gb300 import workloads as w
    return oracle.Oracle(w.barrel_calorimeter(), field_T=3.8)
