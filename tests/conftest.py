import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: full-size workloads")


def read_golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, _cite = line.split(" ", 2)
            out[name] = float(value)
    return out


@pytest.fixture(scope="session")
def paper_constants():
    return read_golden_constants()


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library, loaded through its Python binding; GPU tests only."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1803_08601_gb300 as pkg

    pkg.load()
    return pkg
