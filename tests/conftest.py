import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running full-size case")


def read_golden(name):
    """Data lines of a golden fixture (comment lines start with '#')."""
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.rstrip("\n") for ln in fh if ln.strip() and not ln.lstrip().startswith("#")]


def ints(s):
    return tuple(int(x) for x in s.replace(" ", "").split(",") if x != "")


@pytest.fixture(scope="session")
def tl():
    """The CUDA library's Python binding (built in-tree on first use)."""
    from paper_1711_10912_gb300 import build as _build
    import paper_1711_10912_gb300 as tlmod
    _build.build()
    tlmod.load_library()
    return tlmod


@pytest.fixture(scope="session")
def cuda_dev():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    return torch.device("cuda:0")
