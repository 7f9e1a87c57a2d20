import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def read_golden(name):
    """Rows of a whitespace-separated golden fixture (comments skipped)."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture
def golden():
    return read_golden


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def lsq():
    """The CUDA library binding (built on first use); skips without a GPU."""
    if not _cuda_ok():
        pytest.skip("needs a CUDA GPU")
    import importlib.util
    path = os.path.join(ROOT, "paper_2410_06319_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("lsq_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import paper_2410_06319_gb300 as lib
    return lib


@pytest.fixture(scope="session")
def handle(lsq):
    h = lsq.Handle()
    yield h
    h.close()


def dev(a):
    """numpy -> contiguous CUDA float64 tensor."""
    import numpy as np
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def colmajor(Y):
    """s x k numpy matrix -> flat column-major numpy vector (ld = s)."""
    import numpy as np
    return np.ascontiguousarray(np.asarray(Y).T).ravel()


def from_colmajor(t, rows, cols):
    return t.cpu().numpy().reshape(cols, rows).T
