import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def tq():
    """The C-ABI binding with the library loaded; GPU tests only."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2404_13184_gb300 import binding
    binding.load()
    return binding


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="session")
def golden():
    """Load a text fixture from tests/golden: '#' lines are comments (each file
    cites its source), numbers are whitespace separated; a '# complex' line
    means each row holds interleaved (re, im) pairs."""
    import numpy as np

    def load(name):
        path = os.path.join(GOLDEN, name)
        is_complex = False
        rows = []
        with open(path) as f:
            for line in f:
                s = line.strip()
                if s.startswith("#"):
                    if s.lower().startswith("# complex"):
                        is_complex = True
                    continue
                if s:
                    rows.append([float(v) for v in s.split()])
        a = np.array(rows)
        if is_complex:
            a = a[:, 0::2] + 1j * a[:, 1::2]
        return a
    return load
