import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def read_golden(name):
    """Rows of a golden fixture: non-comment lines split on whitespace."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


_SYSTEMS = {}


def oracle_system(dims, n_scales, shear_levels, full_system=False):
    """Session cache of oracle filter systems (building one can take seconds)."""
    from oracle import shearlet_oracle as O
    key = (tuple(dims), int(n_scales), tuple(shear_levels), bool(full_system))
    if key not in _SYSTEMS:
        _SYSTEMS[key] = O.build_system(dims, n_scales, shear_levels, full_system)
    return _SYSTEMS[key]


@pytest.fixture
def golden():
    return read_golden
