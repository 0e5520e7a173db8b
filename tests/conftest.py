import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


_SOLIDS = {}


def solid(name, **kw):
    """Session cache of seeded model solids (dense diagonalisation is not free)."""
    from synth import SPECS, build_model_solid
    key = (name, tuple(sorted(kw.items())))
    if key not in _SOLIDS:
        _SOLIDS[key] = build_model_solid(SPECS[name], **kw)
    return _SOLIDS[key]
