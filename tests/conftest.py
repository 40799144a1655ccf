"""Shared fixtures.  GPU tests carry @pytest.mark.gpu; everything else runs on
the CPU.  Ground states come from the oracle's gradient flow and are cached
per session."""
import functools
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@functools.lru_cache(maxsize=None)
def _ground(w):
    from oracle import ground_state as gs
    V = synth.potential(w)
    phi, mu, res, it = gs.ground_state(w, V, synth.initial_spinor(w), tol=1e-12)
    assert res <= 1e-11, (w.name, res)
    return V, phi, mu


@pytest.fixture(scope="session")
def ground():
    """ground(w) -> (V, phi, mu) from the oracle flow, cached."""
    return _ground


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
