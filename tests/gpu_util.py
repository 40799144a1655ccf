"""Helpers for the GPU tests: oracle problems and library plans side by side."""
import functools

import numpy as np

import synth


def need_torch_cuda():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@functools.lru_cache(maxsize=None)
def oracle_problem(w):
    from oracle import apply as ap
    from oracle import ground_state as gs
    V = synth.potential(w)
    phi, mu, res, it = gs.ground_state(w, V, synth.initial_spinor(w), tol=1e-12)
    op = ap.Operator(w, phi, V, mu)
    return V, phi, mu, op


def make_plan(w, V, phi, mu=None, **kw):
    from paper_2506_08308_gb300 import bdg
    prm = bdg.params_from(w, mu=mu, **kw)
    return bdg.Plan(prm, V, phi)


def rel_l2(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
