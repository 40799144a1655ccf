"""Parity of bdg_solve at the size the benchmark times: the 2-D instance on a
256^2 grid (box [-12, 12)^2, beta_n = 100, beta_s = -2, q = 0.1), the 32
smallest excitations with a block of m = 48 (eq. lrep-d), FP64 and mixed
precision, against values written by tests/golden/make_solve_2d_n256.py from
the CPU oracle alone (its eigenvalues, and its ground state, from which the
oracle operator of the test is built).  A 32^2 grid of the same physics, solved with the same
k and m, is compared with the oracle's dense solution as well.

Checks per solve:
  - every pair's relative residual |M x - omega x| / (|omega| |x|)
    (reading P9) recomputed with the oracle's FFT product is at the 1e-10
    tolerance (to 10 %: the device and numpy FFTs round differently);
  - the normalization and bi-orthogonality h^d (u_i.u_j - v_i.v_j) = delta_ij
    (eq. constrain, Theorem "Biorthogonality") to 1e-8;
  - the eigenvalues against the oracle's to 1e-10 relative.
"""
import json
import os

import numpy as np
import pytest

import synth
from gpu_util import make_plan, need_torch_cuda, oracle_problem

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
W = synth.W2D_N256
W32 = synth.small(synth.W2D_N256, 32)


def _oracle_2d_n256(gold):
    """The oracle's operator of the instance from the oracle's stored ground
    state; its chemical potentials must be the recorded ones."""
    from oracle import apply as ap
    from oracle import spin1
    phi = np.load(os.path.join(HERE, "golden", "phi_2d_n256.npz"))["phi"]
    V = synth.potential(W)
    mu = spin1.chemical_potentials(phi, spin1.hamiltonian(phi, V, W, W.beta_n, W.beta_s, W.p, W.q))
    np.testing.assert_allclose(mu, gold["mu"], rtol=1e-10)
    return V, phi, mu, ap.Operator(W, phi, V, mu)


def _checks(w, op, om, UV, om_ref):
    from oracle import lrep
    k = w.k
    uv = UV[:k].cpu().numpy().real
    r = lrep.residual_uv(op, uv, om[:k])
    assert r.max() <= 1.1e-10, r
    U = uv[:, :3].reshape(k, -1)
    V = uv[:, 3:].reshape(k, -1)
    gram = lrep.weight(w) * (U @ U.T - V @ V.T)
    assert np.abs(gram - np.eye(k)).max() < 1e-8, np.abs(gram - np.eye(k)).max()
    np.testing.assert_allclose(om[:k], om_ref[:k], rtol=1e-10, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_2d_n256_against_oracle(prec):
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    with open(os.path.join(HERE, "golden", "solve_2d_n256.json")) as fh:
        gold = json.load(fh)
    V, phi, mu, op = _oracle_2d_n256(gold)
    plan = make_plan(W, V, phi, prec=bdg.FP64 if prec == "fp64" else bdg.MIXED, tol=1e-10, maxit=600)
    X0 = torch.from_numpy(synth.random_block(W, W.m, complex_=True)).cuda()
    om, UV, resid, nconv = plan.solve(W.k, W.m, X0=X0)
    plan.close()
    assert nconv == W.k and np.all(resid <= 1e-10), resid
    _checks(W, op, om, UV, np.array(gold["omega"]))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_2d_n32_block48_against_dense(prec):
    torch = need_torch_cuda()
    from oracle import lrep
    from paper_2506_08308_gb300 import bdg
    V, phi, mu, op = oracle_problem(W32)
    om_d, _, _ = lrep.dense_solve_fg(op, W32.k + 6)
    plan = make_plan(W32, V, phi, prec=bdg.FP64 if prec == "fp64" else bdg.MIXED, tol=1e-10, maxit=600)
    X0 = torch.from_numpy(synth.random_block(W32, W32.m, complex_=True)).cuda()
    om, UV, resid, nconv = plan.solve(W32.k, W32.m, X0=X0)
    plan.close()
    assert nconv == W32.k and np.all(resid <= 1e-10), resid
    _checks(W32, op, om, UV, om_d)


def test_inner_graph_replay_gives_identical_results(monkeypatch):
    """On the 256^2 grid the inner PCG of the search directions replays CUDA
    graphs captured on the second call of each block width: eigenvalues,
    residuals, iteration counts and vectors equal those of direct launches
    (BDG_INNER_GRAPHS=0) bit for bit, in mixed and FP64 precision."""
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    with open(os.path.join(HERE, "golden", "solve_2d_n256.json")) as fh:
        gold = json.load(fh)
    V, phi, mu, op = _oracle_2d_n256(gold)
    X0 = torch.from_numpy(synth.random_block(W, 12, complex_=True)).cuda()
    for prec in (bdg.MIXED, bdg.FP64):
        plan = make_plan(W, V, phi, prec=prec, tol=1e-10, maxit=600)
        out = {}
        for graphs in ("0", "1"):
            monkeypatch.setenv("BDG_INNER_GRAPHS", graphs)
            om, UV, resid, nconv = plan.solve(8, 12, X0=X0)
            out[graphs] = (om.copy(), resid.copy(), nconv, plan.stats()["iterations"], UV.cpu().numpy())
        plan.close()
        assert out["0"][2] == out["1"][2] == 8
        assert out["0"][3] == out["1"][3]
        for a, b in zip(out["0"][:2] + out["0"][4:], out["1"][:2] + out["1"][4:]):
            assert np.array_equal(a, b)
