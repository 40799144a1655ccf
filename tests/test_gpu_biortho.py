"""bdg_biortho (CUDA) against the oracle's bi-orthogonal Gram-Schmidt (Section
3.2, Theorem "Biorthogonality"): F^H G = I, bi-orthogonality to a locked pair,
the kept rank, and the oblique projector F G^H -- the one basis-independent
result, since the SVD of S = F^H G fixes F and G only up to unitary mixing
inside degenerate singular values -- on complex blocks in FP64 and FP32."""
import numpy as np
import pytest

import synth
from gpu_util import make_plan, need_torch_cuda, oracle_problem

pytestmark = pytest.mark.gpu

W1 = synth.Workload("s1d_n64", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.0, 0.0, 0.0, k=8, m=12, gs_seed=101)
W2 = synth.Workload("s2d_16", (16, 16), (-6.0, -6.0), (6.0, 6.0), (1.0, 1.4), 12.0, -1.0, 0.05, 0.3, gs_seed=8)


def _blocks(w, ncol, seed):
    rng = np.random.default_rng(seed)
    n = 3 * w.npts
    F = rng.standard_normal((n, ncol)) + 1j * rng.standard_normal((n, ncol))
    G = F + 0.5 * (rng.standard_normal((n, ncol)) + 1j * rng.standard_normal((n, ncol)))
    return F, G


def _to_dev(M, dtype):
    import torch
    ncol = M.shape[1]
    return torch.from_numpy(np.ascontiguousarray(M.T.reshape(ncol, 3, -1))).to(dtype).cuda()


def _from_dev(t, r):
    a = t.cpu().numpy().astype(np.complex128)
    return a.reshape(a.shape[0], -1).T[:, :r]


@pytest.mark.parametrize("w", [W1, W2], ids=lambda w: w.name)
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_biortho_matches_oracle(w, prec):
    torch = need_torch_cuda()
    from oracle import lrep
    V, phi, mu, op = oracle_problem(w)
    plan = make_plan(w, V, phi)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    tol = 1e-10 if prec == "c128" else 2e-4
    rtol = 1e-12 if prec == "c128" else 1e-6
    ncol, nlock = 10, 4
    Fl0, Gl0 = _blocks(w, nlock, 11)
    Fl, Gl, _ = lrep.biortho(Fl0, Gl0, rtol=1e-12)           # a locked bi-orthonormal pair
    F0, G0 = _blocks(w, ncol, 12)
    Fo, Go, ro = lrep.biortho(F0, G0, Fl, Gl, rtol=rtol)     # oracle
    F, G = _to_dev(F0, dt), _to_dev(G0, dt)
    for call in range(2):                                     # a second call on fresh inputs
        if call:
            F, G = _to_dev(F0, dt), _to_dev(G0, dt)
        r = plan.biortho(F, G, _to_dev(Fl, dt), _to_dev(Gl, dt))
        assert r == ro
        Fg, Gg = _from_dev(F, r), _from_dev(G, r)
        assert np.abs(Fg.conj().T @ Gg - np.eye(r)).max() < tol
        assert np.abs(Gl.conj().T @ Fg).max() < tol * np.abs(Fg).max() * 10
        assert np.abs(Fl.conj().T @ Gg).max() < tol * np.abs(Gg).max() * 10
        z = np.random.default_rng(3).standard_normal(F0.shape[0]) + 0j
        pz, pzo = Fg @ (Gg.conj().T @ z), Fo @ (Go.conj().T @ z)
        assert np.linalg.norm(pz - pzo) < 10 * tol * np.linalg.norm(pzo)
        rest = F.cpu().numpy()[r:]
        assert not rest.size or np.abs(rest).max() == 0
    plan.close()


def test_biortho_rank_deficient():
    """A column of F orthogonal to every column of G has no partner: the rank
    drops by one and F^H G = I holds on the rest."""
    torch = need_torch_cuda()
    w = W1
    V, phi, mu, op = oracle_problem(w)
    plan = make_plan(w, V, phi)
    F0, G0 = _blocks(w, 6, 21)
    Q, _ = np.linalg.qr(G0)
    v = np.random.default_rng(5).standard_normal(F0.shape[0]) + 0j
    v -= Q @ (Q.conj().T @ v)
    F0[:, 5] = v / np.linalg.norm(v)
    F, G = _to_dev(F0, torch.complex128), _to_dev(G0, torch.complex128)
    r = plan.biortho(F, G)
    assert r == 5
    Fg, Gg = _from_dev(F, r), _from_dev(G, r)
    assert np.abs(Fg.conj().T @ Gg - np.eye(r)).max() < 1e-10
    plan.close()


def test_biortho_limits():
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    w = W1
    V, phi, mu, op = oracle_problem(w)
    plan = make_plan(w, V, phi)
    F = torch.zeros((41, 3, w.npts), dtype=torch.complex128, device="cuda")
    with pytest.raises(bdg.BdgError) as e:
        plan.biortho(F, F.clone())
    assert e.value.status == bdg.ERR_UNSUPPORTED
    with pytest.raises(bdg.BdgError) as e:
        plan.biortho(F[:4], F[:4].clone())       # S = 0
    assert e.value.status == bdg.ERR_BREAKDOWN
    plan.close()
