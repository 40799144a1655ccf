"""Parity of bdg_solve (CUDA) with the oracle's dense FP64 solution of
eq. lrep-d: the k smallest positive excitations to 1e-10 relative, the
amplitudes per degenerate cluster to 1e-8 (projector metric of Section 4.1),
residuals <= 1e-10 in FP64, and the normalization / bi-orthogonality
h^d (u_i.u_j - v_i.v_j) = delta_ij (eq. constrain, Theorem
"Biorthogonality"); FP64 and mixed precision, 1-D, 2-D and 3-D, odd and even
block sizes, a start block passed in and the internal seeded one, and an
antiferromagnetic state whose deflation space holds S_x Phi."""
import numpy as np
import pytest

import synth
from gpu_util import make_plan, need_torch_cuda, oracle_problem

pytestmark = pytest.mark.gpu

W1 = synth.Workload("s1d_n64", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.0, 0.0, 0.0, k=8, m=12,
                    gs_seed=101, block_seed=7)
W1Q = synth.Workload("s1d_n64_q", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.0, 0.0, 0.1, k=8, m=11,
                     gs_seed=102, block_seed=9)
W2 = synth.Workload("s2d_16", (16, 16), (-6.0, -6.0), (6.0, 6.0), (1.0, 1.4), 12.0, -1.0, 0.05, 0.3, k=10, m=14,
                    gs_seed=8, block_seed=3)
W3 = synth.Workload("s3d_8", (8, 8, 8), (-4.0,) * 3, (4.0,) * 3, (1.0, 1.2, 1.5), 8.0, -0.5, 0.02, 0.2, k=6,
                    m=10, gs_seed=31, block_seed=32)
WC1 = synth.W1D_N256
# Table 1's antiferromagnetic instance at h0/2 (p = q = 0): its ground state
# (phi_1, 0, phi_-1) puts S_x Phi in null(H_-), a third column of Z_f
WAFM = synth.Workload("t1a_64", (64,), (-16.0,), (16.0,), (1.0,), 240.8, 7.5, 0.0, 0.0, k=8, m=16,
                      gs_seed=17, block_seed=18)


def _dense(op, k):
    from oracle import lrep
    return lrep.dense_solve_fg(op, k + 6)


def _check(w, op, om, UV, resid, k, dense):
    from oracle import lrep
    om_d, F, G = dense
    assert np.all(resid[:k] <= 1e-10), resid
    assert np.allclose(om[:k], om_d[:k], rtol=1e-10, atol=0), (om[:k], om_d[:k])
    U = UV[:k, :3].reshape(k, -1)
    V = UV[:k, 3:].reshape(k, -1)
    hd = lrep.weight(w)
    gram = hd * (U @ U.T - V @ V.T)
    assert np.allclose(gram, np.eye(k), atol=1e-8), np.abs(gram - np.eye(k)).max()
    # amplitudes per cluster of (relative gap < 1e-8) eigenvalues, the cluster
    # fully inside the first k
    Ud = (F + G)[:, :, :].reshape(len(om_d), -1)
    Vd = (F - G).reshape(len(om_d), -1)
    i = 0
    while i < k:
        j = i + 1
        while j < len(om_d) and abs(om_d[j] - om_d[i]) < 1e-8 * om_d[i]:
            j += 1
        if j <= k:
            Q, _ = np.linalg.qr(np.concatenate([Ud[i:j], Vd[i:j]], axis=1).T)
            X = np.concatenate([U[i:j], V[i:j]], axis=1).T
            err = np.linalg.norm(X - Q @ (Q.T @ X)) / np.linalg.norm(X)
            assert err < 1e-8, (i, j, err)
        i = j
    r = lrep.residual_uv(op, UV[:k], om[:k])
    assert r.max() < 1e-9, r


@pytest.mark.parametrize("w", [W1, W1Q, W2, W3, WAFM], ids=lambda w: w.name)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_matches_dense(w, prec):
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    V, phi, mu, op = oracle_problem(w)
    plan = make_plan(w, V, phi, prec=bdg.FP64 if prec == "fp64" else bdg.MIXED, tol=1e-10, maxit=600)
    X0 = torch.from_numpy(synth.random_block(w, w.m, complex_=True)).cuda()
    om, UV, resid, nconv = plan.solve(w.k, w.m, X0=X0)
    assert nconv == w.k
    _check(w, op, om, UV.cpu().numpy().real, resid, w.k, _dense(op, w.k))
    st = plan.stats()
    assert st["iterations"] > 0
    if prec == "mixed":
        assert st["iterations_fp32"] > 0 and st["applies_fp32"] > 0
    plan.close()


def test_solve_1d_n256_full_size():
    """The 1-D workload as specified: N = 256, k = 16, m = 24, FP64, seeded
    internal start block."""
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    w = WC1
    V, phi, mu, op = oracle_problem(w)
    plan = make_plan(w, V, phi, prec=bdg.FP64, tol=1e-10, maxit=800, seed=w.block_seed)
    om, UV, resid, nconv = plan.solve(w.k, w.m)
    assert nconv == w.k
    dense = _dense(op, w.k)
    _check(w, op, om, UV.cpu().numpy().real, resid, w.k, dense)
    # the Kohn mode omega = gamma_x = 1 is among the excitations (Theorem
    # "Analytical eigenpairs")
    assert np.min(np.abs(om - 1.0)) < 1e-9
    plan.close()


def test_solve_rejects_bad_sizes():
    need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    V, phi, mu, op = oracle_problem(W1)
    plan = make_plan(W1, V, phi)
    with pytest.raises(bdg.BdgError) as e:
        plan.solve(5, 4)
    assert e.value.status == bdg.ERR_INVALID
    with pytest.raises(bdg.BdgError) as e:
        plan.solve(8, 200)
    assert e.value.status == bdg.ERR_UNSUPPORTED
    # the largest block the header allows is 52; 53 is refused before any work
    with pytest.raises(bdg.BdgError) as e:
        plan.solve(8, 53)
    assert e.value.status == bdg.ERR_UNSUPPORTED and "52" in str(e.value)
    plan.close()


def test_solve_at_the_largest_block():
    """A full solve with the largest block the header allows (m = 52), on a
    2-D grid whose problem holds enough directions (16 x 16 x 3 f-side
    unknowns): the basis reaches its 156-column maximum without overflowing
    the projected eigensolver, and the pairs match the dense solution."""
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    import dataclasses
    w = dataclasses.replace(W2, name="s2d_16_m52", k=30, m=52)
    V, phi, mu, op = oracle_problem(w)
    plan = make_plan(w, V, phi, prec=bdg.FP64, tol=1e-10, maxit=600)
    X0 = torch.from_numpy(synth.random_block(w, w.m, complex_=True)).cuda()
    om, UV, resid, nconv = plan.solve(w.k, w.m, X0=X0)
    assert nconv == w.k
    _check(w, op, om, UV.cpu().numpy().real, resid, w.k, _dense(op, w.k))
    plan.close()


def test_solve_batched_matches_single_solves():
    """bdg_solve_batched over three independent problems of different grids
    (1-D, 2-D, 3-D): each entry equals its own bdg_solve and the dense FP64
    eigenvalues."""
    need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    cases = [W1, W2, W3]
    plans, dense = [], []
    for w in cases:
        V, phi, mu, op = oracle_problem(w)
        plans.append(make_plan(w, V, phi, prec=bdg.FP64, tol=1e-10, maxit=600, seed=w.block_seed + 11))
        dense.append(_dense(op, w.k))
    out = bdg.solve_batched(plans, [w.k for w in cases], [w.m for w in cases])
    for w, plan, (om, UV, resid, nconv), dn in zip(cases, plans, out, dense):
        assert nconv == w.k
        np.testing.assert_allclose(om, dn[0][:w.k], rtol=1e-10, atol=0)
        om1, _, _, nconv1 = plan.solve(w.k, w.m, want_vectors=False)
        assert nconv1 == w.k
        np.testing.assert_allclose(om, om1, rtol=1e-10, atol=0)
        assert np.all(resid <= 1e-10)
    for p in plans:
        p.close()


def test_solve_batched_work_queue_matches_serial(monkeypatch):
    """Ten instances of different grids and interactions (16^2 and 32^2, FM
    and AFM draws) served by four host threads with a stream each give the
    eigenvalues, residuals and convergence counts of the same call with one
    worker, and a plan listed twice is refused."""
    need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    rng = np.random.default_rng(77)
    cases = []
    for i in range(10):
        n = 16 if i % 2 else 32
        cases.append(synth.Workload(f"q{i}", (n, n), (-6.0, -6.0), (6.0, 6.0), (1.0, 1.3),
                                    float(rng.uniform(8.0, 20.0)), float(rng.uniform(-2.0, 2.0)), 0.0,
                                    float(rng.uniform(0.05, 0.4)), k=6, m=10, gs_seed=200 + i, block_seed=300 + i))
    plans = []
    for w in cases:
        V, phi, mu, op = oracle_problem(w)
        plans.append(make_plan(w, V, phi, prec=bdg.MIXED, tol=1e-10, maxit=600, seed=w.block_seed))
    ks, ms_ = [w.k for w in cases], [w.m for w in cases]
    monkeypatch.setenv("BDG_BATCH_WORKERS", "1")
    serial = bdg.solve_batched(plans, ks, ms_, want_vectors=False)
    monkeypatch.setenv("BDG_BATCH_WORKERS", "4")
    queued = bdg.solve_batched(plans, ks, ms_, want_vectors=False)
    for (om1, _, r1, c1), (om4, _, r4, c4), w in zip(serial, queued, cases):
        assert c1 == c4 == w.k
        np.testing.assert_allclose(om4, om1, rtol=1e-12, atol=0)
        assert np.all(r4 <= 1e-10)
    with pytest.raises(RuntimeError, match="twice"):
        bdg.solve_batched([plans[0], plans[1], plans[0]], ks[:3], ms_[:3], want_vectors=False)
    for p in plans:
        p.close()


def test_second_lane_gives_identical_results(monkeypatch):
    """The previous-update block's Gram-Schmidt on the second lane (its own
    stream and scratch, overlapped with the inner PCG of the directions)
    touches buffers disjoint from the directions' and reduces in a fixed
    order: eigenvalues, residuals and iteration counts equal the one-lane
    solve's bit for bit, in mixed and FP64 precision."""
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    w = synth.Workload("s2d_32", (32, 32), (-6.0, -6.0), (6.0, 6.0), (1.0, 1.3), 20.0, -1.0, 0.0, 0.1, k=8,
                       m=12, gs_seed=3, block_seed=4)
    V, phi, mu, op = oracle_problem(w)
    X0 = torch.from_numpy(synth.random_block(w, w.m, complex_=True)).cuda()
    for prec in (bdg.MIXED, bdg.FP64):
        plan = make_plan(w, V, phi, prec=prec, tol=1e-10, maxit=600)
        out = {}
        for lanes in ("0", "1"):
            monkeypatch.setenv("BDG_OVERLAP", lanes)
            om, UV, resid, nconv = plan.solve(w.k, w.m, X0=X0)
            out[lanes] = (om.copy(), resid.copy(), nconv, plan.stats()["iterations"], UV.cpu().numpy())
        assert out["0"][2] == out["1"][2] == w.k
        assert out["0"][3] == out["1"][3]
        assert np.array_equal(out["0"][0], out["1"][0]) and np.array_equal(out["0"][1], out["1"][1])
        assert np.array_equal(out["0"][4], out["1"][4])
        plan.close()
