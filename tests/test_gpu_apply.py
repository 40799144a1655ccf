"""Parity of bdg_apply (CUDA, FP64 and FP32) with the FP64 oracle
(eqs. BdG-d / lrep-d): element-wise relative L2 of 1e-12 (FP64) and 1e-5
relative to |M| |x| (FP32, |M| estimated by the largest kinetic symbol plus
the largest pointwise entry), on seeded inputs spanning several tiles and
ragged tails, every dimension, both forms; sampled vectors at the full 2-D
256^2 workload with the m = 48 block; chemical potentials of eq.
chem-formula computed on the device."""
import numpy as np
import pytest

import synth
from gpu_util import make_plan, need_torch_cuda, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

CASES = [
    synth.Workload("1d_n256", (256,), (-16.0,), (16.0,), (1.0,), 10.0, -1.0, 0.0, 0.0, gs_seed=101),
    synth.Workload("1d_n64", (64,), (-8.0,), (8.0,), (1.0,), 5.0, 0.7, 0.02, 0.1, gs_seed=5),
    synth.Workload("2d_8x8", (8, 8), (-4.0, -4.0), (4.0, 4.0), (1.0, 1.0), 3.0, -0.5, 0.0, 0.1, gs_seed=6),
    synth.Workload("2d_32x64", (32, 64), (-6.0, -8.0), (6.0, 8.0), (1.0, 0.8), 20.0, -1.0, 0.05, 0.1, gs_seed=7),
    synth.Workload("2d_64x16", (64, 16), (-8.0, -4.0), (8.0, 4.0), (0.8, 1.5), 12.0, 1.0, 0.0, 0.3, gs_seed=8),
    synth.Workload("3d_16x8x32", (16, 8, 32), (-4.0, -3.0, -5.0), (4.0, 3.0, 5.0), (1.0, 1.5, 0.8),
                   10.0, -1.0, 0.05, 0.2, gs_seed=9),
]


def _opnorm(w, op):
    kin = 0.5 * sum((np.pi * n / (hi - lo)) ** 2 for n, lo, hi in zip(w.n, w.lo, w.hi))
    pt = np.max(np.abs(op.Apt).sum(axis=2) + np.abs(op.Bpt).sum(axis=2))
    return kin + pt


@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
@pytest.mark.parametrize("nvec", [1, 3])
def test_apply_matches_oracle(w, nvec):
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    V, phi, mu, op = oracle_problem(w)
    plan = make_plan(w, V, phi)
    assert np.allclose(plan.mu, mu, rtol=1e-10, atol=1e-12)
    x = synth.random_block(w, nvec, seed=11 + nvec)
    norm = _opnorm(w, op)
    for mode in (bdg.UV, bdg.FG):
        ref = op.apply_fft(x, mode)
        y64 = plan.apply(torch.from_numpy(x).cuda(), mode).cpu().numpy()
        assert rel_l2(y64, ref) < 1e-12, (mode, rel_l2(y64, ref))
        y32 = plan.apply(torch.from_numpy(x.astype(np.complex64)).cuda(), mode).cpu().numpy()
        err = np.linalg.norm((y32 - ref).ravel()) / (norm * np.linalg.norm(x.ravel()))
        assert err < 1e-5, (mode, err)
    plan.close()


def test_apply_full_2d_block_sampled():
    """The 2-D 256^2 workload, m = 48 vectors per call as timed by the
    benchmark; vectors 0 and 47 checked against the oracle."""
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    from oracle import apply as ap
    w = synth.W2D_N256
    V = synth.potential(w)
    rng = np.random.default_rng(3)
    # any real spinor is a valid operator input; a Gaussian keeps it smooth
    phi = synth.initial_spinor(w) * 0.3
    mu = np.array([1.1, 0.9, 1.3])
    op = ap.Operator(w, phi, V, mu)
    plan = make_plan(w, V, phi, mu=mu)
    x = synth.random_block(w, w.m, complex_=True)
    xt = torch.from_numpy(x).cuda()
    for mode in (bdg.UV, bdg.FG):
        y64 = plan.apply(xt, mode).cpu().numpy()
        y32 = plan.apply(xt.to(torch.complex64), mode).cpu().numpy()
        norm = _opnorm(w, op)
        for i in (0, w.m - 1):
            ref = op.apply_fft(x[i:i + 1], mode)[0]
            assert rel_l2(y64[i], ref) < 1e-12
            assert np.linalg.norm(y32[i] - ref) / (norm * np.linalg.norm(x[i])) < 1e-5
    plan.close()



def _lines_through(grid, nodes):
    """lines[a][s] = the (6, N_a) fields of grid (6, n_1, .., n_d) on the line
    through node s along axis a, as complex128 host arrays."""
    lines = []
    for a in range(grid.dim() - 1):
        per = []
        for nd in nodes:
            sl = list(nd)
            sl[a] = slice(None)
            per.append(grid[(slice(None),) + tuple(sl)].cpu().numpy().astype(np.complex128))
        lines.append(np.stack(per))
    return lines


@pytest.mark.parametrize("w", [synth.W3D_N128, synth.W3D_N256], ids=lambda w: w.name)
def test_apply_full_3d_sampled(w):
    """The 3-D workloads in the launch configuration the benchmark times for
    their products: FG products of the workload's m vectors in c64 and in
    c128 (m / 2 of them in c128 at 256^3: 1.6e9 entries next to the 3.2e9
    of the c64 block), the blocks drawn on the device.  At 40 seeded nodes
    (corners and the trap centre included) of the first, a middle and the
    last vector the result is compared with the oracle's product at those
    nodes, formed from the grid lines through them: the per-node error
    relative to |M| times the vector's RMS entry below 1e-5 (c64) and 1e-12
    (c128), the per-entry form of the whole-vector bounds above."""
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    from oracle import apply as ap
    phi = synth.initial_spinor(w)
    phi = phi / np.sqrt(np.prod(w.h) * np.sum(phi ** 2))
    V = synth.potential(w)
    mu = np.array([1.0, 1.0, 1.0])
    plan = make_plan(w, V, phi.reshape(-1), mu=mu)
    rng = np.random.default_rng(41)
    n0, n1, n2 = w.n
    nodes = [(0, 0, 0), (n0 - 1, n1 - 1, n2 - 1), (n0 // 2, n1 // 2, n2 // 2), (n0 // 2, 0, n2 - 1),
             (1, n1 - 2, n2 // 2 - 1)] + [tuple(int(rng.integers(0, nn)) for nn in w.n) for _ in range(35)]
    flat = [int(np.ravel_multi_index(nd, w.n)) for nd in nodes]
    ph = phi.reshape(3, -1)[:, flat]
    Vn = V.reshape(-1)[flat]
    del phi
    # |M|: the largest kinetic symbol plus the largest pointwise row sum over
    # the nodes, which include the trap centre (where rho, and with it the
    # pointwise part, is largest)
    from oracle import spin1
    kin = 0.5 * sum((np.pi * n / (hi - lo)) ** 2 for n, lo, hi in zip(w.n, w.lo, w.hi))
    Apt, Bpt = spin1.pointwise_blocks(ph, Vn, w.beta_n, w.beta_s, mu, w.p, w.q)
    norm = kin + float(np.max(np.abs(Apt.real).sum(axis=2) + np.abs(Bpt.real).sum(axis=2)))
    gen = torch.Generator(device="cuda")
    m64 = w.m if w.npts < (1 << 24) else w.m // 2
    for dt, m, tol in ((torch.complex64, w.m, 1e-5), (torch.complex128, m64, 1e-12)):
        gen.manual_seed(w.block_seed)
        x = torch.randn((m, 6, w.npts), dtype=dt, device="cuda", generator=gen)
        y = plan.apply(x, bdg.FG)
        torch.cuda.synchronize()
        for v in (0, m // 2 + 1, m - 1):
            xv = x[v].view((6,) + w.n)
            yv = y[v].view((6,) + w.n)
            rms = float(torch.linalg.vector_norm(x[v].to(torch.complex128))) / np.sqrt(6 * w.npts)
            ref = ap.apply_at_nodes(w, ph, Vn, mu, _lines_through(xv, nodes), nodes, ap.FG)
            got = np.stack([yv[(slice(None),) + nd].cpu().numpy() for nd in nodes])
            err = np.abs(got - ref).max() / (norm * rms)
            assert err < tol, (str(dt), v, err)
        del x, y
        torch.cuda.empty_cache()
    plan.close()


def test_apply_edge_cases():
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    w = CASES[1]
    V, phi, mu, op = oracle_problem(w)
    plan = make_plan(w, V, phi)
    x = torch.zeros((2, 6, w.npts), dtype=torch.complex128, device="cuda")
    # zero in, zero out
    assert float(plan.apply(x).abs().max()) == 0.0
    # overlapping buffers are rejected
    with pytest.raises(bdg.BdgError) as e:
        plan.apply(x, out=x)
    assert e.value.status == bdg.ERR_INVALID
    # nvec = 0 is a no-op
    assert plan.apply(x[:0]).shape[0] == 0
    plan.close()


def test_linearity_and_realness():
    """M is real and linear: M(a x + i b x') = a M x + i b M x'."""
    torch = need_torch_cuda()
    w = CASES[3]
    V, phi, mu, op = oracle_problem(w)
    plan = make_plan(w, V, phi)
    xr = synth.random_block(w, 2, complex_=False, seed=5)
    yr = plan.apply(torch.from_numpy(xr[0:1] + 0j).cuda()).cpu().numpy()
    yi = plan.apply(torch.from_numpy(1j * xr[1:2]).cuda()).cpu().numpy()
    yc = plan.apply(torch.from_numpy(xr[0:1] + 1j * xr[1:2]).cuda()).cpu().numpy()
    assert np.abs(yr.imag).max() < 1e-13 * np.abs(yr.real).max()
    assert rel_l2(yc, yr + yi) < 1e-14
    plan.close()
