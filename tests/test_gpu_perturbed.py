"""Parity of bdg_perturbed_density (CUDA) with the oracle's perturbed
densities (Section 4.2, "2D Case" example; eq. waveAssump with one mode):
element by element on seeded complex amplitudes over 1-D, 2-D and 3-D grids
(a ragged single tile, several tiles, a grid-stride loop), on the amplitudes
bdg_solve returns, and on sampled points of the 256^2 workload with its 32
modes; plus the no-op and argument checks.

Tolerances: FP64 path 1e-13 of max n (a few roundings of terms of size max n);
FP32 path 1e-6 of max n against the oracle evaluated on the same FP32-rounded
inputs (phi and the amplitudes), i.e. a few FP32 roundings."""
import math

import numpy as np
import pytest

import synth
from gpu_util import make_plan, need_torch_cuda, oracle_problem
from oracle.perturbed import perturbed_density

pytestmark = pytest.mark.gpu

GRIDS = [
    synth.Workload("pd_1d_8", (8,), (-4.0,), (4.0,), (1.0,), 10.0, -1.0, block_seed=41),
    synth.Workload("pd_2d_64", (64, 64), (-6.0, -6.0), (6.0, 6.0), (1.0, 1.3), 10.0, -1.0, block_seed=42),
    synth.Workload("pd_3d_16", (16, 16, 16), (-5.0,) * 3, (5.0,) * 3, (1.0, 1.2, 1.5), 10.0, -1.0, block_seed=43),
]


def _phi(w):
    phi = synth.initial_spinor(w)
    return (phi / np.sqrt(np.prod(w.h) * np.sum(phi ** 2))).reshape(3, -1)


def _plan(w, phi):
    return make_plan(w, synth.potential(w), phi.reshape(-1), mu=(1.0, 1.0, 1.0))


def _check(got, expect, tol):
    scale = float(np.max(np.abs(expect)))
    err = float(np.max(np.abs(got - expect)))
    assert err <= tol * scale, (err, scale)


@pytest.mark.parametrize("w", GRIDS, ids=lambda w: w.name)
def test_random_amplitudes_fp64(w):
    torch = need_torch_cuda()
    phi = _phi(w)
    plan = _plan(w, phi)
    UV = synth.random_block(w, 3) * 0.5
    om = np.array([0.37, 1.0, 2.9])
    times = np.array([0.0, 0.8, 10.6, -3.1])
    eps = 0.1
    out = plan.perturbed_density(torch.from_numpy(UV).cuda(), om, times, eps)
    assert out.dtype == torch.float64 and tuple(out.shape) == (3, 4, 3, w.npts)
    expect = perturbed_density(phi, UV[:, :3], UV[:, 3:], om, times, eps)
    _check(out.cpu().numpy(), expect, 1e-13)
    plan.close()


@pytest.mark.parametrize("w", GRIDS, ids=lambda w: w.name)
def test_random_amplitudes_fp32(w):
    torch = need_torch_cuda()
    phi = _phi(w)
    plan = _plan(w, phi)
    UV = (synth.random_block(w, 2) * 0.5).astype(np.complex64)
    om = np.array([0.61, 1.7])
    times = np.array([0.0, 2.5, 10.6])
    eps = 0.2
    out = plan.perturbed_density(torch.from_numpy(UV).cuda(), om, times, eps)
    assert out.dtype == torch.float32
    phi32 = phi.astype(np.float32).astype(np.float64)
    expect = perturbed_density(phi32, UV[:, :3], UV[:, 3:], om, times, eps)
    _check(out.cpu().numpy().astype(np.float64), expect, 1e-6)
    plan.close()


@pytest.mark.parametrize("cdt", [np.complex128, np.complex64], ids=["c128", "c64"])
def test_long_phase_table(cdt):
    """More (mode, time) pairs than travel with the launch (4 x 40 > 128):
    the table goes through device scratch, same results."""
    torch = need_torch_cuda()
    w = GRIDS[1]
    phi = _phi(w)
    plan = _plan(w, phi)
    UV = (synth.random_block(w, 4, seed=77) * 0.5).astype(cdt)
    om = np.array([0.3, 0.9, 1.4, 2.2])
    times = np.linspace(-2.0, 12.0, 40)
    out = plan.perturbed_density(torch.from_numpy(UV).cuda(), om, times, 0.15)
    phi_ref = phi if cdt == np.complex128 else phi.astype(np.float32).astype(np.float64)
    expect = perturbed_density(phi_ref, UV[:, :3], UV[:, 3:], om, times, 0.15)
    _check(out.cpu().numpy().astype(np.float64), expect, 1e-13 if cdt == np.complex128 else 1e-6)
    plan.close()


def test_solver_modes():
    """Densities of the pairs bdg_solve returns (FP64, 1-D workload): the
    paper's eps = 0.1 at t = 10.6 for all modes at once, and each mode at a
    quarter of its period."""
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    w = synth.Workload("s1d_n64", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.0, 0.0, 0.0, k=8, m=12,
                       gs_seed=101, block_seed=7)
    V, phi, mu, op = oracle_problem(w)
    phi = phi.reshape(3, -1)
    plan = make_plan(w, V, phi.reshape(-1), prec=bdg.FP64, tol=1e-10, maxit=600)
    om, UV, resid, nconv = plan.solve(w.k, w.m)
    assert nconv == w.k
    uv = UV.cpu().numpy()
    eps = 0.1
    out = plan.perturbed_density(UV, om, [10.6], eps).cpu().numpy()
    _check(out, perturbed_density(phi, uv[:, :3], uv[:, 3:], om, [10.6], eps), 1e-13)
    for l in range(w.k):
        tq = [0.5 * math.pi / om[l]]
        out = plan.perturbed_density(UV[l:l + 1], om[l:l + 1], tq, eps).cpu().numpy()
        _check(out, perturbed_density(phi, uv[l:l + 1, :3], uv[l:l + 1, 3:], om[l:l + 1], tq, eps), 1e-13)
    plan.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_full_workload_sampled(dtype):
    """The 256^2 workload's 32 modes, one snapshot (the launch the
    benchmark's density line times): 4096 sampled points per mode against
    the oracle evaluated point by point."""
    torch = need_torch_cuda()
    w = synth.W2D_N256
    phi = _phi(w)
    plan = _plan(w, phi)
    UV = synth.random_block(w, w.k, seed=2024) * 0.05
    if dtype == "c64":
        UV = UV.astype(np.complex64)
        phi_ref = phi.astype(np.float32).astype(np.float64)
        tol = 1e-6
    else:
        phi_ref, tol = phi, 1e-13
    om = np.linspace(1.0, 3.0, w.k)
    times = np.array([10.6])
    out = plan.perturbed_density(torch.from_numpy(UV).cuda(), om, times, 0.1)
    idx = np.sort(np.random.default_rng(5).choice(w.npts, 4096, replace=False))
    got = out[:, :, :, torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    expect = perturbed_density(phi_ref[:, idx], UV[:, :3][:, :, idx], UV[:, 3:][:, :, idx], om, times, 0.1)
    _check(got, expect, tol)
    plan.close()


def test_noop_and_argument_checks():
    torch = need_torch_cuda()
    from paper_2506_08308_gb300 import bdg
    w = GRIDS[0]
    phi = _phi(w)
    plan = _plan(w, phi)
    UV = torch.from_numpy(synth.random_block(w, 2)).cuda()
    sentinel = torch.full((2, 0, 3, w.npts), 7.0, dtype=torch.float64, device="cuda")
    # nt == 0: nothing written, status OK
    out = plan.perturbed_density(UV, [1.0, 2.0], [], 0.1, out=sentinel)
    assert out.numel() == 0
    with pytest.raises(bdg.BdgError) as e:
        plan.perturbed_density(UV, [1.0, float("nan")], [0.0], 0.1)
    assert e.value.status == bdg.ERR_INVALID
    with pytest.raises(bdg.BdgError) as e:
        plan.perturbed_density(UV, [1.0, 2.0], [0.0], float("inf"))
    assert e.value.status == bdg.ERR_INVALID
    # out overlapping UV
    big = torch.zeros(2 * 6 * w.npts * 2, dtype=torch.float64, device="cuda")
    uv_view = torch.view_as_complex(big.view(-1, 2)).view(2, 6, w.npts)
    with pytest.raises(bdg.BdgError) as e:
        plan.perturbed_density(uv_view, [1.0, 2.0], [0.0], 0.1, out=big[: 2 * 3 * w.npts].view(2, 1, 3, w.npts))
    assert e.value.status == bdg.ERR_INVALID
    torch.cuda.synchronize()
    plan.close()
