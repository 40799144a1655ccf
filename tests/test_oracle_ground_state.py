"""Pins of the ground-state flow (eq. groundDef on S_M).

- Lemma SMA (FM, beta_s < 0, beta_n + beta_s >= 0, p = q = 0): Phi = a phi_g with
  a = ((1+M)/2, ((1-M^2)/2)^{1/2}, (1-M)/2), equal chemical potentials, and
  phi_g solving the scalar equation with interaction beta_n + beta_s.
- Lemma on the two-component AFM state (beta_s > 0, M != 0): phi_0 = 0.
- Non-interacting limit: the oscillator ground state, mu_j = sum gamma / 2.
- Constraints: mass 1 and magnetization M; NLEP residual <= 1e-12.
"""
import numpy as np
import pytest

import synth
from oracle import discretization as disc
from oracle import ground_state as gs
from oracle import spin1


def _run(w):
    V = synth.potential(w)
    phi, mu, res, it = gs.ground_state(w, V, synth.initial_spinor(w), tol=1e-12)
    return V, phi, mu, res


@pytest.mark.parametrize("M", [0.0, 0.3])
def test_sma_ferromagnetic(M):
    w = synth.Workload("sma", (128,), (-16.0,), (16.0,), (1.0,), 10.0, -1.0, 0.0, 0.0, M=M, gs_seed=5)
    V, phi, mu, res = _run(w)
    assert res <= 1e-12
    a = np.array([(1 + M) / 2, np.sqrt((1 - M * M) / 2), (1 - M) / 2])
    # the sign of a global spin rotation is free: compare |phi|
    ratios = np.abs(phi) / np.abs(phi[1])[None]
    core = np.abs(phi[1]) > 1e-3 * np.abs(phi[1]).max()
    for j in range(3):
        assert np.allclose(ratios[j][core], a[j] / a[1], rtol=1e-9)
    assert np.ptp(mu) < 1e-10
    phig = phi[1] * np.sign(phi[1][np.argmax(np.abs(phi[1]))]) / a[1]
    lap = disc.laplacian_fft(phig, w.lo, w.hi).real
    r = -0.5 * lap + (V + (w.beta_n + w.beta_s) * phig ** 2) * phig - mu[1] * phig
    assert np.abs(r).max() < 1e-10


def test_constraints_and_residual():
    w = synth.Workload("c", (64, 64), (-8.0, -8.0), (8.0, 8.0), (1.0, 1.2), 40.0, -1.0, 0.0, 0.1,
                       M=0.2, gs_seed=9)
    V, phi, mu, res = _run(w)
    cell = float(np.prod(w.h))
    assert res <= 1e-12
    assert abs(cell * np.sum(phi ** 2) - 1) < 1e-12
    assert abs(cell * (np.sum(phi[0] ** 2) - np.sum(phi[2] ** 2)) - 0.2) < 1e-12
    assert abs(mu[0] + mu[2] - 2 * mu[1]) < 1e-10


def test_antiferromagnetic_two_component():
    w = synth.Workload("afm", (128,), (-12.0,), (12.0,), (1.0,), 30.0, 2.0, 0.0, 0.0, M=0.3, gs_seed=3)
    V, phi, mu, res = _run(w)
    assert res <= 1e-12
    cell = w.h[0]
    assert cell * np.sum(phi[1] ** 2) < 1e-16


def test_non_interacting_oscillator():
    w = synth.Workload("free", (64, 32), (-8.0, -6.0), (8.0, 6.0), (1.0, 2.0), 0.0, 0.0, M=0.0, gs_seed=4)
    V, phi, mu, res = _run(w)
    assert res <= 1e-12
    assert np.allclose(mu, 1.5, atol=1e-11)
    x, y = np.meshgrid(*synth.axes(w), indexing="ij")
    g = np.exp(-(1.0 * x * x + 2.0 * y * y) / 2)
    for j in range(3):
        c = np.sum(phi[j] * g) / np.sum(g * g)
        assert np.abs(phi[j] - c * g).max() < 1e-9


def test_chemical_potential_rules():
    phi = np.zeros((3, 4))
    phi[1] = 1.0
    Hphi = 2.5 * phi
    mu = spin1.chemical_potentials(phi, Hphi)
    assert np.allclose(mu, 2.5)
    phi = np.ones((3, 4))
    phi[1] = 0.0
    Hphi = np.stack([1.0 * phi[0], 0 * phi[1], 3.0 * phi[2]])
    assert np.allclose(spin1.chemical_potentials(phi, Hphi), [1.0, 2.0, 3.0])


@pytest.mark.parametrize("M", [0.0, 0.25, -0.6])
def test_project_SM_lands_on_SM(M):
    """The scaling onto S_M: mass h^d sum |phi|^2 = 1, magnetization
    N_1 - N_-1 = M, the scale factors obey sigma_1 sigma_-1 = sigma_0^2, a
    point already on S_M is left unchanged, and a vanishing phi_0 stays zero
    while N_{+-1} = (1 +- M) / 2."""
    rng = np.random.default_rng(21)
    cell = 0.3
    phi = rng.uniform(0.1, 1.0, (3, 16, 12))
    out = gs.project_SM(phi, M, cell)
    N = cell * np.sum(out.reshape(3, -1) ** 2, axis=1)
    assert abs(N.sum() - 1.0) < 1e-13 and abs(N[0] - N[2] - M) < 1e-13
    sig = (out / phi).reshape(3, -1)
    assert np.ptp(sig, axis=1).max() < 1e-13          # one factor per component
    s1, s0, sm = sig[:, 0]
    assert abs(s1 * sm - s0 * s0) < 1e-13 * s0 * s0
    np.testing.assert_allclose(gs.project_SM(out, M, cell), out, rtol=1e-13, atol=0)
    phi[1] = 0.0
    out = gs.project_SM(phi, M, cell)
    N = cell * np.sum(out.reshape(3, -1) ** 2, axis=1)
    assert N[1] == 0.0
    np.testing.assert_allclose(N[[0, 2]], [(1 + M) / 2, (1 - M) / 2], rtol=1e-13)


def test_newton_step_converges_quadratically(ground):
    """The inexact Newton step of the ground-state solver (Hessian H_+ on the
    tangent space of S_M, solved to 1e-13): from a converged state moved by
    delta along a smooth direction and projected back onto S_M, the residual
    after one step falls as the square of the residual before it (the
    observed order between delta = 1e-2 and 1e-3 is 2 within 0.1, and the
    step gains at least a factor 100 at delta = 1e-3).  A wrong Hessian
    converges linearly or not at all."""
    w = synth.Workload("zq1d", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.0, 0.0, 0.1, M=0.2, gs_seed=7)
    V, phi, _ = ground(w)
    V = V.reshape(w.n)
    phi = phi.reshape((3,) + w.n)
    cell = gs.cell_volume(w)
    x = synth.axes(w)[0]
    d = np.stack([np.exp(-0.3 * (x - s) ** 2) * (1 + 0.3 * np.sin(k * x))
                  for s, k in ((0.2, 1.0), (-0.5, 2.0), (0.7, 3.0))])
    r0s, r1s = [], []
    for delta in (1e-2, 1e-3):
        p0 = gs.project_SM(phi + delta * d, w.M, cell)
        r0, _ = gs.nlep_residual(p0, V, w)
        r1, _ = gs.nlep_residual(gs.newton_step(p0, V, w, 10.0, cell, eta=1e-13, maxcg=3000), V, w)
        r0s.append(r0)
        r1s.append(r1)
    order = np.log(r1s[0] / r1s[1]) / np.log(r0s[0] / r0s[1])
    assert abs(order - 2.0) < 0.1, (order, r0s, r1s)
    assert r1s[1] < 1e-2 * r0s[1], (r0s, r1s)


def _smooth(w, seed):
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*synth.axes(w), indexing="ij")
    r2 = sum(g * g for g in grids)
    return np.stack([np.exp(-0.2 * r2) * (0.5 + rng.uniform()) * (1 + 0.2 * np.sin(grids[0] + rng.uniform(0, 6)))
                     for _ in range(3)])


@pytest.mark.parametrize("w", [
    synth.Workload("e1d", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.5, 0.07, 0.2),
    synth.Workload("e2d", (16, 12), (-5.0, -4.0), (5.0, 4.0), (1.0, 1.3), 20.0, 2.0, -0.03, 0.1)],
    ids=lambda w: w.name)
def test_energy_derivative_is_twice_the_hamiltonian(w):
    """eq. energy and eq. NLEP: for real Phi and a real direction d,
    dE(Phi + e d)/de at e = 0 equals 2 h^d <d, H Phi> (central differences
    to 1e-8), the Zeeman terms of reading P1 included.  This ties the
    energy (gradient term by Parseval) to the Hamiltonian (spectral
    Laplacian) through two different formulas."""
    V = synth.potential(w)
    phi = _smooth(w, 3)
    d = _smooth(w, 4) - _smooth(w, 5)
    eps = 1e-5
    fd = (gs.energy(phi + eps * d, V, w) - gs.energy(phi - eps * d, V, w)) / (2 * eps)
    H = spin1.hamiltonian(phi, V, w, w.beta_n, w.beta_s, w.p, w.q)
    exact = 2.0 * gs.cell_volume(w) * np.sum(d * H)
    assert abs(fd - exact) < 1e-8 * abs(exact), (fd, exact)


def test_gradient_flow_is_energy_diminishing():
    """The flow phase of the ground-state solver lowers the energy of
    eq. energy at every step (its docstring's claim; the stabiliser alpha
    keeps the explicit factors non-negative): 40 steps from the seeded start
    on S_M, energies non-increasing to rounding."""
    w = synth.Workload("fl1d", (64,), (-8.0,), (8.0,), (1.0,), 30.0, -2.0, 0.0, 0.1, M=0.2, gs_seed=9)
    V = synth.potential(w)
    phi0 = synth.initial_spinor(w)
    E = []
    for k in range(0, 41, 2):
        phi, _, _, _ = gs.ground_state(w, V, phi0, tol=0.0, maxit=k, newton_start=0.0)
        E.append(gs.energy(phi, V, w))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-13 * np.abs(E[:-1])), E
    assert E[-1] < E[0] - 1e-3 * abs(E[0])


def test_ground_state_minimises_the_energy_on_S_M(ground):
    """eq. groundDef: moving the computed ground state by e d and projecting
    back onto S_M raises the energy, and the rise is of second order in e
    (the first-order term vanishes at a stationary point of E on S_M):
    the observed order between e = 1e-2 and 1e-3 is 2 within 0.05."""
    w = synth.Workload("zq1d", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.0, 0.0, 0.1, M=0.2, gs_seed=7)
    V, phi, _ = ground(w)
    V = V.reshape(w.n)
    phi = phi.reshape((3,) + w.n)
    cell = gs.cell_volume(w)
    E0 = gs.energy(phi, V, w)
    for seed in (6, 7, 8):
        d = _smooth(w, seed) - _smooth(w, seed + 10)
        rise = [gs.energy(gs.project_SM(phi + e * d, w.M, cell), V, w) - E0 for e in (1e-2, 1e-3)]
        assert min(rise) > 0, rise
        order = np.log(rise[0] / rise[1]) / np.log(10.0)
        assert abs(order - 2.0) < 0.05, (seed, rise, order)
