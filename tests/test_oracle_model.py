"""Pins of the spin-1 model and the discrete BdG operator.

- Spin matrices: commutator [S_x, S_y] = i S_z and Casimir S.S = s(s+1) I = 2 I.
- The compact Hamiltonian (eq. GPEs) equals the componentwise GPE (eq. GPE).
- A and B (eqs. def_A, def_B) are the linearization of the componentwise GPE
  at a real Phi: G(Phi + e d) = G(Phi) + e (A d + B conj(d)) + O(e^2),
  checked by central differences with complex d (this fixes A and B entirely).
- H_- Phi = H Phi - Lambda Phi for any real Phi (Section 2.3 proofs).
- The three evaluations of the operator agree; UV and FG forms are related by
  the change of variables (eqs. c-o-v, lrep-d); A, B are symmetric.
- Non-interacting limit: H_+ = H_- = -1/2 Lap + V - mu acting on harmonic
  oscillator states gives the oscillator energies.
"""
import numpy as np
import pytest

import synth
from oracle import apply as ap
from oracle import discretization as disc
from oracle import spin1

from conftest import relerr

W1 = synth.Workload("t1d", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.0, 0.03, 0.07)
W2 = synth.Workload("t2d", (16, 16), (-6.0, -6.0), (6.0, 6.0), (1.0, 1.5), 20.0, 1.5, 0.0, 0.2)


def test_spin_matrices():
    SX, SY, SZ = spin1.SPIN
    assert np.allclose(SX @ SY - SY @ SX, 1j * SZ)
    assert np.allclose(SY @ SZ - SZ @ SY, 1j * SX)
    assert np.allclose(SX @ SX + SY @ SY + SZ @ SZ, 2 * np.eye(3))
    for S in spin1.SPIN:
        assert np.allclose(S, S.conj().T)


def _rand_state(w, seed):
    rng = np.random.default_rng(seed)
    env = np.exp(-0.25 * sum(g ** 2 for g in np.meshgrid(*synth.axes(w), indexing="ij")))
    return np.stack([env * (0.5 + rng.uniform()) for _ in range(3)]) * (
        1 + 0.1 * rng.standard_normal((3,) + w.n))


@pytest.mark.parametrize("w", [W1, W2])
def test_compact_equals_componentwise_gpe(w):
    rng = np.random.default_rng(1)
    psi = _rand_state(w, 2) * np.exp(1j * rng.uniform(0, 2 * np.pi, (3,) + w.n))
    V = synth.potential(w)
    a = spin1.hamiltonian(psi, V, w, w.beta_n, w.beta_s, w.p, w.q)
    b = spin1.gpe_rhs_componentwise(psi, V, w, w.beta_n, w.beta_s, w.p, w.q)
    assert relerr(a, b) < 1e-13


@pytest.mark.parametrize("w", [W1, W2])
def test_A_B_are_the_linearization_of_the_gpe(w):
    rng = np.random.default_rng(5)
    phi = _rand_state(w, 7)
    V = synth.potential(w)
    mu = np.array([1.3, -0.4, 2.2])
    op = ap.Operator(w, phi, V, mu)
    d = rng.standard_normal((3,) + w.n) + 1j * rng.standard_normal((3,) + w.n)
    lam = mu.reshape((3,) + (1,) * w.dim)

    def G(psi):
        return spin1.gpe_rhs_componentwise(psi, V, w, w.beta_n, w.beta_s, w.p, w.q) - lam * psi

    eps = 1e-5
    fd = (G(phi + eps * d) - G(phi - eps * d)) / (2 * eps)
    x = np.concatenate([d.reshape(1, 3, -1), np.conj(d).reshape(1, 3, -1)], axis=1)
    lin = op.apply_fft(x, ap.UV)[0, :3].reshape(fd.shape)
    assert relerr(lin, fd) < 1e-9


@pytest.mark.parametrize("w", [W1, W2])
def test_hminus_phi_is_nlep_residual(w):
    phi = _rand_state(w, 11)
    V = synth.potential(w)
    mu = np.array([0.7, 0.9, 1.1])
    op = ap.Operator(w, phi, V, mu)
    hm = op.hminus(phi.reshape(1, 3, -1))[0]
    r = spin1.hamiltonian(phi, V, w, w.beta_n, w.beta_s, w.p, w.q).reshape(3, -1) - mu[:, None] * phi.reshape(3, -1)
    assert relerr(hm, r) < 1e-13


@pytest.mark.parametrize("w", [W1, W2])
def test_three_applies_agree_and_forms(w):
    phi = _rand_state(w, 13)
    V = synth.potential(w)
    op = ap.Operator(w, phi, V, np.array([0.3, 0.2, 0.1]))
    x = synth.random_block(w, 3, seed=4)
    for mode in (ap.UV, ap.FG):
        y1 = op.apply_fft(x, mode)
        assert relerr(op.apply_dft(x, mode), y1) < 1e-13
        assert relerr(op.apply_dense(x, mode), y1) < 1e-13
    A, B = op.dense_blocks()
    assert np.allclose(A, A.T, atol=1e-12) and np.allclose(B, B.T, atol=1e-12)
    # UV of (f+g, f-g) = [H+f + H-g ; H-g - H+f]
    fg = x
    yfg = op.apply_fft(fg, ap.FG)
    yuv = op.apply_fft(ap.fg_to_uv(fg), ap.UV)
    hf, hg = yfg[:, :3], yfg[:, 3:]
    assert relerr(yuv, np.concatenate([hf + hg, hg - hf], axis=1)) < 1e-13


def test_closed_form_entries_of_A_B():
    """The pointwise A, B of the Pauli form against entries worked out by hand
    (real Phi = (a, b, c), rho = a^2 + b^2 + c^2)."""
    rng = np.random.default_rng(2)
    a, b, c, V = rng.uniform(-1, 1, 4)
    bn, bs, p, q = 3.0, -0.7, 0.2, 0.4
    mu = np.array([0.5, -0.25, 1.5])
    Apt, Bpt = spin1.pointwise_blocks(np.array([[a], [b], [c]]), np.array([V]), bn, bs, mu, p, q)
    rho = a * a + b * b + c * c
    A = np.array([
        [V + q - p - mu[0] + bn * (rho + a * a) + bs * (2 * a * a + b * b - c * c),
         bn * a * b + bs * b * (a + 2 * c), (bn - bs) * a * c],
        [0, V - mu[1] + bn * (rho + b * b) + bs * (a * a + c * c), bn * b * c + bs * b * (2 * a + c)],
        [0, 0, V + q + p - mu[2] + bn * (rho + c * c) + bs * (2 * c * c + b * b - a * a)]])
    A = np.triu(A) + np.triu(A, 1).T
    B = np.array([[(bn + bs) * a * a, (bn + bs) * a * b, bn * a * c + bs * (b * b - a * c)],
                  [0, bn * b * b + 2 * bs * a * c, (bn + bs) * b * c],
                  [0, 0, (bn + bs) * c * c]])
    B = np.triu(B) + np.triu(B, 1).T
    assert np.allclose(Apt[0], A, atol=1e-14) and np.allclose(Bpt[0], B, atol=1e-14)


def test_non_interacting_oscillator_states():
    w = synth.Workload("free", (64,), (-10.0,), (10.0,), (1.3,), 0.0, 0.0)
    x = synth.axes(w)[0]
    g = w.gamma[0]
    phi0 = np.exp(-g * x * x / 2)
    phi = np.stack([phi0, phi0, phi0])
    mu = np.full(3, g / 2)
    op = ap.Operator(w, phi, synth.potential(w), mu)
    # first excited oscillator state: energy 3g/2 -> H_+/- eigenvalue g
    psi1 = x * phi0
    v = np.stack([psi1, 0 * psi1, psi1]).reshape(1, 3, -1)
    for y in (op.hplus(v), op.hminus(v)):
        assert relerr(y, g * v) < 1e-12


def test_vanishing_component_rule_is_relative():
    """Reading P3: a component counts as vanishing when ||phi_j||^2 <
    1e-20 ||Phi||^2 (unweighted sums), and then takes mu_j from
    mu_1 + mu_-1 = 2 mu_0.  The antiferromagnetic state (a, 0, a) with a
    remnant phi_0 = 1e-12 a (relative norm^2 1e-24; an absolute threshold of
    1e-24 would not catch it on a 64-point grid) gives mu_0 = (mu_1 + mu_-1)/2
    exactly, whatever the remnant's shape; a populated phi_0 = 1e-6 a keeps
    its own Rayleigh quotient."""
    w = W1
    V = synth.potential(w)
    x = synth.axes(w)[0]
    a = np.exp(-0.5 * x ** 2)
    for eps, vanishing in ((1e-12, True), (1e-6, False)):
        phi = np.stack([a, eps * a * (1.0 + x), a])
        H = spin1.hamiltonian(phi, V, w, w.beta_n, w.beta_s, w.p, w.q)
        mu = spin1.chemical_potentials(phi, H)
        own0 = np.dot(phi[1], H[1]) / np.dot(phi[1], phi[1])
        if vanishing:
            assert np.sum(phi[1] ** 2) > 1e-24 and abs(mu[1] - 0.5 * (mu[0] + mu[2])) < 1e-12
            assert abs(own0 - mu[1]) > 1e-3
        else:
            assert abs(mu[1] - own0) < 1e-12 * abs(own0)


@pytest.mark.parametrize("w", [W1, W2, synth.Workload("t3d", (8, 6, 10), (-3.0, -2.0, -4.0), (3.0, 2.0, 4.0),
                                                      (1.0, 1.3, 0.7), 15.0, -0.8, 0.02, 0.15)])
def test_apply_at_nodes_matches_the_whole_product(w):
    """The per-node product (rows of the 1-D spectral Laplacians on the grid
    lines through a node, the pointwise blocks at the node) equals the dense
    6P x 6P product at those nodes, both forms, corner nodes included."""
    phi = _rand_state(w, 17)
    V = synth.potential(w)
    mu = np.array([0.4, 0.6, 0.5])
    op = ap.Operator(w, phi, V, mu)
    x = synth.random_block(w, 2, seed=8)
    rng = np.random.default_rng(9)
    nodes = [tuple(0 for _ in w.n), tuple(nn - 1 for nn in w.n)] + \
        [tuple(int(rng.integers(0, nn)) for nn in w.n) for _ in range(10)]
    flat = [int(np.ravel_multi_index(nd, w.n)) for nd in nodes]
    ph = phi.reshape(3, -1)[:, flat]
    Vn = V.reshape(-1)[flat]
    for v in range(2):
        grid = x[v].reshape((6,) + w.n)
        lines = []
        for a in range(w.dim):
            per = []
            for nd in nodes:
                sl = list(nd)
                sl[a] = slice(None)
                per.append(grid[(slice(None),) + tuple(sl)])
            lines.append(np.stack(per))
        for mode in (ap.UV, ap.FG):
            ref = op.apply_dense(x[v:v + 1], mode)[0][:, flat].T
            got = ap.apply_at_nodes(w, ph, Vn, mu, lines, nodes, mode)
            assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max(), (w.name, mode)
