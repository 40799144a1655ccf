"""Pins of the oracle's perturbed densities (Section 4.2, "2D Case" example;
eq. waveAssump with a single mode) against closed forms that do not go
through its formula: single-amplitude modes whose modulus is elementary,
the time average over a period, the analytical Kohn pair (a dipole
oscillation of the density), and brute force with scalar complex
arithmetic on a tiny grid."""
import cmath
import math

import numpy as np

import synth
from oracle import kohn
from oracle.perturbed import perturbed_density

W = synth.Workload("pd1d", (32,), (-6.0,), (6.0,), (1.0,), 10.0, -1.0)


def _gauss_phi(w, widths=(1.0, 1.3, 0.8), shifts=(0.0, 0.4, -0.3)):
    x = synth.axes(w)[0]
    return np.stack([np.exp(-((x - s) / a) ** 2 / 2.0) for a, s in zip(widths, shifts)])


def test_zero_amplitude_gives_ground_density():
    rng = np.random.default_rng(1)
    phi = _gauss_phi(W)
    U = rng.standard_normal((2, 3, W.npts)) + 1j * rng.standard_normal((2, 3, W.npts))
    n = perturbed_density(phi, U, U[::-1], [0.7, 1.9], [0.0, 1.3], 0.0)
    np.testing.assert_allclose(n, np.broadcast_to(phi ** 2, n.shape), rtol=0, atol=0)


def test_single_amplitudes_with_imaginary_factor():
    """u = i c phi, v = 0  and  u = 0, v = i c phi both give
    phi^2 (1 + 2 eps c sin(omega t) + eps^2 c^2): the sign of the sine term
    fixes both the e^{-i omega t} on u and the conjugate on v."""
    phi = _gauss_phi(W)
    c, eps, om = 0.8, 0.1, 1.7
    times = np.array([0.0, 0.3, 1.1, 2.5, 4.0])
    Z = np.zeros((1, 3, W.npts), complex)
    A = (1j * c * phi)[None]
    expect = phi[None] ** 2 * (1.0 + 2 * eps * c * np.sin(om * times)[:, None, None] + (eps * c) ** 2)
    np.testing.assert_allclose(perturbed_density(phi, A, Z, [om], times, eps)[0], expect, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(perturbed_density(phi, Z, A, [om], times, eps)[0], expect, rtol=1e-14, atol=1e-16)


def test_single_real_amplitude():
    """u = c phi (real), v = 0: phi^2 (1 + 2 eps c cos(omega t) + eps^2 c^2)."""
    phi = _gauss_phi(W)
    c, eps, om = -1.3, 0.05, 0.9
    times = np.array([0.0, 0.7, 3.3])
    expect = phi[None] ** 2 * (1.0 + 2 * eps * c * np.cos(om * times)[:, None, None] + (eps * c) ** 2)
    got = perturbed_density(phi, (c * phi)[None], np.zeros((1, 3, W.npts)), [om], times, eps)[0]
    np.testing.assert_allclose(got, expect, rtol=1e-14, atol=1e-16)


def test_period_average():
    """Over one period the terms of first and second harmonic average out:
    the mean of 8 equispaced samples is phi^2 + eps^2 (|u|^2 + |v|^2)."""
    rng = np.random.default_rng(7)
    phi = _gauss_phi(W)
    U = rng.standard_normal((3, 3, W.npts)) + 1j * rng.standard_normal((3, 3, W.npts))
    V = rng.standard_normal((3, 3, W.npts)) + 1j * rng.standard_normal((3, 3, W.npts))
    om = np.array([0.6, 1.0, 2.3])
    eps = 0.2
    for l in range(3):
        times = np.arange(8) * (2 * math.pi / om[l] / 8) + 0.37
        n = perturbed_density(phi, U[l:l + 1], V[l:l + 1], om[l:l + 1], times, eps)[0]
        expect = phi ** 2 + eps ** 2 * (np.abs(U[l]) ** 2 + np.abs(V[l]) ** 2)
        np.testing.assert_allclose(n.mean(0), expect, rtol=1e-13, atol=1e-15)


def test_kohn_mode_is_a_dipole_oscillation():
    """The analytical Kohn pair (Theorem "Analytical eigenpairs":
    f = d_x phi / sqrt(2 gamma), g = -sqrt(gamma/2) x phi, u = f + g,
    v = f - g, omega = gamma): at t = 0 the density is (phi + delta d_x phi)^2,
    delta = eps sqrt(2/gamma), i.e. the condensate displaced by -delta to
    first order; a quarter period later it is phi^2 (1 + 2 gamma eps^2 x^2)."""
    w = synth.Workload("pd_kohn", (64,), (-8.0,), (8.0,), (1.3,), 10.0, -1.0)
    phi = _gauss_phi(w, widths=(1.1, 1.1, 1.1), shifts=(0.0, 0.0, 0.0)) * np.array([[0.5], [0.6], [0.3]])
    (gam, f, g), = kohn.kohn_modes(w, phi)
    U, V = (f + g)[None], (f - g)[None]
    eps = 0.05
    times = np.array([0.0, 0.5 * math.pi / gam])
    n = perturbed_density(phi, U, V, [gam], times, eps)[0]
    x = synth.axes(w)[0]
    dphi = -x / 1.1 ** 2 * phi       # exact derivative of the Gaussian
    delta = eps * math.sqrt(2.0 / gam)
    np.testing.assert_allclose(n[0], (phi + delta * dphi) ** 2, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(n[1], phi ** 2 * (1.0 + 2.0 * gam * eps ** 2 * x ** 2), rtol=1e-12, atol=1e-15)


def test_brute_force_scalar_loops():
    """Scalar cmath evaluation of the ansatz's modulus on four points."""
    rng = np.random.default_rng(3)
    P = 4
    phi = rng.standard_normal((3, P))
    U = rng.standard_normal((2, 3, P)) + 1j * rng.standard_normal((2, 3, P))
    V = rng.standard_normal((2, 3, P)) + 1j * rng.standard_normal((2, 3, P))
    om, times, eps = [0.4, 1.6], [0.0, 0.9, 2.2], 0.3
    n = perturbed_density(phi, U, V, om, times, eps)
    for l in range(2):
        for it, t in enumerate(times):
            for j in range(3):
                for x in range(P):
                    z = complex(phi[j, x]) + eps * (complex(U[l, j, x]) * cmath.exp(complex(0, -om[l] * t))
                                                    + complex(V[l, j, x]).conjugate() * cmath.exp(complex(0, om[l] * t)))
                    assert abs(n[l, it, j, x] - (z.real ** 2 + z.imag ** 2)) <= 1e-13 * max(1.0, abs(z) ** 2)
