"""Perturbed densities of single excitation modes (Section 4.2, the
"2D Case" example; the wave-function ansatz eq. waveAssump with one mode).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU leg, never by the product library.

With one mode l kept in eq. waveAssump, component j of the wave function is

  Psi_j(x, t) = e^{-i mu_j t} [ phi_j(x) + eps ( u_j(x) e^{-i omega t} + conj(v_j(x)) e^{i omega t} ) ],

and the perturbed density is its squared modulus; the global phase
e^{-i mu_j t} drops out, so

  n_j(x, t) = | phi_j(x) + eps ( u_j(x) e^{-i omega t} + conj(v_j(x)) e^{i omega t} ) |^2,  j = 1, 0, -1.

This module evaluates that definition directly in complex FP64 (numpy), one
(mode, time) pair at a time.
"""
from __future__ import annotations

import numpy as np


def perturbed_density(phi, U, V, omega, times, eps):
    """n[l, t, j, x] for modes l (rows of U, V) and times t.

    phi    (3, P) real ground state (phi_1, phi_0, phi_-1).
    U, V   (nmode, 3, P) complex Bogoliubov amplitudes u^l, v^l.
    omega  (nmode,) excitation energies;  times (nt,);  eps the amplitude.
    """
    phi = np.asarray(phi, dtype=np.float64)
    U = np.asarray(U, dtype=np.complex128)
    V = np.asarray(V, dtype=np.complex128)
    omega = np.asarray(omega, dtype=np.float64).reshape(-1)
    times = np.asarray(times, dtype=np.float64).reshape(-1)
    nmode, nt = U.shape[0], times.size
    out = np.empty((nmode, nt) + phi.shape, dtype=np.float64)
    for l in range(nmode):
        for it, t in enumerate(times):
            psi = phi + eps * (U[l] * np.exp(-1j * omega[l] * t) + np.conj(V[l]) * np.exp(1j * omega[l] * t))
            out[l, it] = np.abs(psi) ** 2
    return out
