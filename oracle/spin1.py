"""Spin-1 model: spin matrices, the BdG operators A and B, the GPE and its
stationary (NLEP) form.

Sources (Section 1 and Section 2.1):
  spin-1 matrices S_x, S_y, S_z and the spin vector s(Psi) = (Psi^H S_j Psi);
  GPE, componentwise (eq. GPE) and compact (eq. GPEs);
  NLEP  Lambda Phi = H Phi, H = (L + beta_n rho) I_3 + beta_s S.s(Phi)
  (eq. NLEP), chemical potentials (eq. chem-formula) with mu_1+mu_-1 = 2 mu_0;
  A = (L I - Lambda) + beta_n (rho I + Phi Phi^H)
      + beta_s (S.s(Phi) + sum_j S_j Phi Phi^H S_j^H)           (eq. def_A)
  B = beta_n Phi Phi^T + beta_s sum_j S_j Phi Phi^T S_j^T        (eq. def_B)
and their discrete forms (eqs. def_bfA, def_bfB).

Zeeman terms: the paper has none; this oracle adds the single-particle term
-p S_z + q S_z^2 to L (reading P1), i.e. diag(q-p, 0, q+p) on the diagonal of
H and of A, nothing on B.  Component order is (1, 0, -1).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU leg, never by the product library.
"""
from __future__ import annotations

import numpy as np

from . import discretization as disc

SQ2 = np.sqrt(2.0)
SX = np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]], dtype=np.complex128) / SQ2
SY = 1j * np.array([[0, -1, 0], [1, 0, -1], [0, 1, 0]], dtype=np.complex128) / SQ2
SZ = np.diag([1.0, 0.0, -1.0]).astype(np.complex128)
SPIN = (SX, SY, SZ)


def zeeman_diag(p: float, q: float) -> np.ndarray:
    """Diagonal of -p S_z + q S_z^2 (reading P1)."""
    return (-p * SZ + q * (SZ @ SZ)).diagonal().real


def spin_vector(phi: np.ndarray) -> np.ndarray:
    """s_j(Phi) = Phi^H S_j Phi at every point; phi has shape (3, ...)."""
    return np.stack([np.einsum("a...,ab,b...->...", phi.conj(), S, phi) for S in SPIN])


def pointwise_blocks(phi: np.ndarray, V: np.ndarray, beta_n: float, beta_s: float,
                     mu, p: float = 0.0, q: float = 0.0):
    """Pointwise 3x3 parts of A and B at every node, built literally from the
    Pauli-matrix expressions of eqs. def_A / def_B (the -1/2 Laplacian is not
    included).  Returns (Apt, Bpt), each of shape (P, 3, 3) complex, where
    P = number of nodes and phi has shape (3, P)."""
    phi = np.asarray(phi, dtype=np.complex128).reshape(3, -1)
    npts = phi.shape[1]
    V = np.asarray(V, dtype=np.float64).reshape(-1)
    rho = np.sum(np.abs(phi) ** 2, axis=0)
    s = spin_vector(phi)
    z = zeeman_diag(p, q)
    I3 = np.eye(3)
    S = np.stack(SPIN)                                   # (3 spins, 3, 3)
    ff_h = np.einsum("ap,bp->pab", phi, phi.conj())      # Phi Phi^H per node
    ff_t = np.einsum("ap,bp->pab", phi, phi)             # Phi Phi^T per node
    sdots = np.einsum("jp,jab->pab", s, S)               # S . s(Phi)
    sum_a = np.einsum("jac,pcd,jbd->pab", S, ff_h, S.conj())   # sum_j S_j Phi Phi^H S_j^H
    sum_b = np.einsum("jac,pcd,jbd->pab", S, ff_t, S)          # sum_j S_j Phi Phi^T S_j^T
    diag = np.diag(z) - np.diag(np.asarray(mu, dtype=np.float64))
    Apt = (V[:, None, None] * I3 + diag
           + beta_n * (rho[:, None, None] * I3 + ff_h) + beta_s * (sdots + sum_a))
    Bpt = beta_n * ff_t + beta_s * sum_b
    return Apt, Bpt


def hamiltonian(phi: np.ndarray, V: np.ndarray, w, beta_n: float, beta_s: float,
                p: float = 0.0, q: float = 0.0) -> np.ndarray:
    """H Phi of eq. NLEP (compact form, eq. GPEs) with the spectral Laplacian;
    phi has shape (3,)+grid, real or complex."""
    lap = disc.laplacian_fft(phi, w.lo, w.hi)
    if not np.iscomplexobj(phi):
        lap = lap.real
    rho = np.sum(np.abs(phi) ** 2, axis=0)
    s = spin_vector(phi.reshape(3, -1)).reshape((3,) + phi.shape[1:])
    out = -0.5 * lap + (V + beta_n * rho)[None] * phi
    z = zeeman_diag(p, q)
    for j in range(3):
        out = out + beta_s * np.einsum("ab,...,b...->a...", SPIN[j], s[j], phi)
    out = out + z.reshape((3,) + (1,) * (phi.ndim - 1)) * phi
    if not np.iscomplexobj(phi):
        out = out.real
    return out


def gpe_rhs_componentwise(psi: np.ndarray, V: np.ndarray, w, beta_n: float,
                          beta_s: float, p: float = 0.0, q: float = 0.0) -> np.ndarray:
    """Right-hand side of the componentwise GPE (eq. GPE), with the Zeeman
    diagonal of reading P1; psi complex of shape (3,)+grid.  Written from the
    three printed equations, independently of the compact Pauli form."""
    p1, p0, pm = psi
    lap = disc.laplacian_fft(psi, w.lo, w.hi)
    rho = np.abs(p1) ** 2 + np.abs(p0) ** 2 + np.abs(pm) ** 2
    rhoz = np.abs(p1) ** 2 - np.abs(pm) ** 2
    z = zeeman_diag(p, q)
    r1 = (-0.5 * lap[0] + (V + beta_n * rho + beta_s * (np.abs(p0) ** 2 + rhoz)) * p1
          + beta_s * p0 ** 2 * np.conj(pm) + z[0] * p1)
    r0 = (-0.5 * lap[1] + (V + beta_n * rho + beta_s * (np.abs(p1) ** 2 + np.abs(pm) ** 2)) * p0
          + 2 * beta_s * pm * np.conj(p0) * p1 + z[1] * p0)
    rm = (-0.5 * lap[2] + (V + beta_n * rho + beta_s * (np.abs(p0) ** 2 - rhoz)) * pm
          + beta_s * np.conj(p1) * p0 ** 2 + z[2] * pm)
    return np.stack([r1, r0, rm])


ZERO_COMPONENT = 1e-20


def chemical_potentials(phi: np.ndarray, Hphi: np.ndarray) -> np.ndarray:
    """mu_j = <phi_j, (H Phi)_j> / ||phi_j||^2 (eq. chem-formula), with the
    relation mu_1 + mu_-1 = 2 mu_0 filling components that vanish
    (||phi_j||^2 < 1e-20 ||Phi||^2 on unweighted grid sums; reading P3).  A
    component that small is the decayed remnant of a ground-state iteration;
    its own Rayleigh quotient is the energy of its slowest mode, not a
    Lagrange multiplier of the stationary state."""
    phi = phi.reshape(3, -1)
    Hphi = Hphi.reshape(3, -1)
    nrm = np.sum(np.abs(phi) ** 2, axis=1)
    small = nrm < ZERO_COMPONENT * np.sum(nrm)
    mu = np.full(3, np.nan)
    for j in range(3):
        if not small[j]:
            mu[j] = np.real(np.vdot(phi[j], Hphi[j])) / nrm[j]
    z1, z0, zm = small
    if z0 and not z1 and not zm:
        mu[1] = 0.5 * (mu[0] + mu[2])
    elif z1 and zm and not z0:
        mu[0] = mu[2] = mu[1]
    elif z1 and not zm and not z0:
        mu[0] = 2 * mu[1] - mu[2]
    elif zm and not z1 and not z0:
        mu[2] = 2 * mu[1] - mu[0]
    return mu
