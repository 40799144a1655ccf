"""Ground state on S_M by a normalized gradient flow (eq. groundDef).

The paper computes Phi_g with a PCG method that it cites but does not
describe; this oracle reaches the same minimizer with the normalized gradient
flow of the cited spin-1 literature, discretized in the Fourier
pseudospectral basis of Section 3.1:

  flow    (1/tau + alpha - 1/2 Lap) Phi* = (1/tau + alpha) Phi^n - N(Phi^n) Phi^n,
          Phi^{n+1} = projection of Phi* onto S_M,
          where N(Phi) Phi = H Phi + 1/2 Lap Phi is the non-kinetic part of
          eq. NLEP (trap, density, spin and Zeeman terms) and alpha a
          stabilizing constant above max N; the kinetic term and alpha are implicit and
          diagonal in Fourier space.  The flow diminishes the energy but its
          fixed point carries an O(tau) bias, so it only brings Phi near the
          minimizer.
  project phi_j = sigma_j phi*_j with ||Phi||^2 = 1, ||phi_1||^2 - ||phi_-1||^2 = M
          and sigma_1 sigma_-1 = sigma_0^2, solved in closed form.
  Newton  inexact Newton steps on S_M with the Hessian H_+ = A + B of the
          Lagrangian (eqs. def_A + def_B at a real Phi), solved by projected
          PCG with the Fourier preconditioner (alpha - 1/2 Lap)^-1 -- a
          preconditioned conjugate gradient method in the spirit of the PCG
          solver the paper uses.  Multipliers mu_j = mu + j lambda are the
          least-squares fit of H Phi ~ (mu + lambda S_z) Phi, which keeps
          mu_1 + mu_-1 = 2 mu_0.
  stop    max_j max_x |(H Phi)_j - mu_j phi_j| <= tol with mu_j from
          eq. chem-formula.

Norms carry the quadrature weight h^d (the discrete inner product of
Section 3.3 with n = 0..N-1).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU leg, never by the product library.
"""
from __future__ import annotations

import numpy as np

from . import discretization as disc
from . import spin1


def cell_volume(w) -> float:
    return float(np.prod(w.h))


def project_SM(phi: np.ndarray, M: float, cell: float) -> np.ndarray:
    """Scale the three components onto S_M: returns sigma_j phi_j with
    sum_j sigma_j^2 N_j = 1, sigma_1^2 N_1 - sigma_-1^2 N_-1 = M and
    sigma_1 sigma_-1 = sigma_0^2, N_j = h^d ||phi_j||^2.  A component with
    N_j = 0 stays zero."""
    N = np.array([cell * np.sum(phi[j] ** 2) for j in range(3)])
    N1, N0, Nm = N
    s = (1.0 - M * M) / (N0 + np.sqrt(M * M * N0 * N0 + 4.0 * (1.0 - M * M) * N1 * Nm))
    sig = np.zeros(3)
    sig[1] = np.sqrt(s)
    if N1 > 0:
        sig[0] = np.sqrt(max(1.0 + M - s * N0, 0.0) / (2.0 * N1))
    if Nm > 0:
        sig[2] = np.sqrt(max(1.0 - M - s * N0, 0.0) / (2.0 * Nm))
    if N1 == 0 and Nm == 0:
        sig[1] = 1.0 / np.sqrt(N0)
    return sig.reshape((3,) + (1,) * (phi.ndim - 1)) * phi


def energy(phi, V, w) -> float:
    """The energy of eq. energy on the grid, for a real spinor phi of shape
    (3,)+grid: h^d sum_n [ 1/2 |grad phi_j|^2 + V |phi_j|^2 + beta_n/2 rho^2
    + beta_s/2 |s(Phi)|^2 ], the gradient term through Parseval as
    1/2 sum_k |mu_k|^2 |phi~_k|^2 (the interpolant's gradient, eq.
    laplace_approx), plus the Zeeman energy sum (q - p) |phi_1|^2 +
    (q + p) |phi_-1|^2 of reading P1.  Its derivative along a real d is
    2 h^d <d, H Phi>, and the ground state minimises it on S_M (eq. groundDef)."""
    phi = np.asarray(phi, dtype=np.float64)
    d = len(w.n)
    cell = cell_volume(w)
    npts = int(np.prod(w.n))
    axes = tuple(range(1, d + 1))
    spec = np.fft.fftn(phi, axes=axes) / npts
    k2 = np.zeros(w.n)
    for i in range(d):
        mu = disc.wavenumbers(w.n[i], w.lo[i], w.hi[i])
        shape = [1] * d
        shape[i] = w.n[i]
        k2 = k2 + (mu ** 2).reshape(shape)
    kinetic = 0.5 * npts * np.sum(k2[None] * np.abs(spec) ** 2)
    rho = np.sum(phi ** 2, axis=0)
    s = spin1.spin_vector(phi.reshape(3, -1)).real
    z = spin1.zeeman_diag(w.p, w.q)
    local = np.sum(np.asarray(V).reshape(w.n) * rho + 0.5 * w.beta_n * rho ** 2) + \
        0.5 * w.beta_s * np.sum(s ** 2) + np.sum(z.reshape((3,) + (1,) * d) * phi ** 2)
    return float(cell * (kinetic + local))


def nonkinetic(phi, V, w):
    """N(Phi) Phi: everything of H Phi except -1/2 Lap (eq. NLEP)."""
    rho = np.sum(phi ** 2, axis=0)
    s = spin1.spin_vector(phi.reshape(3, -1)).real.reshape((3,) + phi.shape[1:])
    out = (V + w.beta_n * rho)[None] * phi
    # real Phi: s_y(Phi) = 0, so only S_x and S_z (both real) contribute
    for j in (0, 2):
        out = out + w.beta_s * np.einsum("ab,...,b...->a...", spin1.SPIN[j].real, s[j], phi)
    z = spin1.zeeman_diag(w.p, w.q)
    return out + z.reshape((3,) + (1,) * (phi.ndim - 1)) * phi


def nlep_residual(phi, V, w):
    """(max |H Phi - Lambda Phi|, mu) for a real spinor phi of shape (3,)+grid."""
    Hphi = spin1.hamiltonian(phi, V, w, w.beta_n, w.beta_s, w.p, w.q)
    mu = spin1.chemical_potentials(phi, Hphi)
    r = Hphi - mu.reshape((3,) + (1,) * (phi.ndim - 1)) * phi
    return float(np.max(np.abs(r))), mu


def multipliers(phi, V, w, cell):
    """(mu + lambda, mu, mu - lambda): the least-squares fit of
    H Phi ~ (mu + lambda S_z) Phi in the weighted l2 norm."""
    Hphi = spin1.hamiltonian(phi, V, w, w.beta_n, w.beta_s, w.p, w.q)
    szphi = np.stack([phi[0], 0.0 * phi[1], -phi[2]])
    g = np.array([[np.sum(phi * phi), np.sum(phi * szphi)],
                  [np.sum(szphi * phi), np.sum(szphi * szphi)]]) * cell
    r = np.array([np.sum(phi * Hphi), np.sum(szphi * Hphi)]) * cell
    if g[1, 1] < 1e-300:
        mu, lam = r[0] / g[0, 0], 0.0
    else:
        mu, lam = np.linalg.solve(g, r)
    return np.array([mu + lam, mu, mu - lam])


def _weighted_Z(phi, cell):
    """Orthonormal (weighted) basis of span{Phi, S_z Phi}, the normal space of S_M."""
    szphi = np.stack([phi[0], 0.0 * phi[1], -phi[2]])
    cols = []
    for v in (phi, szphi):
        for c in cols:
            v = v - c * (cell * np.sum(c * v))
        nv = np.sqrt(cell * np.sum(v * v))
        if nv > 1e-10 * np.sqrt(cell * np.sum(phi * phi)):
            cols.append(v / nv)
    return cols


def _hplus_real(phi, mu, V, w, d):
    """H_+ d for real d: the linearization of H Phi - Lambda Phi at Phi
    (eqs. def_A + def_B with real perturbations), through the oracle apply."""
    from .apply import Operator
    op = Operator(w, phi, V, mu)
    return op.hplus(d.reshape(1, 3, -1))[0].reshape(d.shape)


def newton_step(phi, V, w, c, cell, eta=1e-2, maxcg=500):
    """One inexact Newton step on S_M: with r = H Phi - (mu + lambda S_z) Phi
    (least-squares multipliers) and P the projector onto the tangent space
    {d : <Phi, d> = <S_z Phi, d> = 0}, solve P H_+ P d = -r by preconditioned
    CG (preconditioner P (c - 1/2 Lap)^-1 P) to relative accuracy eta, then
    Phi <- project_SM(Phi + d).  H_+ is the Hessian of the Lagrangian on the
    tangent space; it is positive at the minimizer."""
    mu = multipliers(phi, V, w, cell)
    Hphi = spin1.hamiltonian(phi, V, w, w.beta_n, w.beta_s, w.p, w.q)
    lam = mu.reshape((3,) + (1,) * len(w.n))
    r = Hphi - lam * phi
    Z = _weighted_Z(phi, cell)

    def P(v):
        for z in Z:
            v = v - z * (cell * np.sum(z * v))
        return v

    def prec(v):
        return P(disc.inverse_kdiag(P(v), lambda k2: 1.0 / (c + 0.5 * k2), w.lo, w.hi))

    def A(v):
        return P(_hplus_real(phi, mu, V, w, P(v)))

    b = -P(r)
    x = np.zeros_like(b)
    res = b.copy()
    z = prec(res)
    p = z.copy()
    rz = np.sum(res * z)
    b0 = np.sqrt(np.sum(b * b))
    for _ in range(maxcg):
        Ap = A(p)
        pAp = np.sum(p * Ap)
        if pAp <= 0:
            break
        a = rz / pAp
        x = x + a * p
        res = res - a * Ap
        if np.sqrt(np.sum(res * res)) <= eta * b0:
            break
        z = prec(res)
        rz_new = np.sum(res * z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return project_SM(phi + x, w.M, cell)


def ground_state(w, V, phi0, tol: float = 1e-12, tau: float = 1.0, alpha=None,
                 maxit: int = 100000, verbose: bool = False, newton_start: float = 1e-3):
    """Ground state on S_M from phi0 (shape (3,)+grid); returns
    (phi, mu, residual, steps).

    Phase 1: the energy-diminishing flow with alpha = max_x of the
    non-kinetic potential (refreshed every 50 steps), which keeps every
    explicit factor (1/tau + alpha - N) non-negative, until the residual is below
    newton_start * (1 + max|mu|) or falls by less than 1% per 50 steps.
    Phase 2: inexact Newton steps on S_M (newton_step); if a Newton step does
    not reduce the residual the flow resumes for 50 steps."""
    V = np.asarray(V, dtype=np.float64).reshape(w.n)
    cell = cell_volume(w)
    phi = project_SM(np.array(phi0, dtype=np.float64).reshape((3,) + w.n), w.M, cell)

    def stab(phi):
        if alpha is not None:
            return alpha
        rho = np.sum(phi ** 2, axis=0)
        return float(np.max(V + (w.beta_n + abs(w.beta_s)) * rho)) + abs(w.p) + abs(w.q)

    it = 0
    res, mu = nlep_residual(phi, V, w)
    c = 1.0 / tau + stab(phi)
    phase, flow_left, last = 1, 0, np.inf
    while it < maxit and res > tol:
        if phase == 1 or flow_left > 0:
            rhs = c * phi - nonkinetic(phi, V, w)
            phi = project_SM(disc.inverse_kdiag(rhs, lambda k2: 1.0 / (c + 0.5 * k2), w.lo, w.hi),
                             w.M, cell)
            flow_left = max(flow_left - 1, 0)
            it += 1
            res, mu = nlep_residual(phi, V, w)
            if it % 50 == 0:
                c = 1.0 / tau + stab(phi)
                if phase == 1 and res > 0.99 * last:
                    phase = 2
                last = res
            if phase == 1 and res < newton_start * (1 + np.max(np.abs(mu))):
                phase = 2
        else:
            trial = newton_step(phi, V, w, c, cell)
            it += 1
            rt, mt = nlep_residual(trial, V, w)
            if rt < res:
                phi, res, mu = trial, rt, mt
            else:
                flow_left = 50
        if verbose and it % 50 == 0:
            print(it, phase, res)
    return phi, mu, res, it
