"""Analytical eigenpairs for harmonic traps (Theorem "Analytical eigenpairs",
eq. eig-pair) and the error metrics of Section 4.1.

  omega_alpha = gamma_alpha,
  f_alpha = (1/sqrt2) gamma^{-1/2} d_alpha Phi_g,  g_alpha = -(1/sqrt2) gamma^{1/2} x_alpha Phi_g,
  u = f + g, v = f - g.
  e_omega = |omega_N - omega| / |omega|,
  e_uv = |u_N - P_u u_N| / |u_N| + |v_N - P_v v_N| / |v_N|, P the l2
  projector onto the analytical eigenspace of that eigenvalue.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU leg, never by the product library.
"""
from __future__ import annotations

import numpy as np

from . import discretization as disc


def kohn_modes(w, phi):
    """[(omega_alpha, f, g)] for alpha over the axes; f, g of shape (3, P)."""
    phi = np.asarray(phi, dtype=np.float64).reshape((3,) + tuple(w.n))
    grids = np.meshgrid(*[lo + np.arange(nn) * (hi - lo) / nn
                          for nn, lo, hi in zip(w.n, w.lo, w.hi)], indexing="ij")
    out = []
    for ax, gam in enumerate(w.gamma):
        d = np.stack([disc.spectral_derivative(phi[j], ax, w.lo, w.hi) for j in range(3)])
        f = d / np.sqrt(2.0 * gam)
        g = -np.sqrt(gam / 2.0) * grids[ax][None] * phi
        out.append((gam, f.reshape(3, -1), g.reshape(3, -1)))
    return out


def e_omega(om_num, om_exact):
    return abs(om_num - om_exact) / abs(om_exact)


def e_uv(u_num, v_num, U_exact, V_exact):
    """Projector error of Section 4.1 for one computed pair against the span of
    the analytical vectors (columns of U_exact / V_exact)."""
    def proj_err(x, B):
        Q, _ = np.linalg.qr(B)
        return np.linalg.norm(x - Q @ (Q.conj().T @ x)) / np.linalg.norm(x)
    return proj_err(u_num, U_exact) + proj_err(v_num, V_exact)
