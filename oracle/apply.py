"""The discrete BdG operator (Section 3.1, eqs. def_bfA, def_bfB, BdG-d, lrep-d).

  A = -1/2 [[Lap]] (x) I_3 + blockdiag_n Apt(x_n),  B = blockdiag_n Bpt(x_n),
  UV form  [[A, B], [-B, -A]] [u; v]                       (eq. BdG-d)
  FG form  (H_+ f, H_- g) with H_+ = A + B, H_- = A - B     (eq. lrep-d)
with the pointwise parts Apt, Bpt from `spin1.pointwise_blocks` (the Pauli
form of eqs. def_A / def_B, real ground state).

Three independent evaluations:
  dense_matrix / apply_dense   the explicit 6P x 6P matrix (small P only);
  apply_dft                    the Laplacian by dense per-axis DFT matrices;
  apply_fft                    the Laplacian by numpy.fft;
and, for grids too large for those, apply_at_nodes: the product at chosen
nodes from the grid lines through them.
Vectors have shape (nvec, 6, P) with components (u_1, u_0, u_-1, v_1, v_0,
v_-1) in UV form and (f_1, f_0, f_-1, g_1, g_0, g_-1) in FG form, P the number
of nodes in C order.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU leg, never by the product library.
"""
from __future__ import annotations

import numpy as np

from . import discretization as disc
from . import spin1

UV, FG = 0, 1


class Operator:
    """The pointwise data of one BdG problem: Apt, Bpt (P,3,3), the grid."""

    def __init__(self, w, phi, V, mu):
        self.w = w
        self.shape = tuple(w.n)
        self.npts = int(np.prod(self.shape))
        Apt, Bpt = spin1.pointwise_blocks(np.asarray(phi).reshape(3, -1), V,
                                          w.beta_n, w.beta_s, mu, w.p, w.q)
        assert np.max(np.abs(Apt.imag)) < 1e-12 and np.max(np.abs(Bpt.imag)) < 1e-12
        self.Apt = Apt.real
        self.Bpt = Bpt.real
        self.mu = np.asarray(mu, dtype=np.float64)

    # ---- pointwise parts -------------------------------------------------
    def _point(self, x, mat):
        # x: (nvec, 3, P) -> sum_b mat[p, a, b] x[:, b, p]
        return np.einsum("pab,nbp->nap", mat, x)

    def _assemble(self, x, lap, mode):
        kin = -0.5 * lap
        a, b = x[:, :3], x[:, 3:]
        ka, kb = kin[:, :3], kin[:, 3:]
        if mode == UV:
            yu = ka + self._point(a, self.Apt) + self._point(b, self.Bpt)
            yv = -(kb + self._point(b, self.Apt) + self._point(a, self.Bpt))
            return np.concatenate([yu, yv], axis=1)
        yf = ka + self._point(a, self.Apt + self.Bpt)
        yg = kb + self._point(b, self.Apt - self.Bpt)
        return np.concatenate([yf, yg], axis=1)

    def apply_fft(self, x, mode=UV):
        x = np.asarray(x)
        grid = x.reshape(x.shape[:2] + self.shape)
        lap = disc.laplacian_fft(grid, self.w.lo, self.w.hi).reshape(x.shape)
        if not np.iscomplexobj(x):
            lap = lap.real
        return self._assemble(x, lap, mode)

    def apply_dft(self, x, mode=UV):
        x = np.asarray(x)
        grid = x.reshape(x.shape[:2] + self.shape)
        lap = disc.laplacian_dft(grid, self.w.lo, self.w.hi).reshape(x.shape)
        if not np.iscomplexobj(x):
            lap = lap.real
        return self._assemble(x, lap, mode)

    # ---- dense -----------------------------------------------------------
    def dense_blocks(self):
        """(A, B) as dense 3P x 3P real matrices, component-major ordering
        (index = component * P + node)."""
        P = self.npts
        lapm = disc.laplacian_matrix(self.shape, self.w.lo, self.w.hi)
        A = np.zeros((3 * P, 3 * P))
        B = np.zeros((3 * P, 3 * P))
        for c in range(3):
            A[c * P:(c + 1) * P, c * P:(c + 1) * P] += -0.5 * lapm
        for a in range(3):
            for b in range(3):
                A[a * P:(a + 1) * P, b * P:(b + 1) * P] += np.diag(self.Apt[:, a, b])
                B[a * P:(a + 1) * P, b * P:(b + 1) * P] += np.diag(self.Bpt[:, a, b])
        return A, B

    def dense_matrix(self, mode=UV):
        A, B = self.dense_blocks()
        if mode == UV:
            return np.block([[A, B], [-B, -A]])
        Z = np.zeros_like(A)
        return np.block([[A + B, Z], [Z, A - B]])

    def apply_dense(self, x, mode=UV):
        m = self.dense_matrix(mode)
        x = np.asarray(x)
        flat = x.reshape(x.shape[0], -1)
        return (flat @ m.T).reshape(x.shape)

    # ---- f/g helpers -----------------------------------------------------
    def hplus(self, f):
        """H_+ f for f of shape (ncol, 3, P)."""
        x = np.concatenate([f, np.zeros_like(f)], axis=1)
        return self.apply_fft(x, FG)[:, :3]

    def hminus(self, g):
        """H_- g for g of shape (ncol, 3, P)."""
        x = np.concatenate([np.zeros_like(g), g], axis=1)
        return self.apply_fft(x, FG)[:, 3:]


def uv_to_fg(x):
    """f = (u+v)/2, g = (u-v)/2 (eq. c-o-v-h)."""
    u, v = x[:, :3], x[:, 3:]
    return np.concatenate([0.5 * (u + v), 0.5 * (u - v)], axis=1)


def fg_to_uv(x):
    """u = f+g, v = f-g (eq. c-o-v)."""
    f, g = x[:, :3], x[:, 3:]
    return np.concatenate([f + g, f - g], axis=1)


def apply_at_nodes(w, phi_nodes, V_nodes, mu, lines, nodes, mode=UV):
    """The product (eq. BdG-d in UV form, eq. lrep-d in FG form) at a few nodes
    only, for grids too large for the whole-vector evaluations.

    nodes      S grid indices (n_1, ..., n_d);
    lines[a]   (S, 6, N_a): the six fields of x on the grid line through node
               s along axis a;
    phi_nodes  (3, S) real ground state and V_nodes (S,) potential at the nodes.

    At node s the Laplacian is the sum over the axes of row n_a of the dense
    1-D spectral Laplacian matrix (eq. laplace_approx, a Kronecker sum on the
    tensor grid) applied to the line along axis a; the pointwise parts are
    the blocks of eqs. def_bfA / def_bfB at the node.  Returns (S, 6)."""
    S = len(nodes)
    Apt, Bpt = spin1.pointwise_blocks(np.asarray(phi_nodes).reshape(3, S), V_nodes,
                                      w.beta_n, w.beta_s, mu, w.p, w.q)
    Apt, Bpt = Apt.real, Bpt.real
    lap = np.zeros((S, 6), dtype=np.complex128)
    for a in range(len(w.n)):
        row = disc.laplacian_matrix_1d(w.n[a], w.lo[a], w.hi[a])
        for s in range(S):
            lap[s] += np.asarray(lines[a][s]) @ row[nodes[s][a]]
    x = np.stack([np.asarray(lines[0][s])[:, nodes[s][0]] for s in range(S)])
    kin = -0.5 * lap
    a, b = x[:, :3], x[:, 3:]

    def pt(mat, v):
        return np.einsum("sab,sb->sa", mat, v)
    if mode == UV:
        yu = kin[:, :3] + pt(Apt, a) + pt(Bpt, b)
        yv = -(kin[:, 3:] + pt(Apt, b) + pt(Bpt, a))
        return np.concatenate([yu, yv], axis=1)
    yf = kin[:, :3] + pt(Apt + Bpt, a)
    yg = kin[:, 3:] + pt(Apt - Bpt, b)
    return np.concatenate([yf, yg], axis=1)
