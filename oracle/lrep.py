"""Linear-response eigenproblem of the discrete BdG operator (Sections 2.2,
3.1, 3.2, 3.4).

  [[0, H_-], [H_+, 0]] [f; g] = omega [f; g]        (eq. lrep-d)
  weak/pencil form  a(Phi, Psi) = omega b(Phi, Psi) with
  a = <H_+ f, xi> + <H_- g, eta>, b = <g, xi> + <f, eta>   (eqs. BdG-wf, BdG-wf-a)

Contents
  dense_eig_uv         eigenvalues of the full [[A,B],[-B,-A]] (eq. BdG-d), scipy.linalg.eig.
  dense_solve_fg       the same spectrum by the symmetric route: H_+ = L L^T on its
                       range, eigh(L^T H_- L) = omega^2 (eq. lrep-d).
  biortho              bi-orthogonal Gram-Schmidt: CGS2 against locked pairs, SVD
                       of the in-block S = F^H G with rank cut (Theorem
                       "Biorthogonality" motivates the basis; Section 3.2).
  small_lrep           the projected pencil of eq. BdG-wf-a on a bi-orthonormal
                       basis, K_+ = U^T H_+ U, K_- = V^T H_- V, by Cholesky of K_+ and
                       eigh of L^T K_- L.
  deflation_bases      Z_f = span{Phi, S_z Phi} (in null(H_-)), Z_g = span{-i S_y Phi}
                       when it lies in null(H_+) (Section 2.3; reading P7).
  solve_iterative      block structure-preserving subspace iteration (reading P8).
  residuals, normalize_fg, fg_to_uv.
  pair_gram            S = F^T G over real columns (real, imaginary part) of two blocks
                       of complex columns: the Gram of the bi-orthogonal Gram-Schmidt
                       (Theorem "Biorthogonality") and of the projected matrices.

The inner products here are the unweighted Euclidean ones; the weight h^d
enters only the normalization <f, g> = 1/4 of eq. constrainfg (reading P11).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU leg, never by the product library.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import discretization as disc
from .apply import FG, UV


def weight(w) -> float:
    return float(np.prod(w.h))


# --------------------------------------------------------------------------
# dense routes
# --------------------------------------------------------------------------
def dense_eig_uv(op):
    """All eigenvalues of the dense UV matrix (complex, unsorted)."""
    return sla.eig(op.dense_matrix(UV), right=False)


def dense_solve_fg(op, k, zero_tol=1e-5):
    """k smallest positive eigenpairs by the symmetric route.  Returns
    (omega[k], f[k,3,P], g[k,3,P]) with h^d <f_i, g_i> = 1/4."""
    A, B = op.dense_blocks()
    Hp, Hm = A + B, A - B
    lam, Q = np.linalg.eigh(0.5 * (Hp + Hp.T))
    keep = lam > 1e-9 * np.max(np.abs(lam))
    L = Q[:, keep] * np.sqrt(lam[keep])
    C = L.T @ Hm @ L
    w2, Y = np.linalg.eigh(0.5 * (C + C.T))
    pos = w2 > zero_tol ** 2
    w2, Y = w2[pos], Y[:, pos]
    om = np.sqrt(w2[:k])
    Y = Y[:, :k]
    F = (Q[:, keep] / np.sqrt(lam[keep])) @ Y
    G = (L @ Y) / om
    F, G = normalize_fg(F, G, weight(op.w))
    P = op.npts
    return om, F.T.reshape(-1, 3, P), G.T.reshape(-1, 3, P)


def normalize_fg(F, G, hd):
    """Scale column pairs so that h^d f_i^T g_i = 1/4 (eq. constrainfg), the
    largest-|.| entry of u = f + g made positive (reading P12)."""
    F = F.copy()
    G = G.copy()
    for i in range(F.shape[1]):
        d = hd * np.vdot(F[:, i], G[:, i]).real
        s = np.sqrt(0.25 / abs(d))
        F[:, i] *= s
        G[:, i] *= s * np.sign(d)
        u = F[:, i] + G[:, i]
        j = np.argmax(np.abs(u))
        ph = np.conj(u[j]) / abs(u[j])
        F[:, i] *= ph
        G[:, i] *= ph
    return F, G


# --------------------------------------------------------------------------
# bi-orthogonal Gram-Schmidt and the projected pencil
# --------------------------------------------------------------------------
def biortho(F, G, Fl=None, Gl=None, rtol=1e-12):
    """Make the column blocks F, G (n x c, real or complex) bi-orthonormal,
    F^H G = I_r, and bi-orthogonal to a locked bi-orthonormal pair (Fl, Gl):
      twice: F <- F - Fl (Gl^H F),  G <- G - Gl (Fl^H G)     (CGS2)
      S = F^H G = X Sigma Y^H,  keep sigma_i >= rtol * sigma_max,
      F <- F X_r Sigma_r^{-1/2},  G <- G Y_r Sigma_r^{-1/2}.
    Returns (F, G, r)."""
    F = np.array(F, copy=True)
    G = np.array(G, copy=True)
    if Fl is not None and Fl.shape[1] > 0:
        for _ in range(2):
            F = F - Fl @ (Gl.conj().T @ F)
            G = G - Gl @ (Fl.conj().T @ G)
    S = F.conj().T @ G
    X, sig, Yh = np.linalg.svd(S)
    if sig.size == 0 or sig[0] == 0:
        return F[:, :0], G[:, :0], 0
    r = int(np.sum(sig >= rtol * sig[0]))
    sc = 1.0 / np.sqrt(sig[:r])
    return F @ (X[:, :r] * sc), G @ (Yh[:r].conj().T * sc), r


def small_lrep(Kp, Km, zero_tol=1e-8, rank_tol=1e-10):
    """Eigenpairs of the projected pencil: K_- q = omega p, K_+ p = omega q
    with K_+ = L L^T, eigh(L^T K_- L) = Z diag(omega^2) Z^T, p = L^-T z,
    q = L z / omega, scaled so p_i^T q_i = 1.  Returns (omega, Pc, Qc) for the
    omega > zero_tol, ascending.

    K_+ is only semidefinite when the basis holds a direction of null(H_+)
    (the spin rotations of a ground state with full spin symmetry leave such
    directions outside Z_f).  The factor is therefore rank-revealing, as in
    reading P17: with D = diag(K_+)^-1/2 and D K_+ D = Q diag(lam) Q^T,
    L = D^-1 Q_r lam_r^1/2 over the lam > rank_tol max(lam), and L^-T is
    the pseudo-inverse D Q_r lam_r^-1/2 on that subspace."""
    Kp = 0.5 * (Kp + Kp.T)
    Km = 0.5 * (Km + Km.T)
    dd = np.sqrt(np.maximum(np.diag(Kp), 0.0))
    live = dd > 1e-150 * max(dd.max(), 1e-300)      # zero columns stay out
    d = np.where(live, 1.0 / np.where(live, dd, 1.0), 0.0)
    lam, Q = np.linalg.eigh((Kp * d[:, None]) * d[None, :])
    keep = lam > rank_tol * lam.max()
    lam, Q = lam[keep], Q[:, keep]
    L = (Q * np.sqrt(lam)) * dd[:, None]
    Lit = (Q / np.sqrt(lam)) * d[:, None]
    C = L.T @ Km @ L
    w2, Z = np.linalg.eigh(0.5 * (C + C.T))
    pos = w2 > zero_tol ** 2
    w2, Z = w2[pos], Z[:, pos]
    om = np.sqrt(w2)
    Pc = Lit @ Z
    Qc = (L @ Z) / om
    s = np.sqrt(om)          # p^T q = z^T z / omega = 1 / omega before scaling
    return om, Pc * s, Qc * s


# --------------------------------------------------------------------------
# deflation
# --------------------------------------------------------------------------
def deflation_bases(op, phi, par_tol=1e-12, null_tol=1e-8):
    """Orthonormal Z_f (n x 1..3) and Z_g (n x 0..1), n = 3P (reading P7):
    Phi and S_z Phi always, S_x Phi and -i S_y Phi when numerically null."""
    phi = np.asarray(phi, dtype=np.float64).reshape(3, -1)
    P = phi.shape[1]
    z1 = phi.ravel() / np.linalg.norm(phi)
    sz = np.concatenate([phi[0], 0.0 * phi[1], -phi[2]])
    cols = [z1]
    r = sz - z1 * (z1 @ sz)
    if np.linalg.norm(r) > par_tol * max(np.linalg.norm(sz), 1e-300) and np.linalg.norm(sz) > par_tol:
        r = r - z1 * (z1 @ r)
        cols.append(r / np.linalg.norm(r))
    # S_x Phi = (1/sqrt2) (phi_0, phi_1 + phi_-1, phi_0): the rotation about x
    # is a symmetry too when the state is symmetric enough (antiferromagnetic
    # or polar states at p = q = 0); kept when its part outside
    # span{Phi, S_z Phi} is numerically in null(H_-)
    sx = np.concatenate([phi[1], phi[0] + phi[2], phi[1]]) / np.sqrt(2.0)
    nsx = np.linalg.norm(sx)
    if nsx > par_tol * np.linalg.norm(phi):
        r = sx.copy()
        for _ in range(2):
            for c in cols:
                r = r - c * (c @ r)
        nr = np.linalg.norm(r)
        if nr > 1e-6 * nsx:
            r = r / nr
            hr = op.hminus(r.reshape(1, 3, P)).ravel()
            if np.linalg.norm(hr) < null_tol:
                cols.append(r)
    Zf = np.stack(cols, axis=1)
    # -i S_y Phi = (1/sqrt2) (-phi_0, phi_1 - phi_-1, phi_0)
    y = np.concatenate([-phi[1], phi[0] - phi[2], phi[1]]) / np.sqrt(2.0)
    Zg = np.zeros((3 * P, 0))
    ny = np.linalg.norm(y)
    if ny > par_tol * np.linalg.norm(phi):
        hy = op.hplus(y.reshape(1, 3, P)).ravel()
        if np.linalg.norm(hy) / ny < null_tol:
            Zg = (y / ny)[:, None]
    return Zf, Zg


# --------------------------------------------------------------------------
# residuals and the iterative solver
# --------------------------------------------------------------------------
def pair_gram(A, B):
    """Gram matrix of real columns: A (P, n) and B (Q, n) complex rows are
    taken as 2P and 2Q real vectors (real part, imaginary part), and
    S[2i+s, 2j+t] = sum_r part_s(A[i, r]) part_t(B[j, r]) in FP64, together
    with S_abs, the same sums of absolute products (the scale of its
    rounding).  This is the inner product of the bi-orthogonality relations
    (Theorem "Biorthogonality") on packed real vectors."""
    Ar = np.stack([A.real, A.imag], axis=1).reshape(2 * A.shape[0], -1).astype(np.float64)
    Br = np.stack([B.real, B.imag], axis=1).reshape(2 * B.shape[0], -1).astype(np.float64)
    return Ar @ Br.T, np.abs(Ar) @ np.abs(Br).T


def residuals(op, F, G, om):
    """r_i = sqrt(|H_+ f - w g|^2 + |H_- g - w f|^2) / (w sqrt(|f|^2 + |g|^2)),
    which equals |M x - w x| / (|w| |x|) for x = (u, v) (reading P9).
    F, G: (k, 3, P)."""
    hf = op.hplus(F)
    hg = op.hminus(G)
    out = []
    for i in range(len(om)):
        a = np.linalg.norm(hf[i] - om[i] * G[i]) ** 2 + np.linalg.norm(hg[i] - om[i] * F[i]) ** 2
        b = np.linalg.norm(F[i]) ** 2 + np.linalg.norm(G[i]) ** 2
        out.append(np.sqrt(a) / (abs(om[i]) * np.sqrt(b)))
    return np.array(out)


def residual_uv(op, UVv, om):
    """|M x - w x| / (|w| |x|) computed with the UV operator directly."""
    y = op.apply_fft(UVv, UV)
    out = []
    for i in range(len(om)):
        out.append(np.linalg.norm(y[i] - om[i] * UVv[i]) / (abs(om[i]) * np.linalg.norm(UVv[i])))
    return np.array(out)


def _cols(x, P):
    return np.asarray(x).reshape(x.shape[0], 3 * P).T


def _vecs(X, P):
    return X.T.reshape(-1, 3, P)


def solve_iterative(op, k, m, X0, Zf, Zg, tol=1e-10, maxit=1000, sigma=None,
                    rtol=1e-5, refresh_every=20, verbose=False, inner=0):
    """Block structure-preserving subspace iteration (reading P8; after the
    LOBP4dCG family the paper cites for BOSP).  Real arithmetic.

    Basis per side: [F, D, P] with F the current Ritz block, D the
    preconditioned residual directions of the unconverged columns and P the
    previous update; CGS2 of [D, P] against (F, G), SVD bi-orthonormalization
    inside [D, P], then the projected pencil (small_lrep).  With f kept
    orthogonal to Z_f and g to Z_g, the pencil does not see the components
    of g along Z_f or of f along Z_g; after each Rayleigh-Ritz step they are
    set by the residual-minimizing closed form
    g <- g + Z_f Z_f^T (H_+ f - w g) / w  (and symmetrically for f).  Preconditioner
    T_sigma = IDFT (1/2|mu|^2 + sigma)^-1 DFT (reading P10).  The
    bi-orthonormalization keeps singular values >= rtol sigma_max (reading
    P16), and the images H X are recomputed every refresh_every iterations.

    inner > 0 replaces T_sigma by that many steps of preconditioned conjugate
    gradients (preconditioner T_sigma, start 0) on H_+ d_f = r_f over the
    complement of Z_g, and on H_- d_g = r_g over the complement of Z_f (the
    null spaces of H_+ and H_-, reading P7): an approximation of the exact
    preconditioner (H_+^-1, H_-^-1) of the minimization principle, under
    which the search space grows like block inverse iteration on H_- H_+
    (reading P10; the paper names no preconditioner, and any one leaves the
    converged pairs unchanged).

    X0: (m, 6, P) real FG start.  Returns (omega[k], F[k,3,P], G[k,3,P],
    resid[k], iterations)."""
    w = op.w
    P = op.npts
    if sigma is None:
        sigma = max(float(np.mean(op.mu)), 1.0)

    def hp(X):
        return _cols(op.hplus(_vecs(X, P)), P)

    def hm(X):
        return _cols(op.hminus(_vecs(X, P)), P)

    def prec(X):
        g = _vecs(X, P).reshape((-1, 3) + tuple(w.n))
        out = disc.inverse_kdiag(g, lambda k2: 1.0 / (0.5 * k2 + sigma), w.lo, w.hi)
        return out.reshape(-1, 3, P).reshape(-1, 3 * P).T

    def defl(X, Z):
        return X - Z @ (Z.T @ X) if Z.shape[1] else X

    def pcg(hop, B, Z):
        """inner steps of PCG for hop(X) = B, column by column, on Z^perp."""
        B = defl(B, Z)
        X = np.zeros_like(B)
        R = B.copy()
        Zr = defl(prec(R), Z)
        D = Zr.copy()
        rz = np.sum(R * Zr, 0)
        for _ in range(inner):
            HD = defl(hop(D), Z)
            dhd = np.sum(D * HD, 0)
            ok = dhd > 0
            a = np.where(ok, rz / np.where(ok, dhd, 1.0), 0.0)
            X = X + D * a
            R = R - HD * a
            Zr = defl(prec(R), Z)
            rz_new = np.sum(R * Zr, 0)
            b = np.where(rz != 0, rz_new / np.where(rz != 0, rz, 1.0), 0.0)
            D = Zr + D * b
            rz = rz_new
        return X

    F = defl(_cols(np.asarray(X0)[:, :3], P), Zf)
    G = defl(_cols(np.asarray(X0)[:, 3:], P), Zg)
    F, G, r = biortho(F, G, rtol=rtol)
    U, V, HU, HV = F, G, hp(F), hm(G)
    nF = 0
    Pf = Pg = HPf = HPg = None
    resid = np.full(m, np.inf)
    om = None
    for it in range(1, maxit + 1):
        Kp = U.T @ HU
        Km = V.T @ HV
        om_all, Pc, Qc = small_lrep(Kp, Km)
        mm = min(m, om_all.size)
        om, Pc, Qc = om_all[:mm], Pc[:, :mm], Qc[:, :mm]
        F, G, HF, HG = U @ Pc, V @ Qc, HU @ Pc, HV @ Qc
        if it % refresh_every == 0:
            # the images carried by linear combination drift from H X by
            # rounding; recompute them (and drop the previous update, whose
            # images drifted the same way)
            HF, HG = hp(F), hm(G)
            nF = 0
            Pf = Pg = HPf = HPg = None
        if nF > 0:
            Pf, HPf = U[:, nF:] @ Pc[nF:], HU[:, nF:] @ Pc[nF:]
            Pg, HPg = V[:, nF:] @ Qc[nF:], HV[:, nF:] @ Qc[nF:]
        # Components of g along Z_f (in null(H_-)) and of f along Z_g (in
        # null(H_+)) are invisible to the projected pencil; they are fixed in
        # closed form by minimizing |H_+ f - w g| and |H_- g - w f|.
        G = G + Zf @ (Zf.T @ (HF - G * om)) / om
        if Zg.shape[1]:
            F = F + Zg @ (Zg.T @ (HG - F * om)) / om
        Rf = HF - G * om
        Rg = HG - F * om
        resid = np.sqrt(np.sum(Rf ** 2, 0) + np.sum(Rg ** 2, 0)) / (
            om * np.sqrt(np.sum(F ** 2, 0) + np.sum(G ** 2, 0)))
        if verbose:
            print(it, om[:k].min(), resid[:k].max())
        if mm >= k and np.all(resid[:k] <= tol):
            break
        act = np.nonzero(resid > tol)[0]
        if inner > 0:
            Df = defl(pcg(hp, Rf[:, act], Zg), Zf)
            Dg = defl(pcg(hm, Rg[:, act], Zf), Zg)
        else:
            Df = defl(prec(Rf[:, act]), Zf)
            Dg = defl(prec(Rg[:, act]), Zg)
        Bf, Bg, HBf, HBg = Df, Dg, hp(Df), hm(Dg)
        if Pf is not None:
            Bf = np.concatenate([Bf, Pf[:, act]], 1)
            Bg = np.concatenate([Bg, Pg[:, act]], 1)
            HBf = np.concatenate([HBf, HPf[:, act]], 1)
            HBg = np.concatenate([HBg, HPg[:, act]], 1)
        for _ in range(2):
            cf = G.T @ Bf
            cg = F.T @ Bg
            Bf, HBf = Bf - F @ cf, HBf - HF @ cf
            Bg, HBg = Bg - G @ cg, HBg - HG @ cg
        S = Bf.T @ Bg
        X, sig, Yh = np.linalg.svd(S)
        rr = int(np.sum(sig >= rtol * sig[0]))
        sx = X[:, :rr] / np.sqrt(sig[:rr])
        sy = Yh[:rr].T / np.sqrt(sig[:rr])
        U = np.concatenate([F, Bf @ sx], 1)
        V = np.concatenate([G, Bg @ sy], 1)
        HU = np.concatenate([HF, HBf @ sx], 1)
        HV = np.concatenate([HG, HBg @ sy], 1)
        nF = F.shape[1]
    om, F, G = om[:k], F[:, :k], G[:, :k]
    F, G = normalize_fg(F, G, weight(w))
    return om, _vecs(F, P), _vecs(G, P), resid[:k], it


def fg_to_uv(F, G):
    """(u, v) = (f + g, f - g) (eq. c-o-v), stacked as (k, 6, P)."""
    return np.concatenate([F + G, F - G], axis=1)
