"""Planted mistakes: each case puts one plausible error into the oracle (on
the CPU, through monkeypatch, for the duration of the case) and checks that
at least one of the named pins fails on it.  This is the evidence that the
pins of the oracle are sensitive to the mistakes they are meant to catch:
a dropped term, a wrong sign, factor or index, a transposed operand.

The pins are the functions of the other test_oracle_* modules, called
directly.  Ground states that a pin takes from the session fixture are always
computed with the oracle unmodified (the mistake is lifted while one is
computed), so that a pin sees the planted error only in the function under
test; pins that compute their own ground state see the error throughout.

Sources of the pins: Section 2.1 (spin matrices, eqs. def_A / def_B), Section
3.1 (eqs. FT_3, laplace_approx, BdG-d, lrep-d, constrainfg), Theorem
"Analytical eigenpairs", Section 4.1 (Table 1), Section 4.2 (eq. waveAssump),
and the readings P1, P3, P6, P7 and P9 of the paper."""
import numpy as np
import pytest

import synth
import test_oracle_discretization as tdisc
import test_oracle_ground_state as tgs
import test_oracle_lrep as tl
import test_oracle_model as tmod
import test_oracle_perturbed as tper
from oracle import apply as ap
from oracle import discretization as disc
from oracle import ground_state as gs
from oracle import kohn, lrep, perturbed, spin1


# ---------------------------------------------------------------------------
# the planted mistakes: plant(mp) applies one through the monkeypatch mp
# ---------------------------------------------------------------------------
def _kinetic_without_half(mp):
    orig = ap.Operator._assemble
    mp.setattr(ap.Operator, "_assemble", lambda self, x, lap, mode: orig(self, x, 2.0 * lap, mode))


def _wavenumbers_of_half_box(mp):
    orig = disc.wavenumbers
    mp.setattr(disc, "wavenumbers", lambda n, lo, hi: 2.0 * orig(n, lo, hi))


def _nyquist_dropped(mp):
    orig = disc.wavenumbers

    def wn(n, lo, hi):
        mu = orig(n, lo, hi).copy()
        mu[n // 2] = 0.0
        return mu
    mp.setattr(disc, "wavenumbers", wn)


def _dft_sign_flipped(mp):
    mp.setattr(disc, "dft_matrix", lambda n: disc.idft_matrix(n) / n)


def _spin_y_sign(mp):
    SX, SY, SZ = spin1.SPIN
    mp.setattr(spin1, "SPIN", (SX, -SY, SZ))


def _spin_x_unnormalised(mp):
    SX, SY, SZ = spin1.SPIN
    mp.setattr(spin1, "SPIN", (SX * np.sqrt(2.0), SY, SZ))


def _wrap_blocks(mp, change):
    orig = spin1.pointwise_blocks

    def blocks(phi, V, beta_n, beta_s, mu, p=0.0, q=0.0):
        Apt, Bpt = orig(phi, V, beta_n, beta_s, mu, p, q)
        return change(np.asarray(phi, dtype=np.complex128).reshape(3, -1), beta_n, beta_s, p, q,
                      Apt.copy(), Bpt.copy())
    mp.setattr(spin1, "pointwise_blocks", blocks)


def _density_term_of_A_dropped(mp):
    def change(phi, bn, bs, p, q, Apt, Bpt):
        return Apt - bn * np.einsum("ap,bp->pab", phi, phi.conj()), Bpt
    _wrap_blocks(mp, change)


def _B_with_hermitian_adjoint(mp):
    # sum_j S_j Phi Phi^T S_j^H in place of S_j Phi Phi^T S_j^T
    def change(phi, bn, bs, p, q, Apt, Bpt):
        S = np.stack(spin1.SPIN)
        ff_t = np.einsum("ap,bp->pab", phi, phi)
        wrong = np.einsum("jac,pcd,jbd->pab", S, ff_t, S.conj())
        right = np.einsum("jac,pcd,jbd->pab", S, ff_t, S)
        return Apt, Bpt + bs * (wrong - right)
    _wrap_blocks(mp, change)


def _exchange_sum_of_A_dropped(mp):
    def change(phi, bn, bs, p, q, Apt, Bpt):
        S = np.stack(spin1.SPIN)
        ff_h = np.einsum("ap,bp->pab", phi, phi.conj())
        return Apt - bs * np.einsum("jac,pcd,jbd->pab", S, ff_h, S.conj()), Bpt
    _wrap_blocks(mp, change)


def _zeeman_on_B(mp):
    def change(phi, bn, bs, p, q, Apt, Bpt):
        z = np.diag(spin1.zeeman_diag(p, q))
        return Apt - z, Bpt + z
    _wrap_blocks(mp, change)


def _uv_lower_left_sign(mp):
    orig = ap.Operator.dense_matrix

    def dense(self, mode=ap.UV):
        m = orig(self, mode).copy()
        if mode == ap.UV:
            n = m.shape[0] // 2
            m[n:, :n] *= -1.0
        return m
    mp.setattr(ap.Operator, "dense_matrix", dense)


def _residual_without_omega(mp):
    r_fg, r_uv = lrep.residuals, lrep.residual_uv
    mp.setattr(lrep, "residuals", lambda op, F, G, om: r_fg(op, F, G, om) * np.abs(om))
    mp.setattr(lrep, "residual_uv", lambda op, X, om: r_uv(op, X, om) * np.abs(om))


def _residual_with_squared_norm(mp):
    r_fg, r_uv = lrep.residuals, lrep.residual_uv

    def fg(op, F, G, om):
        n = np.sqrt(np.sum(np.abs(F.reshape(len(om), -1)) ** 2, 1) + np.sum(np.abs(G.reshape(len(om), -1)) ** 2, 1))
        return r_fg(op, F, G, om) / n

    def uv(op, X, om):
        return r_uv(op, X, om) / np.linalg.norm(np.asarray(X).reshape(len(om), -1), axis=1) * np.sqrt(2.0)
    mp.setattr(lrep, "residuals", fg)
    mp.setattr(lrep, "residual_uv", uv)


def _residual_of_one_half(mp):
    # only |H_- g - w f| enters, in both routes
    def fg(op, F, G, om):
        hg = op.hminus(G)
        return np.array([np.linalg.norm(hg[i] - om[i] * F[i]) /
                         (abs(om[i]) * np.sqrt(np.linalg.norm(F[i]) ** 2 + np.linalg.norm(G[i]) ** 2))
                         for i in range(len(om))])

    def uv(op, X, om):
        X = np.asarray(X)
        F, G = 0.5 * (X[:, :3] + X[:, 3:]), 0.5 * (X[:, :3] - X[:, 3:])
        return fg(op, F, G, om)
    mp.setattr(lrep, "residuals", fg)
    mp.setattr(lrep, "residual_uv", uv)


def _biortho_without_conjugate(mp):
    def bi(F, G, Fl=None, Gl=None, rtol=1e-12):
        F = np.array(F, copy=True)
        G = np.array(G, copy=True)
        if Fl is not None and Fl.shape[1] > 0:
            for _ in range(2):
                F = F - Fl @ (Gl.T @ F)
                G = G - Gl @ (Fl.T @ G)
        X, sig, Yh = np.linalg.svd(F.T @ G)
        r = int(np.sum(sig >= rtol * sig[0]))
        sc = 1.0 / np.sqrt(sig[:r])
        return F @ (X[:, :r] * sc), G @ (Yh[:r].conj().T * sc), r
    mp.setattr(lrep, "biortho", bi)


def _pencil_operands_swapped(mp):
    orig = lrep.small_lrep
    mp.setattr(lrep, "small_lrep", lambda Kp, Km, **kw: orig(Km, Kp, **kw))


def _normalised_to_one(mp):
    orig = lrep.normalize_fg

    def nf(F, G, hd):
        F, G = orig(F, G, hd)
        return 2.0 * F, 2.0 * G
    mp.setattr(lrep, "normalize_fg", nf)


def _kohn_g_sign(mp):
    orig = kohn.kohn_modes
    mp.setattr(kohn, "kohn_modes", lambda w, phi: [(g, f, -gg) for g, f, gg in orig(w, phi)])


def _kohn_f_power_of_gamma(mp):
    # f = sqrt(gamma / 2) d Phi in place of d Phi / sqrt(2 gamma)
    orig = kohn.kohn_modes
    mp.setattr(kohn, "kohn_modes", lambda w, phi: [(g, g * f, gg) for g, f, gg in orig(w, phi)])


def _e_uv_u_part_only(mp):
    def euv(u_num, v_num, U_exact, V_exact):
        Q, _ = np.linalg.qr(U_exact)
        return np.linalg.norm(u_num - Q @ (Q.conj().T @ u_num)) / np.linalg.norm(u_num)
    mp.setattr(kohn, "e_uv", euv)


def _patch_density(mp, change):
    # the pins import the function by name, so both bindings are replaced
    orig = perturbed.perturbed_density

    def pd(phi, U, V, omega, times, eps):
        return orig(*change(phi, U, V, omega, times, eps))
    mp.setattr(perturbed, "perturbed_density", pd)
    mp.setattr(tper, "perturbed_density", pd)


def _density_without_conjugate_on_v(mp):
    _patch_density(mp, lambda phi, U, V, om, t, eps: (phi, U, np.conj(np.asarray(V, dtype=np.complex128)),
                                                       om, t, eps))


def _density_time_sign(mp):
    _patch_density(mp, lambda phi, U, V, om, t, eps: (phi, U, V, om, -np.asarray(t, dtype=np.float64), eps))


def _chemical_fill_without_half(mp):
    orig = spin1.chemical_potentials

    def cp(phi, Hphi):
        mu = orig(phi, Hphi)
        p = np.asarray(phi).reshape(3, -1)
        nrm = np.sum(np.abs(p) ** 2, axis=1)
        if nrm[1] < spin1.ZERO_COMPONENT * nrm.sum() and nrm[0] > 0 and nrm[2] > 0:
            mu = mu.copy()
            mu[1] = mu[0] + mu[2]
        return mu
    mp.setattr(spin1, "chemical_potentials", cp)


def _magnetisation_ignored(mp):
    orig = gs.project_SM
    mp.setattr(gs, "project_SM", lambda phi, M, cell: orig(phi, 0.0, cell))


def _spin_coupling_sign_in_hamiltonian(mp):
    orig = spin1.hamiltonian
    mp.setattr(spin1, "hamiltonian",
               lambda phi, V, w, bn, bs, p=0.0, q=0.0: orig(phi, V, w, bn, -bs, p, q))


def _sz_phi_not_deflated(mp):
    orig = lrep.deflation_bases

    def db(op, phi, **kw):
        Zf, Zg = orig(op, phi, **kw)
        return np.delete(Zf, 1, axis=1), Zg
    mp.setattr(lrep, "deflation_bases", db)


def _pair_gram_parts_swapped(mp):
    orig = lrep.pair_gram
    mp.setattr(lrep, "pair_gram", lambda A, B: orig(1j * np.conj(A), B))


def _kdiag_symbol_of_modulus(mp):
    # the symbol evaluated at |mu| for |mu|^2
    orig = disc.inverse_kdiag
    mp.setattr(disc, "inverse_kdiag", lambda f, symbol, lo, hi: orig(f, lambda k2: symbol(np.sqrt(k2)), lo, hi))


def _derivative_sign(mp):
    orig = disc.spectral_derivative
    mp.setattr(disc, "spectral_derivative", lambda f, ax, lo, hi: -orig(f, ax, lo, hi))


def _projection_of_mass_only(mp):
    mp.setattr(gs, "project_SM", lambda phi, M, cell: phi / np.sqrt(cell * np.sum(phi ** 2)))


def _pencil_pseudo_inverse_scaled_wrong(mp):
    # the pseudo-inverse L^-T built with D^-1 for D (the diagonal scaling of
    # K_+ applied the wrong way round)
    def small(Kp, Km, zero_tol=1e-8, rank_tol=1e-10):
        Kp = 0.5 * (Kp + Kp.T)
        Km = 0.5 * (Km + Km.T)
        dd = np.sqrt(np.maximum(np.diag(Kp), 0.0))
        d = 1.0 / dd
        lam, Q = np.linalg.eigh((Kp * d[:, None]) * d[None, :])
        keep = lam > rank_tol * lam.max()
        lam, Q = lam[keep], Q[:, keep]
        L = (Q * np.sqrt(lam)) * dd[:, None]
        Lit = (Q / np.sqrt(lam)) * dd[:, None]
        w2, Z = np.linalg.eigh(L.T @ Km @ L)
        pos = w2 > zero_tol ** 2
        om = np.sqrt(w2[pos])
        Z = Z[:, pos]
        s = np.sqrt(om)
        return om, (Lit @ Z) * s, ((L @ Z) / om) * s
    mp.setattr(lrep, "small_lrep", small)


def _e_uv_squared(mp):
    def euv(u_num, v_num, U_exact, V_exact):
        def err(x, B):
            Q, _ = np.linalg.qr(B)
            return (np.linalg.norm(x - Q @ (Q.conj().T @ x)) / np.linalg.norm(x)) ** 2
        return err(u_num, U_exact) + err(v_num, V_exact)
    mp.setattr(kohn, "e_uv", euv)


def _node_product_first_axis_only(mp):
    # the per-node Laplacian summed over the first axis only
    orig = ap.apply_at_nodes

    def at(w, phi_nodes, V_nodes, mu, lines, nodes, mode=ap.UV):
        kept = [lines[0]] + [np.zeros_like(np.asarray(li)) for li in lines[1:]]
        return orig(w, phi_nodes, V_nodes, mu, kept, nodes, mode)
    mp.setattr(ap, "apply_at_nodes", at)


def _uv_from_fg_sign(mp):
    # v = g - f for v = f - g
    orig = ap.fg_to_uv

    def f2u(x):
        y = np.array(orig(x), copy=True)
        y[:, 3:] *= -1.0
        return y
    mp.setattr(ap, "fg_to_uv", f2u)


def _kronecker_order_reversed(mp):
    def lapm(shape, lo, hi):
        mats = [disc.laplacian_matrix_1d(nn, a, b) for nn, a, b in zip(shape, lo, hi)]
        total = 0.0
        for ax, mat in enumerate(mats):
            term = np.ones((1, 1))
            for bx in reversed(range(len(mats))):
                term = np.kron(term, mat if bx == ax else np.eye(shape[bx]))
            total = total + term
        return total
    mp.setattr(disc, "laplacian_matrix", lapm)


def _gpe_exchange_term_dropped(mp):
    # the beta_s phi_0^2 conj(phi_-1) term of the phi_1 equation left out
    orig = spin1.gpe_rhs_componentwise

    def rhs(psi, V, w, bn, bs, p=0.0, q=0.0):
        r = np.array(orig(psi, V, w, bn, bs, p, q), copy=True)
        r[0] -= bs * psi[1] ** 2 * np.conj(psi[2])
        return r
    mp.setattr(spin1, "gpe_rhs_componentwise", rhs)


def _spin_vector_conjugate_side(mp):
    # Phi^T S_j conj(Phi) for Phi^H S_j Phi
    mp.setattr(spin1, "spin_vector",
               lambda phi: np.stack([np.einsum("a...,ab,b...->...", phi, S, phi.conj()) for S in spin1.SPIN]))


def _dense_g_without_omega(mp):
    # g = L y in place of L y / omega (then normalised as usual)
    orig = lrep.dense_solve_fg

    def dense(op, k, zero_tol=1e-5):
        om, F, G = orig(op, k, zero_tol)
        n = len(om)
        Fm = F.reshape(n, -1).T
        Gm = (G * om[:, None, None]).reshape(n, -1).T
        Fm, Gm = lrep.normalize_fg(Fm, Gm, lrep.weight(op.w))
        return om, Fm.T.reshape(F.shape), Gm.T.reshape(G.shape)
    mp.setattr(lrep, "dense_solve_fg", dense)


def _g_side_never_deflated(mp):
    orig = lrep.deflation_bases

    def db(op, phi, **kw):
        Zf, Zg = orig(op, phi, **kw)
        return Zf, Zg[:, :0]
    mp.setattr(lrep, "deflation_bases", db)


def _newton_with_hminus(mp):
    # the Newton step's Hessian built from H_- for H_+
    def hess(phi, mu, V, w, d):
        op = ap.Operator(w, phi, V, mu)
        return op.hminus(d.reshape(1, 3, -1))[0].reshape(d.shape)
    mp.setattr(gs, "_hplus_real", hess)


def _energy_density_without_half(mp):
    # beta_n rho^2 for beta_n / 2 rho^2 in eq. energy
    orig = gs.energy

    def energy(phi, V, w):
        rho = np.sum(np.asarray(phi) ** 2, axis=0)
        return orig(phi, V, w) + gs.cell_volume(w) * 0.5 * w.beta_n * float(np.sum(rho ** 2))
    mp.setattr(gs, "energy", energy)


# ---------------------------------------------------------------------------
# the cases: (name, plant, pins); a pin is (function, needs ground, args)
# ---------------------------------------------------------------------------
G = True
CASES = [
    ("kinetic term without its 1/2", _kinetic_without_half,
     [(tmod.test_non_interacting_oscillator_states, False, ())]),
    ("wavenumbers pi k / (L/2)", _wavenumbers_of_half_box,
     [(tdisc.test_gaussian_second_derivative_spectral_accuracy, False, ())]),
    ("Nyquist wavenumber dropped (reading P6)", _nyquist_dropped,
     [(tdisc.test_plane_waves_are_exact_eigenfunctions, False, (16, -4.0, 4.0))]),
    ("DFT with the wrong exponent sign", _dft_sign_flipped,
     [(tdisc.test_dft_matrix_matches_explicit_sum_and_numpy, False, (8,))]),
    ("S_y with the wrong sign", _spin_y_sign, [(tmod.test_spin_matrices, False, ())]),
    ("S_x without 1/sqrt2", _spin_x_unnormalised, [(tmod.test_spin_matrices, False, ())]),
    ("beta_n Phi Phi^H dropped from A", _density_term_of_A_dropped,
     [(tmod.test_closed_form_entries_of_A_B, False, ()), (tl.test_fm_generalized_nullspace, G, ())]),
    ("S_j^H in place of S_j^T in B", _B_with_hermitian_adjoint,
     [(tmod.test_closed_form_entries_of_A_B, False, ()),
      (tmod.test_A_B_are_the_linearization_of_the_gpe, False, (tmod.W2,))]),
    ("sum_j S_j Phi Phi^H S_j^H dropped from A", _exchange_sum_of_A_dropped,
     [(tmod.test_A_B_are_the_linearization_of_the_gpe, False, (tmod.W1,))]),
    ("Zeeman diagonal on B instead of A (reading P1)", _zeeman_on_B,
     [(tmod.test_closed_form_entries_of_A_B, False, ())]),
    ("UV form with +B in the lower-left block", _uv_lower_left_sign,
     [(tl.test_pm_pairing_and_two_dense_routes, G, (tl.WFM,))]),
    ("residual without the |omega| divisor (reading P9)", _residual_without_omega,
     [(tl.test_residuals_closed_forms_on_unconverged_pairs, G, ())]),
    ("residual divided by |x|^2 (reading P9)", _residual_with_squared_norm,
     [(tl.test_residuals_closed_forms_on_unconverged_pairs, G, ())]),
    ("residual of the H_- half only (reading P9)", _residual_of_one_half,
     [(tl.test_residuals_closed_forms_on_unconverged_pairs, G, ())]),
    ("bi-orthogonalisation with F^T G for F^H G", _biortho_without_conjugate,
     [(tl.test_biortho_properties, False, ())]),
    ("projected pencil with K_+ and K_- swapped", _pencil_operands_swapped,
     [(tl.test_small_lrep_against_scipy, False, ())]),
    ("pairs normalised to h^d f.g = 1 (eq. constrainfg)", _normalised_to_one,
     [(tl.test_biorthogonality_and_normalization, G, (tl.WFM,))]),
    ("Kohn pair with the wrong sign of g", _kohn_g_sign, [(tl.test_kohn_mode, G, ())]),
    ("Kohn pair with f scaled by gamma^(1/2) for gamma^(-1/2)", _kohn_f_power_of_gamma,
     [(tper.test_kohn_mode_is_a_dipole_oscillation, False, ())]),
    ("e_uv without its v part", _e_uv_u_part_only, [(tl.test_table1_case1, G, ("fm", 885.4, -4.1))]),
    ("perturbed density without the conjugate on v", _density_without_conjugate_on_v,
     [(tper.test_single_amplitudes_with_imaginary_factor, False, ())]),
    ("perturbed density with e^{+i omega t} on u", _density_time_sign,
     [(tper.test_single_amplitudes_with_imaginary_factor, False, ())]),
    ("vanishing mu_0 filled as mu_1 + mu_-1 (reading P3)", _chemical_fill_without_half,
     [(tgs.test_chemical_potential_rules, False, ()), (tmod.test_vanishing_component_rule_is_relative, False, ())]),
    ("ground state projected with M = 0", _magnetisation_ignored,
     [(tgs.test_sma_ferromagnetic, False, (0.3,))]),
    ("compact Hamiltonian with -beta_s", _spin_coupling_sign_in_hamiltonian,
     [(tmod.test_compact_equals_componentwise_gpe, False, (tmod.W1,))]),
    ("S_z Phi left out of Z_f (reading P7)", _sz_phi_not_deflated,
     [(tl.test_deflation_and_iterative_solver_afm_case, G, ())]),
    ("pair Gram with real and imaginary parts swapped", _pair_gram_parts_swapped,
     [(tl.test_pair_gram_brute_force_and_complex_identity, False, ())]),
    ("T_sigma symbol of |mu| for |mu|^2", _kdiag_symbol_of_modulus,
     [(tdisc.test_inverse_kdiag_on_plane_waves, False, ())]),
    ("spectral derivative with -i mu", _derivative_sign,
     [(tdisc.test_spectral_derivative_of_sines_and_cosines, False, ()), (tl.test_kohn_mode, G, ())]),
    ("ground state projected by mass only", _projection_of_mass_only,
     [(tgs.test_project_SM_lands_on_SM, False, (0.25,))]),
    ("pseudo-inverse of the K_+ factor scaled by D^-1 for D", _pencil_pseudo_inverse_scaled_wrong,
     [(tl.test_small_lrep_semidefinite_Kplus, False, ())]),
    ("e_uv with squared projector errors", _e_uv_squared, [(tl.test_e_uv_closed_forms, False, ())]),
    ("per-node product with the Laplacian of the first axis only", _node_product_first_axis_only,
     [(tmod.test_apply_at_nodes_matches_the_whole_product, False, (tmod.W2,))]),
    ("UV from FG with v = g - f (eq. c-o-v)", _uv_from_fg_sign,
     [(tmod.test_three_applies_agree_and_forms, False, (tmod.W1,))]),
    ("dense Laplacian with the Kronecker factors reversed", _kronecker_order_reversed,
     [(tdisc.test_laplacian_forms_agree_2d_3d, False, ())]),
    ("componentwise GPE without beta_s phi_0^2 conj(phi_-1)", _gpe_exchange_term_dropped,
     [(tmod.test_compact_equals_componentwise_gpe, False, (tmod.W1,))]),
    ("spin vector Phi^T S conj(Phi)", _spin_vector_conjugate_side,
     [(tmod.test_compact_equals_componentwise_gpe, False, (tmod.W2,))]),
    ("dense route with g = L y (no 1/omega)", _dense_g_without_omega,
     [(tl.test_biorthogonality_and_normalization, G, (tl.WFM,))]),
    ("-i S_y Phi never deflated (reading P7)", _g_side_never_deflated,
     [(tl.test_residuals_closed_forms_on_unconverged_pairs, G, ())]),
    ("ground-state Newton step with the Hessian H_-", _newton_with_hminus,
     [(tgs.test_newton_step_converges_quadratically, G, ())]),
    ("energy with beta_n rho^2 for beta_n/2 rho^2 (eq. energy)", _energy_density_without_half,
     [(tgs.test_energy_derivative_is_twice_the_hamiltonian, False, (synth.Workload(
         "e1d", (64,), (-8.0,), (8.0,), (1.0,), 10.0, -1.5, 0.07, 0.2),))]),
]


@pytest.mark.parametrize("name, plant, pins", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(name, plant, pins, ground, monkeypatch):
    def clean_ground(w):
        monkeypatch.undo()
        try:
            return ground(w)
        finally:
            plant(monkeypatch)

    plant(monkeypatch)
    caught = []
    for fn, needs_ground, args in pins:
        try:
            fn(clean_ground, *args) if needs_ground else fn(*args)
        except AssertionError:
            caught.append(fn.__name__)
    monkeypatch.undo()
    assert caught, f"no pin caught the planted mistake: {name}"
