"""CPU FP64 oracle for the spin-1 BdG Fourier-spectral eigensolver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, NumPy/SciPy
restatement of what the paper defines, used to check the CUDA library.  Only
the test-suite, the smoke check and the CPU-baseline leg of the benchmark may
import it; the product library never does, and it shares no code with the CUDA
path (both take their inputs from the seeded-input module `synth`).

Modules, each citing the passages it follows:
  discretization  Fourier pseudospectral grid, DFT (eq. FT_3), Laplacian
                  (eq. laplace_approx) in three independent forms.
  spin1           spin-1 matrices, the operators A, B (eqs. def_A, def_B,
                  def_bfA, def_bfB), the GPE right-hand side (eq. GPE), the
                  Hamiltonian of eq. NLEP and the chemical potentials
                  (eq. chem-formula).
  ground_state    the energy of eq. energy and the ground state on S_M
                  (eq. groundDef): normalized
                  gradient flow, then inexact Newton steps with the Hessian
                  H_+ (projected CG); the paper cites its PCG method without
                  describing it.
  apply           the discrete BdG operator of eq. BdG-d / eq. lrep-d as a
                  dense matrix, by DFT matrices, by numpy.fft, and at chosen
                  nodes from the grid lines through them (large grids).
  lrep            dense solves, the bi-orthogonal Gram-Schmidt, the
                  structure-preserving Rayleigh-Ritz step, the iterative
                  subspace solver, residuals, the Gram of packed real
                  columns and the normalization of eq. constrainfg.
  kohn            the analytical eigenpairs of Theorem "Analytical eigenpairs"
                  (eq. eig-pair) and the error metrics of Section 4.1.
  perturbed       the perturbed densities of single modes (Section 4.2,
                  eq. waveAssump with one mode).

Parity status: every function is pinned by a `-m "not gpu"` test against
closed forms, invariants or library routines, except the iterates of the
subspace solver (the paper does not give its algorithm; only its converged
result is pinned) -- parity unpinned for the iteration history.  The tests
in tests/test_oracle_planted_mistakes.py plant plausible slips in these
functions and check that a pin fails on each.
"""
