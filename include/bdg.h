/*
 * bdg.h -- C ABI of the GB300 spin-1 Bogoliubov-de Gennes (BdG) library.
 *
 * The library computes low-lying excitations of a spin-1 Bose-Einstein
 * condensate around a real ground state Phi_g, following the Fourier
 * spectral BdG solver of arXiv 2506.08308:
 *
 *   [[A, B], [-B, -A]] [u; v] = omega [u; v]                 (Section 3.1, eq. BdG-d)
 *   [[0, H_-], [H_+, 0]] [f; g] = omega [f; g],  H_+- = A +- B (eq. lrep-d)
 *
 * with A, B the Fourier-pseudospectral discretizations of the operators of
 * eqs. def_A / def_B (Section 2.1) on a periodic grid, the Laplacian taken
 * spectrally (eq. laplace_approx).  Every computation runs in CUDA kernels
 * on the calling process's current device; there is no CPU fallback.
 *
 * Conventions for every call:
 *   - Grids: dim = 1..3 axes, n[a] points per axis (powers of two, 8..1024,
 *     at most 2^27 points in total), box [lo[a], hi[a]); node x_j = lo + j h,
 *     h = (hi - lo)/n (Section 3.1).  Grid arrays are C-ordered, axis 0 = x
 *     slowest, the last axis fastest.
 *   - Vectors: a block of nvec 6-component vectors is stored [nvec][6][N_p]
 *     with N_p = prod n, complex interleaved (re, im).  Components are
 *     (u_1, u_0, u_-1, v_1, v_0, v_-1) in the UV form and
 *     (f_1, f_0, f_-1, g_1, g_0, g_-1) in the FG form (eq. c-o-v-h).
 *     Complex element type: BDG_C128 = 2 x double, BDG_C64 = 2 x float.
 *   - Streams: every call is ordered on the given cudaStream_t (passed as
 *     void*, NULL = legacy default stream).  Device pointers must be valid
 *     device (or managed) memory on the current device.  Calls on one plan
 *     from several host threads at once are not supported.
 *   - Errors: every call returns a bdg_status; none aborts or exits.  On an
 *     error the output buffers are unspecified; bdg_last_error(plan) (or
 *     bdg_last_error(NULL) for a failed bdg_plan_create) returns a message.
 *   - Ownership: the plan deep-copies Phi and V to device memory it owns
 *     and frees in bdg_plan_destroy; the caller owns every buffer it passes.
 */
#ifndef BDG_H
#define BDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bdg_plan_s* bdg_plan_t;

typedef enum {
  BDG_OK = 0,
  BDG_ERR_INVALID = 1,        /* bad argument (size, pointer, enum, alias) */
  BDG_ERR_NOMEM = 2,          /* device or host allocation failed */
  BDG_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  BDG_ERR_BREAKDOWN = 4,      /* bi-orthogonalization lost rank / pencil not definite */
  BDG_ERR_NOT_CONVERGED = 5,  /* maxit reached; outputs hold the best pairs so far */
  BDG_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
  BDG_ERR_NAN = 7,            /* a NaN/Inf appeared in an input or an iterate */
  BDG_ERR_UNSUPPORTED = 8     /* valid request this build does not implement */
} bdg_status;

typedef enum { BDG_FP64 = 0, BDG_MIXED = 1 } bdg_precision;
typedef enum { BDG_C128 = 0, BDG_C64 = 1 } bdg_dtype;
typedef enum { BDG_UV = 0, BDG_FG = 1 } bdg_mode;

typedef struct {
  int dim;                 /* 1, 2 or 3 */
  int n[3];                /* points per axis (unused axes ignored) */
  double lo[3], hi[3];     /* box per axis */
  double beta_n, beta_s;   /* density and spin-exchange interaction (eq. GPE) */
  double p, q;             /* linear / quadratic Zeeman: adds -p S_z + q S_z^2 to L */
  double mu[3];            /* chemical potentials (mu_1, mu_0, mu_-1); NaN => computed
                              from Phi by eq. chem-formula with mu_1 + mu_-1 = 2 mu_0
                              filling vanishing components */
  int prec;                /* bdg_precision of bdg_solve */
  double tol;              /* relative residual target of bdg_solve (e.g. 1e-10) */
  int maxit;               /* iteration cap of bdg_solve */
  unsigned long long seed; /* seed of the internal start block when X0 == NULL */
  int flags;               /* reserved, 0 */
} bdg_params;

/*
 * bdg_plan_create -- set up one BdG problem (Section 3.1).
 *   out     [out] receives the plan handle (NULL on failure).
 *   p       [in, host] problem parameters, validated (dim, n, box, finite scalars).
 *   V       [in, host] trap potential on the grid, double[N_p].
 *   phi     [in, host] real ground state (phi_1, phi_0, phi_-1), double[3][N_p];
 *           eq. NLEP should hold to the accuracy wanted from the spectrum.
 *   stream  [in] cudaStream_t used for the set-up copies and kernels.
 * The chemical potentials (eq. chem-formula, with the vanishing-component
 * rule) and the deflation vectors of the null spaces of H_- and H_+
 * (Section 2.3) are computed on the device.  Returns BDG_OK or an error.
 */
bdg_status bdg_plan_create(bdg_plan_t* out, const bdg_params* p, const double* V,
                           const double* phi, void* stream);

/* bdg_plan_destroy -- free the plan and its device memory (synchronizes the
 * plan's last stream).  NULL is accepted. */
bdg_status bdg_plan_destroy(bdg_plan_t plan);

/* bdg_plan_mu -- copy the chemical potentials the plan uses into mu[3] (host). */
bdg_status bdg_plan_mu(bdg_plan_t plan, double* mu);

/*
 * bdg_apply -- y = M x for a block of nvec vectors (Section 3.2: the
 * matrix-free product by FFTs and pointwise multiplications).
 *   mode  BDG_UV: y = [[A, B], [-B, -A]] [u; v]            (eq. BdG-d)
 *         BDG_FG: y = (H_+ f, H_- g)                        (eq. lrep-d)
 *   dtype BDG_C128 or BDG_C64 (the arithmetic precision of the product).
 *   x, y  device, [nvec][6][N_p] complex of dtype; x and y must not overlap.
 *   nvec  >= 0 (0 is a no-op).
 */
bdg_status bdg_apply(bdg_plan_t plan, int mode, int dtype, const void* x, void* y, int nvec,
                     void* stream);

/*
 * bdg_biortho -- stable bi-orthogonal Gram-Schmidt (Section 3.2; Theorem
 * "Biorthogonality"): make the f-block F and the g-block G (each
 * [ncol][3][N_p] complex of dtype, device, updated in place) satisfy
 * F^H G = I and be bi-orthogonal to a locked bi-orthonormal pair (Fl, Gl)
 * (each [nlock][3][N_p], device, may be NULL when nlock == 0):
 *   twice  F <- F - Fl (Gl^H F),  G <- G - Gl (Fl^H G)
 *   S = F^H G = X Sigma Y^H,  keep sigma_i >= rtol sigma_max,
 *   F <- F X Sigma^-1/2,  G <- G Y Sigma^-1/2,
 * with rtol = 1e-12 (C128) or 1e-6 (C64).  The first *rank columns of F and G
 * hold the result; the rest are zeroed.  Gram entries are accumulated in
 * FP64; the SVD comes from the Hermitian matrix [[0, S], [S^H, 0]].
 * Limits: ncol <= 40, nlock <= 256 (BDG_ERR_UNSUPPORTED beyond).  F and G
 * must not overlap.  Returns BDG_ERR_BREAKDOWN (with *rank = 0) if S is zero.
 */
bdg_status bdg_biortho(bdg_plan_t plan, int dtype, void* F, void* G, int ncol, const void* Fl,
                       const void* Gl, int nlock, int* rank, void* stream);

/*
 * bdg_gram -- the Gram matrix of two blocks of complex columns taken as
 * real columns (real part, imaginary part): G = A^T B, the contraction of
 * the bi-orthogonal Gram-Schmidt (S = F^H G, Theorem "Biorthogonality") and
 * of the projected matrices U^H H_+ U, V^H H_- V of the Rayleigh-Ritz step
 * (Section 3.2).
 *   A, B    device, ncol_a (ncol_b) complex columns of n elements, column
 *           stride lda (ldb) elements, interleaved complex of dtype.
 *   G       device, double[2 ncol_a][2 ncol_b] row-major:
 *           G[2i+s][2j+t] = sum_{r<n} part_s(A_i[r]) part_t(B_j[r]),
 *           part_0 the real and part_1 the imaginary part.
 *   engine  BDG_GRAM_SIMT: FP32 (C64) or double-float with about 1e-15 of
 *           sum |a b| (C128) on the CUDA cores, row chunks summed in FP64;
 *           BDG_GRAM_TENSOR: every element split into three BF16 slices,
 *           the six leading slice products accumulated in FP32 by the
 *           tensor cores (tcgen05), row chunks summed in FP64: FP32 accuracy
 *           (about 1e-6 of sum |a b|) for either dtype; needs 2 ncol_b <= 160
 *           (BDG_ERR_UNSUPPORTED beyond).
 * Sums are taken in a fixed order (repeated calls give identical G).  The
 * workspace is allocated and freed in stream order on `stream`.
 * ncol_a or ncol_b == 0 is a no-op; n == 0 gives G = 0 (A and B may then
 * be NULL).
 */
typedef enum { BDG_GRAM_SIMT = 0, BDG_GRAM_TENSOR = 1 } bdg_gram_engine;
bdg_status bdg_gram(int dtype, int engine, const void* A, long long lda, int ncol_a, const void* B, long long ldb,
                    int ncol_b, long long n, double* G, void* stream);

/*
 * bdg_solve -- the k smallest positive excitation energies and their
 * Bogoliubov amplitudes (Sections 3.1-3.2; solver details are this library's
 * own, see the design notes).
 *   k       number of wanted pairs, 1 <= k <= m.
 *   m       block size, k <= m <= 52 (the projected problem of three
 *           blocks of m rounded up to even, at most 156 columns, must fit the
 *           160-column on-chip eigensolver; BDG_ERR_UNSUPPORTED beyond).
 *   X0      optional device start block, [m][6][N_p] C128 in the FG form (only
 *           the real parts are used); NULL => seeded internal block.
 *   omega   [out, host] double[k], ascending.
 *   UV      [out, device, may be NULL] [k][6][N_p] C128, (u, v) normalized to
 *           h^d (|u|^2 - |v|^2) = 1 (eqs. constrain, constrainfg), imaginary
 *           parts zero (the operator is real for a real Phi_g).
 *   resid   [out, host, may be NULL] double[k], relative residuals
 *           |M x - omega x| / (|omega| |x|) evaluated in FP64.
 *   nconv   [out, host] number of leading pairs with resid <= tol.
 * Precision: BDG_FP64 runs every kernel in FP64; BDG_MIXED runs the bulk
 * iteration in FP32 and finishes with FP64 refinement.  The call returns
 * after the outputs are written (it synchronizes the stream).  Returns
 * BDG_ERR_NOT_CONVERGED if fewer than k pairs reached tol within maxit.
 */
bdg_status bdg_solve(bdg_plan_t plan, int k, int m, const void* X0, double* omega, void* UV,
                     double* resid, int* nconv, void* stream);

/*
 * bdg_solve_batched -- the k[i] smallest positive excitations of count
 * independent problems (the batched workload: many parameter sets and grids,
 * eqs. lrep-d and constrain for each).  Each entry behaves as
 * bdg_solve(plans[i], k[i], m[i], NULL, omega[i], UV ? UV[i] : NULL,
 * resid ? resid[i] : NULL, &nconv[i], s) with the plan's seeded start
 * block.  The instances form a work queue (largest grids first) served by
 * up to 8 host threads (environment BDG_BATCH_WORKERS), each solving on a
 * stream of its own that starts after the work queued on `stream`; with a
 * grid above 2^20 points the instances are solved one at a time on
 * `stream`.  The plans must be distinct (BDG_ERR_INVALID otherwise) and on
 * the current device.  Every plan is attempted; the first failing status
 * (in plan order) is returned (bdg_last_error(NULL) names the plan), and
 * nconv[i] is filled for all entries.  Returns after every output is
 * written.
 */
bdg_status bdg_solve_batched(bdg_plan_t* plans, int count, const int* k, const int* m, double** omega,
                             void** UV, double** resid, int* nconv, void* stream);

/* Counters of the last bdg_solve on this plan. */
typedef struct {
  int iterations;          /* outer iterations (both phases) */
  int iterations_fp32;     /* iterations with FP32 products */
  int applies_fp32;        /* vector-products in FP32 */
  int applies_fp64;        /* vector-products in FP64 */
  double seconds;          /* wall time of the call */
  double flops_update_df;  /* algorithmic FLOPs (2 per multiply-add) of the FP64 block
                              updates, which run in double-float arithmetic */
} bdg_solve_stats;
bdg_status bdg_get_solve_stats(bdg_plan_t plan, bdg_solve_stats* st);

/*
 * bdg_ground_state -- ground state on S_M (eq. groundDef) for the problem in
 * p (mu ignored) with magnetization M, by a normalized gradient flow followed
 * by inexact Newton steps whose Hessian is H_+ = A + B (eqs. def_A + def_B),
 * all on the device in FP64.
 *   V      [in, host] double[N_p];  phi0 [in, host] start spinor double[3][N_p].
 *   phi    [out, host] double[3][N_p];  mu [out, host] double[3].
 *   resid  [out, host] max_j max_x |(H Phi)_j - mu_j phi_j|;  iters [out, host].
 *   tol    target of resid;  maxit  cap on flow steps + Newton-CG products.
 */
bdg_status bdg_ground_state(const bdg_params* p, double M, const double* V, const double* phi0,
                            double tol, int maxit, double* phi, double* mu, double* resid,
                            int* iters, void* stream);

/*
 * bdg_chemical_potentials_noalloc -- the chemical potentials mu_j of the
 * plan's Phi by eq. chem-formula (the values bdg_plan_create computes when
 * p->mu[j] is NaN), whatever mu the plan itself uses.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory during the call (a memory budget or caching allocator that
 * forbids implicit cudaMalloc, a loop that cannot afford an allocation's
 * synchronization).  It allocates nothing: its scratch is one fixed device
 * array of about 3.1 MB inside the library, held by every GPU that loads the
 * library until the process exits.
 *   mu     [out, host] double[3].
 * Limits and caveats:
 *   - grids of at most 16384 points (e.g. 128^2, 16 x 32^2, or 1-D up to
 *     1024); larger plans return BDG_ERR_UNSUPPORTED with the limit in
 *     bdg_last_error.
 *   - all calls share the array: calls that overlap on the GPU (several
 *     streams, threads or plans at once) race and must be serialized.
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and should come before any stream capture on
 *     that device.  The address is kept until the process exits: after a
 *     cudaDeviceReset of that device, do not call this entry point on it.
 * The call synchronizes the stream before it returns.
 */
bdg_status bdg_chemical_potentials_noalloc(bdg_plan_t plan, double* mu, void* stream);

/*
 * bdg_perturbed_density -- perturbed densities of excitation modes
 * (Section 4.2, the "2D Case" example; the ansatz eq. waveAssump with one
 * mode l kept):
 *   n_j^l(x, t) = | phi_j(x) + eps ( u_j^l(x) e^{-i omega_l t}
 *                                   + conj(v_j^l(x)) e^{i omega_l t} ) |^2,
 * j = 1, 0, -1, with phi the plan's ground state, for nmode modes and nt times.
 *   dtype  BDG_C128: FP64 arithmetic, double output;  BDG_C64: FP32
 *          arithmetic (phi rounded to FP32), float output.  The phases
 *          (eps cos omega t, eps sin omega t) are formed in FP64 on the host
 *          (and rounded to FP32 for BDG_C64).
 *   UV     [in, device] [nmode][6][N_p] complex of dtype in the UV form
 *          (u_1, u_0, u_-1, v_1, v_0, v_-1), e.g. as bdg_solve writes it.
 *   omega  [in, host] double[nmode];  times [in, host] double[nt].
 *   eps    the amplitude of the perturbation (finite).
 *   out    [out, device] [nmode][nt][3][N_p] real of dtype's precision;
 *          must not overlap UV.
 * nmode == 0 or nt == 0 is a no-op; nmode <= 65535.  Non-finite omega,
 * times or eps return BDG_ERR_INVALID.  With nmode * nt <= 128 the phase
 * table is passed with the launch and the call does not wait for the
 * stream.  Longer tables are copied from pageable host memory into plan
 * scratch: that copy first waits for the stream, and consecutive calls on
 * one plan must then be stream-ordered.
 */
bdg_status bdg_perturbed_density(bdg_plan_t plan, int dtype, const void* UV, int nmode, const double* omega,
                                 const double* times, int nt, double eps, void* out, void* stream);

/* bdg_last_error -- message of the last failing call on plan (NULL: of the
 * last failing plan-less call on this thread).  Never NULL. */
const char* bdg_last_error(bdg_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* BDG_H */
