/*
 * xs.h -- C ABI of libxs, the GB300 (sm_103a) semiempirical excited-state library.
 *
 * The library computes the lowest singlet excitations (and, beyond the paper,
 * the spin-adapted triplets) of closed-shell molecules at the CIS
 * (Tamm-Dancoff) and TDHF/RPA level on top of an NDDO ground state, following
 * arXiv:2505.24807 ("PySEQM 2.0"):
 *   - ground state: F C = C eps with S = I, restricted closed shell (Eq. 1);
 *   - RPA eigenproblem [[A,B],[B,A]][X;Y] = omega diag(I,-I)[X;Y] (Eq. rpa_eqn),
 *     CIS A X = omega X (Eq. cis_eqn);
 *   - Davidson iterations built on the product
 *       (A V)_ia = (eps_a - eps_i) V_ia + sum_{mu nu} C_mu,i Ft_mu,nu C_nu,a
 *     with Ft = sum [(mu nu|lam sig) - (mu lam|nu sig)] R_lam sig and
 *     R = C_occ V C_vir^T (Eqs. cis_matrix_vector, ftilde), Coulomb on the
 *     diagonal atom blocks and exchange called with the symmetric and
 *     antisymmetric parts of R (Section "GPU Implementation");
 *   - the batched Davidson steps 1-6 of the same section;
 *   - transition dipoles and oscillator strengths, and the absorption
 *     spectrum by Gaussian broadening (Section "Results and discussion").
 * Spin: singlet adaptation, A = d eps + 2(ia|jb) - (ij|ab),
 * B = 2(ia|jb) - (ib|ja) (the paper omits spin indices).
 *
 * Conventions
 *   - Units: energies in eV, lengths in Angstrom, oscillator strengths
 *     dimensionless (atomic units).
 *   - AO order = atom order; a heavy atom (Z = 6, 7, 8) carries s, px, py, pz,
 *     hydrogen (Z = 1) carries s.
 *   - Matrices are row-major float64.  C is n x n with MOs in columns;
 *     amplitudes X, Y are nocc x nvir row-major (index i * nvir + a).
 *   - Every function returns XS_OK (0) or a negative status; the message of
 *     the last failure is available from xs_last_error().  No C++ exception
 *     crosses this boundary.
 *   - The caller owns every host array it passes; the library copies what it
 *     needs and owns all device memory it allocates.  Pointers documented as
 *     "host or device" may point to either (unified addressing decides).
 *   - One context per host thread; calls on one context are not re-entrant.
 */
#ifndef XS_H
#define XS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define XS_OK 0
#define XS_EINVAL -1     /* bad argument (also odd electron counts: closed shell only) */
#define XS_ENOMEM -2     /* device allocation failed */
#define XS_ESCF -3       /* SCF did not converge, or HOMO-LUMO gap below the floor */
#define XS_EUNSTABLE -4  /* A - B not positive definite: unstable reference for TDHF */
#define XS_ENOCONV -5    /* Davidson not converged: outputs hold best estimates and residuals */
#define XS_ECUDA -6      /* CUDA runtime or library error */
#define XS_ETIMEOUT -7   /* a bounded device-side wait gave up */
#define XS_ESTATE -8     /* call order violated (e.g. excited before ground state) */

/* methods, precisions, product kinds */
#define XS_CIS 0
#define XS_TDHF 1

#define XS_FP64 0   /* every step in float64 */
#define XS_MIXED 1  /* split-precision tensor-core transforms, float32 G build, float64 subspace */

#define XS_KIND_A 0    /* A X          (CIS)  */
#define XS_KIND_APB 1  /* (A + B) X    (TDHF) */
#define XS_KIND_AMB 2  /* (A - B) X    (TDHF) */
#define XS_KIND_G 3    /* G_CIS(R) = 2 J(R) - K(R) of an n x n AO matrix R */
#define XS_KIND_A_TRIPLET 4    /* A_T X = de X - C_occ^T K(R) C_vir (triplet CIS) */
#define XS_KIND_APB_TRIPLET 5  /* (A_T + B_T) X (triplet TDHF); (A_T - B_T) = (A - B): XS_KIND_AMB */

/* Spin of the computed states (xs_ex_opts.spin).  The paper computes
 * closed-shell singlets; triplets use the spin-adapted A_T = de - (ij|ab),
 * B_T = -(ib|ja) (no Coulomb terms in G) and have zero oscillator strength. */
#define XS_SINGLET 0
#define XS_TRIPLET 1

#define XS_GUESS_PLAIN 0    /* unit vectors on the lowest orbital-energy gaps */
#define XS_GUESS_LEARNED 1  /* MLP-predicted guess and diagonal shift (plain fallback) */
#define XS_SUBSPACE_AUTO 0
#define XS_SUBSPACE_FP64 1
#define XS_SUBSPACE_EMULATED 2

/* Number of per-element parameter fields, in this order:
 * Uss, Upp, beta_s, beta_p, gss, gsp, gpp, gp2, hsp, D1, D2, zeta_s, zeta_p
 * (eV for energies, Angstrom for D1/D2, 1/Angstrom for zeta).  Rows are the
 * elements H, C, N, O. */
#define XS_NPARAM 13
#define XS_NELEM 4

typedef struct xs_ctx xs_ctx;

typedef struct {
  int n_mol;
  int max_scf_iter_used; /* largest SCF iteration count over the molecules */
  double seconds;        /* wall time of the call */
} xs_gs_info;

typedef struct {
  int method;        /* XS_CIS or XS_TDHF */
  int nroots;        /* roots per molecule (>= 1) */
  double tol;        /* residual 2-norm threshold in eV.  XS_MIXED solves apply max(tol, 1e-4 eV):
                        their products carry ~1e-6 relative rounding, so residuals stall near 1e-5 eV,
                        while the energies (quadratic in the residual, then refined by a float32
                        Rayleigh-Ritz step) still land within ~5e-6 eV.  The threshold applied is
                        returned in xs_solve_info.tol_used */
  int precision;     /* XS_FP64 or XS_MIXED */
  int guess;         /* XS_GUESS_PLAIN or XS_GUESS_LEARNED */
  int max_subspace;  /* subspace cap per molecule (0: library default) */
  int max_iter;      /* Davidson iteration cap (0: library default) */
  int batched;       /* 0: molecules one after another (each with its own launch sequence);
                        1: lock-step batch -- every molecule of the last xs_ground_state call advances
                        one Davidson iteration per replay of one captured CUDA graph whose kernels walk
                        device-side work lists over all molecules (no zero padding; converged molecules
                        retire on the device); up to 16 roots, subspaces of at most 128 vectors, products
                        in float32 SIMT (XS_MIXED) or float64 (XS_FP64), float64 subspace; the learned
                        guess is scored for all molecules in one network pass;
                        2: molecules concurrently, each on its own stream and host thread */
  int subspace;      /* float64 subspace products: XS_SUBSPACE_AUTO (0), XS_SUBSPACE_FP64 (1, the
                        float64 pipe) or XS_SUBSPACE_EMULATED (2, exact digit splitting on the tensor
                        cores, see xs_subspace_gram); AUTO = EMULATED for XS_MIXED solves of
                        molecules with nocc * nvir >= 32768, else FP64 */
  double memory_limit; /* bytes the subspace arrays of one molecule may occupy (V and its products in
                          float64, their digit operands when emulated); the subspace cap is lowered to
                          fit.  0: the device's free memory at the call, plus the context's reusable
                          subspace buffers, less a reserve for the other work buffers.  XS_ENOMEM when
                          not even the initial guess block and one block of new vectors fit */
  int spin;            /* XS_SINGLET (0) or XS_TRIPLET (1); triplet solves use the plain guess */
} xs_ex_opts;

typedef struct {
  int iterations;       /* Davidson iterations of the slowest molecule */
  long long products;   /* trial vectors multiplied (sum over molecules) */
  int converged;        /* 1 if every root of every molecule converged */
  int polished;         /* 1 if a float32-SIMT Rayleigh-Ritz step followed a mixed solve */
  int learned;          /* 1 if the learned guess and diagonal shift were used */
  int fallback;         /* 1 if the learned shift was dropped because a residual stalled */
  double seconds;       /* wall time of the call */
  double seconds_products;  /* of which in A*X products */
  int max_subspace_used;    /* subspace cap in effect (largest over the molecules) */
  double tol_used;          /* residual threshold applied (eV): opts->tol, or its mixed-precision floor */
  long long graph_launches; /* lock-step batched solves (batched = 1): CUDA graph replays, one per iteration */
} xs_solve_info;

/* Create a context on CUDA device `device`.  `stream` is a cudaStream_t to
 * borrow (the caller keeps ownership) or NULL for a library-owned stream. */
int xs_create(xs_ctx** out, int device, void* stream);
int xs_destroy(xs_ctx* ctx);

/* Message of the last failure on this context ("" if none).  Valid until the
 * next call on the context. */
const char* xs_last_error(const xs_ctx* ctx);

/* Set the per-element NDDO parameters: `table` is XS_NELEM x XS_NPARAM
 * float64 (rows H, C, N, O; fields as listed at XS_NPARAM).  The paper's
 * Hamiltonians (MNDO/AM1/PM3/PM6, Section "Overview") use tabulated sets of
 * this kind; the library copies the table. */
int xs_set_params(xs_ctx* ctx, const double* table, int n_elem);

/* Ground state of n_mol molecules: integrals (two-centre multipole model,
 * one-centre parameters), core Hamiltonian and the closed-shell SCF of Eq. 1
 * (Pulay DIIS; converged when max|dD| < scf_tol and max|FD - DF| < 10 scf_tol eV).
 * natoms[n_mol]; Z and xyz (Angstrom, 3 per atom) concatenated over the
 * molecules, host memory.  Returns XS_ESCF if a molecule does not converge
 * or its HOMO-LUMO gap is below 0.5 eV, XS_EINVAL for odd electron counts or
 * unsupported elements. */
int xs_ground_state(xs_ctx* ctx, int n_mol, const int* natoms, const int* Z, const double* xyz,
                    double scf_tol, int max_iter, xs_gs_info* info);

/* Sizes of molecule `mol` after xs_ground_state. */
int xs_get_sizes(const xs_ctx* ctx, int mol, int* nao, int* nocc, int* natoms);

/* The model of molecule `mol` as the library built it (on the device): the
 * two-centre product supermatrix W (nprod x nprod, nprod = 10 per heavy atom +
 * 1 per hydrogen; rows and columns are the on-atom AO products mu <= nu in
 * atom order, (s,s), (s,px), (s,py), (s,pz), (px,px), (px,py), (px,pz),
 * (py,py), (py,pz), (pz,pz) on a heavy atom; W[p][q] = (mu nu|lam sig) for
 * products on different atoms, zero inside an atom's own block) and the core
 * Hamiltonian H (n x n): paper, Section "Ground-state wavefunction
 * calculation".  Either pointer may be NULL; host or device memory; nprod is
 * returned in *nprod when it is not NULL. */
int xs_get_model(const xs_ctx* ctx, int mol, double* W, double* H, int* nprod);

/* Read (get) or replace (set) the MO coefficients C (n x n, row-major, MOs in
 * columns) and orbital energies eps (n, eV) of molecule `mol`; host or
 * device pointers.  Replacing them lets a caller run the products on its own
 * orbitals. */
int xs_get_orbitals(const xs_ctx* ctx, int mol, double* C, double* eps);
int xs_set_orbitals(xs_ctx* ctx, int mol, const double* C, const double* eps);

/* Apply a response product to nvec vectors of molecule `mol`
 * (Eqs. cis_matrix_vector and ftilde):
 *   kind XS_KIND_A / APB / AMB / A_TRIPLET / APB_TRIPLET: in and out are nvec x (nocc*nvir);
 *   kind XS_KIND_G: in and out are nvec x (n*n) AO matrices, out = 2J(R) - K(R).
 * `precision` selects XS_FP64 or XS_MIXED.  Host or device pointers. */
int xs_apply(xs_ctx* ctx, int mol, int kind, int nvec, const double* in, double* out, int precision);

/* Excited states of every molecule loaded by xs_ground_state (paper,
 * batched Davidson steps 1-6; RPA in the symmetric subspace form of
 * Stratmann, Scuseria and Frisch).  Outputs are host or device arrays of
 * n_mol * nroots entries: omega (eV), osc (oscillator strengths), resid
 * (final residual norms, eV); iters has n_mol entries.  A molecule has
 * nocc * nvir roots at most: entries past them are 0.  Any output may be
 * NULL.  Returns XS_ENOCONV with best estimates filled if the iteration cap
 * is reached, XS_EUNSTABLE if A - B is not positive definite (TDHF). */
int xs_excited(xs_ctx* ctx, const xs_ex_opts* opts, double* omega, double* osc, int* iters,
               double* resid, xs_solve_info* info);

/* Amplitudes of root `root` of molecule `mol` from the last xs_excited:
 * X (and Y for TDHF; Y may be NULL) of nocc*nvir float64 each, normalised
 * |X|^2 - |Y|^2 = 1.  `ov` must equal nocc*nvir.  Host or device pointers. */
int xs_get_amplitudes(const xs_ctx* ctx, int mol, int root, double* X, double* Y, size_t ov);

/* ---- learned Davidson guess and preconditioner ----------------------------
 * Not in the paper: a small MLP (XS_MLP_FEATURES -> 256 -> 256 -> 256 -> 2,
 * gelu, weights rounded to bfloat16, float32 accumulation) maps per-pair
 * features of the lowest orbital-energy gaps to (0) the diagonal shift
 * A_ia,ia - (eps_a - eps_i) = 2(ia|ia) - (ij|ab)|_{j=i,b=a}, used as the
 * preconditioner r / (omega - d eps - shift), and (1) log10 of the pair's
 * weight sum_n X_n,ia^2 in the lowest roots, used to pick the start vectors.
 * xs_excited uses it when opts->guess == XS_GUESS_LEARNED and a network is
 * loaded; the plain Davidson still decides convergence and the shift is
 * dropped when a residual stalls, so converged roots do not change. */
#define XS_MLP_FEATURES 11

/* number of float32 parameters of the network (weights and biases, layer by
 * layer: W (out x in) row-major, then b) */
int xs_mlp_nparams(void);
/* initialise the context's network (uniform +-1/sqrt(fan_in) weights, zero biases) */
int xs_mlp_init(xs_ctx* ctx, unsigned long long seed);
/* copy the parameters out / in (host or device, xs_mlp_nparams() floats) */
int xs_mlp_get_weights(xs_ctx* ctx, float* w);
int xs_mlp_set_weights(xs_ctx* ctx, const float* w);
/* features of the npairs lowest-gap pairs of molecule `mol`: features
 * (npairs x XS_MLP_FEATURES float32) and the pairs (flattened i * nvir + a);
 * returns the number of pairs written in *count (<= npairs) */
int xs_mlp_features(xs_ctx* ctx, int mol, int npairs, float* features, long long* pairs, int* count);
/* training targets of the given pairs (npairs x 2 float32): exact diagonal
 * shift (eV) and log10(max(sum over the last solve's roots of (X+Y)_ia^2, 1e-6)) */
int xs_mlp_targets(xs_ctx* ctx, int mol, int npairs, const long long* pairs, float* targets);
/* network outputs (rows x 2) for the given features */
int xs_mlp_forward(xs_ctx* ctx, int rows, const float* features, float* out);
/* gradient of the weighted loss (see xs_mlp_train) with respect to every
 * parameter (xs_mlp_nparams() floats, host or device), and the loss */
int xs_mlp_grad(xs_ctx* ctx, int rows, const float* features, const float* targets, float* grad, float* loss);
/* Adam training on the GPU: `epochs` passes over rows samples in minibatches
 * of `batch` rows (in the given order), learning rate lr, loss weights 0.01
 * (shift, eV^2) and 1 (log-weight); mean loss per epoch in loss (epochs). */
int xs_mlp_train(xs_ctx* ctx, int rows, const float* features, const float* targets, int epochs, int batch,
                 float lr, float* loss);

/* Allocation-free G(R) build: the same G = 2J(R) - K(R) as
 * xs_apply(ctx, mol, XS_KIND_G, nvec, R, G, XS_FP64), for callers that cannot
 * call cudaMalloc during the call: a process whose device memory is reserved
 * up front by another allocator's pool (a framework's caching allocator), or
 * a latency-critical loop that must not meet cudaMalloc's implicit device
 * synchronisation.  No counterpart in the paper.
 *   R, G: DEVICE pointers to nvec n x n row-major float64 matrices, owned by
 *   the caller (molecule `mol` must have its ground state already).
 * Scratch comes from one fixed device array of 2^18 doubles (2 MiB) compiled
 * into the library, held by every GPU that loads the library until the
 * process exits.  A call needs 2 * nprod * nvec doubles of it (nprod = 10 per
 * heavy atom + 1 per hydrogen); larger requests return XS_EINVAL.  The first
 * call on a device looks the array's device address up once; make that first
 * call before any stream capture.  The call is asynchronous on the context's
 * stream.  Every call shares the one array: calls that overlap on the GPU
 * (other streams or contexts on the same device) race.  Nothing in the array
 * needs clearing -- each call writes every element it later reads.  The call
 * makes no cudaMalloc, cudaFree or allocating library call. */
int xs_gbuild_noalloc(xs_ctx* ctx, int mol, int nvec, const double* R, double* G);

/* ---- float64 subspace products (the Davidson step, Section "GPU
 * Implementation": projected matrices V^T A V, Gram-Schmidt against V, Ritz
 * vectors and residuals V x) ----------------------------------------------
 * The solver uses these internally; they are exported so that the products
 * can be checked and timed on their own.  emulated != 0 runs them on the
 * BF16 tensor cores by exact digit splitting (Ozaki et al., Numer. Algorithms
 * 59 (2012) 95): every float64 row is cut into eight base-128 digits scaled
 * by a per-row power of two, digit products are summed exactly in float32
 * chunks of 4096 and assembled in float64 -- float64 accuracy (an error of
 * the order of a float64 GEMM's) at tensor-core speed.  emulated == 0 runs
 * the float64-pipe GEMM.  Pointers may be host or device memory, row-major,
 * owned by the caller; the call is synchronous.  Errors: XS_EINVAL for bad
 * sizes, XS_ECUDA for a non-finite input (emulated) or a CUDA failure,
 * XS_ETIMEOUT when a bounded device wait gave up. */
/* C (M x N) = A B^T, A: M x L, B: N x L */
int xs_subspace_gram(xs_ctx* ctx, int M, int N, long long L, const double* A, const double* B, double* C,
                     int emulated);
/* Y (nout x L) = sum_{b<nb} coef_b^T X_b, X: nb x S x L, coef: nb x S x nout, 1 <= nb <= 3 */
int xs_subspace_combine(xs_ctx* ctx, int nb, int S, int nout, long long L, const double* X, const double* coef,
                        double* Y, int emulated);

/* The Rayleigh-Ritz eigensolver of the Davidson step on its own (paper,
 * batched step 3: diagonalise the projected matrix, keep the lowest K):
 * the k lowest eigenpairs of the symmetric S x S float64 matrix A (row-major,
 * 1 <= k <= S <= 1024), eigenvalues ascending in w (k entries), eigenvectors
 * in the columns of Z (S x k, row-major: Z[i * k + t]).  Householder
 * tridiagonalisation, float32 Sturm multisection, float64 inverse iteration
 * (clusters of close eigenvalues orthogonalised as they are found), one CTA.
 * Host or device pointers owned by the caller; synchronous.  XS_EINVAL for bad
 * sizes. */
int xs_subspace_eig(xs_ctx* ctx, int S, int k, const double* A, double* w, double* Z);

/* Parameter derivatives of a CIS or TDHF excitation energy (paper, Section
 * "Overview of the capabilities of PySEQM": the semiempirical parameters are
 * learned by differentiating through the model).  After a singlet xs_excited,
 * grad (XS_NELEM x XS_NPARAM float64, host or device; rows H, C, N, O, fields
 * as listed at XS_NPARAM) receives d omega_root / d parameter in eV per unit
 * of the parameter, including the response of the ground-state orbitals: one
 * adjoint solve (A+B) Z = L by conjugate gradients on float64 (A+B) products,
 * then the derivatives of the core Hamiltonian, one-centre and two-centre
 * integrals contracted with the relaxed difference density.  cg_iterations
 * (may be NULL) receives the adjoint solve's iteration count.  XS_ESTATE if
 * the molecule has no singlet solution, XS_EINVAL for a bad root,
 * XS_EUNSTABLE if A+B is not positive definite, XS_ENOCONV if the adjoint
 * solve does not converge in 500 iterations. */
int xs_gradient(xs_ctx* ctx, int mol, int root, double* grad, int* cg_iterations);

/* Absorption spectrum (paper, Section "Results and discussion": the computed
 * states' oscillator strengths broadened by Gaussians of width 0.1 eV):
 *   out[g] = sum_{i<n} f[i] exp(-(grid[g] - omega[i])^2 / (2 width^2)) / (width sqrt(2 pi))
 * omega, grid and width in eV; width is the Gaussian's standard deviation
 * (each line has unit area, so the spectrum integrates to sum f).  omega and
 * f (n values), grid and out (ngrid values) may be host or device memory,
 * owned by the caller; n = 0 gives zeros.  XS_EINVAL for negative counts,
 * null arrays with positive counts, or a width that is not positive and
 * finite.  Synchronous. */
int xs_spectrum(xs_ctx* ctx, int n, const double* omega, const double* f, double width, int ngrid,
                const double* grid, double* out);

/* Per-kernel timing.  xs_profile(ctx, 1) clears and enables it: every
 * instrumented kernel launch of later calls is bracketed by CUDA events on
 * the launching stream; xs_profile(ctx, 2) clears and enables counting only
 * (launches, algorithmic bytes and flops, host phases; no CUDA events, ms = 0
 * for kernels), which leaves device timings undisturbed; xs_profile(ctx, 3)
 * is mode 1 plus entries "gap:<kernel>" holding the device idle time between
 * the previous instrumented launch and each launch of <kernel> (a timeline of
 * the launching stream); xs_profile(ctx, 0) disables it.  xs_profile_read
 * synchronises the context's stream and copies up to max_entries entries
 * (one per kernel name: launches, summed device milliseconds, summed
 * algorithmic bytes and flops) and the number of entries into *count.
 * Entries named "host:<phase>" hold host wall milliseconds of the excited-
 * state solver's phases instead (setup, learned_guess, loop, finish; fetch_wait and
 * sync_wait: time blocked on the device; launches = times entered), and
 * "all_launches" counts every kernel launch of the library.  No counterpart
 * in the paper (measurement plumbing). */
typedef struct {
  char name[32];
  int launches;
  double ms;
  double bytes;
  double flops;
} xs_prof_entry;

int xs_profile(xs_ctx* ctx, int enable);
int xs_profile_read(xs_ctx* ctx, xs_prof_entry* out, int max_entries, int* count);

#ifdef __cplusplus
}
#endif

#endif /* XS_H */
