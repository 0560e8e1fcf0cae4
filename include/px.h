/*
 * px.h -- C ABI of the GB300 (sm_103a) wFQ / wFQFmu linear-response library.
 *
 * The library solves, for every frequency w of a sweep and every field
 * polarisation e, the complex linear system of the wFQ model (Eq. 1)
 *
 *     [ Kbar T^qq - z_q(w) I_N ] q(w) = -Kbar V(w)
 *
 * or of the wFQFmu model (Eq. 7)
 *
 *     [ diag(Kbar, I_3N) T - diag(z_q(w) I_N, z_mu(w) I_3N) ] (q; mu)
 *                                         = diag(Kbar, I_3N) (-V; E),
 *
 * with K the Fermi-damped Drude bond weights (Eq. 3, Eq. 4), Kbar its Laplacian
 * form (Eq. 2), T the Gaussian-smeared Coulomb kernels (Eq. 5 and its
 * derivatives, Sec. 2.2), z_q the Drude shift (Eq. 6) and z_mu = -1/alpha^IB
 * (Eq. 8), and returns the induced charges and dipoles, the complex
 * polarisability alpha_kl = d d_k / d E_l with d = sum q_i r_i (+ sum mu_i) and
 * the absorption cross-section 4 pi w / (3c) Tr Im alpha (Sec. "Observables").
 *
 * All frequencies and polarisations of one call form one block of right-hand
 * sides that is solved together on the GPU (restarted GMRES with FP64
 * orthogonalisation and FP64 true-residual refinement around a low-precision
 * block matvec; Sec. "Solvers" describes the per-frequency GMRES this batches).
 *
 * Conventions for every function below:
 *   - Every function returns px_status; none aborts, throws or exits.
 *   - Inputs are read (and copied where the handle keeps them) during the call;
 *     the caller keeps ownership of every buffer it passes.
 *   - Outputs go to caller-allocated buffers; a NULL output pointer skips that
 *     output.
 *   - Complex numbers are interleaved (re, im) doubles.
 *   - Units at the boundary: Angstrom for positions, eV for frequencies,
 *     atomic units for everything else (bohr, hartree, bohr^3 for alpha, bohr^2
 *     for cross-sections).  Inside, everything is in atomic units.
 *   - On failure px_last_error(h) holds a human-readable message.
 *   - One handle must not be used by two host threads at the same time.
 */
#ifndef PX_H
#define PX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PX_ABI_VERSION 2

typedef enum {
  PX_OK = 0,
  PX_EINVAL = 1,     /* bad argument: NULL where required, size <= 0, NaN, duplicate atoms */
  PX_ENOMEM = 2,     /* device allocation failed or the HBM budget is exceeded */
  PX_ENOTCONV = 3,   /* at least one column missed the tolerance; see status[] */
  PX_ETIMEOUT = 4,   /* a bounded wait ran out */
  PX_ECUDA = 5,      /* a CUDA runtime call failed (message in px_last_error) */
  PX_EBUSY = 6,      /* the server queue is full */
  PX_ENOTIMPL = 7,   /* valid request that the library does not support */
  PX_ENOTFOUND = 8   /* unknown request id */
} px_status;

typedef enum {
  PX_WFQ = 0,           /* Eq. 1: charges only, N unknowns */
  PX_WFQFMU = 1,        /* Eq. 7: charges and dipoles, 4N unknowns; one n, tau for all types */
  PX_WFQFMU_HETERO = 2  /* Eq. 9 with Eq. 10 (alloys, core-shell): atom types may differ in
                           drude_n_au and tau_au; z_q is the charge's own type's (Eq. 6), the
                           conductance block is 1/2 (Kbar + Hbar(w)) with
                           H_ij = (n_j tau_j)/(n_i tau_i) (1 - i w tau_i)/(1 - i w tau_j) K_ji, and
                           each atom's alpha^IB is Eq. 10's weighted harmonic mean over the
                           atom and its nearest neighbours (atoms within the pair's Fermi
                           midpoint s r0).  PX_FP32 or PX_FP64 matvecs, materialised T */
} px_model;

/* Arithmetic of the block matvec Y = T X inside the Krylov iteration.  The
 * Hessenberg least squares, the true residual and the refinement are FP64 (or
 * double-FP32, ~48 bits) in every mode; the storage of the Krylov basis is
 * chosen by px_basis. */
typedef enum {
  PX_FP64 = 0,       /* FP64 matvec (plain double-precision solve) */
  PX_FP32 = 1,       /* FP32 matvec on the CUDA cores */
  PX_BF16SPLIT = 2,  /* T = T_hi + T_lo, X = X_hi + X_lo in bf16; tcgen05 MMA with FP32
                        accumulation of T_hi X_hi + T_hi X_lo + T_lo X_hi (~16 bits) */
  PX_FP16SPLIT = 3   /* the same three tcgen05 products on power-of-two scaled fp16 parts,
                        lo parts scaled by 2^11 into a second accumulator (~22 bits) */
} px_precision;

/* Storage and arithmetic of the Krylov basis V and the Gram-Schmidt sweeps over it
 * (the sweeps are bound by HBM bandwidth, so the element size sets their cost). */
typedef enum {
  PX_BASIS_AUTO = 0,  /* PX_FP64: FP64; low-precision matvecs: FP32 */
  PX_BASIS_FP64 = 1,  /* FP64 complex, 16 bytes per entry */
  PX_BASIS_FF32 = 2,  /* double-FP32 complex (hi + lo pairs, ~48 bits), 16 bytes per
                         entry; arithmetic on the FP32 pipe with error-free transforms */
  PX_BASIS_FP32 = 3   /* FP32 complex, 8 bytes per entry; low-precision matvecs only:
                         each refinement round asks the inner iteration for a modest
                         reduction (inner_tol), which the FP32 basis delivers, and the
                         FP64 true residual corrects what it loses */
} px_basis;

typedef enum {
  PX_MODE_AUTO = 0,         /* materialise T if it fits the HBM budget, else matrix-free */
  PX_MODE_MATFREE = 1,      /* generate T tiles on the fly inside the matvec ("on the fly") */
  PX_MODE_MATERIALISED = 2  /* store T once per structure ("on memory") */
} px_mode;

/* How the columns of a sweep are solved. */
typedef enum {
  PX_SOLVER_BATCHED = 0,  /* every (frequency, direction) column is its own restarted GMRES;
                             all columns share one block matvec (both models) */
  PX_SOLVER_SHIFTED = 1   /* PX_WFQ only: Eq. 1's frequency enters as the scalar shift
                             z_q(w) I (Eq. 6) and its right-hand side does not depend on w,
                             so one real Arnoldi process of Kbar T per field direction
                             serves every frequency (shifted GMRES, unrestarted, in
                             double-FP32 throughout: matvec on T held as two FP32 planes,
                             basis, orthogonalisation).  Columns whose FP64-class true
                             residual misses tol_rel afterwards (basis limit reached) continue
                             in the batched refinement with the handle's precision.  Needs
                             the materialised T */
} px_solver;

/* Per-atom-type parameters (Eqs. 3-6 and the Gaussian widths of Secs. 2.1, 2.2).
 * Pair values of r0, d and s are the arithmetic means of the two atoms' types. */
typedef struct {
  double r0_ang;      /* nearest-neighbour distance r^0 of the lattice, Angstrom (Eq. 4) */
  double d;           /* Fermi steepness d (Eq. 4) */
  double s;           /* Fermi scale s (Eq. 4) */
  double area_bohr2;  /* effective area A_i, bohr^2, > 0 (Eq. 3) */
  double Rq_bohr;     /* Gaussian charge width R_q, bohr, > 0 (Sec. 2.1) */
  double Rmu_bohr;    /* Gaussian dipole width R_mu, bohr, > 0 (Sec. 2.2; wFQFmu only) */
  double drude_n_au;  /* density n of Eq. 6, a.u., > 0; equal for all types */
  double tau_au;      /* scattering time tau of Eq. 6, a.u., > 0; equal for all types */
} px_atom_type;

typedef struct {
  int precision;            /* px_precision; default PX_FP32 */
  int mode;                 /* px_mode; default PX_MODE_AUTO */
  int restart_m;            /* Krylov basis length per restart cycle; 0 (default) = automatic:
                               60 for low-precision PX_WFQ solves, 100 for PX_WFQFMU and for
                               PX_FP64 solves; a cycle whose active set has shrunk uses a
                               longer restart (up to 400) in the same memory */
  int max_iter;             /* cap on matvecs per column over the whole solve; default 20000 */
  int max_cycles;           /* cap on restart cycles (inner cycles of all rounds); default 200 */
  int max_refine;           /* FP64 refinement rounds after the first low-precision solve;
                               0 returns the first round's result; default 20 */
  int gs_passes;            /* Gram-Schmidt passes (1 = CGS, 2 = CGS2); default 1 */
  int basis;                /* px_basis; default PX_BASIS_AUTO.  PX_FP64 accepts only
                               AUTO and PX_BASIS_FP64 */
  int gemm_tiles;           /* tile shape of the tensor-core matvec: 0 (default) = autotuned
                               per (rows, columns) shape on first use, cached per process;
                               1 = 128 x 256 tiles, 2-stage ring (where the padded operand
                               column count is a multiple of 256, else 2 runs); 2 = 128 x 128
                               tiles, 3-stage ring.  Every choice gives bit-identical results */
  int cycle_graphs;         /* 1 (default): each restart cycle is one CUDA graph launch whose
                               device-side while loop runs the Krylov steps (matvec, shift,
                               Gram-Schmidt, Givens, normalisation) until every column stopped
                               or the basis is full; graphs are cached per handle and shape.
                               0: one launch per kernel with a per-step host poll.  profile = 1
                               always uses the latter (events around every matvec) */
  int sort_atoms;           /* 1 (default): the device reorders atoms along a Morton curve of
                               their positions (neighbours at nearby indices); per-atom
                               inputs and outputs stay in the caller's order.  0: keep the
                               caller's order */
  double tol_rel;           /* per-column target ||b - A x||_2 / ||b||_2 in FP64; default 1e-7 */
  double inner_tol;         /* per-cycle reduction asked of the low-precision inner
                               iteration (ignored in PX_FP64); default 1e-3 */
  double kcut_eps;          /* keep bond pairs with 1 - f(r) >= kcut_eps; default 1e-6 */
  int mu_self_term;         /* 1: Gaussian self term on the T^mumu diagonal; default 0 */
  int profile;              /* 1: time every matvec launch with CUDA events; default 0 */
  size_t hbm_budget_bytes;  /* device memory the handle may use; 0 = 90% of free memory */
  double device_wait_limit_s; /* bound on any host wait for device progress; default 600 */
  int solver;               /* px_solver; default PX_SOLVER_BATCHED */
  int shift_krylov_max;     /* PX_SOLVER_SHIFTED: largest basis per field direction; 0 (default)
                               = automatic, min(n_u, 2500) further limited so that the basis,
                               the per-shift triangular factors and the products T V fit in
                               40% of the free device memory */
} px_options;

/* Host-side results of px_solve.  F = n_freq, P = n_pol, N = n_atoms.  Column
 * (f, p) is one spectrum point.  Every pointer may be NULL. */
typedef struct {
  double* alpha;         /* [F][3][P] complex: alpha_kp = d_k / E0 for field along pol p */
  double* sigma_abs;     /* [F]: 4 pi w/(3c) Tr Im alpha (orientation average); only when
                            P == 3.  The full alpha tensor is A E^-1 (A = alpha[f] as written
                            here, E = the 3 x 3 matrix whose columns are the field
                            directions), so any three linearly independent directions work;
                            linearly dependent ones (|det E| < 1e-6) with sigma_abs
                            requested make px_solve return PX_EINVAL */
  double* sigma_abs_pol; /* [F][P]: 4 pi w / c Im(e_p . alpha e_p) */
  double* q;             /* [F][P][N] complex induced charges, caller's atom order */
  double* mu;            /* [F][P][N][3] complex induced dipoles (wFQFmu) */
  double* rel_residual;  /* [F][P]: final ||b - A x|| / ||b||, FP64 */
  int* iters;            /* [F][P]: low-precision matvecs spent on the column */
  int* status;           /* [F][P]: PX_OK or PX_ENOTCONV */
} px_result;

/* Timing and work counters of the last px_solve on a handle. */
typedef struct {
  double setup_ms;         /* px_set_structure device time (neighbour list, T build) */
  double solve_ms;         /* px_solve device time, staging to observables */
  double matvec_ms;        /* summed CUDA-event durations of the low-precision matvec
                              launches (only with options.profile) */
  long long matvec_launches;
  double matvec_flops;     /* algorithmic flops of those launches: 4 n_u^2 B_active each */
  double matvec_bytes;     /* algorithmic bytes of those launches (T once + X + Y) */
  double resid_ms;         /* summed durations of the FP64 true-residual matvecs (profile) */
  long long resid_launches;
  double resid_flops;
  long long kernel_launches; /* every kernel this library launched in the last px_solve */
  long long setup_launches;  /* kernels launched by the last px_set_structure */
  int cycles;              /* restart/refinement cycles run */
  long long total_iters;   /* sum over cycles of the inner iterations run */
  long long n_unknowns;    /* n_u: N (wFQ) or 4N (wFQFmu) */
  int used_mode;           /* px_mode actually used */
  int used_precision;      /* px_precision actually used */
  int gemm_tiles_used;     /* tensor-core matvec tile shape of the first (widest) cycle:
                              1 or 2 as in px_options.gemm_tiles; 0 without that matvec */
  long long graph_launches; /* restart cycles run as one graph launch each */
  long long graphs_built;   /* of those, cycles whose graph was captured and instantiated
                               (the others reused a cached graph) */
  int solver_used;          /* px_solver of the last px_solve */
  long long shift_steps;    /* PX_SOLVER_SHIFTED: Arnoldi steps, summed over direction groups */
  long long shift_matvec_launches;  /* double-FP32 matvecs on <= 4 columns (one per step) */
  double shift_matvec_ms;   /* their summed CUDA-event durations (only with options.profile) */
  double shift_matvec_bytes;  /* their algorithmic bytes: T's two FP32 planes once, n_u^2 8 */
  double shift_ms;          /* device time of the shifted phase, start to true residual */
} px_stats;

typedef struct px_handle px_handle;

/* Library ABI version (PX_ABI_VERSION). */
int px_abi_version(void);

/* Fill *opt with the defaults listed in px_options.  PX_EINVAL if opt is NULL. */
px_status px_options_default(px_options* opt);

/* Create a handle on the current CUDA device.  opt may be NULL (defaults).
 * The handle owns all device memory it allocates and one CUDA stream.
 * PX_EINVAL for bad options, PX_ECUDA if no device is usable. */
px_status px_create(px_handle** h, const px_options* opt);

/* Replace the handle's options (validated as in px_create). */
px_status px_set_options(px_handle* h, const px_options* opt);

/* Load a structure (Sec. "Specify the Nanostructure": atom positions in
 * Angstrom) and build its device-resident operators: the CSR of K (Eq. 3) with
 * the diagonal of Kbar (Eq. 2), and T (Eq. 5, Sec. 2.2) in the storage the
 * options select.
 *   model     PX_WFQ (n_u = N unknowns), PX_WFQFMU or PX_WFQFMU_HETERO (n_u = 4N).
 *   xyz_ang   [n_atoms][3] doubles, Angstrom.
 *   type_idx  [n_atoms] ints in [0, n_types).
 *   types     [n_types] parameter records (all share drude_n_au and tau_au except
 *             under PX_WFQFMU_HETERO).
 * Errors: PX_EINVAL (NULL, n_atoms < 1, bad type index, non-finite or
 * non-positive parameter, two atoms closer than 1e-6 Angstrom), PX_ENOMEM,
 * PX_ENOTIMPL (PX_WFQFMU_HETERO with a split precision), PX_ECUDA.  Synchronous:
 * returns after the device work finished. */
px_status px_set_structure(px_handle* h, px_model model, int n_atoms, const double* xyz_ang,
                           const int* type_idx, const px_atom_type* types, int n_types);

/* Solve the loaded structure for every (frequency, polarisation) column and
 * write the observables (Sec. "Observables") to host buffers.
 *   n_freq, omega_ev  [n_freq] frequencies in eV, > 0.
 *   alpha_ib          [n_types][n_freq] complex interband polarisabilities
 *                     alpha^IB(w), a.u. (Eq. 8); required for PX_WFQFMU and
 *                     PX_WFQFMU_HETERO (per type: Eq. 10 forms each atom's value),
 *                     ignored (may be NULL) for PX_WFQ.
 *   n_pol, pol_dir    [n_pol][3] unit field directions.
 *   e0                field amplitude E0, a.u. (> 0; the response is linear).
 *   out               host result buffers (see px_result).
 *   cuda_stream       cudaStream_t to order the work on, or NULL for the
 *                     handle's own stream.  The call is synchronous.
 * Returns PX_OK, or PX_ENOTCONV when some column missed options.tol_rel within
 * the iteration caps (its status[] entry says so; its outputs hold the last
 * iterate), PX_EINVAL, PX_ENOMEM, PX_ECUDA, PX_ETIMEOUT. */
px_status px_solve(px_handle* h, int n_freq, const double* omega_ev, const double* alpha_ib,
                   int n_pol, const double* pol_dir, double e0, px_result* out,
                   void* cuda_stream);

/* Same computation, with the per-column results left in DEVICE memory owned by
 * the caller (for callers that keep results on the GPU, e.g. PyTorch tensors):
 *   d_alpha   device [F][3][P] complex (may be NULL)
 *   d_q       device [F][P][N] complex (may be NULL)
 *   d_mu      device [F][P][N][3] complex (may be NULL)
 *   d_relres  device [F][P] doubles (may be NULL)
 * Host-side inputs are as in px_solve.  Returns after the device work finished. */
px_status px_solve_device(px_handle* h, int n_freq, const double* omega_ev,
                          const double* alpha_ib, int n_pol, const double* pol_dir, double e0,
                          double* d_alpha, double* d_q, double* d_mu, double* d_relres,
                          void* cuda_stream);

/* No-allocation residual check.  The paper has no counterpart: this is a service for
 * callers that cannot allocate device memory at the point of the call (callers whose
 * memory pool -- a framework's caching allocator, another library's arena -- owns all
 * free device memory, and latency-bound loops that must not enter the driver's
 * allocator, which can synchronise the device).  It computes,
 * exactly as px_solve_device does for its own solution, the FP64 relative residual
 * ||b - A x|| / ||b|| of every (frequency, polarisation) column for a solution the
 * caller holds in device memory:
 *   d_q      device [F][P][N] complex charges (the layout px_solve_device writes)
 *   d_mu     device [F][P][N][3] complex dipoles (PX_WFQFMU; ignored for PX_WFQ)
 *   d_relres device [F][P] doubles, written
 * Host-side inputs are as in px_solve.  All work space comes from one fixed device
 * array of 32 MiB inside the library (held by every GPU that loads it until the
 * process exits); problems that need more return PX_EINVAL with the required size.
 * The call performs no device allocation.  Each call made outside a stream capture
 * looks up the array's address on the current device (cudaGetSymbolAddress); a call
 * under a capture reuses the address of that device's last uncaptured call, so make
 * the first call on a device before any stream capture (a captured first call returns
 * PX_ECUDA).  Inputs are validated as in px_solve.  Every call shares the array: calls that overlap
 * on the GPU (two host threads, or two streams) race.  The call is synchronous.
 * A structure must be loaded with px_set_structure (PX_WFQ or PX_WFQFMU; a
 * PX_WFQFMU_HETERO structure returns PX_ENOTIMPL). */
px_status px_relres_device_noalloc(px_handle* h, int n_freq, const double* omega_ev,
                                   const double* alpha_ib, int n_pol, const double* pol_dir,
                                   double e0, const double* d_q, const double* d_mu,
                                   double* d_relres, void* cuda_stream);

/* Induced density, potential and field maps (Sec. "Post-process Analysis") of solved
 * columns at probe points, for the loaded structure.  The model's charges and dipoles
 * are Gaussian densities (Secs. 2.1, 2.2): atom i carries q_i g(x; R_q,i) and
 * -mu_i . grad g(x; R_mu,i), g(x; R) = (pi R^2)^(-3/2) exp(-|x|^2/R^2), x = r - r_i, whose
 * potential is erf(|x|/R)/|x| (the kernel of Eq. 5).  For every column c and point m:
 *   rho = sum_i q_i g(x; R_q,i) + (2/R_mu,i^2)(mu_i . x) g(x; R_mu,i)
 *   phi = sum_i q_i G(x; R_q,i) - mu_i . grad G(x; R_mu,i),   G = erf(|x|/R)/|x|
 *   E   = -grad phi
 * (atomic units; points may sit on atom centres, where the limits are used).
 *   points_ang  host [n_points][3] probe points, Angstrom
 *   d_q         device [n_cols][N] complex charges, caller's atom order (the layout
 *               px_solve_device writes: n_cols = F P)
 *   d_mu        device [n_cols][N][3] complex dipoles (PX_WFQFMU), or NULL (no dipoles)
 *   d_rho, d_phi  device [n_cols][n_points] complex outputs, d_E device
 *               [n_cols][n_points][3] complex; each may be NULL (skipped)
 * Pair terms are evaluated in FP32 and accumulated in FP64 (relative error ~1e-5 of the
 * largest map value).  Synchronous; allocates the points' device copy for the call.
 * PX_EINVAL for NULL / non-finite inputs or d_mu with a PX_WFQ structure. */
px_status px_fields(px_handle* h, int n_points, const double* points_ang, int n_cols,
                    const double* d_q, const double* d_mu, double* d_rho, double* d_phi,
                    double* d_E, void* cuda_stream);

/* The frequency-independent dense system of the loaded structure, for callers that
 * factorise it themselves (e.g. a direct LU per frequency, the "inversion" solver of
 * Sec. "Solvers"): A0 = Kbar T (Eq. 1) or diag(Kbar, I_3N) T (Eq. 7), so that
 * A(w) = A0 - z_q(w) I (wFQ) or A0 - diag(z_q(w) I_N, z_mu(w) I_3N) (wFQFmu), and the
 * real right-hand sides b (-Kbar V; E) of the field directions.
 *   d_A0    device [n_u][ld_A0] doubles (row-major, ld_A0 >= n_u), or NULL
 *   d_b     device [n_u][n_pol] doubles, or NULL
 * Unknowns in the caller's atom order: charges 0..N-1, then the dipole components
 * N + 3 i + k (the order of px_result's q and mu).
 * Needs the materialised FP64 T (not PX_MODE_MATFREE); PX_ENOTIMPL for
 * PX_WFQFMU_HETERO (its conductance block depends on the frequency).  Allocates a
 * transient n_u^2 FP64 buffer.  Synchronous. */
px_status px_system_device(px_handle* h, int n_pol, const double* pol_dir, double e0,
                           double* d_A0, size_t ld_A0, double* d_b, void* cuda_stream);

/* Boundary-element formulations (Sec. 2.3). */
typedef enum {
  PX_BEM_DPCM = 0,    /* Eq. 11 */
  PX_BEM_IEFPCM = 1   /* Eq. 12 */
} px_bem_formulation;

/* Boundary-element surface of a dielectric or metal particle (Sec. 2.3): replaces any
 * loaded structure.  Tessera i has barycentre s_i, outward unit normal n_i and area A_i.
 * PX_BEM_DPCM solves the normal-field form of Eq. 11 for the surface charge densities,
 *   (Ft - Lambda(w) I) sigma = -E0 e . n,   Lambda(w) = 2 pi (e2 + e1)/(e2 - e1),
 *   Ft_ij = A_j (s_i - s_j).n_i / |s_i - s_j|^3 (i != j),  Ft_ii = +1.0694 sqrt(4 pi A_i)/(2R),
 * which is the printed equation read dimensionally (the area matrix on the diagonal term
 * dropped, F taken with the receiving tessera's normal).  PX_BEM_IEFPCM solves Eq. 12 for
 * the tesserae's charges q in two steps,
 *   (F + Lambda(w) I) y = -(2 pi I + F) V,   then   (S A^-1) q = y,
 *   F_ij = A_j (s_i - s_j).n_j / |s_i - s_j|^3 (i != j),  F_ii = -1.0694 sqrt(4 pi A_i)/(2R),
 *   (S A^-1)_ij = 1/|s_i - s_j| (i != j),  (S A^-1)_ii = 1.0694 sqrt(4 pi / A_i),
 *   V_i = -E0 e . s_i,
 * with the self term of F taken with the sign of the off-diagonal double-layer sum (with
 * the printed positive sign a refined sphere converges only slowly).  Both converge on a
 * sphere to the exact quasistatic polarisability R^3 (e2 - e1)/(e2 + 2 e1).  The operators
 * are dense and frequency-independent, built once in FP64 (plus the planes the selected
 * precision and solver read), and every frequency is a column shift, exactly as z_q(w) in
 * Eq. 1: PX_SOLVER_BATCHED and PX_SOLVER_SHIFTED both apply to DPCM and to IEFPCM's first
 * step; the second step (complex right-hand sides) runs batched.
 *   pos_ang      host [n_tess][3] barycentres, Angstrom
 *   normals      host [n_tess][3] outward unit normals
 *   area_ang2    host [n_tess] areas, Angstrom^2 (> 0)
 *   radius_ang   R of the self term: the radius of the sphere enclosing the mesh, Angstrom
 *   formulation  PX_BEM_DPCM or PX_BEM_IEFPCM
 * PX_EINVAL for NULL / non-finite inputs, non-unit normals, non-positive areas or R, or an
 * unknown formulation; PX_ENOTIMPL in PX_MODE_MATFREE; PX_ECUDA when the n_tess^2 operator
 * planes (two operators for IEFPCM) do not fit.  Tesserae keep the caller's order.
 * px_fields, px_system_device and px_relres_device_noalloc return PX_ENOTIMPL while a
 * mesh is loaded. */
px_status px_set_mesh(px_handle* h, int n_tess, const double* pos_ang, const double* normals,
                      const double* area_ang2, double radius_ang, int formulation);

/* Solve the loaded mesh (px_set_mesh) for F frequencies x P field directions.
 *   omega_ev  host [F] frequencies, eV (> 0; they enter sigma_abs only)
 *   eps       host [F][4] doubles: Re e2, Im e2, Re e1, Im e1 -- the particle's and the
 *             medium's permittivities at each frequency (finite, e2 != e1)
 * Everything else is as in px_solve: out->q holds the tesserae's charges (A_i sigma_i for
 * DPCM; there are no dipoles: out->mu is left untouched), out->alpha the dipole
 * sum_i q_i s_i / E0 (bohr^3), out->sigma_abs 4 pi w/(3c) Im Tr(alpha) for three
 * independent directions.  For IEFPCM rel_residual is the larger of the two steps'
 * relative residuals, iters their sum, and the statistics cover both steps.
 * PX_EINVAL when no mesh is loaded. */
px_status px_solve_bem(px_handle* h, int n_freq, const double* omega_ev, const double* eps,
                       int n_pol, const double* pol_dir, double e0, px_result* out,
                       void* cuda_stream);

/* Counters of the last px_solve / px_set_structure. */
px_status px_get_stats(const px_handle* h, px_stats* st);

/* Release all device memory and the stream.  NULL is accepted. */
px_status px_destroy(px_handle* h);

/* Message of the last failure on h (or of the last failed px_create when h is
 * NULL).  The string is owned by the library and valid until the next call on h. */
const char* px_last_error(const px_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* PX_H */
