// Internal declarations shared by the px CUDA translation units.
//
// Data layout in device memory (one structure, one block of B columns):
//   positions      pos64 [N][3] double (bohr)
//   per atom       Rq, Rmu, area [N] double; type [N] int
//   K (Eq. 3)      CSR of the off-diagonal bond weights: rowptr [N+1], col [nnz],
//                  val64 [nnz] double, val32 [nnz] float.  The Laplacian form of
//                  Eq. 2 is applied as (Kbar y)_i = sum_j K_ij (y_j - y_i), which is
//                  the same sum with the diagonal folded in (exact for constants).
//   T (Eq. 5 + derivatives)  row-major [np][np], np = n_u rounded up to 128, zero
//                  padded; T64 (double), T32 (float), Thi/Tlo (bf16 split).
//   columns        column c = f * P + p (frequency-major).  Work arrays hold only the
//                  B_act active columns, compacted, column index fastest.
//   complex data   double2 (re, im); the matvec operands X / Y are real matrices
//                  [np][ldx] whose columns 2a, 2a+1 are the re / im parts of column a.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>

#include "px.h"

namespace px {

constexpr int kTile = 128;   // padding granularity of T and of the matvec operands
constexpr int kMaxRestart = 400;  // largest Krylov basis per restart cycle

inline size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------- structure
struct DevStructure {
  int model = 0;      // 0 wFQ, 1 wFQFmu
  int N = 0;          // atoms
  int nu = 0;         // unknowns
  int np = 0;         // padded unknowns (multiple of kTile)
  int ntypes = 0;
  int nnz = 0;
  double* pos64 = nullptr;
  double* Rq = nullptr;
  double* Rmu = nullptr;
  double* area = nullptr;
  int* type = nullptr;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* val64 = nullptr;
  float* val32 = nullptr;
  double* T64 = nullptr;
  float* T32 = nullptr;
  float* Tffh = nullptr;       // double-FP32 planes of T64 (true residual of the
  float* Tffl = nullptr;       //   low-precision modes): T = Tffh + Tffl
  float4* pos4f = nullptr;     // matrix-free: x, y, z, R_q^2 (FP32)
  double* pos4d = nullptr;     // matrix-free: [N][4] x, y, z, R_q^2 (FP64)
  float* rm2f = nullptr;       // matrix-free wFQFmu: R_mu^2 (FP32)
  double* rm2d = nullptr;      // matrix-free wFQFmu: R_mu^2 (FP64)
  float4* pos4tc = nullptr;    // matrix-free split (tensor-core pair kernel): positions and
                               //   R_q^2 scaled by 2^-op_scale_exp, padded to np
  float tc_wmax = 0.f;         //   the largest scaled R_q^2
  int mu_self = 0;             // Gaussian self term on the T^mumu diagonal (options at set-up)
  bool matfree = false;
  int* perm = nullptr;         // [N] caller's index of internal (Morton-sorted) atom i
  // tensor-core planes Thi / Tlo hold M = diag(Kbar, I) T (split-precision modes), fp16
  // parts scaled by 2^op_scale_exp; the FP64 T, the FP32 T and the double-FP32 planes
  // stay T
  bool op_has_kbar = false;
  int op_scale_exp = 12;
  uint16_t* Thi = nullptr;     // hi part of M: bf16, or fp16 of 2^e M (e = op_scale_exp)
  uint16_t* Tlo = nullptr;     // lo part of M: bf16, or fp16 of (2^e M - hi) 2^11
  bool t_f16 = false;          // the split planes are fp16 (else bf16)
  // heterogeneous wFQFmu (Eqs. 9-10; model stays 1): per-type Drude parameters and the
  // nearest-neighbour counts of Eq. 10
  bool hetero = false;
  double* tpar = nullptr;      // [ntypes][3] n, tau, area of each type
  int* nncnt = nullptr;        // [N][ntypes] nearest neighbours of each type (r <= s r0)
  int* ident = nullptr;        // [N] 0..N-1: per-atom indexing of the dipole shifts
  // boundary elements (Sec. 2.3): the "atoms" are tesserae; T holds the DPCM operator Ft
  bool bem = false;
  int bem_stage = 0;           // 0 DPCM; 1, 2 the two steps of IEFPCM (Eq. 12)
  double* nrm = nullptr;       // [N][3] outward normals
  double* tarea = nullptr;     // [N] tessera areas (bohr^2)
};

// ---------------------------------------------------------------- launch wrappers
// Every wrapper enqueues its kernels on `s` and adds the number of kernel
// launches to *nl.  They never synchronise.

// Structure staging: xyz_ang [N][3] (Angstrom), tidx [N] and types [ntypes] on the
// device, in the caller's order -> pos (bohr), type, Rq, Rmu, area in internal order
// and perm[i] = caller index of internal atom i.  sort: Morton order (needs
// stage_scratch_bytes(N) of scratch), else the caller's order (perm = identity).
size_t stage_scratch_bytes(int N);
cudaError_t launch_stage_atoms(const double* xyz_ang, const int* tidx, const px_atom_type* types,
                               int N, bool sort, void* scratch, size_t scratch_bytes, int* perm,
                               double* pos, int* type, double* Rq, double* Rmu, double* area,
                               cudaStream_t s, long long* nl);

// Neighbour list + CSR of K.  rcut2 / r0 / dd / ss are [ntypes][ntypes] pair tables.
cudaError_t launch_neigh_count(const double* pos, int N, const int* type, int ntypes,
                               const double* rcut2, int* counts, cudaStream_t s, long long* nl);
cudaError_t launch_scan(const int* counts, int N, int* rowptr, cudaStream_t s, long long* nl);
cudaError_t launch_neigh_fill(const double* pos, int N, const int* type, int ntypes,
                              const double* rcut2, const double* r0, const double* dd,
                              const double* ss, const double* area, const int* rowptr,
                              int* col, double* val64, float* val32, cudaStream_t s,
                              long long* nl);
// Dense T in FP64 (Eq. 5; wFQFmu adds the 4x4 blocks of Sec. 2.2).
cudaError_t launch_build_T64(const DevStructure& d, int mu_self_term, cudaStream_t s,
                             long long* nl);
// T32 = float(T64) (the FP32 CUDA-core matvec's operator).
cudaError_t launch_convert_T(const DevStructure& d, cudaStream_t s, long long* nl);
// M = diag(Kbar, I) T in FP64 (charge rows: M_ik = sum_j K_ij (T_jk - T_ik), Eq. 2 applied
// to T; dipole and padding rows copy T), and *absmax_bits = bits of max |M| (a
// non-negative double, so its bit pattern orders like its value; zero it first).
cudaError_t launch_build_M64(const DevStructure& d, double* M64,
                             unsigned long long* absmax_bits, cudaStream_t s, long long* nl);
// Operator M [np][np] (internal order) -> A [nu][lda] in the caller's atom order, and
// right-hand sides b [nu][P] (internal) -> bout [nu][P] (caller's order); either may be null.
cudaError_t launch_unpermute_system(const double* M, int np, int nu, int N, const int* perm,
                                    double* A, size_t lda, const double* b, int P, double* bout,
                                    cudaStream_t s, long long* nl);
// Thi / Tlo split of an FP64 operator A [np][np]: bf16 hi/lo, or (f16) fp16 hi of
// 2^scale_exp A and fp16 lo of the remainder times 2^11.
cudaError_t launch_split_op(const double* A, size_t n, uint16_t* hi, uint16_t* lo, bool f16,
                            int scale_exp, cudaStream_t s, long long* nl);

// Matvec Y[np][ldy] = T[np][np] X[np][ldx], columns ncols (multiple of kTile).
cudaError_t launch_sgemm(const float* T, int np, const float* X, int ldx, float* Y, int ldy,
                         int ncols, cudaStream_t s, long long* nl);
cudaError_t launch_dgemm(const double* T, int np, const double* X, int ldx, double* Y, int ldy,
                         int ncols, cudaStream_t s, long long* nl);
// The same product with K split over blocks when the output has fewer than ~2 waves
// of tiles (small N): partial products in part [nz][np][ncols] (part_elems doubles;
// nz = dgemm_splits(np, ncols)), summed in a fixed order into Y.  Falls back to
// launch_dgemm when nz == 1 or part is too small.
int dgemm_splits(int np, int ncols);
cudaError_t launch_dgemm_splitk(const double* T, int np, const double* X, int ldx, double* Y,
                                int ldy, int ncols, double* part, size_t part_elems, cudaStream_t s,
                                long long* nl);
// FP64-class matvec Y = (Th + Tl)(Xh + Xl) in double-FP32 arithmetic (FP64 result);
// np % 64 == 0, ncols % 64 == 0.
cudaError_t launch_ffgemm(const float* Th, const float* Tl, int np, const float* Xh,
                          const float* Xl, int ldx, double* Y, int ldy, int ncols, cudaStream_t s,
                          long long* nl);
// Xh = fl32(X), Xl = fl32(X - Xh) over n FP64 values.
cudaError_t launch_split_ff(const double* X, size_t n, float* Xh, float* Xl, cudaStream_t s,
                            long long* nl);
// Matrix-free matvecs: T generated from the staged positions (wFQ, Eq. 5).
cudaError_t launch_sgemm_mf(const float4* pos, int n, int np, const float* X, int ldx, float* Y,
                            int ldy, int ncols, cudaStream_t s, long long* nl);
// FP64-class on-the-fly wFQ matvec for the true residual: T in FP64 per pair, the
// contraction in double-FP32 with the operand as FP32 hi / lo planes [np][ldx].
cudaError_t launch_ffgemm_mf(const double* pos4, int n, int np, const float* Xh, const float* Xl,
                             int ldx, double* Y, int ldy, int ncols, cudaStream_t s, long long* nl);
cudaError_t launch_dgemm_mf(const double* pos4, int n, int np, const double* X, int ldx,
                            double* Y, int ldy, int ncols, cudaStream_t s, long long* nl);
// wFQFmu matrix-free matvecs: the 4 x 4 blocks of T (Sec. 2.2) generated per atom pair;
// rows in the charges-first order of the unknowns; unknown rows of Y beyond 4N untouched.
cudaError_t launch_sgemm_mf4(const float4* pos, const float* rm2, int N, int mu_self,
                             const float* X, int ldx, float* Y, int ldy, int ncols, cudaStream_t s,
                             long long* nl);
cudaError_t launch_dgemm_mf4(const double* pos4, const double* rm2, int N, int mu_self,
                             const double* X, int ldx, double* Y, int ldy, int ncols,
                             cudaStream_t s, long long* nl);
// pos4f / pos4d (and rm2f / rm2d when set) of a structure from pos64, R_q and R_mu.
cudaError_t launch_stage_pos4(const DevStructure& d, cudaStream_t s, long long* nl);
// FP64 matvec for nc <= 8 real operand columns (bandwidth/FP64-pipe bound GEMV).
cudaError_t launch_dgemv(const double* T, int np, const double* X, int ldx, double* Y, int ldy,
                         int nc, cudaStream_t s, long long* nl);
// Tensor-core split-precision matvec Y = T X from hi/lo 16-bit parts of T and X
// (bf16, or scaled fp16 when f16).  Xh / Xl are the transposed operand [ncols][np]
// (K-major); np % 128 == 0, ncols % 128 == 0.  *err is set to 1 if a pipeline wait
// ran out of time.  variant: 0 = 128 x 256 tiles (2-stage ring; only when ncols % 256
// == 0, else variant 1 runs), 1 = 128 x 128 tiles (3-stage ring), -1 = autotuned: the
// first call of a (np, ncols, f16) shape times every variant that fits on its operands
// (synchronising the stream once) and caches the fastest.  *used (may be NULL) receives
// the variant launched.
cudaError_t launch_tc_gemm(const uint16_t* Th, const uint16_t* Tl, int np, const uint16_t* Xh,
                           const uint16_t* Xl, int ncols, float* Y, int ldy, bool f16, int* err,
                           cudaStream_t s, long long* nl, int variant, int* used);
// The autotuner's cached variant for a shape on the current device, or -1.
int tc_tuned_variant(int np, int ncols, bool f16);
// Matrix-free wFQ block matvec Y = T X on the tensor cores: T^qq tiles generated from the
// scaled, padded positions of launch_tc_mf_positions (wmax: their largest R_q^2) into shared
// memory as split planes and contracted with the split operand (Xh / Xl as for
// launch_tc_gemm).  f16: the tiles hold 2^scale_exp T (2^scale_exp max|T| <= 2^14; bf16:
// scale_exp = 0); Y is returned unscaled.  128 x 256 or 128 x 128 tiles (only 128 when
// ncols % 256 != 0; else the faster of the two for the shape, timed on its first call
// outside a stream capture).  *err as for launch_tc_gemm.
cudaError_t launch_tc_mf(const float4* pos, int np, float wmax, const uint16_t* Xh,
                         const uint16_t* Xl, int ncols, float* Y, int ldy, bool f16, int scale_exp,
                         int* err, cudaStream_t s, long long* nl);
// Matrix-free wFQFmu block matvec Y = T X on the tensor cores (Sec. 2.2): the 4 x 4 blocks
// of T^qq / T^qmu / T^muq / T^mumu generated from the positions of launch_tc_mf4_positions
// into shared memory as split planes (f16: 2^scale_exp T, 2^scale_exp max|T| <= 2^14; bf16:
// scale_exp unused), contracted with the atom-blocked split operand of launch_split_xt_mu;
// Y (charges-first rows, unscaled) is written for the rows of the N real atoms only.
// mu_self: the Gaussian dipole self term on the T^mumu diagonal.  Tile widths and *err as
// for launch_tc_mf; np % 128 == 0, N <= np / 4.
cudaError_t launch_tc_mf4(const float4* pos, int np, int N, int mu_self, const uint16_t* Xh,
                          const uint16_t* Xl, int ncols, float* Y, int ldy, bool f16, int scale_exp,
                          int* err, cudaStream_t s, long long* nl);
// The pair kernel's tile width chosen for a shape on the current device (256 or 128), or -1
// before the first uncaptured call of that shape (which times both widths); mu: wFQFmu.
int tc_mf_tuned_width(int np, int ncols, bool f16, bool mu = false);
// Its positions: pos (bohr) and Rq in internal order -> out (np / 2 atom pairs of 8 floats,
// [-x0 -x1 -y0 -y1 -z0 -z1 w0 w1], w = R_q^2) scaled by 2^-scale_exp (w by 2^-2 scale_exp),
// atoms n .. np-1 distinct far-away dummies.
cudaError_t launch_tc_mf_positions(const double* pos, const double* Rq, int n, int np,
                                   int scale_exp, float4* out, cudaStream_t s, long long* nl);
// wFQFmu positions: pos (bohr), Rq, Rmu in internal order -> out[2 a] = (x, y, z, R_q^2),
// out[2 a + 1] = (R_mu^2, 0, 0, 0) for the np / 4 atoms of the padded tiles (atoms n and
// beyond distinct far-away dummies).
cudaError_t launch_tc_mf4_positions(const double* pos, const double* Rq, const double* Rmu, int n,
                                    int np, float4* out, cudaStream_t s, long long* nl);
// Xh[c][k], Xl[c][k] from X[k][c] (k < np, c < ncols): bf16 hi/lo, or fp16 hi/lo of 2^8 X.
cudaError_t launch_split_xt(const float* X, int ldx, int np, int ncols, uint16_t* Xh,
                            uint16_t* Xl, bool f16, cudaStream_t s, long long* nl);
// The same split of a wFQFmu operand (charges-first rows of N atoms) into the atom-blocked K
// order of launch_tc_mf4: K index 64 g + w is the charge of atom 16 g + w (w < 16), else
// dipole component (w - 16) % 3 of atom 16 g + (w - 16) / 3; 0 beyond atom N.
cudaError_t launch_split_xt_mu(const float* X, int ldx, int np, int ncols, int N, uint16_t* Xh,
                               uint16_t* Xl, bool f16, cudaStream_t s, long long* nl);

// ---------------------------------------------------------------- Krylov workspace
// The Krylov basis V and the work vector W hold complex numbers in one of three
// element types (kBasis*): FP64 (double2); double-FP32 (float4 = re_hi, im_hi, re_lo,
// im_lo: value = hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits, whose
// arithmetic runs on the FP32 pipe with error-free transformations -- GB300's FP64
// pipe is 1/64 of its FP32 rate); or FP32 (float2, half the bytes of the other two,
// for low-precision inner iterations whose refinement rounds each need only a modest
// residual reduction).  The Gram-Schmidt sweeps are bound by HBM bandwidth, so the
// element size sets their cost.
constexpr int kBasisF64 = 0, kBasisFF = 1, kBasisF32 = 2;
inline size_t basis_bytes(int basis) { return basis == kBasisF32 ? 8 : 16; }
// Element type for the options' precision and px_basis choice (validated): FP64 solves
// keep an FP64 basis; low-precision solves default to FP32.
inline int basis_kind(int precision, int basis) {
  if (precision == PX_FP64 || basis == PX_BASIS_FP64) return kBasisF64;
  if (basis == PX_BASIS_FF32) return kBasisFF;
  return kBasisF32;   // PX_BASIS_FP32 or automatic
}

struct KrylovArgs {
  int nu, Bact, m, nblk;
  int basis;           // kBasisF64 (double2), kBasisFF (float4) or kBasisF32 (float2)
  void* V;             // [m+1][nu][Bact]
  void* W;             // [nu][Bact]
  double2* h;          // [2][m+1][Bact] projections of each Gram-Schmidt pass
  double2* part;       // [nblk][m+1][Bact] per-row-block partial projections
  double* normpart;    // [nblk][Bact] per-row-block partial |W|^2
  double2* R;          // [m][m+1][Bact] rotated Hessenberg columns (column-major by step)
  double2* g;          // [m+1][Bact] rotated right-hand side
  double* cs;          // [m][Bact] Givens cosines
  double2* sn;         // [m][Bact] Givens sines
  double* target;      // [Bact] absolute residual at which a column stops this cycle
  int* jconv;          // [Bact] basis size used (0 while the column still iterates)
  double* inv_h;       // [Bact] scale of the next basis vector (0 after the column stopped)
  int* active_count;   // [m] columns still iterating after step j
  double2* y;          // [m][Bact] least-squares solution
  double2* u;          // [m+1][Bact] coefficients of the implicit residual V u
  // wFQFmu right preconditioner M = diag(I_N, alpha^IB I_3N) (mu = alpha^IB nu): the
  // Krylov space is built for A M; operands of dipole rows are scaled by alpha^IB and
  // the solution update is M V y.  amu = nullptr disables it (wFQ).
  int N;               // atoms (dipole rows start at N)
  const int* type;     // [N] atom types
  const double2* amu;  // [ntypes][Bact] alpha^IB = -1 / z_mu of each active column
  // Step index: kernels take j as an argument, or, when jdev is set (a restart cycle
  // captured as one graph with a device-side loop), read it from *jdev.
  const int* jdev;
};

// Conductance + shift apply of one Krylov step (Eq. 1 / Eq. 7 on a block):
//   W[i][a] = (Kbar Y)_i - z_q X[i][a]         charge rows (i < N)
//   W[i][a] = Y_i - z_mu(type) X[i][a]         dipole rows (wFQFmu)
// with X = V_j and Y = T X from the matvec ([np][ldy] real, re/im in columns 2a, 2a+1).
// When the matvec applied M = diag(Kbar, I) T instead (kbar_in_y), every row is
// W = yscale Y - z X (yscale undoes a power-of-two operator scaling).
struct ShiftArgs {
  int nu, N, model, Bact, nblk, basis;
  const int* rowptr; const int* col; const double* val64; const float* val32;
  const int* type;
  const void* Y; int ldy; bool y_is_f32;
  const void* X;                                // V_j (basis element type), stride Bact
  const double2* zq;                            // [Bact]
  const double2* zmu;                           // [ntypes][Bact] (wFQFmu)
  const int* jconv;                             // columns with jconv > 0 are skipped
  int precond_mu;                               // 1: dipole rows use the right preconditioner
  void* W;
  const int* jdev;                              // set: X is V_0 and the step is *jdev
  int kbar_in_y;                                // 1: Y = M X already holds Kbar T X
  float yscale;                                 // power of two applied to Y (kbar_in_y)
  // heterogeneous wFQFmu (Eq. 9): charge rows use z_q of their atom's type (zq [ntypes][Bact]
  // indexed by qtype) and the complex bond weights K_ij kappa[t_i][t_j][col] of
  // 1/2 (Kbar + Hbar(w)); null for the homogeneous models
  const int* qtype; int ntypes; const double2* kappa;
};
cudaError_t launch_shift(const ShiftArgs& a, cudaStream_t s, long long* nl);

// FP64 true residual of the active columns: R[i][act[a]] = b[i][pol] - (A x)[i] with
// (A x) from Y = T64 x (FP64), plus per-row-block partial |R|^2 in normpart.
struct ResidArgs {
  int nu, N, model, Bact, P, B, nblk;
  const int* rowptr; const int* col; const double* val64; const int* type;
  const double* Y; int ldy;
  const double2* x; const int* act; const double* b;
  const double2* zq; const double2* zmu;
  double2* R; double* normpart;
  // heterogeneous wFQFmu: as in ShiftArgs, plus the complex right-hand side of every
  // column bc [nu][B] (replaces b)
  const int* qtype; int ntypes; const double2* kappa; const double2* bc;
  int op_full;   // boundary elements: Y already holds the whole operator; every row w = Y - z x
};
cudaError_t launch_resid(const ResidArgs& a, cudaStream_t s, long long* nl);

// ---- boundary elements (Sec. 2.3; Eq. 11 in the normal-field DPCM form, Eq. 12)
// Operators [np][np] (zero padded) of a mesh: pos, nrm [n][3] (bohr, unit), area [n]
// (bohr^2), R the radius of the enclosing sphere.  Stored transposed (S[j][i] = Op[i][j]);
// ief selects Eq. 12's F instead of Eq. 11's Ft.
cudaError_t launch_build_F(const double* pos, const double* nrm, const double* area, double R,
                           int n, int np, bool ief, double* S, cudaStream_t s, long long* nl);
// S A^-1 of Eq. 12 (symmetric)
cudaError_t launch_build_G(const double* pos, const double* area, int n, int np, double* G,
                           cudaStream_t s, long long* nl);
// M = S^T and max |M| (bits of the double, atomicMax)
cudaError_t launch_transpose_absmax(const double* S, int np, double* M,
                                    unsigned long long* absmax_bits, cudaStream_t s, long long* nl);
// zq[c] = Lambda(w_f) = 2 pi (e2 + e1)/(e2 - e1) from eps [F][4] = (Re e2, Im e2, Re e1, Im e1),
// and b[i][p] = -e0 e_p . n_i: the system (Ft - Lambda I) sigma = -E . n.
// stage 0: DPCM (z = Lambda, b = -E0 e . n); 1: first IEFPCM step (z = -Lambda, b = c from
// the transposed operator S); 2: second IEFPCM step (z = 0, b unused)
cudaError_t launch_bem_setup(int F, int P, int n, int np, int stage, const double* eps,
                             const double* nrm, const double* S, const double* pos,
                             const double* pol, double e0, double2* zq, double* b, cudaStream_t s,
                             long long* nl);

// ---- heterogeneous wFQFmu (Eqs. 9-10)
// nn[i][t] = atoms of type t within the Fermi midpoint s_ij r0_ij of atom i (Eq. 10's
// nearest neighbours), from the CSR rows and positions; ident[i] = i.
cudaError_t launch_nn_counts(const double* pos, int N, const int* type, int ntypes,
                             const double* r0t, const double* st, const int* rowptr,
                             const int* col, int* nn, int* ident, cudaStream_t s, long long* nl);
// Per-column tables: zq[t][c] = z_q of type t (Eq. 6 with the type's n, tau),
// kappa[t][u][c] = 1/2 (1 + rho_tu(w) A_u / A_t) with rho_tu = (n_u tau_u)/(n_t tau_t)
// (1 - i w tau_t)/(1 - i w tau_u) (the weight of bond t -> u in 1/2 (Kbar + Hbar), Eq. 9),
// zmu_atom[i][c] = z_mu of atom i: the Eq. 10 weighted mean of the types' z_mu[t][c]
// (weights nn[i][t] + [t == type_i]).  tpar [ntypes][3] = n, tau, area.
cudaError_t launch_hetero_tables(int F, int P, int ntypes, int N, const double* omega_ev,
                                 const double* tpar, const int* type, const int* nn,
                                 const double2* zmu_type, double2* zq, double2* kappa,
                                 double2* zmu_atom, cudaStream_t s, long long* nl);
// Complex right-hand side of Eq. 9 per column, bc[i][c] = (diag(C(w), I) (-V; E))_i, and
// per-column norms bn[c].
cudaError_t launch_rhs_hetero(int N, int F, int P, const int* rowptr, const int* col,
                              const double* val64, const int* type, int ntypes,
                              const double2* kappa, const double* pos, const double* pol,
                              double e0, double2* bc, double* bn, cudaStream_t s, long long* nl);
// out[t][a] = in[t][act[a]] for t < rows
cudaError_t launch_gather_rows(const double2* in, int rows, int B, const int* act, int Bact,
                               double2* out, cudaStream_t s, long long* nl);

// RHS b[i][p] (real): -Kbar V for charge rows, E0 e_p for dipole rows.
cudaError_t launch_rhs(int nu, int N, int model, const int* rowptr, const int* col,
                       const double* val64, const double* pos, const double* pol, int P,
                       double e0, double* b, cudaStream_t s, long long* nl);

// ---------------------------------------------------------------- Arnoldi
cudaError_t launch_dots(const KrylovArgs& a, int j, int pass, cudaStream_t s, long long* nl);
cudaError_t launch_update(const KrylovArgs& a, int j, int pass, bool last, cudaStream_t s,
                          long long* nl);
// End of a Krylov step inside a captured cycle: ++*jdev and set the while-loop
// condition to (another step fits in m) && (some column still iterates).
cudaError_t launch_step_advance(int* jdev, const int* active_count, int m,
                                cudaGraphConditionalHandle loop, cudaStream_t s, long long* nl);
cudaError_t launch_givens(const KrylovArgs& a, int j, int passes, cudaStream_t s,
                          long long* nl);
// V[j+1] = W * inv_h; also writes the matvec operand of V[j+1] (X32 hi parts, or X64).
cudaError_t launch_normalize(const KrylovArgs& a, int j, float* X32, double* X64, int ldx,
                             cudaStream_t s, long long* nl);
// Cycle start: g_0 = beta[act[a]], target[a] = target_all[act[a]], freeze flags, and
// V[0][i][a] = r[i][act[a]] / beta[act[a]] with its matvec operand.
cudaError_t launch_cycle_start(const KrylovArgs& a, const int* act, const double2* r, int B,
                               const double* beta, const double* target_all, float* X32,
                               double* X64, int ldx, cudaStream_t s, long long* nl);
// Cycle end: y = R^-1 g, u = Omega^H (0..0, gamma) per column; x[., act[a]] += V y,
// r[., act[a]] = V u (the residual of the inner iteration; r must not be NULL),
// beta[act[a]] = ||V u|| (measured, not |gamma|, so a basis that lost orthogonality
// cannot mis-scale the next cycle), iters[act[a]] += basis size used.
cudaError_t launch_cycle_end(const KrylovArgs& a, int jend, const int* act, double2* x,
                             double2* r, int B, double* beta, int* iters, cudaStream_t s,
                             long long* nl);
// rnorm[act[a]] = sqrt(sum_blk normpart[blk][a]); beta[act[a]] = rnorm[act[a]];
// target_all[act[a]] = max(inner_tol * rnorm, tol_abs_frac * ||b_p||).
cudaError_t launch_norm_finish(const double* normpart, int nblk, int Bact, const int* act,
                               int P, const double* bnorm, double inner_tol, double tol_abs_frac,
                               double* rnorm, double* beta, double* target_all, cudaStream_t s,
                               long long* nl);
// Gather x[., act[a]] into the f64 matvec operand.
cudaError_t launch_gather_x(const double2* x, int B, const int* act, int Bact, int nu,
                            double* X64, int ldx, cudaStream_t s, long long* nl);

// Per-column shifts z_q(w) = -w (w tau + i) / (2 n tau) (Eq. 6) and, per atom type,
// z_mu(w) = -1 / alpha^IB(w) (Eq. 8); omega in eV, alpha_ib [ntypes][F] complex.
cudaError_t launch_shifts(int F, int P, int ntypes, int model, const double* omega_ev,
                          const double* alpha_ib, double n, double tau, double2* zq,
                          double2* zmu, cudaStream_t s, long long* nl);
// zq_act[a] = zq[act[a]], zmu_act[t][a] = zmu[t][act[a]], and (when amu_act is not null)
// amu_act[t][a] = -1 / zmu_act[t][a] = alpha^IB.
cudaError_t launch_gather_shifts(const double2* zq, const double2* zmu, int ntypes, int B,
                                 const int* act, int Bact, double2* zq_act, double2* zmu_act,
                                 double2* amu_act, cudaStream_t s, long long* nl);
// bnorm[p] = ||b[., p]||_2
// ||bc_c|| of complex right-hand sides bc [nu][B]
cudaError_t launch_col_norms_c(const double2* bc, int nu, int B, double* bn, cudaStream_t s,
                               long long* nl);
cudaError_t launch_col_norms(const double* b, int nu, int P, double* bnorm, cudaStream_t s,
                             long long* nl);
// x = 0: r[i][c] = b[i][c % P], rnorm[c] = beta[c] = bnorm[c % P],
// target_all[c] = max(inner_tol * rnorm[c], tol_abs_frac * bnorm[c % P]).
cudaError_t launch_init_residual(const double* b, int nu, int P, int B, const double* bnorm,
                                 double inner_tol, double tol_abs_frac, double2* r,
                                 double* rnorm, double* beta, double* target_all, cudaStream_t s,
                                 long long* nl);
// The same from a per-column complex right-hand side bc [nu][B] with norms bn [B].
cudaError_t launch_init_residual_c(const double2* bc, int nu, int B, const double* bn,
                                   double inner_tol, double tol_abs_frac, double2* r,
                                   double* rnorm, double* beta, double* target_all, cudaStream_t s,
                                   long long* nl);
// bn[c] = bnorm[c % P]: per-column right-hand-side norms of the real right-hand sides.
cudaError_t launch_bnorm_cols(const double* bnorm, int P, int B, double* bn, cudaStream_t s,
                              long long* nl);
cudaError_t launch_relres(const double* rnorm, const double* bnorm, int B, int P, double* out,
                          cudaStream_t s, long long* nl);

// ---------------------------------------------------------------- observables
// alpha[f][k][p] = (sum_i q_i r_ik + sum_i mu_ik) / e0 (Sec. "Observables");
// sigma_pol[f][p] = 4 pi w / c Im(e_p . alpha e_p); sigma[f] = 4 pi w/(3c) Tr Im alpha_full
// (written when P == 3 and pol_inv, the host-side row-major inverse of the 3 x 3 matrix whose
// columns are the field directions, is given); q / mu copied out as [F][P][N] / [F][P][N][3].
cudaError_t launch_observables(int N, int model, int F, int P, const double* pos,
                               const int* perm, const double2* x, double e0, const double* omega_ev,
                               const double* pol, double2* alpha, double2* qout, double2* muout,
                               double* sigma_pol, double* sigma, const double* pol_inv,
                               const double* weight, cudaStream_t s, long long* nl);
// Row-major inverse of E = [e_0 e_1 e_2] (columns = the three field directions pol[3][3]);
// false when the directions are not linearly independent (|det E| < 1e-6).
bool pol_triple_inverse(const double* pol, double* inv);

int reduction_blocks(int nu);

// ---------------------------------------------------------------- shifted Krylov (wFQ)
// One real Arnoldi process of A0 = Kbar T per field direction serves every frequency
// (Eq. 1: the shift z_q(w) I is scalar, the right-hand side does not depend on w).  A
// group holds NP <= 4 directions p0 .. p0+NP-1, i.e. the Bg = F NP systems s = f NP + pl
// (global column c = f P + p0 + pl).  Everything in double-FP32; layouts in k_shifted.cu.
struct SkMatvecPlan {
  int grid = 0;      // persistent blocks (2 per SM)
  int S = 1;         // column segments; partial products part [S][np][NP]
  int seg_cols = 128;
  int St = 1;        // transposed operator: row segments, partials part [St][np][NP]
  int seg_rows = 32;
  int parts() const { return S > St ? S : St; }
};
SkMatvecPlan sk_matvec_plan(int np);
struct SkGroup {
  int n = 0, NP = 0, P = 0, p0 = 0, Bg = 0, m = 0;   // m: largest basis (Krylov steps)
  int np = 0;                 // n rounded up to 128
  float* vp = nullptr;        // [2 NP][np] the current basis vector, planar hi / lo (matvec operand)
  double* H = nullptr;        // [m][m+2][NP] Hessenberg columns
  double* inv_h = nullptr;    // [NP] scale of the next basis vector (0: invariant subspace)
  const double2* zq = nullptr;  // [B] z_q of every global column
  double* cs = nullptr;       // [m][Bg]
  double2* sn = nullptr;      // [m][Bg]
  double2* g = nullptr;       // [m+1][Bg]
  double2* R = nullptr;       // [Bg][rstride] rotated triangular factors, packed by columns
  size_t rstride = 0;         // m (m+1) / 2
  double* target = nullptr;   // [Bg] absolute least-squares residual that stops a system
  int* jconv = nullptr;       // [Bg] 0 iterating, > 0 basis size at stop, -1 zero rhs
  int* active = nullptr;      // [m] systems still iterating after step j
};
// U = T v in double-FP32 (T = Th + Tl planes [np][np]; v as planar hi / lo rows vp [2 NP][np],
// zero beyond n; U [n][NP] float2), via partial products over column segments
// (part [S][np][NP]).  trans: the planes hold T transposed (U = planes^T v, partial products
// over row segments, part [St][np][NP]).
cudaError_t launch_sk_matvec(const float* Th, const float* Tl, int n, int np, int NP,
                             const SkMatvecPlan& pl, bool trans, const float* vp, float2* part,
                             float2* U, cudaStream_t s, long long* nl);
// W = Kbar U (Eq. 2), double-FP32 arithmetic (K = val64 split as val32 + remainder).
cudaError_t launch_sk_kbar(int n, int NP, const int* rowptr, const int* col, const double* val,
                           const float* val32, const float2* U, float2* W, cudaStream_t s,
                           long long* nl);
int sk_row_blocks(int n);        // row blocks of the projection kernel (dpart rows)
int sk_update_chunks(int m);     // basis-vector chunks of the update kernel (upart rows)
// One classical Gram-Schmidt pass against V_0..V_j: h = V^T W (dpart [nrb][m1][NP] partials,
// h [m1][NP]), W -= V h (upart [chunks][n][NP] partials); `last` adds |W|^2 partials npart
// [(n+255)/256][NP].
cudaError_t launch_sk_gs_pass(const float2* V, float2* W, int n, int NP, int j, int m1,
                              double* dpart, double* h, float2* upart, bool last, double* npart,
                              cudaStream_t s, long long* nl);
// Hessenberg column j (from the passes' projections h [passes][m+1][NP] and npart), the
// per-shift Givens step with its stop test, and V_{j+1} = W / h_{j+1,j}.
cudaError_t launch_sk_step_end(const SkGroup& G, int j, const double* h, int passes,
                               const double* npart, float2* V, const float2* W, cudaStream_t s,
                               long long* nl);
// V_0 = b_p / ||b_p||, g_0, targets (tol_abs_frac ||b_p||) and stop flags of the group.
cudaError_t launch_sk_start(const SkGroup& G, const double* b, const double* bnorm,
                            double tol_abs_frac, float2* V, cudaStream_t s, long long* nl);
// y = R^-1 g per system (y [jend][Bg]), x[., c] = V y and (T x)[., c] = U y into the
// residual operand layout Y [np][ldy] (columns 2c, 2c+1), iters[c] += basis size.
cudaError_t launch_sk_solution(const SkGroup& G, int jend, const float2* V, const float2* U,
                               double2* y, double2* x, int B, double* Y, int ldy, int* iters,
                               cudaStream_t s, long long* nl);

// Inner-iteration target of one refinement round: the requested reduction
// inner_tol * ||r||, but never below the floor (a fraction of tol * ||b||).  Each
// round contracts the true residual by about max(inner_tol, eps_op * kappa) with
// eps_op the relative error of the low-precision operator, so a deeper inner solve
// than that buys nothing.
__host__ __device__ inline double round_target(double reduce_to, double floor_abs) {
  return reduce_to > floor_abs ? reduce_to : floor_abs;
}

}  // namespace px
