// Per-column bookkeeping kernels: frequency shifts (Eq. 6, Eq. 8), right-hand-side
// norms, the x = 0 initial residual, relative residuals and the observables of
// Sec. "Observables" (dipole, polarisability, absorption cross-section).
#include "px_internal.cuh"

#include <cmath>

namespace px {

namespace {

// One block per column c = f * P + p: dipole, polarisability and per-polarisation
// absorption (Sec. "Observables").
__global__ void k_observables(int N, int model, int F, int P, const double* __restrict__ pos,
                              const int* __restrict__ perm, const double2* __restrict__ x, double e0,
                              const double* __restrict__ omega_ev, const double* __restrict__ pol,
                              double2* alpha, double2* qout, double2* muout, double* sigma_pol,
                              const double* __restrict__ weight) {
  const int c = blockIdx.x;
  const int B = F * P;
  const int f = c / P, p = c % P;
  double d[6] = {0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double2 q = x[(size_t)i * B + c];
    if (weight) {   // boundary elements: the tessera's charge A_i sigma_i
      q.x *= weight[i];
      q.y *= weight[i];
    }
    for (int k = 0; k < 3; ++k) {
      d[2 * k] += q.x * pos[3 * i + k];
      d[2 * k + 1] += q.y * pos[3 * i + k];
    }
    const int io = perm[i];   // per-atom outputs in the caller's atom order
    if (qout) qout[(size_t)c * N + io] = q;
    if (model == 1) {
      for (int k = 0; k < 3; ++k) {
        double2 mu = x[(size_t)(N + 3 * i + k) * B + c];
        d[2 * k] += mu.x;
        d[2 * k + 1] += mu.y;
        if (muout) muout[((size_t)c * N + io) * 3 + k] = mu;
      }
    }
  }
  __shared__ double sh[6][256];
  for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] = d[k];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
      for (int k = 0; k < 6; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double im = 0.0;
    for (int k = 0; k < 3; ++k) {
      double2 a = make_double2(sh[2 * k][0] / e0, sh[2 * k + 1][0] / e0);
      if (alpha) alpha[((size_t)f * 3 + k) * P + p] = a;
      im += pol[3 * p + k] * a.y;
    }
    const double w = omega_ev[f] / 27.211386245988;
    const double c_au = 137.035999084;
    if (sigma_pol) sigma_pol[(size_t)f * P + p] = 4.0 * 3.141592653589793 * w / c_au * im;
  }
}

// sigma[f] = 4 pi w / (3c) Tr Im alpha_full (Sec. "Observables").  The solve measures
// A = alpha_full E column by column (E = [e_1 e_2 e_3], one column per field direction),
// so alpha_full = A E^-1 and Tr alpha_full = sum_kp A_kp (E^-1)_pk for any three linearly
// independent directions; einv holds E^-1 row-major.
struct Mat3 { double m[9]; };
__global__ void k_sigma_total(int F, const double2* alpha, const double* omega_ev, Mat3 einv,
                              double* sigma) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  double t = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int p = 0; p < 3; ++p) t += alpha[((size_t)f * 3 + k) * 3 + p].y * einv.m[p * 3 + k];
  const double w = omega_ev[f] / 27.211386245988;
  sigma[f] = 4.0 * 3.141592653589793 * w / (3.0 * 137.035999084) * t;
}

__global__ void k_shifts(int F, int P, int ntypes, int model, const double* omega_ev,
                         const double* alpha_ib, double n, double tau, double2* zq, double2* zmu) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int B = F * P;
  if (c >= B) return;
  int f = c / P;
  double w = omega_ev[f] / 27.211386245988;
  // z_q = -w (w tau + i) / (2 n tau)
  double den = 2.0 * n * tau;
  zq[c] = make_double2(-w * w * tau / den, -w / den);
  if (model == 1) {
    for (int t = 0; t < ntypes; ++t) {
      double ar = alpha_ib[2 * ((size_t)t * F + f)], ai = alpha_ib[2 * ((size_t)t * F + f) + 1];
      double m2 = ar * ar + ai * ai;
      // -1 / (ar + i ai) = (-ar + i ai) / |a|^2
      zmu[(size_t)t * B + c] = make_double2(-ar / m2, ai / m2);
    }
  }
}

__global__ void k_gather_shifts(const double2* zq, const double2* zmu, int ntypes, int B,
                                const int* act, int Bact, double2* zq_act, double2* zmu_act,
                                double2* amu_act) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Bact) return;
  int c = act[a];
  zq_act[a] = zq[c];
  if (zmu)
    for (int t = 0; t < ntypes; ++t) {
      const double2 z = zmu[(size_t)t * B + c];
      zmu_act[(size_t)t * Bact + a] = z;
      if (amu_act) {
        const double m2 = z.x * z.x + z.y * z.y;   // -1/z = (-zr + i zi) / |z|^2
        amu_act[(size_t)t * Bact + a] = make_double2(-z.x / m2, z.y / m2);
      }
    }
}

__global__ void k_col_norms(const double* b, int nu, int P, double* bnorm) {
  int p = blockIdx.x;
  double t = 0.0;
  for (int i = threadIdx.x; i < nu; i += blockDim.x) {
    double v = b[(size_t)i * P + p];
    t += v * v;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) bnorm[p] = sqrt(sh[0]);
}

__global__ void k_init_residual(const double* b, int nu, int P, int B, const double* bnorm,
                                double inner_tol, double tol_abs_frac, double2* r, double* rnorm,
                                double* beta, double* target_all) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nu * B) return;
  int i = (int)(idx / B), c = (int)(idx % B);
  r[idx] = make_double2(b[(size_t)i * P + c % P], 0.0);
  if (i == 0) {
    const double bn = bnorm[c % P];
    rnorm[c] = bn;
    beta[c] = bn;
    target_all[c] = round_target(inner_tol * bn, tol_abs_frac * bn);
  }
}

__global__ void k_relres(const double* rnorm, const double* bnorm, int B, int P, double* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= B) return;
  double bn = bnorm[c % P];
  out[c] = bn > 0.0 ? rnorm[c] / bn : 0.0;
}

// ---- heterogeneous wFQFmu (Eqs. 9-10)
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// zq[t][c], kappa[t][u][c]: one thread per column
__global__ void k_hetero_cols(int F, int P, int ntypes, const double* omega_ev,
                              const double* tpar, double2* zq, double2* kappa) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int B = F * P;
  if (c >= B) return;
  const double w = omega_ev[c / P] / 27.211386245988;
  for (int t = 0; t < ntypes; ++t) {
    const double nt = tpar[3 * t], taut = tpar[3 * t + 1], At = tpar[3 * t + 2];
    const double den = 2.0 * nt * taut;
    zq[(size_t)t * B + c] = make_double2(-w * w * taut / den, -w / den);   // Eq. 6
    for (int u = 0; u < ntypes; ++u) {
      const double nu_ = tpar[3 * u], tauu = tpar[3 * u + 1], Au = tpar[3 * u + 2];
      // rho_tu = (n_u tau_u)/(n_t tau_t) (1 - i w tau_t)/(1 - i w tau_u)
      const double2 r = cdiv(make_double2(1.0, -w * taut), make_double2(1.0, -w * tauu));
      const double f = (nu_ * tauu) / (nt * taut) * Au / At;
      kappa[((size_t)t * ntypes + u) * B + c] = make_double2(0.5 * (1.0 + f * r.x), 0.5 * f * r.y);
    }
  }
}

// zmu_atom[i][c] = sum_t wt_it zmu[t][c] / sum_t wt_it, wt_it = nn[i][t] + [t == type_i]
// (Eq. 10: the inverse interband polarisability is the weighted mean of the types')
__global__ void k_hetero_zmu(int N, int B, int ntypes, const int* type, const int* nn,
                             const double2* zmu, double2* zmu_atom) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * B) return;
  const int i = (int)(idx / B), c = (int)(idx % B);
  double sw = 0.0, zr = 0.0, zi = 0.0;
  for (int t = 0; t < ntypes; ++t) {
    const double wt = (double)nn[(size_t)i * ntypes + t] + (type[i] == t ? 1.0 : 0.0);
    const double2 z = zmu[(size_t)t * B + c];
    sw += wt;
    zr += wt * z.x;
    zi += wt * z.y;
  }
  zmu_atom[idx] = make_double2(zr / sw, zi / sw);
}

__global__ void k_gather_rows(const double2* in, int rows, int B, const int* act, int Bact,
                              double2* out) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)rows * Bact) return;
  const int t = (int)(idx / Bact), a = (int)(idx % Bact);
  out[idx] = in[(size_t)t * B + act[a]];
}

__global__ void k_bnorm_cols(const double* bnorm, int P, int B, double* bn) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < B) bn[c] = bnorm[c % P];
}

__global__ void k_init_residual_c(const double2* bc, int nu, int B, const double* bn,
                                  double inner_tol, double tol_abs_frac, double2* r,
                                  double* rnorm, double* beta, double* target_all) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nu * B) return;
  const int i = (int)(idx / B), c = (int)(idx % B);
  r[idx] = bc[idx];
  if (i == 0) {
    const double b = bn[c];
    rnorm[c] = b;
    beta[c] = b;
    target_all[c] = round_target(inner_tol * b, tol_abs_frac * b);
  }
}

// Boundary elements (Sec. 2.3): the scalar shift of every column from Lambda(w_f) =
// 2 pi (e2 + e1) / (e2 - e1): z = +Lambda for DPCM, (Ft - Lambda I) sigma = -E0 e . n
// (Eq. 11); z = -Lambda for the first IEFPCM step, (F + Lambda I) y = c (Eq. 12); z = 0 for
// the second, (S A^-1) q = y.
__global__ void k_bem_shifts(int F, int P, const double* eps, double sign, double2* zq) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= F * P) return;
  const int f = c / P;
  const double2 e2 = make_double2(eps[4 * f], eps[4 * f + 1]);
  const double2 e1 = make_double2(eps[4 * f + 2], eps[4 * f + 3]);
  const double2 num = make_double2(e2.x + e1.x, e2.y + e1.y);
  const double2 den = make_double2(e2.x - e1.x, e2.y - e1.y);
  const double2 q = cdiv(num, den);
  const double k = sign * 2.0 * 3.141592653589793;
  zq[c] = make_double2(k * q.x, k * q.y);
}

// DPCM right-hand side b_i = -E0 e_p . n_i
__global__ void k_rhs_bem(int n, const double* nrm, const double* pol, int P, double e0, double* b) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * P) return;
  const int i = idx / P, p = idx - i * P;
  b[idx] = -e0 * (pol[3 * p] * nrm[3 * i] + pol[3 * p + 1] * nrm[3 * i + 1] + pol[3 * p + 2] * nrm[3 * i + 2]);
}

// IEFPCM right-hand side c = -(2 pi I + F) V with V_j = -E0 e_p . s_j, i.e.
// c_i = E0 (2 pi e_p . s_i + sum_j F_ij e_p . s_j); F is stored transposed (S[j][i] = F_ij),
// so thread i walks column i of S (coalesced across the block's threads).
__global__ void __launch_bounds__(128) k_rhs_ief(int n, int np, const double* __restrict__ S,
                                                 const double* __restrict__ pos,
                                                 const double* __restrict__ pol, int P, double e0,
                                                 double* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  const double ex = pol[3 * p], ey = pol[3 * p + 1], ez = pol[3 * p + 2];
  double acc = 0.0;
  if (i < n)
    for (int j = 0; j < n; ++j)
      acc = fma(S[(size_t)j * np + i], ex * pos[3 * j] + ey * pos[3 * j + 1] + ez * pos[3 * j + 2], acc);
  if (i < n)
    b[(size_t)i * P + p] =
        e0 * (2.0 * 3.141592653589793 * (ex * pos[3 * i] + ey * pos[3 * i + 1] + ez * pos[3 * i + 2]) + acc);
}

}  // namespace

cudaError_t launch_bem_setup(int F, int P, int n, int np, int stage, const double* eps,
                             const double* nrm, const double* S, const double* pos,
                             const double* pol, double e0, double2* zq, double* b, cudaStream_t s,
                             long long* nl) {
  if (stage == 2) {
    cudaError_t e = cudaMemsetAsync(zq, 0, sizeof(double2) * (size_t)F * P, s);
    if (e != cudaSuccess) return e;
    return cudaSuccess;
  }
  k_bem_shifts<<<(F * P + 127) / 128, 128, 0, s>>>(F, P, eps, stage == 0 ? 1.0 : -1.0, zq);
  if (stage == 0) k_rhs_bem<<<(n * P + 255) / 256, 256, 0, s>>>(n, nrm, pol, P, e0, b);
  else k_rhs_ief<<<dim3((n + 127) / 128, P), 128, 0, s>>>(n, np, S, pos, pol, P, e0, b);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_hetero_tables(int F, int P, int ntypes, int N, const double* omega_ev,
                                 const double* tpar, const int* type, const int* nn,
                                 const double2* zmu_type, double2* zq, double2* kappa,
                                 double2* zmu_atom, cudaStream_t s, long long* nl) {
  const int B = F * P;
  k_hetero_cols<<<(B + 127) / 128, 128, 0, s>>>(F, P, ntypes, omega_ev, tpar, zq, kappa);
  const size_t n = (size_t)N * B;
  k_hetero_zmu<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(N, B, ntypes, type, nn, zmu_type, zmu_atom);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const double2* in, int rows, int B, const int* act, int Bact,
                               double2* out, cudaStream_t s, long long* nl) {
  const size_t n = (size_t)rows * Bact;
  k_gather_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, rows, B, act, Bact, out);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_bnorm_cols(const double* bnorm, int P, int B, double* bn, cudaStream_t s,
                              long long* nl) {
  k_bnorm_cols<<<(B + 127) / 128, 128, 0, s>>>(bnorm, P, B, bn);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_init_residual_c(const double2* bc, int nu, int B, const double* bn,
                                   double inner_tol, double tol_abs_frac, double2* r,
                                   double* rnorm, double* beta, double* target_all, cudaStream_t s,
                                   long long* nl) {
  const size_t n = (size_t)nu * B;
  k_init_residual_c<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(bc, nu, B, bn, inner_tol, tol_abs_frac,
                                                                r, rnorm, beta, target_all);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_observables(int N, int model, int F, int P, const double* pos,
                               const int* perm, const double2* x, double e0, const double* omega_ev,
                               const double* pol, double2* alpha, double2* qout, double2* muout,
                               double* sigma_pol, double* sigma, const double* pol_inv,
                               const double* weight, cudaStream_t s, long long* nl) {
  k_observables<<<F * P, 256, 0, s>>>(N, model, F, P, pos, perm, x, e0, omega_ev, pol, alpha, qout,
                                      muout, sigma_pol, weight);
  ++*nl;
  if (sigma && alpha && pol_inv && P == 3) {
    Mat3 ei;
    for (int k = 0; k < 9; ++k) ei.m[k] = pol_inv[k];
    k_sigma_total<<<(F + 127) / 128, 128, 0, s>>>(F, alpha, omega_ev, ei, sigma);
    ++*nl;
  }
  return cudaGetLastError();
}

bool pol_triple_inverse(const double* pol, double* inv) {
  // E[k][p] = pol[3 p + k]: column p is field direction p
  auto E = [&](int k, int p) { return pol[3 * p + k]; };
  const double det = E(0, 0) * (E(1, 1) * E(2, 2) - E(1, 2) * E(2, 1)) -
                     E(0, 1) * (E(1, 0) * E(2, 2) - E(1, 2) * E(2, 0)) +
                     E(0, 2) * (E(1, 0) * E(2, 1) - E(1, 1) * E(2, 0));
  if (!(std::fabs(det) >= 1e-6)) return false;
  // inverse = adjugate / det, row-major
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      const int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
      inv[3 * r + c] = (E(r1, c1) * E(r2, c2) - E(r1, c2) * E(r2, c1)) / det;
    }
  return true;
}

cudaError_t launch_shifts(int F, int P, int ntypes, int model, const double* omega_ev,
                          const double* alpha_ib, double n, double tau, double2* zq,
                          double2* zmu, cudaStream_t s, long long* nl) {
  int B = F * P;
  k_shifts<<<(B + 127) / 128, 128, 0, s>>>(F, P, ntypes, model, omega_ev, alpha_ib, n, tau, zq,
                                           zmu);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_gather_shifts(const double2* zq, const double2* zmu, int ntypes, int B,
                                 const int* act, int Bact, double2* zq_act, double2* zmu_act,
                                 double2* amu_act, cudaStream_t s, long long* nl) {
  k_gather_shifts<<<(Bact + 127) / 128, 128, 0, s>>>(zq, zmu, ntypes, B, act, Bact, zq_act,
                                                     zmu_act, amu_act);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_col_norms(const double* b, int nu, int P, double* bnorm, cudaStream_t s,
                             long long* nl) {
  k_col_norms<<<P, 256, 0, s>>>(b, nu, P, bnorm);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_init_residual(const double* b, int nu, int P, int B, const double* bnorm,
                                 double inner_tol, double tol_abs_frac, double2* r,
                                 double* rnorm, double* beta, double* target_all, cudaStream_t s,
                                 long long* nl) {
  size_t n = (size_t)nu * B;
  k_init_residual<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b, nu, P, B, bnorm, inner_tol,
                                                              tol_abs_frac, r, rnorm, beta,
                                                              target_all);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_relres(const double* rnorm, const double* bnorm, int B, int P, double* out,
                          cudaStream_t s, long long* nl) {
  k_relres<<<(B + 127) / 128, 128, 0, s>>>(rnorm, bnorm, B, P, out);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace px
