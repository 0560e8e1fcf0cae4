// Per-column restarted GMRES on a block of columns: conductance + shift apply,
// FP64 classical Gram-Schmidt (one or two passes), Givens least squares, cycle
// start/end, FP64 true residual, right-hand sides and observables.
//
// Work arrays hold the B_act active columns, column index fastest, so every
// kernel below maps a warp onto 32 consecutive columns of one row and reads /
// writes 32 consecutive complex numbers (512 contiguous bytes for FP64).
#include "px_internal.cuh"

namespace px {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------- conductance + shift
// (Kbar y)_i = sum_j K_ij (y_j - y_i)  (Eq. 2 with the diagonal folded in).
template <bool F32, int MODE>
__global__ void __launch_bounds__(256) k_shift(ShiftArgs a) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int col = blockIdx.x * 32 + tx;
  const bool valid = col < a.Bact;
  double nrm = 0.0;
  if (valid) {
    const int gcol = (MODE == 1) ? a.act[col] : col;
    const double2 zq = a.zq[col];
    for (int i = blockIdx.y * 8 + ty; i < a.nu; i += 8 * gridDim.y) {
      double2 xv = (MODE == 1) ? a.X[(size_t)i * a.B + gcol] : a.X[(size_t)i * a.ldx_c + col];
      double2 w;
      if (i < a.N) {
        double ar, ai;
        if (F32) {
          const float* Y = static_cast<const float*>(a.Y);
          float yr = Y[(size_t)i * a.ldy + 2 * col], yi = Y[(size_t)i * a.ldy + 2 * col + 1];
          float sr = 0.f, si = 0.f;
          for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
            int j = a.col[e];
            float k = a.val32[e];
            sr = fmaf(k, Y[(size_t)j * a.ldy + 2 * col] - yr, sr);
            si = fmaf(k, Y[(size_t)j * a.ldy + 2 * col + 1] - yi, si);
          }
          ar = sr;
          ai = si;
        } else {
          const double* Y = static_cast<const double*>(a.Y);
          double yr = Y[(size_t)i * a.ldy + 2 * col], yi = Y[(size_t)i * a.ldy + 2 * col + 1];
          double sr = 0.0, si = 0.0;
          for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
            int j = a.col[e];
            double k = a.val64[e];
            sr = fma(k, Y[(size_t)j * a.ldy + 2 * col] - yr, sr);
            si = fma(k, Y[(size_t)j * a.ldy + 2 * col + 1] - yi, si);
          }
          ar = sr;
          ai = si;
        }
        double2 zx = cmul(zq, xv);
        w = make_double2(ar - zx.x, ai - zx.y);
      } else {
        int atom = (i - a.N) / 3;
        double2 zm = a.zmu[(size_t)a.type[atom] * a.Bact + col];
        double yr, yi;
        if (F32) {
          const float* Y = static_cast<const float*>(a.Y);
          yr = Y[(size_t)i * a.ldy + 2 * col];
          yi = Y[(size_t)i * a.ldy + 2 * col + 1];
        } else {
          const double* Y = static_cast<const double*>(a.Y);
          yr = Y[(size_t)i * a.ldy + 2 * col];
          yi = Y[(size_t)i * a.ldy + 2 * col + 1];
        }
        double2 zx = cmul(zm, xv);
        w = make_double2(yr - zx.x, yi - zx.y);
      }
      if (MODE == 0) {
        a.W[(size_t)i * a.ldw_c + col] = w;
      } else {
        double bv = a.b[(size_t)i * a.P + (gcol % a.P)];
        double2 r = make_double2(bv - w.x, -w.y);
        a.R[(size_t)i * a.B + gcol] = r;
        nrm += r.x * r.x + r.y * r.y;
      }
    }
  }
  if (MODE == 1) {
    __shared__ double sh[8][32];
    sh[ty][tx] = nrm;
    __syncthreads();
    if (ty == 0 && valid) {
      double t = 0.0;
      for (int k = 0; k < 8; ++k) t += sh[k][tx];
      a.normpart[(size_t)blockIdx.y * a.Bact + col] = t;
    }
  }
}

// RHS (real): charge rows -Kbar V = E0 sum_j K_ij e.(r_j - r_i) (V_i = -E0 e.r_i);
// dipole rows E0 e.
__global__ void k_rhs(int nu, int N, const int* __restrict__ rowptr, const int* __restrict__ col,
                      const double* __restrict__ val, const double* __restrict__ pos,
                      const double* __restrict__ pol, int P, double e0, double* b) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nu * P) return;
  int i = idx / P, p = idx % P;
  const double* e = pol + 3 * p;
  double v;
  if (i < N) {
    double ei = e[0] * pos[3 * i] + e[1] * pos[3 * i + 1] + e[2] * pos[3 * i + 2];
    double s = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int j = col[k];
      double ej = e[0] * pos[3 * j] + e[1] * pos[3 * j + 1] + e[2] * pos[3 * j + 2];
      s = fma(val[k], ej - ei, s);
    }
    v = e0 * s;
  } else {
    v = e0 * e[(i - N) % 3];
  }
  b[(size_t)i * P + p] = v;
}

// ---------------------------------------------------------------- Gram-Schmidt
// Partial projections part[blk][k][a] = sum_{rows of blk} conj(V_k[i][a]) W[i][a]
// for k in [0, j]; groups of 8 basis vectors per sweep over the rows.
__global__ void __launch_bounds__(256) k_dots(ArnoldiArgs a, int j) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int col = blockIdx.x * 32 + tx;
  const bool valid = col < a.Bact;
  __shared__ double2 sh[8][8][32];
  const size_t vstride = (size_t)a.nu * a.Bact;
  for (int k0 = 0; k0 <= j; k0 += 8) {
    const int nk = min(8, j + 1 - k0);
    double2 acc[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) acc[kk] = make_double2(0.0, 0.0);
    if (valid) {
      for (int i = blockIdx.y * 8 + ty; i < a.nu; i += 8 * gridDim.y) {
        size_t off = (size_t)i * a.Bact + col;
        double2 w = a.W[off];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          if (kk < nk) {
            double2 v = a.V[(size_t)(k0 + kk) * vstride + off];
            double2 p = cconjmul(v, w);
            acc[kk].x += p.x;
            acc[kk].y += p.y;
          }
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) sh[ty][kk][tx] = acc[kk];
    __syncthreads();
    if (valid && ty < nk) {
      double2 t = make_double2(0.0, 0.0);
      for (int r = 0; r < 8; ++r) {
        t.x += sh[r][ty][tx].x;
        t.y += sh[r][ty][tx].y;
      }
      reinterpret_cast<double2*>(a.part)[((size_t)blockIdx.y * (a.m + 1) + k0 + ty) * a.Bact + col] = t;
    }
    __syncthreads();
  }
}

// h[pass][k][a] = sum_blk part[blk][k][a]
__global__ void k_dots_reduce(ArnoldiArgs a, int j, int pass) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (j + 1) * a.Bact) return;
  int k = idx / a.Bact, col = idx % a.Bact;
  const double2* p = reinterpret_cast<const double2*>(a.part);
  double2 t = make_double2(0.0, 0.0);
  for (int b = 0; b < a.nblk; ++b) {
    double2 v = p[((size_t)b * (a.m + 1) + k) * a.Bact + col];
    t.x += v.x;
    t.y += v.y;
  }
  a.h[((size_t)pass * (a.m + 1) + k) * a.Bact + col] = t;
}

// W[i][a] -= sum_k V_k[i][a] h[pass][k][a]; with `last`, also |W|^2 partials.
__global__ void __launch_bounds__(256) k_update(ArnoldiArgs a, int j, int pass, int last) {
  extern __shared__ double2 shh[];   // [(j+1)][32]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int col = blockIdx.x * 32 + tx;
  const bool valid = col < a.Bact;
  for (int k = ty; k <= j; k += 8)
    shh[k * 32 + tx] = valid ? a.h[((size_t)pass * (a.m + 1) + k) * a.Bact + col]
                             : make_double2(0.0, 0.0);
  __syncthreads();
  double nrm = 0.0;
  const size_t vstride = (size_t)a.nu * a.Bact;
  if (valid) {
    for (int i = blockIdx.y * 8 + ty; i < a.nu; i += 8 * gridDim.y) {
      size_t off = (size_t)i * a.Bact + col;
      double2 w = a.W[off];
      for (int k = 0; k <= j; ++k) {
        double2 v = a.V[(size_t)k * vstride + off];
        double2 hk = shh[k * 32 + tx];
        w.x -= v.x * hk.x - v.y * hk.y;
        w.y -= v.x * hk.y + v.y * hk.x;
      }
      a.W[off] = w;
      nrm += w.x * w.x + w.y * w.y;
    }
  }
  if (last) {
    __syncthreads();
    double* shn = reinterpret_cast<double*>(shh);
    shn[ty * 32 + tx] = nrm;
    __syncthreads();
    if (ty == 0 && valid) {
      double t = 0.0;
      for (int r = 0; r < 8; ++r) t += shn[r * 32 + tx];
      a.normpart[(size_t)blockIdx.y * a.Bact + col] = t;
    }
  }
}

// One thread per column: new Hessenberg column, previous rotations, new rotation,
// residual estimate |g_{j+1}|, freeze test.
__global__ void k_givens(ArnoldiArgs a, int j, int passes) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= a.Bact) return;
  const int B = a.Bact, m1 = a.m + 1;
  if (a.jconv[col] > 0) {
    a.inv_h[col] = 0.0;
    return;
  }
  double hn2 = 0.0;
  for (int b = 0; b < a.nblk; ++b) hn2 += a.normpart[(size_t)b * B + col];
  double hnext = sqrt(hn2);
  double2* Rc = a.R + (size_t)j * m1 * B;   // column j of the rotated Hessenberg
  double colnorm2 = hn2;
  for (int k = 0; k <= j; ++k) {
    double2 hk = a.h[(size_t)k * B + col];
    if (passes > 1) {
      double2 h2 = a.h[((size_t)m1 + k) * B + col];
      hk.x += h2.x;
      hk.y += h2.y;
    }
    colnorm2 += hk.x * hk.x + hk.y * hk.y;
    Rc[(size_t)k * B + col] = hk;
  }
  // previous rotations
  for (int k = 0; k < j; ++k) {
    double c = a.cs[(size_t)k * B + col];
    double2 s = a.sn[(size_t)k * B + col];
    double2 x0 = Rc[(size_t)k * B + col], x1 = Rc[(size_t)(k + 1) * B + col];
    double2 sx1 = cmul(s, x1);
    double2 csx0 = make_double2(-(s.x * x0.x + s.y * x0.y), -(s.x * x0.y - s.y * x0.x));  // -conj(s) x0
    Rc[(size_t)k * B + col] = make_double2(c * x0.x + sx1.x, c * x0.y + sx1.y);
    Rc[(size_t)(k + 1) * B + col] = make_double2(csx0.x + c * x1.x, csx0.y + c * x1.y);
  }
  // new rotation zeroing (hnext) under a = Rc[j]
  double2 av = Rc[(size_t)j * B + col];
  double aa = sqrt(av.x * av.x + av.y * av.y);
  double rho = sqrt(aa * aa + hn2);
  double c;
  double2 s, r;
  if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
    r = make_double2(hnext, 0.0);
  } else {
    double2 ph = make_double2(av.x / aa, av.y / aa);   // a / |a|
    c = aa / rho;
    s = make_double2(ph.x * hnext / rho, ph.y * hnext / rho);   // (a/|a|) conj(b) / rho, b real
    r = make_double2(ph.x * rho, ph.y * rho);
  }
  a.cs[(size_t)j * B + col] = c;
  a.sn[(size_t)j * B + col] = s;
  Rc[(size_t)j * B + col] = r;
  double2 gj = a.g[(size_t)j * B + col];
  double2 gn = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
  a.g[(size_t)j * B + col] = make_double2(c * gj.x, c * gj.y);
  a.g[(size_t)(j + 1) * B + col] = gn;
  double res = sqrt(gn.x * gn.x + gn.y * gn.y);
  bool breakdown = hnext <= 1e-14 * sqrt(colnorm2);
  if (res <= a.target[col] || breakdown || j + 1 == a.m) {
    a.jconv[col] = j + 1;
    a.inv_h[col] = 0.0;
  } else {
    a.inv_h[col] = 1.0 / hnext;
    atomicAdd(&a.active_count[j], 1);
  }
}

__global__ void __launch_bounds__(256) k_normalize(ArnoldiArgs a, int j, float* X32, double* X64,
                                                   int ldx) {
  const int col = blockIdx.x * 32 + threadIdx.x;
  if (col >= a.Bact) return;
  const double s = a.inv_h[col];
  double2* Vn = a.V + (size_t)(j + 1) * a.nu * a.Bact;
  for (int i = blockIdx.y * 8 + threadIdx.y; i < a.nu; i += 8 * gridDim.y) {
    size_t off = (size_t)i * a.Bact + col;
    double2 w = a.W[off];
    double2 v = make_double2(w.x * s, w.y * s);
    Vn[off] = v;
    if (X32) *reinterpret_cast<float2*>(X32 + (size_t)i * ldx + 2 * col) = make_float2((float)v.x, (float)v.y);
    if (X64) *reinterpret_cast<double2*>(X64 + (size_t)i * ldx + 2 * col) = v;
  }
}

__global__ void k_cycle_init(ArnoldiArgs a, const int* act, const double* rnorm,
                             const double* bnorm, int P, double inner_tol, double tol_frac) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= a.Bact) return;
  int gc = act[col];
  double beta = rnorm[gc];
  a.g[col] = make_double2(beta, 0.0);
  a.target[col] = fmax(inner_tol * beta, tol_frac * bnorm[gc % P]);
  a.jconv[col] = 0;
  a.inv_h[col] = beta > 0.0 ? 1.0 / beta : 0.0;
}

__global__ void __launch_bounds__(256) k_cycle_start(ArnoldiArgs a, const int* act,
                                                     const double2* r, int B, const double* rnorm,
                                                     float* X32, double* X64, int ldx) {
  const int col = blockIdx.x * 32 + threadIdx.x;
  if (col >= a.Bact) return;
  const int gc = act[col];
  const double beta = rnorm[gc];
  const double s = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int i = blockIdx.y * 8 + threadIdx.y; i < a.nu; i += 8 * gridDim.y) {
    double2 rv = r[(size_t)i * B + gc];
    double2 v = make_double2(rv.x * s, rv.y * s);
    a.V[(size_t)i * a.Bact + col] = v;
    if (X32) *reinterpret_cast<float2*>(X32 + (size_t)i * ldx + 2 * col) = make_float2((float)v.x, (float)v.y);
    if (X64) *reinterpret_cast<double2*>(X64 + (size_t)i * ldx + 2 * col) = v;
  }
}

// y = R^{-1} g (upper triangular, size jc) per column.
__global__ void k_backsolve(ArnoldiArgs a, int jend, const int* act, int* iters) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= a.Bact) return;
  const int B = a.Bact, m1 = a.m + 1;
  int jc = a.jconv[col] > 0 ? a.jconv[col] : jend;
  for (int k = jc - 1; k >= 0; --k) {
    double2 t = a.g[(size_t)k * B + col];
    for (int l = k + 1; l < jc; ++l) {
      double2 rl = a.R[((size_t)l * m1 + k) * B + col];
      double2 yl = a.y[(size_t)l * B + col];
      double2 p = cmul(rl, yl);
      t.x -= p.x;
      t.y -= p.y;
    }
    double2 d = a.R[((size_t)k * m1 + k) * B + col];
    double den = d.x * d.x + d.y * d.y;
    double2 yk = den > 0.0 ? make_double2((t.x * d.x + t.y * d.y) / den, (t.y * d.x - t.x * d.y) / den)
                           : make_double2(0.0, 0.0);
    a.y[(size_t)k * B + col] = yk;
  }
  a.jconv[col] = jc;
  iters[act[col]] += jc;
}

__global__ void __launch_bounds__(256) k_xupdate(ArnoldiArgs a, const int* act, double2* x,
                                                 int B) {
  const int col = blockIdx.x * 32 + threadIdx.x;
  if (col >= a.Bact) return;
  const int gc = act[col];
  const int jc = a.jconv[col];
  const size_t vstride = (size_t)a.nu * a.Bact;
  for (int i = blockIdx.y * 8 + threadIdx.y; i < a.nu; i += 8 * gridDim.y) {
    size_t off = (size_t)i * a.Bact + col;
    double2 acc = x[(size_t)i * B + gc];
    for (int k = 0; k < jc; ++k) {
      double2 p = cmul(a.V[(size_t)k * vstride + off], a.y[(size_t)k * a.Bact + col]);
      acc.x += p.x;
      acc.y += p.y;
    }
    x[(size_t)i * B + gc] = acc;
  }
}

__global__ void __launch_bounds__(256) k_gather_x(const double2* x, int B, const int* act,
                                                  int Bact, int nu, double* X64, int ldx) {
  const int col = blockIdx.x * 32 + threadIdx.x;
  if (col >= Bact) return;
  const int gc = act[col];
  for (int i = blockIdx.y * 8 + threadIdx.y; i < nu; i += 8 * gridDim.y)
    *reinterpret_cast<double2*>(X64 + (size_t)i * ldx + 2 * col) = x[(size_t)i * B + gc];
}

__global__ void k_norm_finish(const double* normpart, int nblk, int Bact, const int* act,
                              double* rnorm) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= Bact) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t += normpart[(size_t)b * Bact + col];
  rnorm[act[col]] = sqrt(t);
}

// One block per column c = f * P + p: dipole, polarisability and per-polarisation
// absorption (Sec. "Observables").
__global__ void k_observables(int N, int model, int F, int P, const double* __restrict__ pos,
                              const double2* __restrict__ x, double e0,
                              const double* __restrict__ omega_ev, const double* __restrict__ pol,
                              double2* alpha, double2* qout, double2* muout, double* sigma_pol) {
  const int c = blockIdx.x;
  const int B = F * P;
  const int f = c / P, p = c % P;
  double d[6] = {0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double2 q = x[(size_t)i * B + c];
    for (int k = 0; k < 3; ++k) {
      d[2 * k] += q.x * pos[3 * i + k];
      d[2 * k + 1] += q.y * pos[3 * i + k];
    }
    if (qout) qout[(size_t)c * N + i] = q;
    if (model == 1) {
      for (int k = 0; k < 3; ++k) {
        double2 mu = x[(size_t)(N + 3 * i + k) * B + c];
        d[2 * k] += mu.x;
        d[2 * k + 1] += mu.y;
        if (muout) muout[((size_t)c * N + i) * 3 + k] = mu;
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

// sigma[f] = (1/3) sum_p sigma_pol[f][p] = 4 pi w / (3c) Tr Im alpha for P = 3 orthonormal fields
__global__ void k_sigma_total(int F, int P, const double* sigma_pol, double* sigma) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  double t = 0.0;
  for (int p = 0; p < P; ++p) t += sigma_pol[(size_t)f * P + p];
  sigma[f] = t / 3.0;
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
                                const int* act, int Bact, double2* zq_act, double2* zmu_act) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= Bact) return;
  int c = act[a];
  zq_act[a] = zq[c];
  if (zmu)
    for (int t = 0; t < ntypes; ++t) zmu_act[(size_t)t * Bact + a] = zmu[(size_t)t * B + c];
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
                                double2* r, double* rnorm) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nu * B) return;
  int i = (int)(idx / B), c = (int)(idx % B);
  r[idx] = make_double2(b[(size_t)i * P + c % P], 0.0);
  if (i == 0) rnorm[c] = bnorm[c % P];
}

__global__ void k_relres(const double* rnorm, const double* bnorm, int B, int P, double* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= B) return;
  double bn = bnorm[c % P];
  out[c] = bn > 0.0 ? rnorm[c] / bn : 0.0;
}

inline dim3 col_grid(int Bact, int nblk) { return dim3((Bact + 31) / 32, nblk); }

}  // namespace

int reduction_blocks(int nu) {
  int nb = (nu + 63) / 64;
  if (nb > 128) nb = 128;
  if (nb < 1) nb = 1;
  return nb;
}

cudaError_t launch_shift(const ShiftArgs& a, int mode, cudaStream_t s, long long* nl) {
  dim3 grd = col_grid(a.Bact, a.nblk), blk(32, 8);
  if (mode == 0) {
    if (a.y_is_f32) k_shift<true, 0><<<grd, blk, 0, s>>>(a);
    else k_shift<false, 0><<<grd, blk, 0, s>>>(a);
  } else {
    if (a.y_is_f32) k_shift<true, 1><<<grd, blk, 0, s>>>(a);
    else k_shift<false, 1><<<grd, blk, 0, s>>>(a);
  }
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_rhs(int nu, int N, int model, const int* rowptr, const int* col,
                       const double* val64, const double* pos, const double* pol, int P,
                       double e0, double* b, cudaStream_t s, long long* nl) {
  (void)model;
  int n = nu * P;
  k_rhs<<<(n + 255) / 256, 256, 0, s>>>(nu, N, rowptr, col, val64, pos, pol, P, e0, b);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_dots(const ArnoldiArgs& a, int j, int pass, cudaStream_t s, long long* nl) {
  k_dots<<<col_grid(a.Bact, a.nblk), dim3(32, 8), 0, s>>>(a, j);
  int n = (j + 1) * a.Bact;
  k_dots_reduce<<<(n + 255) / 256, 256, 0, s>>>(a, j, pass);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_update(const ArnoldiArgs& a, int j, int pass, bool last, cudaStream_t s,
                          long long* nl) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxRestart * 32 * (int)sizeof(double2));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  size_t smem = (size_t)(j + 1) * 32 * sizeof(double2);
  if (smem < 8 * 32 * sizeof(double)) smem = 8 * 32 * sizeof(double);
  k_update<<<col_grid(a.Bact, a.nblk), dim3(32, 8), smem, s>>>(a, j, pass, last ? 1 : 0);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_givens(const ArnoldiArgs& a, int j, int passes, cudaStream_t s, long long* nl) {
  k_givens<<<(a.Bact + 127) / 128, 128, 0, s>>>(a, j, passes);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_normalize(const ArnoldiArgs& a, int j, float* X32, double* X64, int ldx,
                             cudaStream_t s, long long* nl) {
  k_normalize<<<col_grid(a.Bact, a.nblk), dim3(32, 8), 0, s>>>(a, j, X32, X64, ldx);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_cycle_start(const ArnoldiArgs& a, const int* act, const double2* r, int B,
                               const double* rnorm, float* X32, double* X64, int ldx,
                               cudaStream_t s, long long* nl) {
  k_cycle_start<<<col_grid(a.Bact, a.nblk), dim3(32, 8), 0, s>>>(a, act, r, B, rnorm, X32, X64,
                                                                   ldx);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_cycle_init(const ArnoldiArgs& a, const int* act, const double* rnorm,
                              const double* bnorm, int P, double inner_tol, double tol_frac,
                              cudaStream_t s, long long* nl) {
  k_cycle_init<<<(a.Bact + 127) / 128, 128, 0, s>>>(a, act, rnorm, bnorm, P, inner_tol, tol_frac);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_cycle_end(const ArnoldiArgs& a, int jend, const int* act, double2* x, int B,
                             int* iters, cudaStream_t s, long long* nl) {
  k_backsolve<<<(a.Bact + 127) / 128, 128, 0, s>>>(a, jend, act, iters);
  k_xupdate<<<col_grid(a.Bact, a.nblk), dim3(32, 8), 0, s>>>(a, act, x, B);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_gather_x(const double2* x, int B, const int* act, int Bact, int nu,
                            double* X64, int ldx, cudaStream_t s, long long* nl) {
  int nblk = reduction_blocks(nu);
  k_gather_x<<<col_grid(Bact, nblk), dim3(32, 8), 0, s>>>(x, B, act, Bact, nu, X64, ldx);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_norm_finish(const double* normpart, int nblk, int Bact, const int* act,
                               double* rnorm, cudaStream_t s, long long* nl) {
  k_norm_finish<<<(Bact + 127) / 128, 128, 0, s>>>(normpart, nblk, Bact, act, rnorm);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_observables(int N, int model, int F, int P, const double* pos,
                               const double2* x, double e0, const double* omega_ev,
                               const double* pol, double2* alpha, double2* qout, double2* muout,
                               double* sigma_pol, double* sigma, cudaStream_t s, long long* nl) {
  k_observables<<<F * P, 256, 0, s>>>(N, model, F, P, pos, x, e0, omega_ev, pol, alpha, qout,
                                      muout, sigma_pol);
  ++*nl;
  if (sigma && sigma_pol && P == 3) {
    k_sigma_total<<<(F + 127) / 128, 128, 0, s>>>(F, P, sigma_pol, sigma);
    ++*nl;
  }
  return cudaGetLastError();
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
                                 cudaStream_t s, long long* nl) {
  k_gather_shifts<<<(Bact + 127) / 128, 128, 0, s>>>(zq, zmu, ntypes, B, act, Bact, zq_act,
                                                     zmu_act);
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
                                 double2* r, double* rnorm, cudaStream_t s, long long* nl) {
  size_t n = (size_t)nu * B;
  k_init_residual<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(b, nu, P, B, bnorm, r, rnorm);
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
