// Per-column restarted GMRES on a block of columns: conductance + shift apply,
// classical Gram-Schmidt (one or two passes), Givens least squares, cycle start /
// end with the implicit inner residual, and the FP64 true residual.
//
// Work arrays hold the B_act active columns, column index fastest, so every
// kernel maps a warp onto 32 consecutive columns of one row (512 contiguous
// bytes of 16-byte complex elements).
//
// Element types of the basis: double2 (FP64 complex), float4 (double-FP32 complex:
// re_hi, im_hi, re_lo, im_lo) or float2 (FP32 complex).  Double-FP32 products and
// sums use the error-free transformations TwoSum (Knuth) and TwoProduct via FMA, so
// each product a*b of two double-FP32 numbers carries ~48 significant bits (the
// lo*lo term, below 2^-48 relative, is dropped).  FP32 sums run over at most a few
// dozen rows per thread before the partial sums continue in FP64.
#include "px_internal.cuh"

namespace px {

namespace {

// ------------------------------------------------------------ double-FP32 arithmetic
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// (h, l) += (ah + al)(bh + bl); h carries the running sum, l its accumulated error
__device__ __forceinline__ void ff_mac(float& h, float& l, float ah, float al, float bh, float bl) {
  float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float s, t;
  two_sum(h, p, s, t);
  h = s;
  l = __fadd_rn(l, __fadd_rn(t, e));
}
__device__ __forceinline__ float2 split_d(double v) {
  float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double join_f(float h, float l) { return (double)h + (double)l; }

// ------------------------------------------------------------ element traits
struct AccD { double re, im; };
struct AccF { float rh, rl, ih, il; };
struct AccS { float re, im; };

template <class E> struct Tr;

template <> struct Tr<double2> {
  using Acc = AccD;
  using Coef = double2;
  static __device__ __forceinline__ Acc zero() { return {0.0, 0.0}; }
  static __device__ __forceinline__ Coef coef(double2 h) { return h; }
  // a += conj(v) w
  static __device__ __forceinline__ void conj_mac(Acc& a, double2 v, double2 w) {
    a.re = fma(v.x, w.x, fma(v.y, w.y, a.re));
    a.im = fma(v.x, w.y, fma(-v.y, w.x, a.im));
  }
  // a += v h
  static __device__ __forceinline__ void mac(Acc& a, double2 v, Coef h) {
    a.re = fma(v.x, h.x, fma(-v.y, h.y, a.re));
    a.im = fma(v.x, h.y, fma(v.y, h.x, a.im));
  }
  static __device__ __forceinline__ void norm_mac(Acc& a, double2 w) {
    a.re = fma(w.x, w.x, fma(w.y, w.y, a.re));
  }
  static __device__ __forceinline__ double2 to_d2(const Acc& a) { return make_double2(a.re, a.im); }
  static __device__ __forceinline__ double norm_d(const Acc& a) { return a.re; }
  static __device__ __forceinline__ double2 sub(double2 w, const Acc& a) {
    return make_double2(w.x - a.re, w.y - a.im);
  }
  static __device__ __forceinline__ double2 scale(double2 w, double s) {
    return make_double2(w.x * s, w.y * s);
  }
  static __device__ __forceinline__ double2 from_d2(double2 v) { return v; }
  static __device__ __forceinline__ double2 to_c(double2 v) { return v; }
  static __device__ __forceinline__ float2 hi(double2 v) {
    return make_float2((float)v.x, (float)v.y);
  }
  // w = y - z x
  static __device__ __forceinline__ double2 axpy_shift(double yr, double yi, double2 z, double2 x) {
    return make_double2(yr - (z.x * x.x - z.y * x.y), yi - (z.x * x.y + z.y * x.x));
  }
};

template <> struct Tr<float4> {
  using Acc = AccF;
  using Coef = float4;   // (re_hi, im_hi, re_lo, im_lo)
  static __device__ __forceinline__ Acc zero() { return {0.f, 0.f, 0.f, 0.f}; }
  static __device__ __forceinline__ Coef coef(double2 h) {
    float2 r = split_d(h.x), i = split_d(h.y);
    return make_float4(r.x, i.x, r.y, i.y);
  }
  static __device__ __forceinline__ void conj_mac(Acc& a, float4 v, float4 w) {
    ff_mac(a.rh, a.rl, v.x, v.z, w.x, w.z);
    ff_mac(a.rh, a.rl, v.y, v.w, w.y, w.w);
    ff_mac(a.ih, a.il, v.x, v.z, w.y, w.w);
    ff_mac(a.ih, a.il, -v.y, -v.w, w.x, w.z);
  }
  static __device__ __forceinline__ void mac(Acc& a, float4 v, Coef h) {
    ff_mac(a.rh, a.rl, v.x, v.z, h.x, h.z);
    ff_mac(a.rh, a.rl, -v.y, -v.w, h.y, h.w);
    ff_mac(a.ih, a.il, v.x, v.z, h.y, h.w);
    ff_mac(a.ih, a.il, v.y, v.w, h.x, h.z);
  }
  static __device__ __forceinline__ void norm_mac(Acc& a, float4 w) {
    ff_mac(a.rh, a.rl, w.x, w.z, w.x, w.z);
    ff_mac(a.rh, a.rl, w.y, w.w, w.y, w.w);
  }
  static __device__ __forceinline__ double2 to_d2(const Acc& a) {
    return make_double2(join_f(a.rh, a.rl), join_f(a.ih, a.il));
  }
  static __device__ __forceinline__ double norm_d(const Acc& a) { return join_f(a.rh, a.rl); }
  // w - a, renormalised
  static __device__ __forceinline__ float4 sub(float4 w, const Acc& a) {
    float sr, er, si, ei;
    two_sum(w.x, -a.rh, sr, er);
    er = __fadd_rn(er, __fsub_rn(w.z, a.rl));
    two_sum(w.y, -a.ih, si, ei);
    ei = __fadd_rn(ei, __fsub_rn(w.w, a.il));
    float rh, rl, ih, il;
    fast_two_sum(sr, er, rh, rl);
    fast_two_sum(si, ei, ih, il);
    return make_float4(rh, ih, rl, il);
  }
  // w * s for a real FP64 scale s
  static __device__ __forceinline__ float4 scale(float4 w, double s) {
    float2 ss = split_d(s);
    AccF a = zero();
    ff_mac(a.rh, a.rl, w.x, w.z, ss.x, ss.y);
    ff_mac(a.ih, a.il, w.y, w.w, ss.x, ss.y);
    float rh, rl, ih, il;
    fast_two_sum(a.rh, a.rl, rh, rl);
    fast_two_sum(a.ih, a.il, ih, il);
    return make_float4(rh, ih, rl, il);
  }
  static __device__ __forceinline__ float4 from_d2(double2 v) {
    float2 r = split_d(v.x), i = split_d(v.y);
    return make_float4(r.x, i.x, r.y, i.y);
  }
  static __device__ __forceinline__ double2 to_c(float4 v) {
    return make_double2(join_f(v.x, v.z), join_f(v.y, v.w));
  }
  static __device__ __forceinline__ float2 hi(float4 v) { return make_float2(v.x, v.y); }
  // w = y - z x in double-FP32, y the FP32 conductance sum (re, im)
  static __device__ __forceinline__ float4 axpy_shift(double yr, double yi, float4 z, float4 x) {
    AccF a = {(float)yr, 0.f, (float)yi, 0.f};
    // -(z x): re = -(zr xr - zi xi), im = -(zr xi + zi xr)
    ff_mac(a.rh, a.rl, -z.x, -z.z, x.x, x.z);
    ff_mac(a.rh, a.rl, z.y, z.w, x.y, x.w);
    ff_mac(a.ih, a.il, -z.x, -z.z, x.y, x.w);
    ff_mac(a.ih, a.il, -z.y, -z.w, x.x, x.z);
    float rh, rl, ih, il;
    fast_two_sum(a.rh, a.rl, rh, rl);
    fast_two_sum(a.ih, a.il, ih, il);
    return make_float4(rh, ih, rl, il);
  }
};

template <> struct Tr<float2> {
  using Acc = AccS;
  using Coef = float2;
  static __device__ __forceinline__ Acc zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ Coef coef(double2 h) {
    return make_float2(__double2float_rn(h.x), __double2float_rn(h.y));
  }
  static __device__ __forceinline__ void conj_mac(Acc& a, float2 v, float2 w) {
    a.re = fmaf(v.x, w.x, fmaf(v.y, w.y, a.re));
    a.im = fmaf(v.x, w.y, fmaf(-v.y, w.x, a.im));
  }
  static __device__ __forceinline__ void mac(Acc& a, float2 v, Coef h) {
    a.re = fmaf(v.x, h.x, fmaf(-v.y, h.y, a.re));
    a.im = fmaf(v.x, h.y, fmaf(v.y, h.x, a.im));
  }
  static __device__ __forceinline__ void norm_mac(Acc& a, float2 w) {
    a.re = fmaf(w.x, w.x, fmaf(w.y, w.y, a.re));
  }
  static __device__ __forceinline__ double2 to_d2(const Acc& a) { return make_double2(a.re, a.im); }
  static __device__ __forceinline__ double norm_d(const Acc& a) { return a.re; }
  static __device__ __forceinline__ float2 sub(float2 w, const Acc& a) {
    return make_float2(w.x - a.re, w.y - a.im);
  }
  static __device__ __forceinline__ float2 scale(float2 w, double s) {
    const float f = __double2float_rn(s);
    return make_float2(w.x * f, w.y * f);
  }
  static __device__ __forceinline__ float2 from_d2(double2 v) {
    return make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  }
  static __device__ __forceinline__ double2 to_c(float2 v) { return make_double2(v.x, v.y); }
  static __device__ __forceinline__ float2 hi(float2 v) { return v; }
  static __device__ __forceinline__ float2 axpy_shift(double yr, double yi, float2 z, float2 x) {
    return make_float2(fmaf(-z.x, x.x, fmaf(z.y, x.y, (float)yr)),
                       fmaf(-z.x, x.y, fmaf(-z.y, x.x, (float)yi)));
  }
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Matvec operand of basis entry v in row i of column col: v, or alpha^IB v on the
// dipole rows when the wFQFmu right preconditioner is on.
template <class E>
__device__ __forceinline__ void write_operand(const KrylovArgs& a, int i, int col, E v, float* X32,
                                              double* X64, int ldx) {
  using TT = Tr<E>;
  if (a.amu && i >= a.N) {
    const double2 m = a.amu[(size_t)a.type[(i - a.N) / 3] * a.Bact + col];
    const double2 w = cmul(m, TT::to_c(v));
    if (X32) *reinterpret_cast<float2*>(X32 + (size_t)i * ldx + 2 * col) = make_float2((float)w.x, (float)w.y);
    if (X64) *reinterpret_cast<double2*>(X64 + (size_t)i * ldx + 2 * col) = w;
    return;
  }
  if (X32) *reinterpret_cast<float2*>(X32 + (size_t)i * ldx + 2 * col) = TT::hi(v);
  if (X64) *reinterpret_cast<double2*>(X64 + (size_t)i * ldx + 2 * col) = TT::to_c(v);
}

// ------------------------------------------------------------ conductance + shift
// (Kbar y)_i = sum_j K_ij (y_j - y_i)  (Eq. 2 with the diagonal folded in).
template <class E, bool F32Y>
__global__ void __launch_bounds__(256) k_shift(ShiftArgs a) {
  using TT = Tr<E>;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int col = blockIdx.x * 32 + tx;
  if (col >= a.Bact) return;
  if (a.jconv && a.jconv[col] > 0) return;   // column stopped at an earlier step
  const E* X = static_cast<const E*>(a.X) + (a.jdev ? (size_t)*a.jdev * a.nu * a.Bact : 0);
  E* W = static_cast<E*>(a.W);
  const auto zq = TT::coef(a.zq[col]);
  for (int i = blockIdx.y * 8 + ty; i < a.nu; i += 8 * gridDim.y) {
    const size_t off = (size_t)i * a.Bact + col;
    const E xv = X[off];
    double yr, yi;
    // heterogeneous wFQFmu: z_q of the charge's own type (Eq. 9)
    auto zz = (a.qtype && i < a.N) ? TT::coef(a.zq[(size_t)a.qtype[i] * a.Bact + col]) : zq;
    if (i < a.N && a.kbar_in_y) {
      // the matvec applied M = diag(Kbar, I) T: no conductance gather
      if (F32Y) {
        const float* Y = static_cast<const float*>(a.Y);
        yr = Y[(size_t)i * a.ldy + 2 * col] * a.yscale;
        yi = Y[(size_t)i * a.ldy + 2 * col + 1] * a.yscale;
      } else {
        const double* Y = static_cast<const double*>(a.Y);
        yr = Y[(size_t)i * a.ldy + 2 * col] * (double)a.yscale;
        yi = Y[(size_t)i * a.ldy + 2 * col + 1] * (double)a.yscale;
      }
    } else if (i < a.N) {
      if (F32Y) {
        const float* Y = static_cast<const float*>(a.Y);
        const float y0r = Y[(size_t)i * a.ldy + 2 * col], y0i = Y[(size_t)i * a.ldy + 2 * col + 1];
        float sr = 0.f, si = 0.f;
        if (a.kappa) {
          // complex bond weights K_ij kappa[t_i][t_j] of 1/2 (Kbar + Hbar(w)) (Eq. 9)
          const double2* kr = a.kappa + (size_t)a.qtype[i] * a.ntypes * a.Bact + col;
          for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
            const int j = a.col[e];
            const size_t jo = (size_t)j * a.ldy + 2 * col;
            const double2 kp = kr[(size_t)a.qtype[j] * a.Bact];
            const float k = a.val32[e];
            const float wr = k * (float)kp.x, wi = k * (float)kp.y;
            const float dr = Y[jo] - y0r, di = Y[jo + 1] - y0i;
            sr = fmaf(wr, dr, fmaf(-wi, di, sr));
            si = fmaf(wr, di, fmaf(wi, dr, si));
          }
        } else {
          for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
            const size_t jo = (size_t)a.col[e] * a.ldy + 2 * col;
            const float k = a.val32[e];
            sr = fmaf(k, Y[jo] - y0r, sr);
            si = fmaf(k, Y[jo + 1] - y0i, si);
          }
        }
        yr = sr;
        yi = si;
      } else {
        const double* Y = static_cast<const double*>(a.Y);
        const double y0r = Y[(size_t)i * a.ldy + 2 * col], y0i = Y[(size_t)i * a.ldy + 2 * col + 1];
        double sr = 0.0, si = 0.0;
        if (a.kappa) {
          const double2* kr = a.kappa + (size_t)a.qtype[i] * a.ntypes * a.Bact + col;
          for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
            const int j = a.col[e];
            const size_t jo = (size_t)j * a.ldy + 2 * col;
            const double2 kp = kr[(size_t)a.qtype[j] * a.Bact];
            const double k = a.val64[e];
            const double wr = k * kp.x, wi = k * kp.y;
            const double dr = Y[jo] - y0r, di = Y[jo + 1] - y0i;
            sr = fma(wr, dr, fma(-wi, di, sr));
            si = fma(wr, di, fma(wi, dr, si));
          }
        } else {
          for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
            const size_t jo = (size_t)a.col[e] * a.ldy + 2 * col;
            const double k = a.val64[e];
            sr = fma(k, Y[jo] - y0r, sr);
            si = fma(k, Y[jo + 1] - y0i, si);
          }
        }
        yr = sr;
        yi = si;
      }
    } else {
      const int atom = (i - a.N) / 3;
      // with the dipole preconditioner the operand was alpha^IB v, and
      // -z_mu alpha^IB v = +v: the shift term becomes +v
      zz = a.precond_mu ? TT::coef(make_double2(-1.0, 0.0))
                        : TT::coef(a.zmu[(size_t)a.type[atom] * a.Bact + col]);
      const float ys = a.kbar_in_y ? a.yscale : 1.0f;
      if (F32Y) {
        const float* Y = static_cast<const float*>(a.Y);
        yr = Y[(size_t)i * a.ldy + 2 * col] * ys;
        yi = Y[(size_t)i * a.ldy + 2 * col + 1] * ys;
      } else {
        const double* Y = static_cast<const double*>(a.Y);
        yr = Y[(size_t)i * a.ldy + 2 * col] * (double)ys;
        yi = Y[(size_t)i * a.ldy + 2 * col + 1] * (double)ys;
      }
    }
    W[off] = TT::axpy_shift(yr, yi, zz, xv);
  }
}

// FP64 true residual r = b - A x (Eq. 1 / Eq. 7) with Y = T64 x.
__global__ void __launch_bounds__(256) k_resid(ResidArgs a) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int col = blockIdx.x * 32 + tx;
  const bool valid = col < a.Bact;
  double nrm = 0.0;
  if (valid) {
    const int gc = a.act[col];
    for (int i = blockIdx.y * 8 + ty; i < a.nu; i += 8 * gridDim.y) {
      const double2 xv = a.x[(size_t)i * a.B + gc];
      const double y0r = a.Y[(size_t)i * a.ldy + 2 * col], y0i = a.Y[(size_t)i * a.ldy + 2 * col + 1];
      double2 w;
      if (a.op_full) {
        // boundary elements: Y = Ft x is the whole operator (Eq. 11): w = Y - Lambda x
        const double2 zx = cmul(a.zq[col], xv);
        w = make_double2(y0r - zx.x, y0i - zx.y);
      } else if (i < a.N) {
        double sr = 0.0, si = 0.0;
        if (a.kappa) {
          // 1/2 (Kbar + Hbar(w)) with complex bond weights (Eq. 9)
          const double2* kr = a.kappa + (size_t)a.qtype[i] * a.ntypes * a.Bact + col;
          for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
            const int j = a.col[e];
            const size_t jo = (size_t)j * a.ldy + 2 * col;
            const double2 kp = kr[(size_t)a.qtype[j] * a.Bact];
            const double k = a.val64[e];
            const double wr = k * kp.x, wi = k * kp.y;
            const double dr = a.Y[jo] - y0r, di = a.Y[jo + 1] - y0i;
            sr = fma(wr, dr, fma(-wi, di, sr));
            si = fma(wr, di, fma(wi, dr, si));
          }
        } else {
          for (int e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
            const size_t jo = (size_t)a.col[e] * a.ldy + 2 * col;
            const double k = a.val64[e];
            sr = fma(k, a.Y[jo] - y0r, sr);
            si = fma(k, a.Y[jo + 1] - y0i, si);
          }
        }
        const double2 zq = a.qtype ? a.zq[(size_t)a.qtype[i] * a.Bact + col] : a.zq[col];
        const double2 zx = cmul(zq, xv);
        w = make_double2(sr - zx.x, si - zx.y);
      } else {
        const int atom = (i - a.N) / 3;
        const double2 zx = cmul(a.zmu[(size_t)a.type[atom] * a.Bact + col], xv);
        w = make_double2(y0r - zx.x, y0i - zx.y);
      }
      const double2 bv = a.bc ? a.bc[(size_t)i * a.B + gc]
                              : make_double2(a.b[(size_t)i * a.P + (gc % a.P)], 0.0);
      const double2 r = make_double2(bv.x - w.x, bv.y - w.y);
      a.R[(size_t)i * a.B + gc] = r;
      nrm += r.x * r.x + r.y * r.y;
    }
  }
  __shared__ double sh[8][32];
  sh[ty][tx] = nrm;
  __syncthreads();
  if (ty == 0 && valid) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += sh[k][tx];
    a.normpart[(size_t)blockIdx.y * a.Bact + col] = t;
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

// Right-hand side of Eq. 9 per column: charge rows (C(w) (-V))_i = E0 sum_j w_ij(w) e.(r_j -
// r_i) with the bond weights w_ij = K_ij kappa[t_i][t_j][c] of C = 1/2 (Kbar + Hbar(w));
// dipole rows E0 e.  bn[c] (written by the first thread of each column's block row) is
// computed by k_col_norms_c.
__global__ void k_rhs_hetero(int N, int F, int P, const int* __restrict__ rowptr,
                             const int* __restrict__ col, const double* __restrict__ val,
                             const int* __restrict__ type, int ntypes,
                             const double2* __restrict__ kappa, const double* __restrict__ pos,
                             const double* __restrict__ pol, double e0, double2* bc) {
  const int B = F * P;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nu = 4 * N;
  if (idx >= (size_t)nu * B) return;
  const int i = (int)(idx / B), c = (int)(idx % B);
  const double* e = pol + 3 * (c % P);
  double2 v = make_double2(0.0, 0.0);
  if (i < N) {
    const double ei = e[0] * pos[3 * i] + e[1] * pos[3 * i + 1] + e[2] * pos[3 * i + 2];
    const int ti = type[i];
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int j = col[k];
      const double ej = e[0] * pos[3 * j] + e[1] * pos[3 * j + 1] + e[2] * pos[3 * j + 2];
      const double2 kap = kappa[((size_t)ti * ntypes + type[j]) * B + c];
      const double d = val[k] * (ej - ei);
      v.x = fma(d, kap.x, v.x);
      v.y = fma(d, kap.y, v.y);
    }
    v.x *= e0;
    v.y *= e0;
  } else {
    v.x = e0 * e[(i - N) % 3];
  }
  bc[idx] = v;
}

// bn[c] = || bc[., c] ||_2, one block per column
__global__ void k_col_norms_c(const double2* bc, int nu, int B, double* bn) {
  const int c = blockIdx.x;
  double t = 0.0;
  for (int i = threadIdx.x; i < nu; i += blockDim.x) {
    const double2 v = bc[(size_t)i * B + c];
    t += v.x * v.x + v.y * v.y;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) bn[c] = sqrt(sh[0]);
}

// ------------------------------------------------------------ Gram-Schmidt
// part[blk][k][a] = sum over the rows of row block blk of conj(V_k[i][a]) W[i][a],
// k in [0, j], in groups of 8 basis vectors per sweep over the rows.
template <class E>
__global__ void __launch_bounds__(256) k_dots(KrylovArgs a, int j) {
  using TT = Tr<E>;
  if (a.jdev) j = *a.jdev;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int col = blockIdx.x * 32 + tx;
  const bool valid = col < a.Bact && a.jconv[col] == 0;   // skip columns that stopped
  __shared__ double2 sh[8][8][32];
  const E* V = static_cast<const E*>(a.V);
  const E* W = static_cast<const E*>(a.W);
  const size_t vstride = (size_t)a.nu * a.Bact;
  // contiguous row range of this block, interleaved over the 8 row lanes
  const int rows_per_blk = (a.nu + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * rows_per_blk;
  const int r1 = min(a.nu, r0 + rows_per_blk);
  for (int k0 = 0; k0 <= j; k0 += 8) {
    const int nk = min(8, j + 1 - k0);   // uniform over the block
    typename TT::Acc acc[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) acc[kk] = TT::zero();
    if (valid) {
      const E* Vk = V + (size_t)k0 * vstride;
      for (int i = r0 + ty; i < r1; i += 8) {
        const size_t off = (size_t)i * a.Bact + col;
        const E w = W[off];
        E v[8];
        // issue every load of this row before any arithmetic
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          if (kk < nk) v[kk] = __ldcs(Vk + (size_t)kk * vstride + off);   // streamed: keep W in L2
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          if (kk < nk) TT::conj_mac(acc[kk], v[kk], w);
      }
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) sh[ty][kk][tx] = TT::to_d2(acc[kk]);
    __syncthreads();
    if (valid && ty < nk) {
      double2 t = make_double2(0.0, 0.0);
      for (int r = 0; r < 8; ++r) {
        t.x += sh[r][ty][tx].x;
        t.y += sh[r][ty][tx].y;
      }
      a.part[((size_t)blockIdx.y * (a.m + 1) + k0 + ty) * a.Bact + col] = t;
    }
    __syncthreads();
  }
}

// h[pass][k][a] = sum_blk part[blk][k][a]
__global__ void k_dots_reduce(KrylovArgs a, int j, int pass) {
  if (a.jdev) j = *a.jdev;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (j + 1) * a.Bact) return;
  int k = idx / a.Bact, col = idx % a.Bact;
  double2 t = make_double2(0.0, 0.0);
  for (int b = 0; b < a.nblk; ++b) {
    double2 v = a.part[((size_t)b * (a.m + 1) + k) * a.Bact + col];
    t.x += v.x;
    t.y += v.y;
  }
  a.h[((size_t)pass * (a.m + 1) + k) * a.Bact + col] = t;
}

// W[i][a] -= sum_k V_k[i][a] h[pass][k][a]; with `last`, also |W|^2 partials.
// The coefficients are staged in shared memory kUpdChunk at a time; a step with more
// basis vectors sweeps W once per chunk (fixed shared memory for any restart length).
constexpr int kUpdChunk = 64;

template <class E>
__global__ void __launch_bounds__(256) k_update(KrylovArgs a, int j, int pass, int last) {
  using TT = Tr<E>;
  using C = typename TT::Coef;
  if (a.jdev) j = *a.jdev;
  __shared__ __align__(16) C shh[kUpdChunk * 32];
  __shared__ double shn[8 * 32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int col = blockIdx.x * 32 + tx;
  const bool valid = col < a.Bact && a.jconv[col] == 0;   // skip columns that stopped
  const E* V = static_cast<const E*>(a.V);
  E* W = static_cast<E*>(a.W);
  typename TT::Acc nacc = TT::zero();
  const size_t vstride = (size_t)a.nu * a.Bact;
  const int rows_per_blk = (a.nu + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * rows_per_blk;
  const int r1 = min(a.nu, r0 + rows_per_blk);
  for (int k0 = 0; k0 <= j; k0 += kUpdChunk) {
    const int kend = min(j + 1, k0 + kUpdChunk);   // uniform over the block
    const bool final_chunk = kend == j + 1;
    if (k0 > 0) __syncthreads();                   // previous chunk's coefficients consumed
    for (int k = k0 + ty; k < kend; k += 8)
      shh[(k - k0) * 32 + tx] = TT::coef(valid ? a.h[((size_t)pass * (a.m + 1) + k) * a.Bact + col]
                                               : make_double2(0.0, 0.0));
    __syncthreads();
    if (valid) {
      for (int i = r0 + ty; i < r1; i += 8) {
        const size_t off = (size_t)i * a.Bact + col;
        const E w0 = W[off];
        typename TT::Acc acc = TT::zero();
        int k = k0;
        for (; k + 8 <= kend; k += 8) {
          E v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) v[q] = __ldcs(V + (size_t)(k + q) * vstride + off);
#pragma unroll
          for (int q = 0; q < 8; ++q) TT::mac(acc, v[q], shh[(k - k0 + q) * 32 + tx]);
        }
        for (; k < kend; ++k) TT::mac(acc, __ldcs(V + (size_t)k * vstride + off), shh[(k - k0) * 32 + tx]);
        const E w = TT::sub(w0, acc);
        W[off] = w;
        if (last && final_chunk) TT::norm_mac(nacc, w);
      }
    }
  }
  if (last) {
    shn[ty * 32 + tx] = TT::norm_d(nacc);
    __syncthreads();
    if (ty == 0 && valid) {
      double t = 0.0;
      for (int r = 0; r < 8; ++r) t += shn[r * 32 + tx];
      a.normpart[(size_t)blockIdx.y * a.Bact + col] = t;
    }
  }
}

// One thread per column: new Hessenberg column, previous rotations, new rotation,
// residual estimate |g_{j+1}|, stop test.
__global__ void k_givens(KrylovArgs a, int j, int passes) {
  if (a.jdev) j = *a.jdev;
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= a.Bact) return;
  const int B = a.Bact, m1 = a.m + 1;
  if (a.jconv[col] > 0) {
    a.inv_h[col] = 0.0;
    return;
  }
  double hn2 = 0.0;
  for (int b = 0; b < a.nblk; ++b) hn2 += a.normpart[(size_t)b * B + col];
  const double hnext = sqrt(hn2);
  double2* Rc = a.R + (size_t)j * m1 * B;   // column j of the rotated Hessenberg
  double colnorm2 = hn2;
  auto hcol = [&](int k) {
    double2 hk = a.h[(size_t)k * B + col];
    if (passes > 1) {
      const double2 h2 = a.h[((size_t)m1 + k) * B + col];
      hk.x += h2.x;
      hk.y += h2.y;
    }
    colnorm2 += hk.x * hk.x + hk.y * hk.y;
    return hk;
  };
  // previous rotations G_k = [c, s; -conj(s), c]; the rotated entry k+1 is carried in
  // a register into rotation k+1
  double2 x0 = hcol(0);
  for (int k = 0; k < j; ++k) {
    const double c = a.cs[(size_t)k * B + col];
    const double2 s = a.sn[(size_t)k * B + col];
    const double2 x1 = hcol(k + 1);
    const double2 sx1 = cmul(s, x1);
    const double2 ncs_x0 = make_double2(-(s.x * x0.x + s.y * x0.y), -(s.x * x0.y - s.y * x0.x));
    Rc[(size_t)k * B + col] = make_double2(c * x0.x + sx1.x, c * x0.y + sx1.y);
    x0 = make_double2(ncs_x0.x + c * x1.x, ncs_x0.y + c * x1.y);
  }
  // new rotation zeroing hnext under the rotated entry j
  const double2 av = x0;
  const double aa = sqrt(av.x * av.x + av.y * av.y);
  const double rho = sqrt(aa * aa + hn2);
  double c;
  double2 s, r;
  if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
    r = make_double2(hnext, 0.0);
  } else {
    const double2 ph = make_double2(av.x / aa, av.y / aa);
    c = aa / rho;
    s = make_double2(ph.x * hnext / rho, ph.y * hnext / rho);
    r = make_double2(ph.x * rho, ph.y * rho);
  }
  a.cs[(size_t)j * B + col] = c;
  a.sn[(size_t)j * B + col] = s;
  Rc[(size_t)j * B + col] = r;
  const double2 gj = a.g[(size_t)j * B + col];
  const double2 gn = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
  a.g[(size_t)j * B + col] = make_double2(c * gj.x, c * gj.y);
  a.g[(size_t)(j + 1) * B + col] = gn;
  const double res = sqrt(gn.x * gn.x + gn.y * gn.y);
  const bool breakdown = hnext <= 1e-14 * sqrt(colnorm2);
  a.inv_h[col] = breakdown ? 0.0 : 1.0 / hnext;
  if (res <= a.target[col] || breakdown || j + 1 == a.m) {
    a.jconv[col] = j + 1;
  } else {
    atomicAdd(&a.active_count[j], 1);
  }
}

template <class E>
__global__ void __launch_bounds__(256) k_normalize(KrylovArgs a, int j, float* X32, double* X64,
                                                   int ldx) {
  using TT = Tr<E>;
  if (a.jdev) j = *a.jdev;
  const int col = blockIdx.x * 32 + threadIdx.x;
  if (col >= a.Bact) return;
  const int jc = a.jconv[col];
  if (jc > 0 && jc <= j) return;   // stopped before this step: V[j+1] is never read
  const double s = a.inv_h[col];
  const E* W = static_cast<const E*>(a.W);
  E* Vn = static_cast<E*>(a.V) + (size_t)(j + 1) * a.nu * a.Bact;
  for (int i = blockIdx.y * 8 + threadIdx.y; i < a.nu; i += 8 * gridDim.y) {
    const size_t off = (size_t)i * a.Bact + col;
    const E v = TT::scale(W[off], s);
    Vn[off] = v;
    write_operand<E>(a, i, col, v, X32, X64, ldx);
  }
}

template <class E>
__global__ void __launch_bounds__(256) k_cycle_start(KrylovArgs a, const int* act, const double2* r,
                                                     int B, const double* beta,
                                                     const double* target_all, float* X32,
                                                     double* X64, int ldx) {
  using TT = Tr<E>;
  const int col = blockIdx.x * 32 + threadIdx.x;
  if (col >= a.Bact) return;
  const int gc = act[col];
  const double bt = beta[gc];
  if (blockIdx.y == 0 && threadIdx.y == 0) {
    a.g[col] = make_double2(bt, 0.0);
    a.target[col] = target_all[gc];
    a.jconv[col] = 0;
  }
  const double s = bt > 0.0 ? 1.0 / bt : 0.0;
  E* V0 = static_cast<E*>(a.V);
  for (int i = blockIdx.y * 8 + threadIdx.y; i < a.nu; i += 8 * gridDim.y) {
    const double2 rv = r[(size_t)i * B + gc];
    const E v = TT::from_d2(make_double2(rv.x * s, rv.y * s));
    V0[(size_t)i * a.Bact + col] = v;
    write_operand<E>(a, i, col, v, X32, X64, ldx);
  }
}

// y = R^{-1} g (upper triangular, size jc) and the implicit-residual coefficients
// u = Omega^H (0, ..., 0, gamma): the inner residual is V_{0..jc} u, |u| = |gamma|.
__global__ void k_backsolve(KrylovArgs a, int jend, const int* act, double* beta, int* iters) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= a.Bact) return;
  const int B = a.Bact, m1 = a.m + 1;
  const int jc = a.jconv[col] > 0 ? a.jconv[col] : jend;
  for (int k = jc - 1; k >= 0; --k) {
    double2 t = a.g[(size_t)k * B + col];
    for (int l = k + 1; l < jc; ++l) {
      const double2 p = cmul(a.R[((size_t)l * m1 + k) * B + col], a.y[(size_t)l * B + col]);
      t.x -= p.x;
      t.y -= p.y;
    }
    const double2 d = a.R[((size_t)k * m1 + k) * B + col];
    const double den = d.x * d.x + d.y * d.y;
    a.y[(size_t)k * B + col] =
        den > 0.0 ? make_double2((t.x * d.x + t.y * d.y) / den, (t.y * d.x - t.x * d.y) / den)
                  : make_double2(0.0, 0.0);
  }
  // u: apply G_k^H = [c, -s; conj(s), c] for k = jc-1 .. 0 to gamma e_jc
  const double2 gamma = a.g[(size_t)jc * B + col];
  double2 carry = gamma;   // u_{k+1} before the update at step k
  for (int k = jc - 1; k >= 0; --k) {
    const double c = a.cs[(size_t)k * B + col];
    const double2 s = a.sn[(size_t)k * B + col];
    const double2 sc = cmul(s, carry);
    a.u[(size_t)(k + 1) * B + col] = make_double2(c * carry.x, c * carry.y);
    carry = make_double2(-sc.x, -sc.y);
  }
  a.u[col] = carry;
  a.jconv[col] = jc;
  const int gc = act[col];
  beta[gc] = sqrt(gamma.x * gamma.x + gamma.y * gamma.y);
  iters[gc] += jc;
}

// x[., act[a]] += sum_{k<jc} V_k y_k ;  r[., act[a]] = sum_{k<=jc} V_k u_k  (FP64 sums;
// r is required).  Each thread keeps four rows' sums in registers per sweep over a chunk
// of 32 basis vectors whose y, u coefficients are staged in shared memory, so four loads
// of V are in flight per thread.  Per-row-block partial sums of |r|^2 go to
// normpart[blk][a]: the norm of the implicit residual V u equals |gamma| only while the
// basis is orthonormal, and the next cycle is normalised by the measured norm, so a
// basis that lost orthogonality (FP32 classical Gram-Schmidt on a slowly converging
// column) cannot mis-scale it.
template <class E>
__global__ void __launch_bounds__(256) k_xupdate(KrylovArgs a, const int* act, double2* x,
                                                 double2* r, int B) {
  using TT = Tr<E>;
  constexpr int kXChunk = 32, kRows = 4;
  using C = typename TT::Coef;
  // y and u in the basis's own arithmetic (FP32 for the FP32 basis: GB300's FP64 pipe is
  // 1/64 of its FP32 rate, and the correction needs no more than the basis carries)
  __shared__ C shy[kXChunk][32], shu[kXChunk][32];
  __shared__ double sh[8][32];
  __shared__ int sh_jmax;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int col = blockIdx.x * 32 + tx;
  const bool valid = col < a.Bact;
  const int jc = valid ? a.jconv[col] : 0;
  // basis vectors the block reads: the largest jc of its 32 columns (every warp of the
  // block holds the same columns)
  int jmax = jc;
  for (int o = 16; o > 0; o >>= 1) jmax = max(jmax, __shfl_xor_sync(0xffffffffu, jmax, o));
  if (tx == 0 && ty == 0) sh_jmax = jmax;
  __syncthreads();
  jmax = sh_jmax;
  const size_t vstride = (size_t)a.nu * a.Bact;
  const E* V = static_cast<const E*>(a.V);
  const int rows_per_blk = (a.nu + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * rows_per_blk;
  const int r1 = min(a.nu, r0 + rows_per_blk);
  const int nrows = max(0, (r1 - r0 - ty + 7) / 8);   // rows r0 + ty + 8 q of this thread
  const int gc = valid ? act[col] : 0;
  double nrm = 0.0;
  for (int k0 = 0; k0 <= jmax; k0 += kXChunk) {
    const int kend = min(jmax + 1, k0 + kXChunk);   // uniform over the block
    if (k0 > 0) __syncthreads();                    // previous chunk consumed
    for (int k = k0 + ty; k < kend; k += 8) {
      shy[k - k0][tx] = TT::coef((valid && k < jc) ? a.y[(size_t)k * a.Bact + col] : make_double2(0.0, 0.0));
      shu[k - k0][tx] = TT::coef((valid && k <= jc) ? a.u[(size_t)k * a.Bact + col] : make_double2(0.0, 0.0));
    }
    __syncthreads();
    if (!valid) continue;
    const bool first = k0 == 0, last = kend == jmax + 1;
    for (int rb = 0; rb < nrows; rb += kRows) {
      typename TT::Acc dxa[kRows], ara[kRows];
#pragma unroll
      for (int q = 0; q < kRows; ++q) dxa[q] = ara[q] = TT::zero();
      for (int k = k0; k < kend; ++k) {
        const C yk = shy[k - k0][tx], uk = shu[k - k0][tx];
        E v[kRows];
#pragma unroll
        for (int q = 0; q < kRows; ++q)
          if (rb + q < nrows)
            v[q] = V[(size_t)k * vstride + (size_t)(r0 + ty + 8 * (rb + q)) * a.Bact + col];
#pragma unroll
        for (int q = 0; q < kRows; ++q) {
          if (rb + q >= nrows) continue;
          TT::mac(ara[q], v[q], uk);
          TT::mac(dxa[q], v[q], yk);
        }
      }
#pragma unroll
      for (int q = 0; q < kRows; ++q) {
        if (rb + q >= nrows) continue;
        const int i = r0 + ty + 8 * (rb + q);
        const double2 arq = TT::to_d2(ara[q]);
        // x += M V y with M = alpha^IB on the dipole rows (right preconditioner)
        double2 d = TT::to_d2(dxa[q]);
        if (a.amu && i >= a.N) d = cmul(a.amu[(size_t)a.type[(i - a.N) / 3] * a.Bact + col], d);
        double2 ax = x[(size_t)i * B + gc];
        ax.x += d.x;
        ax.y += d.y;
        x[(size_t)i * B + gc] = ax;
        double2 rv = first ? make_double2(0.0, 0.0) : r[(size_t)i * B + gc];
        rv.x += arq.x;
        rv.y += arq.y;
        r[(size_t)i * B + gc] = rv;
        if (last) nrm += rv.x * rv.x + rv.y * rv.y;
      }
    }
  }
  sh[ty][tx] = nrm;
  __syncthreads();
  if (ty == 0 && valid) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += sh[k][tx];
    a.normpart[(size_t)blockIdx.y * a.Bact + col] = t;
  }
}

// beta[act[a]] = || V u ||, the measured norm of the implicit residual
__global__ void k_beta_measured(KrylovArgs a, const int* act, double* beta) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= a.Bact) return;
  double t = 0.0;
  for (int b = 0; b < a.nblk; ++b) t += a.normpart[(size_t)b * a.Bact + col];
  beta[act[col]] = sqrt(t);
}

__global__ void __launch_bounds__(256) k_gather_x(const double2* x, int B, const int* act,
                                                  int Bact, int nu, double* X64, int ldx) {
  const int col = blockIdx.x * 32 + threadIdx.x;
  if (col >= Bact) return;
  const int gc = act[col];
  for (int i = blockIdx.y * 8 + threadIdx.y; i < nu; i += 8 * gridDim.y)
    *reinterpret_cast<double2*>(X64 + (size_t)i * ldx + 2 * col) = x[(size_t)i * B + gc];
}

// End of one Krylov step inside a captured restart cycle: advance the device step
// index and tell the enclosing while-loop node whether to run another step (some
// column still iterating and the basis not full).  The index grows by one per step, so
// the loop ends after at most m steps whatever the data.
__global__ void k_step_advance(int* jdev, const int* active_count, int m,
                               cudaGraphConditionalHandle loop) {
  const int j = *jdev;
  const bool more = j + 1 < m && active_count[j] > 0;
  *jdev = j + 1;
  cudaGraphSetConditional(loop, more ? 1u : 0u);
}

__global__ void k_norm_finish(const double* normpart, int nblk, int Bact, const int* act, int P,
                              const double* bnorm, double inner_tol, double tol_abs_frac,
                              double* rnorm, double* beta, double* target_all) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= Bact) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t += normpart[(size_t)b * Bact + col];
  const int gc = act[col];
  const double rn = sqrt(t);
  rnorm[gc] = rn;
  beta[gc] = rn;
  target_all[gc] = round_target(inner_tol * rn, tol_abs_frac * bnorm[gc % P]);
}

inline dim3 col_grid(int Bact, int nblk) { return dim3((Bact + 31) / 32, nblk); }

// Calls f with a value of the basis element type selected by `basis`.
template <class F>
void with_basis(int basis, F&& f) {
  if (basis == kBasisFF) f(float4{});
  else if (basis == kBasisF32) f(float2{});
  else f(double2{});
}

}  // namespace

int reduction_blocks(int nu) {
  int nb = (nu + 63) / 64;
  if (nb > 128) nb = 128;
  if (nb < 1) nb = 1;
  return nb;
}

cudaError_t launch_shift(const ShiftArgs& a, cudaStream_t s, long long* nl) {
  dim3 grd = col_grid(a.Bact, a.nblk), blk(32, 8);
  with_basis(a.basis, [&](auto e) {
    using E = decltype(e);
    if (a.y_is_f32) k_shift<E, true><<<grd, blk, 0, s>>>(a);
    else k_shift<E, false><<<grd, blk, 0, s>>>(a);
  });
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_resid(const ResidArgs& a, cudaStream_t s, long long* nl) {
  k_resid<<<col_grid(a.Bact, a.nblk), dim3(32, 8), 0, s>>>(a);
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

cudaError_t launch_rhs_hetero(int N, int F, int P, const int* rowptr, const int* col,
                              const double* val64, const int* type, int ntypes,
                              const double2* kappa, const double* pos, const double* pol,
                              double e0, double2* bc, double* bn, cudaStream_t s, long long* nl) {
  const int B = F * P;
  const size_t n = (size_t)4 * N * B;
  k_rhs_hetero<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(N, F, P, rowptr, col, val64, type, ntypes,
                                                          kappa, pos, pol, e0, bc);
  k_col_norms_c<<<B, 256, 0, s>>>(bc, 4 * N, B, bn);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_col_norms_c(const double2* bc, int nu, int B, double* bn, cudaStream_t s,
                               long long* nl) {
  k_col_norms_c<<<B, 256, 0, s>>>(bc, nu, B, bn);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_dots(const KrylovArgs& a, int j, int pass, cudaStream_t s, long long* nl) {
  with_basis(a.basis, [&](auto e) {
    k_dots<decltype(e)><<<col_grid(a.Bact, a.nblk), dim3(32, 8), 0, s>>>(a, j);
  });
  // with a device step index the reduction grid covers the longest step of the cycle
  int n = ((a.jdev ? a.m : j) + 1) * a.Bact;
  k_dots_reduce<<<(n + 255) / 256, 256, 0, s>>>(a, j, pass);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_update(const KrylovArgs& a, int j, int pass, bool last, cudaStream_t s,
                          long long* nl) {
  with_basis(a.basis, [&](auto e) {
    k_update<decltype(e)><<<col_grid(a.Bact, a.nblk), dim3(32, 8), 0, s>>>(a, j, pass, last);
  });
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_step_advance(int* jdev, const int* active_count, int m,
                                cudaGraphConditionalHandle loop, cudaStream_t s, long long* nl) {
  k_step_advance<<<1, 1, 0, s>>>(jdev, active_count, m, loop);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_givens(const KrylovArgs& a, int j, int passes, cudaStream_t s, long long* nl) {
  k_givens<<<(a.Bact + 127) / 128, 128, 0, s>>>(a, j, passes);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_normalize(const KrylovArgs& a, int j, float* X32, double* X64, int ldx,
                             cudaStream_t s, long long* nl) {
  with_basis(a.basis, [&](auto e) {
    k_normalize<decltype(e)><<<col_grid(a.Bact, a.nblk), dim3(32, 8), 0, s>>>(a, j, X32, X64, ldx);
  });
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_cycle_start(const KrylovArgs& a, const int* act, const double2* r, int B,
                               const double* beta, const double* target_all, float* X32,
                               double* X64, int ldx, cudaStream_t s, long long* nl) {
  with_basis(a.basis, [&](auto e) {
    k_cycle_start<decltype(e)><<<col_grid(a.Bact, a.nblk), dim3(32, 8), 0, s>>>(
        a, act, r, B, beta, target_all, X32, X64, ldx);
  });
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_cycle_end(const KrylovArgs& a, int jend, const int* act, double2* x,
                             double2* r, int B, double* beta, int* iters, cudaStream_t s,
                             long long* nl) {
  k_backsolve<<<(a.Bact + 127) / 128, 128, 0, s>>>(a, jend, act, beta, iters);
  with_basis(a.basis, [&](auto e) {
    k_xupdate<decltype(e)><<<col_grid(a.Bact, a.nblk), dim3(32, 8), 0, s>>>(a, act, x, r, B);
  });
  k_beta_measured<<<(a.Bact + 127) / 128, 128, 0, s>>>(a, act, beta);
  *nl += 3;
  return cudaGetLastError();
}

cudaError_t launch_norm_finish(const double* normpart, int nblk, int Bact, const int* act, int P,
                               const double* bnorm, double inner_tol, double tol_abs_frac,
                               double* rnorm, double* beta, double* target_all, cudaStream_t s,
                               long long* nl) {
  k_norm_finish<<<(Bact + 127) / 128, 128, 0, s>>>(normpart, nblk, Bact, act, P, bnorm, inner_tol,
                                                   tol_abs_frac, rnorm, beta, target_all);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_gather_x(const double2* x, int B, const int* act, int Bact, int nu,
                            double* X64, int ldx, cudaStream_t s, long long* nl) {
  int nblk = reduction_blocks(nu);
  k_gather_x<<<col_grid(Bact, nblk), dim3(32, 8), 0, s>>>(x, B, act, Bact, nu, X64, ldx);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace px
