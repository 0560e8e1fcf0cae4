// Induced density, potential and field maps of solved columns at probe points
// (Sec. "Post-process Analysis": the density and field maps of a structure at a plasmon
// resonance).  An all-pairs kernel, probe points x atoms, on the same Gaussian kernel as
// Eq. 5 and its derivatives (Sec. 2.2), applied to the solved charges and dipoles.
//
// The model's charge on atom i is the normalised Gaussian density q_i g(r - r_i; R_q,i),
// g(x; R) = (pi R^2)^(-3/2) exp(-|x|^2 / R^2), and its dipole the density
// -mu_i . grad g(r - r_i; R_mu,i).  With G(x; R) = erf(|x| / R) / |x|, the potential of
// g (G(0) = 2 / (sqrt(pi) R)):
//     rho(r) = sum_i q_i g(x_i; R_q,i) + (2 / R_mu,i^2) (mu_i . x_i) g(x_i; R_mu,i)
//     phi(r) = sum_i q_i G(x_i; R_q,i) - mu_i . grad G(x_i; R_mu,i)
//     E(r)   = -grad phi(r),                    x_i = r - r_i.
// The paper names the maps without printing formulas; these follow from the densities.
//
// Arithmetic: the radial functions G, G'/r and G'' in FP32 (erff, expf; a Taylor series
// below x = |x_i| / R = 0.25, where the closed forms cancel), per-pair contributions
// summed in FP32 over a tile of 128 atoms and the tile sums accumulated in FP64.  The
// kernel is bound by the FP32 / SFU pipes (about 60 operations per pair plus ~50 per
// column).
#include "px.h"
#include "px_internal.cuh"
#include "px_handle.cuh"
#include "px_radial.cuh"

#include <cmath>
#include <string>
#include <vector>

namespace {

constexpr int kFTile = 128;   // atoms per shared-memory tile
constexpr int kFCols = 2;     // columns per block (grid y covers the rest)
constexpr float kInvSqrtPi = 0.56418958354775628f;

__device__ __forceinline__ void radial(float r, float R, float& G, float& G1r, float& G2,
                                       float& g) {
  px::radial::eval_f(r, R, G, G1r, G2, g);
}

struct FieldArgs {
  int N, M, C;                 // atoms, probe points, columns
  const double* pos;           // [N][3] bohr, internal order
  const double* Rq;            // [N]
  const double* Rmu;           // [N]
  const int* perm;             // [N] caller index of internal atom a
  const double* points;        // [M][3] bohr
  const double2* q;            // [C][N] caller order
  const double2* mu;           // [C][N][3] caller order, or null
  double2* rho;                // [C][M] or null
  double2* phi;                // [C][M] or null
  double2* E;                  // [C][M][3] or null
};

// One thread per probe point, kFCols columns per block row of the grid.
__global__ void __launch_bounds__(128) k_fields(FieldArgs a) {
  __shared__ float4 sp[kFTile];                   // x, y, z, R_q
  __shared__ float sRm[kFTile];
  __shared__ float2 sq[kFCols][kFTile];
  __shared__ float2 smu[kFCols][kFTile][3];
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int c0 = blockIdx.y * kFCols;
  const int nc = min(kFCols, a.C - c0);
  const bool valid = m < a.M;
  // coordinates relative to the block's first probe point, differences taken in FP64:
  // the FP32 pair differences below then lose only ~1e-7 of the block's own extent
  const size_t mref = (size_t)blockIdx.x * blockDim.x;
  const double rx = a.points[3 * mref], ry = a.points[3 * mref + 1], rz = a.points[3 * mref + 2];
  float px = 0.f, py = 0.f, pz = 0.f;
  if (valid) {
    px = (float)(a.points[3 * (size_t)m] - rx);
    py = (float)(a.points[3 * (size_t)m + 1] - ry);
    pz = (float)(a.points[3 * (size_t)m + 2] - rz);
  }
  // FP64 accumulators: rho (2), phi (2), E (6) per column
  double acc[kFCols][10];
#pragma unroll
  for (int c = 0; c < kFCols; ++c)
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[c][k] = 0.0;
  const bool with_mu = a.mu != nullptr;
  for (int t0 = 0; t0 < a.N; t0 += kFTile) {
    const int nt = min(kFTile, a.N - t0);
    __syncthreads();
    for (int k = threadIdx.x; k < nt; k += blockDim.x) {
      const int at = t0 + k;
      sp[k] = make_float4((float)(a.pos[3 * (size_t)at] - rx), (float)(a.pos[3 * (size_t)at + 1] - ry),
                          (float)(a.pos[3 * (size_t)at + 2] - rz), (float)a.Rq[at]);
      sRm[k] = (float)a.Rmu[at];
      const int io = a.perm[at];
      for (int c = 0; c < kFCols; ++c) {
        const double2 qv = c < nc ? a.q[(size_t)(c0 + c) * a.N + io] : make_double2(0.0, 0.0);
        sq[c][k] = make_float2((float)qv.x, (float)qv.y);
        if (with_mu)
          for (int d = 0; d < 3; ++d) {
            const double2 mv =
                c < nc ? a.mu[((size_t)(c0 + c) * a.N + io) * 3 + d] : make_double2(0.0, 0.0);
            smu[c][k][d] = make_float2((float)mv.x, (float)mv.y);
          }
      }
    }
    __syncthreads();
    if (!valid) continue;
    float tacc[kFCols][10];
#pragma unroll
    for (int c = 0; c < kFCols; ++c)
#pragma unroll
      for (int k = 0; k < 10; ++k) tacc[c][k] = 0.f;
    for (int k = 0; k < nt; ++k) {
      const float4 p4 = sp[k];
      const float dx = px - p4.x, dy = py - p4.y, dz = pz - p4.z;
      const float r = sqrtf(dx * dx + dy * dy + dz * dz);
      float Gq, G1q, G2q, gq;
      radial(r, p4.w, Gq, G1q, G2q, gq);
      float Gm = 0.f, G1m = 0.f, G2m = 0.f, gm = 0.f, Rm = 1.f;
      if (with_mu) {
        Rm = sRm[k];
        radial(r, Rm, Gm, G1m, G2m, gm);
      }
#pragma unroll
      for (int c = 0; c < kFCols; ++c) {
        // columns beyond nc hold zeros in shared memory (staged below) and are not written
        const float2 q = sq[c][k];
        // charge: rho += q g; phi += q G; E = -grad(q G) = -q G'(r) x / r
        tacc[c][0] = fmaf(q.x, gq, tacc[c][0]);
        tacc[c][1] = fmaf(q.y, gq, tacc[c][1]);
        tacc[c][2] = fmaf(q.x, Gq, tacc[c][2]);
        tacc[c][3] = fmaf(q.y, Gq, tacc[c][3]);
        tacc[c][4] = fmaf(-q.x * G1q, dx, tacc[c][4]);
        tacc[c][5] = fmaf(-q.y * G1q, dx, tacc[c][5]);
        tacc[c][6] = fmaf(-q.x * G1q, dy, tacc[c][6]);
        tacc[c][7] = fmaf(-q.y * G1q, dy, tacc[c][7]);
        tacc[c][8] = fmaf(-q.x * G1q, dz, tacc[c][8]);
        tacc[c][9] = fmaf(-q.y * G1q, dz, tacc[c][9]);
        if (with_mu) {
          const float2 mx = smu[c][k][0], my = smu[c][k][1], mz = smu[c][k][2];
          // mu . x (complex)
          const float mdr = mx.x * dx + my.x * dy + mz.x * dz;
          const float mdi = mx.y * dx + my.y * dy + mz.y * dz;
          // rho += (2 / R^2) (mu . x) g;  phi += -(mu . x) G'(r) / r
          const float w = 2.0f / (Rm * Rm) * gm;
          tacc[c][0] = fmaf(w, mdr, tacc[c][0]);
          tacc[c][1] = fmaf(w, mdi, tacc[c][1]);
          tacc[c][2] = fmaf(-G1m, mdr, tacc[c][2]);
          tacc[c][3] = fmaf(-G1m, mdi, tacc[c][3]);
          // E = grad((mu . x) G'/r) = (G'/r) mu + (mu . x) x (G'' - G'/r) / r^2, with the
          // r -> 0 limit (G'' - G'/r) / r^2 -> (c/R^2)(4/5) / R^2
          float h;
          if (r * (1.0f / Rm) < 0.25f) {
            const float iR = 1.0f / Rm;
            const float x2 = r * r * iR * iR;
            h = 2.0f * kInvSqrtPi * iR * iR * iR * iR * iR *
                (0.8f - x2 * (4.0f / 7.0f) + x2 * x2 * (2.0f / 9.0f));
          } else {
            h = (G2m - G1m) / (r * r);
          }
          tacc[c][4] = fmaf(G1m, mx.x, fmaf(h * mdr, dx, tacc[c][4]));
          tacc[c][5] = fmaf(G1m, mx.y, fmaf(h * mdi, dx, tacc[c][5]));
          tacc[c][6] = fmaf(G1m, my.x, fmaf(h * mdr, dy, tacc[c][6]));
          tacc[c][7] = fmaf(G1m, my.y, fmaf(h * mdi, dy, tacc[c][7]));
          tacc[c][8] = fmaf(G1m, mz.x, fmaf(h * mdr, dz, tacc[c][8]));
          tacc[c][9] = fmaf(G1m, mz.y, fmaf(h * mdi, dz, tacc[c][9]));
        }
      }
    }
#pragma unroll
    for (int c = 0; c < kFCols; ++c)
#pragma unroll
      for (int k = 0; k < 10; ++k) acc[c][k] += (double)tacc[c][k];
  }
  if (!valid) return;
  for (int c = 0; c < nc; ++c) {
    const size_t o = (size_t)(c0 + c) * a.M + m;
    if (a.rho) a.rho[o] = make_double2(acc[c][0], acc[c][1]);
    if (a.phi) a.phi[o] = make_double2(acc[c][2], acc[c][3]);
    if (a.E)
      for (int d = 0; d < 3; ++d) a.E[o * 3 + d] = make_double2(acc[c][4 + 2 * d], acc[c][5 + 2 * d]);
  }
}

px_status fail_f(px_handle* h, px_status st, const std::string& msg) {
  px_set_error(h, msg);
  return st;
}

}  // namespace

extern "C" px_status px_fields(px_handle* h, int n_points, const double* points_ang, int n_cols,
                               const double* d_q, const double* d_mu, double* d_rho,
                               double* d_phi, double* d_E, void* cuda_stream) {
  if (!h) return PX_EINVAL;
  const px::DevStructure* dsp = px_structure(h);
  if (!dsp) return fail_f(h, PX_EINVAL, "no structure loaded");
  const px::DevStructure& d = *dsp;
  if (d.bem) return fail_f(h, PX_ENOTIMPL, "field maps of a mesh are not implemented");
  if (n_points < 1 || n_cols < 1 || !points_ang || !d_q)
    return fail_f(h, PX_EINVAL, "need n_points >= 1, n_cols >= 1, points_ang and d_q");
  if (d_mu && d.model != PX_WFQFMU) return fail_f(h, PX_EINVAL, "d_mu is only meaningful for PX_WFQFMU");
  if ((long long)n_points * n_cols > (1LL << 31))
    return fail_f(h, PX_EINVAL, "n_points x n_cols too large");
  constexpr double kBohrAng = 0.529177210903;
  std::vector<double> pts(3 * (size_t)n_points);
  for (size_t k = 0; k < pts.size(); ++k) {
    if (!std::isfinite(points_ang[k])) return fail_f(h, PX_EINVAL, "non-finite probe point");
    pts[k] = points_ang[k] / kBohrAng;
  }
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : px_stream(h);
  double* dp = nullptr;
  cudaError_t e = cudaMalloc(&dp, sizeof(double) * pts.size());
  if (e != cudaSuccess) return fail_f(h, PX_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(dp, pts.data(), sizeof(double) * pts.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    FieldArgs a;
    a.N = d.N;
    a.M = n_points;
    a.C = n_cols;
    a.pos = d.pos64;
    a.Rq = d.Rq;
    a.Rmu = d.Rmu;
    a.perm = d.perm;
    a.points = dp;
    a.q = reinterpret_cast<const double2*>(d_q);
    a.mu = reinterpret_cast<const double2*>(d_mu);
    a.rho = reinterpret_cast<double2*>(d_rho);
    a.phi = reinterpret_cast<double2*>(d_phi);
    a.E = reinterpret_cast<double2*>(d_E);
    dim3 grd((n_points + 127) / 128, (n_cols + kFCols - 1) / kFCols);
    k_fields<<<grd, 128, 0, s>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dp);
  if (e != cudaSuccess) return fail_f(h, PX_ECUDA, std::string("px_fields: ") + cudaGetErrorString(e));
  return PX_OK;
}
