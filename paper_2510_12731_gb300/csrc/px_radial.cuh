// Radial functions of the Gaussian kernel of Eq. 5 and its derivatives (Sec. 2.2):
//   G(r) = erf(r/R)/r,   G'(r)/r,   G''(r)   (and the normalised Gaussian g(r; R))
// and the 4 x 4 wFQFmu blocks of an atom pair built from them (FP32).
// For x = r/R below 0.25 the closed forms cancel (G' and G'' are O(x) and O(1) differences
// of O(1/x) terms), so a Taylor series of erf is used there:
//   G    = c (1 - x^2/3 + x^4/10 - x^6/42)
//   G'/r = (c/R^2)(-2/3 + 2x^2/5 - x^4/7 + x^6/27)
//   G''  = (c/R^2)(-2/3 + 6x^2/5 - 5x^4/7 + 7x^6/27),      c = 2 / (sqrt(pi) R)
// (the next terms are below 3e-7 relative at x = 0.25).
#pragma once
#include <cuda_runtime.h>

namespace px {
namespace radial {

constexpr float kInvSqrtPiF = 0.56418958354775628f;

__device__ __forceinline__ void eval_f(float r, float R, float& G, float& G1r, float& G2,
                                       float& g) {
  const float iR = 1.0f / R;
  const float x = r * iR;
  const float x2 = x * x;
  const float ex = __expf(-x2);
  const float c = 2.0f * kInvSqrtPiF * iR;
  g = kInvSqrtPiF * kInvSqrtPiF * kInvSqrtPiF * iR * iR * iR * ex;
  if (x < 0.25f) {
    const float x4 = x2 * x2, x6 = x4 * x2;
    G = c * (1.0f - x2 * (1.0f / 3.0f) + x4 * 0.1f - x6 * (1.0f / 42.0f));
    const float cr = c * iR * iR;
    G1r = cr * (-2.0f / 3.0f + 0.4f * x2 - x4 * (1.0f / 7.0f) + x6 * (1.0f / 27.0f));
    G2 = cr * (-2.0f / 3.0f + 1.2f * x2 - x4 * (5.0f / 7.0f) + x6 * (7.0f / 27.0f));
  } else {
    const float e = erff(x);
    const float ir = 1.0f / r;
    const float gx = 2.0f * kInvSqrtPiF * ex;   // d erf / dx
    G = e * ir;
    const float G1 = (gx * iR - e * ir) * ir;   // G'(r)
    G1r = G1 * ir;
    G2 = (-2.0f * x * gx * iR * iR - 2.0f * gx * iR * ir + 2.0f * e * ir * ir) * ir;
  }
}

// wFQ charge-charge kernel (Eq. 5) in FP32 from (x, y, z, R_q^2) of two atoms (bohr):
// erf(r/R)/r with R^2 = R_q,a^2 + R_q,b^2, the r -> 0 limit sqrt(2/pi)/R_q on the diagonal;
// erf(r/R) = 1 to FP32 precision beyond r/R = 4, where one reciprocal square root remains.
constexpr float kSqrt2OverPiF = 0.79788456080286536f;
__device__ __forceinline__ float tqq_f(float4 a, float4 b, bool same) {
  if (same) return kSqrt2OverPiF * rsqrtf(a.w);
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float R2 = a.w + b.w;
  if (r2 < 16.0f * R2) {
    const float r = sqrtf(r2);
    return erff(r * rsqrtf(R2)) / r;
  }
  return rsqrtf(r2);
}

// The 4 x 4 block of the wFQFmu kernel (Sec. 2.2) of atoms a != b, unknowns (q, mu_x, mu_y,
// mu_z) of each: blk[0][0] = T^qq, blk[0][1+l] = T^qmu_l = -T'(r; R_q,a mu,b) rhat_l,
// blk[1+k][0] = T^muq_k = +T'(r; R_mu,a q,b) rhat_k,
// blk[1+k][1+l] = T^mumu_kl = -[T'' rhat_k rhat_l + (T'/r)(delta_kl - rhat_k rhat_l)],
// rhat = (r_a - r_b)/r, pair widths sqrt(R_a^2 + R_b^2) of the two densities involved.
// With T' rhat = (T'/r) (r_a - r_b), only G'/r and G'' enter.  Equal charge and dipole
// widths (the usual case) need one radial evaluation instead of four.
__device__ __forceinline__ void pair_block_f(float4 pa, float rma2, float4 pb, float rmb2,
                                             float blk[4][4]) {
  const float d[3] = {pa.x - pb.x, pa.y - pb.y, pa.z - pb.z};
  const float r2 = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
  const float r = sqrtf(r2), ir = 1.0f / r;
  float Gqq, t1, t2, g;
  float G1qm, G1mq, G1mm, G2mm;
  radial::eval_f(r, sqrtf(pa.w + pb.w), Gqq, t1, t2, g);
  if (pa.w == rma2 && pb.w == rmb2) {
    G1qm = G1mq = G1mm = t1;
    G2mm = t2;
  } else {
    float u0, u2;
    radial::eval_f(r, sqrtf(pa.w + rmb2), u0, G1qm, u2, g);
    radial::eval_f(r, sqrtf(rma2 + pb.w), u0, G1mq, u2, g);
    radial::eval_f(r, sqrtf(rma2 + rmb2), u0, G1mm, G2mm, g);
  }
  blk[0][0] = Gqq;
  const float rh[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
#pragma unroll
  for (int l = 0; l < 3; ++l) blk[0][1 + l] = -G1qm * d[l];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    blk[1 + k][0] = G1mq * d[k];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const float rr = rh[k] * rh[l];
      blk[1 + k][1 + l] = -(G2mm * rr + G1mm * ((k == l ? 1.0f : 0.0f) - rr));
    }
  }
}

// Diagonal 4 x 4 block of atom a: T^qq self limit, zero charge-dipole coupling, T^mumu = 0 or
// the Gaussian self term 4/(3 sqrt(pi) R^3) I with R = sqrt(2) R_mu (mu_self_term).
__device__ __forceinline__ void self_block_f(float rq2, float rm2, int mu_self, float blk[4][4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int l = 0; l < 4; ++l) blk[k][l] = 0.f;
  blk[0][0] = kSqrt2OverPiF * rsqrtf(rq2);
  if (mu_self) {
    const float R2 = 2.0f * rm2;   // R = sqrt(2) R_mu
    const float v = 4.0f / (3.0f * 1.7724538509055159f) * rsqrtf(R2) / R2;
    blk[1][1] = blk[2][2] = blk[3][3] = v;
  }
}

}  // namespace radial
}  // namespace px
