// Matrix-free block matvec Y = T X: the T tile of every K step is generated from the
// atom positions inside the GEMM ("on the fly", Sec. "Solvers"), never stored.
//
// T_ik = erf(r/R)/r with R^2 = R_q,i^2 + R_q,k^2 (Eq. 5), T_ii = sqrt(2/pi)/R_q,i; the
// erf is evaluated only for close pairs (r/R < 4 in FP32, < 6 in FP64, beyond which
// erf(r/R) = 1 to the working precision), far pairs cost one reciprocal square root.
// Tiling as in k_gemm_simt.cu: the X tile is staged with cp.async, the generated T
// tile is written to shared memory one stage ahead of the FMA loop.  Rows / columns
// beyond the n real atoms generate 0.
#include "px_ff.cuh"
#include "px_internal.cuh"
#include "px_radial.cuh"

namespace px {

namespace {

constexpr double kSqrt2OverPiD = 0.7978845608028654;
using radial::tqq_f;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n"); }

__global__ void __launch_bounds__(256, 2)
k_sgemm_mf(const float4* __restrict__ pos, int n, const float* __restrict__ X, int ldx,
           float* __restrict__ Y, int ldy, int K) {
  constexpr int BM = 128, BN = 128, BK = 16;
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  __shared__ float4 Pi[BM];
  __shared__ float4 Pk[3][BK];   // positions of K blocks kt, kt+1, kt+2 (one barrier per step)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  const float* Bb = X + c0;
  if (tid < BM) Pi[tid] = (i0 + tid < n) ? pos[i0 + tid] : make_float4(0.f, 0.f, 0.f, 1.f);

  auto load_x = [&](int st, int k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int idx = tid + r * 256;
      const int kk = idx >> 5, cc = (idx & 31) * 4;
      cp_async16(&Bs[st][kk][cc], Bb + (size_t)(k0 + kk) * ldx + cc);
    }
    cp_async_commit();
  };
  auto load_pk = [&](int st, int k0) {
    if (tid < BK) Pk[st][tid] = (k0 + tid < n) ? pos[k0 + tid] : make_float4(0.f, 0.f, 0.f, 1.f);
  };
  // each thread generates 8 entries of the BK x BM tile: row ii = tid % 128 of the block,
  // K offsets kk = tid / 128 + 2 q
  const int gi_local = tid & (BM - 1);
  const int kk_base = tid >> 7;
  auto gen = [&](int st, int ps, int k0) {
    const float4 pi = Pi[gi_local];
    const int gi = i0 + gi_local;
#pragma unroll
    for (int q = 0; q < BK / 2; ++q) {
      const int kk = kk_base + 2 * q;
      const int gk = k0 + kk;
      float v = 0.f;
      if (gi < n && gk < n) v = tqq_f(pi, Pk[ps][kk], gi == gk);
      As[st][kk][gi_local] = v;
    }
  };

  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

  const int nk = K / BK;
  load_pk(0, 0);
  load_x(0, 0);
  __syncthreads();
  gen(0, 0, 0);
  if (nk > 1) load_pk(1, BK);
  cp_async_wait_all();
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1, nx = st ^ 1;
    // slot (kt + 2) % 3 was last read by the generation of block kt - 1, before the
    // previous barrier
    if (kt + 2 < nk) load_pk((kt + 2) % 3, (kt + 2) * BK);
    if (kt + 1 < nk) {
      load_x(nx, (kt + 1) * BK);
      gen(nx, (kt + 1) % 3, (kt + 1) * BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[st][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[st][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[st][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[st][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    cp_async_wait_all();
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int row = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
    float* yr = Y + (size_t)row * ldy + c0;
    *reinterpret_cast<float4*>(yr + tx * 4) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    *reinterpret_cast<float4*>(yr + 64 + tx * 4) =
        make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
  }
}

// FP64 variant for the true residual: 64 x 64 output tiles, generated FP64 T tile.
__device__ __forceinline__ double tqq_d(const double* pi, const double* pk, bool same) {
  if (same) return kSqrt2OverPiD / sqrt(pi[3]);
  const double dx = pi[0] - pk[0], dy = pi[1] - pk[1], dz = pi[2] - pk[2];
  const double r2 = dx * dx + dy * dy + dz * dz;
  const double R2 = pi[3] + pk[3];
  const double r = sqrt(r2);
  if (r2 < 36.0 * R2) return erf(r / sqrt(R2)) / r;
  return 1.0 / r;
}

__global__ void __launch_bounds__(256)
k_dgemm_mf(const double* __restrict__ pos /* [n][4]: x y z Rq^2 */, int n,
           const double* __restrict__ X, int ldx, double* __restrict__ Y, int ldy, int K) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ __align__(16) double As[BK][BM];
  __shared__ __align__(16) double Bs[BK][BN];
  __shared__ double Pi[BM][4];
  __shared__ double Pk[BK][4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  if (tid < BM)
    for (int q = 0; q < 4; ++q) Pi[tid][q] = (i0 + tid < n) ? pos[4 * (size_t)(i0 + tid) + q] : 1.0;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  const int nk = K / BK;
  for (int kt = 0; kt < nk; ++kt) {
    const int k0 = kt * BK;
    if (tid < BK)
      for (int q = 0; q < 4; ++q) Pk[tid][q] = (k0 + tid < n) ? pos[4 * (size_t)(k0 + tid) + q] : 1.0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int idx = tid + r * 256;
      const int kk = idx >> 5, cc = (idx & 31) * 2;
      cp_async16(&Bs[kk][cc], X + (size_t)(k0 + kk) * ldx + c0 + cc);
    }
    cp_async_commit();
    __syncthreads();
    // 16 x 64 generated entries, 4 per thread
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      const int kk = e >> 6, ii = e & 63;
      const int gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < n && gk < n) ? tqq_d(Pi[ii], Pk[kk], gi == gk) : 0.0;
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const double2 a0 = *reinterpret_cast<const double2*>(&As[kk][ty * 2]);
      const double2 a1 = *reinterpret_cast<const double2*>(&As[kk][32 + ty * 2]);
      const double2 b0 = *reinterpret_cast<const double2*>(&Bs[kk][tx * 2]);
      const double2 b1 = *reinterpret_cast<const double2*>(&Bs[kk][32 + tx * 2]);
      const double a[4] = {a0.x, a0.y, a1.x, a1.y};
      const double b[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int row = i0 + (r < 2 ? ty * 2 + r : 32 + ty * 2 + (r - 2));
    double* yr = Y + (size_t)row * ldy + c0;
    *reinterpret_cast<double2*>(yr + tx * 2) = make_double2(acc[r][0], acc[r][1]);
    *reinterpret_cast<double2*>(yr + 32 + tx * 2) = make_double2(acc[r][2], acc[r][3]);
  }
}

// FP64-class on-the-fly matvec for the true residual (wFQ): the T tile of every K step
// is evaluated in FP64 (tqq_d) and split into FP32 hi / lo parts in shared memory, the
// contraction runs in double-FP32 (TwoProduct via FMA, TwoSum; ~48 bits per dot) on the
// FP32 pipe, the result is rounded to FP64.  This replaces the FP64 contraction of
// k_dgemm_mf (GB300's FP64 pipe is 1/64 of FP32).  Output tiles of 32 rows x 256 columns
// (256 threads, 8 x 4 outputs each), so each FP64 pair value serves 256 columns; K steps
// of 16 atoms; T symmetric, so the A tile's rows k are T[k][i0 .. i0+31].  X comes as FP32
// hi / lo planes [np][ldx].
__global__ void __launch_bounds__(256)
k_ffgemm_mf(const double* __restrict__ pos /* [n][4]: x y z Rq^2 */, int n,
            const float* __restrict__ Xh, const float* __restrict__ Xl, int ldx, int ncols,
            double* __restrict__ Y, int ldy, int K) {
  constexpr int BM = 32, BN = 256, BK = 16;
  __shared__ __align__(16) float Ah[BK][BM], Al[BK][BM], Bh[BK][BN], Bl[BK][BN];
  __shared__ double Pi[BM][4];
  __shared__ double Pk[BK][4];
  const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;   // columns 4 tx .., rows 8 ty ..
  const int i0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  if (tid < BM * 4) {
    const int ii = tid >> 2, q = tid & 3;
    Pi[ii][q] = (i0 + ii < n) ? pos[(size_t)(i0 + ii) * 4 + q] : (q == 3 ? 1.0 : 0.0);
  }
  float s[8][4], c[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) s[r][q] = c[r][q] = 0.f;
  const int nk = K / BK;
  for (int kt = 0; kt < nk; ++kt) {
    const int k0 = kt * BK;
    if (tid < BK * 4) {
      const int kk = tid >> 2, q = tid & 3;
      Pk[kk][q] = (k0 + kk < n) ? pos[(size_t)(k0 + kk) * 4 + q] : (q == 3 ? 1.0 : 0.0);
    }
    // operand: 16 x 256 floats per plane, four 16-byte chunks per thread and plane
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int id = tid + 256 * u;
      const int kk = id >> 6, cc = (id & 63) * 4;
      const size_t bx = (size_t)(k0 + kk) * ldx + c0 + cc;
      const bool in = c0 + cc < ncols;   // the last tile may be narrower (ncols % 128 == 0)
      *reinterpret_cast<float4*>(&Bh[kk][cc]) =
          in ? *reinterpret_cast<const float4*>(Xh + bx) : make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(&Bl[kk][cc]) =
          in ? *reinterpret_cast<const float4*>(Xl + bx) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    // T tile: 16 x 32 pair values in FP64, two per thread
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int id = tid + 256 * u;
      const int kk = id >> 5, ii = id & 31;
      const int gi = i0 + ii, gk = k0 + kk;
      const double v = (gi < n && gk < n) ? tqq_d(Pi[ii], Pk[kk], gi == gk) : 0.0;
      const float h = __double2float_rn(v);
      Ah[kk][ii] = h;
      Al[kk][ii] = __double2float_rn(v - (double)h);
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < BK; ++kk) {
      const float4 ah0 = *reinterpret_cast<const float4*>(&Ah[kk][ty * 8]);
      const float4 ah1 = *reinterpret_cast<const float4*>(&Ah[kk][ty * 8 + 4]);
      const float4 al0 = *reinterpret_cast<const float4*>(&Al[kk][ty * 8]);
      const float4 al1 = *reinterpret_cast<const float4*>(&Al[kk][ty * 8 + 4]);
      const float4 bh = *reinterpret_cast<const float4*>(&Bh[kk][tx * 4]);
      const float4 bl = *reinterpret_cast<const float4*>(&Bl[kk][tx * 4]);
      const float a_h[8] = {ah0.x, ah0.y, ah0.z, ah0.w, ah1.x, ah1.y, ah1.z, ah1.w};
      const float a_l[8] = {al0.x, al0.y, al0.z, al0.w, al1.x, al1.y, al1.z, al1.w};
      const float b_h[4] = {bh.x, bh.y, bh.z, bh.w}, b_l[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) ff::mac(s[r][q], c[r][q], a_h[r], a_l[r], b_h[q], b_l[q]);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) ff::renorm(s[r][q], c[r][q]);
    __syncthreads();
  }
  if (c0 + tx * 4 >= ncols) return;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    double* yr = Y + (size_t)(i0 + ty * 8 + r) * ldy + c0 + tx * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) yr[q] = (double)s[r][q] + (double)c[r][q];
  }
}

// ---------------------------------------------------------------- wFQFmu on the fly
// Standard (charges first) row of unknown u of a tile whose atoms start at a0 and whose
// first `na` unknowns are those atoms' charges, the next 3 na their dipole components.
__device__ __forceinline__ int std_row(int N, int a0, int na, int u, int* atom) {
  if (u < na) {
    *atom = a0 + u;
    return a0 + u;
  }
  *atom = a0 + (u - na) / 3;
  return N + 3 * a0 + (u - na);
}

__global__ void __launch_bounds__(256, 2)
k_sgemm_mf4(const float4* __restrict__ pos, const float* __restrict__ rm2, int N, int mu_self,
            const float* __restrict__ X, int ldx, float* __restrict__ Y, int ldy) {
  constexpr int BM = 128, BN = 128, BK = 16, AT = 32, KA = 4;
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  __shared__ float4 Pa[AT];
  __shared__ float Ra[AT];
  __shared__ float4 Pb[2][KA];
  __shared__ float Rb[2][KA];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int a0 = blockIdx.y * AT, c0 = blockIdx.x * BN;
  if (tid < AT) {
    const int a = a0 + tid;
    Pa[tid] = a < N ? pos[a] : make_float4(0.f, 0.f, 0.f, 1.f);
    Ra[tid] = a < N ? rm2[a] : 1.f;
  }
  auto load_x = [&](int st, int kb) {
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int idx = tid + rr * 256;
      const int kk = idx >> 5, cc = (idx & 31) * 4;
      int b;
      const int row = std_row(N, kb * KA, KA, kk, &b);
      if (b < N) cp_async16(&Bs[st][kk][cc], X + (size_t)row * ldx + c0 + cc);
      else *reinterpret_cast<float4*>(&Bs[st][kk][cc]) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    cp_async_commit();
  };
  auto load_pb = [&](int st, int kb) {
    if (tid < KA) {
      const int b = kb * KA + tid;
      Pb[st][tid] = b < N ? pos[b] : make_float4(0.f, 0.f, 0.f, 1.f);
      Rb[st][tid] = b < N ? rm2[b] : 1.f;
    }
  };
  auto gen = [&](int st, int kb) {
    if (tid < AT * KA) {
      const int al = tid & (AT - 1), bl = tid >> 5;
      const int a = a0 + al, b = kb * KA + bl;
      float blk[4][4];
      if (a >= N || b >= N) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int l = 0; l < 4; ++l) blk[k][l] = 0.f;
      } else if (a == b) {
        radial::self_block_f(Pa[al].w, Ra[al], mu_self, blk);
      } else {
        radial::pair_block_f(Pa[al], Ra[al], Pb[st][bl], Rb[st][bl], blk);
      }
      // As[st][K unknown][row unknown]
      As[st][bl][al] = blk[0][0];
#pragma unroll
      for (int l = 0; l < 3; ++l) As[st][KA + 3 * bl + l][al] = blk[0][1 + l];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        As[st][bl][AT + 3 * al + k] = blk[1 + k][0];
#pragma unroll
        for (int l = 0; l < 3; ++l) As[st][KA + 3 * bl + l][AT + 3 * al + k] = blk[1 + k][1 + l];
      }
    }
  };
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  const int nk = (N + KA - 1) / KA;
  load_pb(0, 0);
  load_x(0, 0);
  __syncthreads();
  gen(0, 0);
  if (nk > 1) load_pb(1, 1);
  cp_async_wait_all();
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1, nx = st ^ 1;
    if (kt + 1 < nk) {
      load_x(nx, kt + 1);
      gen(nx, kt + 1);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0v = *reinterpret_cast<const float4*>(&As[st][kk][ty * 4]);
      const float4 a1v = *reinterpret_cast<const float4*>(&As[st][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[st][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[st][kk][64 + tx * 4]);
      const float a[8] = {a0v.x, a0v.y, a0v.z, a0v.w, a1v.x, a1v.y, a1v.z, a1v.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    cp_async_wait_all();
    __syncthreads();
    if (kt + 2 < nk) load_pb(st, kt + 2);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int u = r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4);
    int a;
    const int row = std_row(N, a0, AT, u, &a);
    if (a >= N) continue;
    float* yr = Y + (size_t)row * ldy + c0;
    *reinterpret_cast<float4*>(yr + tx * 4) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    *reinterpret_cast<float4*>(yr + 64 + tx * 4) =
        make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
  }
}

// FP64 counterpart (the true residual of matrix-free wFQFmu solves): 64 x 64 output tiles
// (16 atoms), K steps of 4 atoms; the blocks in FP64 closed form, as the materialised FP64
// kernel evaluates them.
struct RadialD { double t1r, t2; };   // T'/r, T''
__device__ __forceinline__ RadialD radial_d(double r, double R) {
  const double x = r / R;
  const double e = erf(x);
  const double g = 1.1283791670955126 * exp(-x * x);
  const double ir = 1.0 / r;
  RadialD o;
  o.t1r = (g * x - e) * ir * ir * ir;
  o.t2 = (2.0 * e - 2.0 * g * x - 2.0 * g * x * x * x) * ir * ir * ir;
  return o;
}

__device__ void pair_block_d(const double* pa, double rma2, const double* pb, double rmb2,
                             double blk[4][4]) {
  const double d[3] = {pa[0] - pb[0], pa[1] - pb[1], pa[2] - pb[2]};
  const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  blk[0][0] = erf(r / sqrt(pa[3] + pb[3])) / r;
  const RadialD qm = radial_d(r, sqrt(pa[3] + rmb2));
  const RadialD mq = radial_d(r, sqrt(rma2 + pb[3]));
  const RadialD mm = radial_d(r, sqrt(rma2 + rmb2));
  const double rh[3] = {d[0] / r, d[1] / r, d[2] / r};
  for (int l = 0; l < 3; ++l) blk[0][1 + l] = -qm.t1r * d[l];
  for (int k = 0; k < 3; ++k) {
    blk[1 + k][0] = mq.t1r * d[k];
    for (int l = 0; l < 3; ++l) {
      const double rr = rh[k] * rh[l];
      blk[1 + k][1 + l] = -(mm.t2 * rr + mm.t1r * ((k == l ? 1.0 : 0.0) - rr));
    }
  }
}

__global__ void __launch_bounds__(256)
k_dgemm_mf4(const double* __restrict__ pos /* [N][4] x y z Rq^2 */, const double* __restrict__ rm2,
            int N, int mu_self, const double* __restrict__ X, int ldx, double* __restrict__ Y,
            int ldy) {
  constexpr int BM = 64, BN = 64, BK = 16, AT = 16, KA = 4;
  __shared__ __align__(16) double As[BK][BM];
  __shared__ __align__(16) double Bs[BK][BN];
  __shared__ double Pa[AT][5];
  __shared__ double Pb[KA][5];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int a0 = blockIdx.y * AT, c0 = blockIdx.x * BN;
  if (tid < AT) {
    const int a = a0 + tid;
    for (int q = 0; q < 4; ++q) Pa[tid][q] = a < N ? pos[4 * (size_t)a + q] : 1.0;
    Pa[tid][4] = a < N ? rm2[a] : 1.0;
  }
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  const int nk = (N + KA - 1) / KA;
  for (int kt = 0; kt < nk; ++kt) {
    if (tid < KA) {
      const int b = kt * KA + tid;
      for (int q = 0; q < 4; ++q) Pb[tid][q] = b < N ? pos[4 * (size_t)b + q] : 1.0;
      Pb[tid][4] = b < N ? rm2[b] : 1.0;
    }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int idx = tid + rr * 256;
      const int kk = idx >> 5, cc = (idx & 31) * 2;
      int b;
      const int row = std_row(N, kt * KA, KA, kk, &b);
      if (b < N) cp_async16(&Bs[kk][cc], X + (size_t)row * ldx + c0 + cc);
      else *reinterpret_cast<double2*>(&Bs[kk][cc]) = make_double2(0.0, 0.0);
    }
    cp_async_commit();
    __syncthreads();
    if (tid < AT * KA) {
      const int al = tid & (AT - 1), bl = tid >> 4;
      const int a = a0 + al, b = kt * KA + bl;
      double blk[4][4];
      for (int k = 0; k < 4; ++k)
        for (int l = 0; l < 4; ++l) blk[k][l] = 0.0;
      if (a < N && b < N) {
        if (a == b) {
          blk[0][0] = kSqrt2OverPiD / sqrt(Pa[al][3]);
          if (mu_self) {
            const double R = 1.4142135623730951 * sqrt(Pa[al][4]);
            blk[1][1] = blk[2][2] = blk[3][3] = 4.0 / (3.0 * 1.7724538509055159 * R * R * R);
          }
        } else {
          pair_block_d(Pa[al], Pa[al][4], Pb[bl], Pb[bl][4], blk);
        }
      }
      As[bl][al] = blk[0][0];
      for (int l = 0; l < 3; ++l) As[KA + 3 * bl + l][al] = blk[0][1 + l];
      for (int k = 0; k < 3; ++k) {
        As[bl][AT + 3 * al + k] = blk[1 + k][0];
        for (int l = 0; l < 3; ++l) As[KA + 3 * bl + l][AT + 3 * al + k] = blk[1 + k][1 + l];
      }
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const double2 a0v = *reinterpret_cast<const double2*>(&As[kk][ty * 2]);
      const double2 a1v = *reinterpret_cast<const double2*>(&As[kk][32 + ty * 2]);
      const double2 b0 = *reinterpret_cast<const double2*>(&Bs[kk][tx * 2]);
      const double2 b1 = *reinterpret_cast<const double2*>(&Bs[kk][32 + tx * 2]);
      const double a[4] = {a0v.x, a0v.y, a1v.x, a1v.y};
      const double b[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int u = r < 2 ? ty * 2 + r : 32 + ty * 2 + (r - 2);
    int a;
    const int row = std_row(N, a0, AT, u, &a);
    if (a >= N) continue;
    double* yr = Y + (size_t)row * ldy + c0;
    *reinterpret_cast<double2*>(yr + tx * 2) = make_double2(acc[r][0], acc[r][1]);
    *reinterpret_cast<double2*>(yr + 32 + tx * 2) = make_double2(acc[r][2], acc[r][3]);
  }
}

}  // namespace

cudaError_t launch_sgemm_mf4(const float4* pos, const float* rm2, int N, int mu_self,
                             const float* X, int ldx, float* Y, int ldy, int ncols, cudaStream_t s,
                             long long* nl) {
  if (ncols % 128) return cudaErrorInvalidValue;
  k_sgemm_mf4<<<dim3(ncols / 128, (N + 31) / 32), 256, 0, s>>>(pos, rm2, N, mu_self, X, ldx, Y, ldy);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_dgemm_mf4(const double* pos4, const double* rm2, int N, int mu_self,
                             const double* X, int ldx, double* Y, int ldy, int ncols,
                             cudaStream_t s, long long* nl) {
  if (ncols % 64) return cudaErrorInvalidValue;
  k_dgemm_mf4<<<dim3(ncols / 64, (N + 15) / 16), 256, 0, s>>>(pos4, rm2, N, mu_self, X, ldx, Y, ldy);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_sgemm_mf(const float4* pos, int n, int np, const float* X, int ldx, float* Y,
                            int ldy, int ncols, cudaStream_t s, long long* nl) {
  if (np % 128 || ncols % 128) return cudaErrorInvalidValue;
  k_sgemm_mf<<<dim3(ncols / 128, np / 128), 256, 0, s>>>(pos, n, X, ldx, Y, ldy, np);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_ffgemm_mf(const double* pos4, int n, int np, const float* Xh, const float* Xl,
                             int ldx, double* Y, int ldy, int ncols, cudaStream_t s, long long* nl) {
  if (np % 32 || ncols % 4 || ldx % 4 || ldx < ncols) return cudaErrorInvalidValue;
  k_ffgemm_mf<<<dim3((ncols + 255) / 256, np / 32), 256, 0, s>>>(pos4, n, Xh, Xl, ldx, ncols, Y, ldy,
                                                                 np);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_dgemm_mf(const double* pos4, int n, int np, const double* X, int ldx,
                            double* Y, int ldy, int ncols, cudaStream_t s, long long* nl) {
  if (np % 64 || ncols % 64) return cudaErrorInvalidValue;
  k_dgemm_mf<<<dim3(ncols / 64, np / 64), 256, 0, s>>>(pos4, n, X, ldx, Y, ldy, np);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace px
