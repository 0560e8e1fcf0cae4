// Matrix-free block matvec Y = T X: the T tile of every K step is generated from the
// atom positions inside the GEMM ("on the fly", Sec. "Solvers"), never stored.
//
// T_ik = erf(r/R)/r with R^2 = R_q,i^2 + R_q,k^2 (Eq. 5), T_ii = sqrt(2/pi)/R_q,i; the
// erf is evaluated only for close pairs (r/R < 4 in FP32, < 6 in FP64, beyond which
// erf(r/R) = 1 to the working precision), far pairs cost one reciprocal square root.
// Tiling as in k_gemm_simt.cu: the X tile is staged with cp.async, the generated T
// tile is written to shared memory one stage ahead of the FMA loop.  Rows / columns
// beyond the n real atoms generate 0.
#include "px_internal.cuh"

namespace px {

namespace {

constexpr float kSqrt2OverPiF = 0.79788456080286536f;
constexpr double kSqrt2OverPiD = 0.7978845608028654;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n"); }

// pos: x, y, z (bohr, FP32) and R_q^2
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

__global__ void __launch_bounds__(256, 2)
k_sgemm_mf(const float4* __restrict__ pos, int n, const float* __restrict__ X, int ldx,
           float* __restrict__ Y, int ldy, int K) {
  constexpr int BM = 128, BN = 128, BK = 16;
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  __shared__ float4 Pi[BM];
  __shared__ float4 Pk[2][BK];
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
  auto gen = [&](int st, int k0) {
    const float4 pi = Pi[gi_local];
    const int gi = i0 + gi_local;
#pragma unroll
    for (int q = 0; q < BK / 2; ++q) {
      const int kk = kk_base + 2 * q;
      const int gk = k0 + kk;
      float v = 0.f;
      if (gi < n && gk < n) v = tqq_f(pi, Pk[st][kk], gi == gk);
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
  gen(0, 0);
  if (nk > 1) load_pk(1, BK);
  cp_async_wait_all();
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1, nx = st ^ 1;
    if (kt + 1 < nk) {
      load_x(nx, (kt + 1) * BK);
      gen(nx, (kt + 1) * BK);
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
    // positions of the K block after next go into the stage just consumed
    if (kt + 2 < nk) load_pk(st, (kt + 2) * BK);
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

}  // namespace

cudaError_t launch_sgemm_mf(const float4* pos, int n, int np, const float* X, int ldx, float* Y,
                            int ldy, int ncols, cudaStream_t s, long long* nl) {
  if (np % 128 || ncols % 128) return cudaErrorInvalidValue;
  k_sgemm_mf<<<dim3(ncols / 128, np / 128), 256, 0, s>>>(pos, n, X, ldx, Y, ldy, np);
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
