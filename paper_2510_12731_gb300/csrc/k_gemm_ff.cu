// FP64-class matvec for the true residual on the CUDA cores: Y = T X with T held as
// two FP32 planes (T = T_hi + T_lo, ~48 significant bits) and X as FP32 hi/lo planes,
// every product and sum in double-FP32 arithmetic (TwoProduct via FMA, TwoSum), the
// result rounded to FP64.  GB300 runs FP32 at ~62x its FP64 rate, so this replaces an
// FP64 GEMM at the accuracy the residual needs (relative error ~2^-44 per dot).
//
// Tiling: 64 x 64 output tile per 256-thread block, 4 x 4 outputs per thread, K steps
// of 16 staged in shared memory (T is symmetric: row segments T[k][i0 : i0+64] are the
// A tile, as in k_gemm_simt.cu).  Operands zero padded to the tile sizes.
#include "px_internal.cuh"

namespace px {

namespace {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// (s, c) += (ah + al)(bh + bl): TwoProduct of the hi parts, cross terms into the error
__device__ __forceinline__ void ff_mac(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float t = __fadd_rn(s, p);
  const float bb = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

__global__ void __launch_bounds__(256)
k_ffgemm(const float* __restrict__ Th, const float* __restrict__ Tl, int ldt,
         const float* __restrict__ Xh, const float* __restrict__ Xl, int ldx,
         double* __restrict__ Y, int ldy, int K) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ __align__(16) float Ah[2][BK][BM], Al[2][BK][BM], Bh[2][BK][BN], Bl[2][BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  auto load = [&](int st, int k0) {
    // 16 x 64 floats = 256 16-byte chunks per plane: one chunk per thread per plane
    const int kk = tid >> 4, cc = (tid & 15) * 4;
    const size_t at = (size_t)(k0 + kk) * ldt + i0 + cc;
    const size_t bx = (size_t)(k0 + kk) * ldx + c0 + cc;
    cp_async16(&Ah[st][kk][cc], Th + at);
    cp_async16(&Al[st][kk][cc], Tl + at);
    cp_async16(&Bh[st][kk][cc], Xh + bx);
    cp_async16(&Bl[st][kk][cc], Xl + bx);
    cp_async_commit();
  };
  float s[4][4], c[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) s[r][q] = c[r][q] = 0.f;
  const int nk = K / BK;
  load(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) {
      load((kt + 1) & 1, (kt + 1) * BK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int st = kt & 1;
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      const float4 ah = *reinterpret_cast<const float4*>(&Ah[st][kk][ty * 4]);
      const float4 al = *reinterpret_cast<const float4*>(&Al[st][kk][ty * 4]);
      const float4 bh = *reinterpret_cast<const float4*>(&Bh[st][kk][tx * 4]);
      const float4 bl = *reinterpret_cast<const float4*>(&Bl[st][kk][tx * 4]);
      const float a_h[4] = {ah.x, ah.y, ah.z, ah.w}, a_l[4] = {al.x, al.y, al.z, al.w};
      const float b_h[4] = {bh.x, bh.y, bh.z, bh.w}, b_l[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) ff_mac(s[r][q], c[r][q], a_h[r], a_l[r], b_h[q], b_l[q]);
    }
    // renormalise the accumulators once per K step so the error term stays below ulp(s)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float t = __fadd_rn(s[r][q], c[r][q]);
        c[r][q] = __fsub_rn(c[r][q], __fsub_rn(t, s[r][q]));
        s[r][q] = t;
      }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    double* yr = Y + (size_t)(i0 + ty * 4 + r) * ldy + c0 + tx * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) yr[q] = (double)s[r][q] + (double)c[r][q];
  }
}

// FP64 -> FP32 hi/lo planes of an FP64 operand (np x ldx)
__global__ void k_split_ff(const double* __restrict__ X, size_t n, float* Xh, float* Xl) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const double v = X[k];
    const float h = __double2float_rn(v);
    Xh[k] = h;
    Xl[k] = __double2float_rn(v - (double)h);
  }
}

}  // namespace

cudaError_t launch_split_ff(const double* X, size_t n, float* Xh, float* Xl, cudaStream_t s,
                            long long* nl) {
  k_split_ff<<<152 * 8, 256, 0, s>>>(X, n, Xh, Xl);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_ffgemm(const float* Th, const float* Tl, int np, const float* Xh,
                          const float* Xl, int ldx, double* Y, int ldy, int ncols, cudaStream_t s,
                          long long* nl) {
  if (np % 64 || ncols % 64 || ldx % 4) return cudaErrorInvalidValue;
  k_ffgemm<<<dim3(ncols / 64, np / 64), 256, 0, s>>>(Th, Tl, np, Xh, Xl, ldx, Y, ldy, np);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace px
