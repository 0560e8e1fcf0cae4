// Block matvec Y = T X on the CUDA cores (FP32 and FP64), T materialised.
//
// T is symmetric, so the rows of T are also its columns: the A-tile of the
// product, T[i0:i0+BM][k0:k0+BK], is read as BK contiguous row segments
// T[k][i0:i0+BM] -- the same access pattern as the X tile X[k][c0:c0+BN].  Both
// tiles are staged into shared memory with 16-byte cp.async copies, double
// buffered.  Operands are zero padded to multiples of 128 (rows, columns, K), so
// the kernels need no bounds checks.
#include "px_internal.cuh"

#include <algorithm>

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

// FP32: BM = BN = 128, BK = 16, 256 threads, 8 x 8 outputs per thread arranged as
// rows {ty*4 + r, 64 + ty*4 + r} and columns {tx*4 + c, 64 + tx*4 + c}.  A 3-stage
// cp.async ring (48 KB): the copy of K block kt + 2 goes into the stage consumed at step
// kt - 1, so one barrier per K step suffices.
__global__ void __launch_bounds__(256, 2)
k_sgemm(const float* __restrict__ T, int ldt, const float* __restrict__ X, int ldx,
        float* __restrict__ Y, int ldy, int K) {
  constexpr int BM = 128, BN = 128, BK = 16, ST = 3;
  __shared__ __align__(16) float As[ST][BK][BM];
  __shared__ __align__(16) float Bs[ST][BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  const float* Ab = T + i0;
  const float* Bb = X + c0;

  auto load = [&](int st, int k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int idx = tid + r * 256;
      int kk = idx >> 5, cc = (idx & 31) * 4;
      cp_async16(&As[st][kk][cc], Ab + (size_t)(k0 + kk) * ldt + cc);
      cp_async16(&Bs[st][kk][cc], Bb + (size_t)(k0 + kk) * ldx + cc);
    }
    cp_async_commit();
  };

  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

  const int nk = K / BK;
  load(0, 0);
  if (nk > 1) load(1, BK);
  for (int kt = 0; kt < nk; ++kt) {
    if (kt + 1 < nk) cp_async_wait<1>();   // block kt landed, kt + 1 may be in flight
    else cp_async_wait<0>();
    __syncthreads();                       // ... for every thread; stage (kt + 2) % 3 is free
    if (kt + 2 < nk) load((kt + 2) % ST, (kt + 2) * BK);
    const int st = kt % ST;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&As[st][kk][ty * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[st][kk][64 + ty * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[st][kk][tx * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[st][kk][64 + tx * 4]);
      float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    int row = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
    float* yr = Y + (size_t)row * ldy + c0;
    *reinterpret_cast<float4*>(yr + tx * 4) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    *reinterpret_cast<float4*>(yr + 64 + tx * 4) =
        make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
  }
}

// FP64: BM = BN = 64, BK = 16, 256 threads, 4 x 4 outputs per thread at rows
// {ty*2 + r, 32 + ty*2 + r} and columns {tx*2 + c, 32 + tx*2 + c}.  Split K: block z of
// gridDim.z sums K tiles [z nk / nz, (z+1) nk / nz) into Y + z zstride (nz = 1: all K).
__global__ void __launch_bounds__(256)
k_dgemm(const double* __restrict__ T, int ldt, const double* __restrict__ X, int ldx,
        double* __restrict__ Y, int ldy, int K, size_t zstride) {
  constexpr int BM = 64, BN = 64, BK = 16;
  Y += blockIdx.z * zstride;
  __shared__ __align__(16) double As[2][BK][BM];
  __shared__ __align__(16) double Bs[2][BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
  const double* Ab = T + i0;
  const double* Bb = X + c0;
  auto load = [&](int st, int k0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int idx = tid + r * 256;          // 512 16-byte chunks = 16 rows x 32 chunks
      int kk = idx >> 5, cc = (idx & 31) * 2;
      cp_async16(&As[st][kk][cc], Ab + (size_t)(k0 + kk) * ldt + cc);
      cp_async16(&Bs[st][kk][cc], Bb + (size_t)(k0 + kk) * ldx + cc);
    }
    cp_async_commit();
  };
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  const int nk_all = K / BK;
  const int kt0 = (int)(((long long)blockIdx.z * nk_all) / gridDim.z);
  const int kt1 = (int)(((long long)(blockIdx.z + 1) * nk_all) / gridDim.z);
  if (kt1 > kt0) load(0, kt0 * BK);
  for (int kt = kt0; kt < kt1; ++kt) {
    if (kt + 1 < kt1) {
      load((kt + 1 - kt0) & 1, (kt + 1) * BK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int st = (kt - kt0) & 1;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double2 a0 = *reinterpret_cast<const double2*>(&As[st][kk][ty * 2]);
      double2 a1 = *reinterpret_cast<const double2*>(&As[st][kk][32 + ty * 2]);
      double2 b0 = *reinterpret_cast<const double2*>(&Bs[st][kk][tx * 2]);
      double2 b1 = *reinterpret_cast<const double2*>(&Bs[st][kk][32 + tx * 2]);
      double a[4] = {a0.x, a0.y, a1.x, a1.y};
      double b[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int row = i0 + (r < 2 ? ty * 2 + r : 32 + ty * 2 + (r - 2));
    double* yr = Y + (size_t)row * ldy + c0;
    *reinterpret_cast<double2*>(yr + tx * 2) = make_double2(acc[r][0], acc[r][1]);
    *reinterpret_cast<double2*>(yr + 32 + tx * 2) = make_double2(acc[r][2], acc[r][3]);
  }
}

// FP64 matvec on nc <= 8 real columns, Y = T X.  GB300's FP64 pipe (~2 FMA per clock per
// SM) bounds it: at 2 columns it needs 2 FMAs per 8-byte element of T, about 3x the time
// of streaming T from HBM.  So the kernel keeps every SM's FP64 pipe fed: each warp owns
// 4 rows and reads 2 consecutive columns per lane per step (16-byte loads, 64 columns per
// warp step) with 4 x 2 x NC independent FMA chains per lane; blocks of 2 warps (8 rows)
// give ~16 blocks per SM at N = 20k, so the last round of blocks is a small fraction.
// X rows are 64 bytes at most and come through L1 / L2.
template <int NC>
__global__ void __launch_bounds__(64) k_dgemv(const double* __restrict__ T, int ldt,
                                              const double* __restrict__ X, int ldx,
                                              double* __restrict__ Y, int ldy, int nrows, int K) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int row0 = warp * 4;
  if (row0 >= nrows) return;
  double acc[4][NC];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[r][c] = 0.0;
  for (int k = 2 * lane; k < K; k += 64) {
    double2 t[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
      t[r] = __ldcs(reinterpret_cast<const double2*>(T + (size_t)(row0 + r) * ldt + k));
    double x0[NC], x1[NC];
    const double* xr0 = X + (size_t)k * ldx;
    const double* xr1 = xr0 + ldx;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      x0[c] = __ldg(xr0 + c);
      x1[c] = __ldg(xr1 + c);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[r][c] = fma(t[r].y, x1[c], fma(t[r].x, x0[c], acc[r][c]));
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], o);
  if (lane == 0)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < NC; ++c) Y[(size_t)(row0 + r) * ldy + c] = acc[r][c];
}

}  // namespace

cudaError_t launch_dgemv(const double* T, int np, const double* X, int ldx, double* Y, int ldy,
                         int nc, cudaStream_t s, long long* nl) {
  // 8 rows per 64-thread block; np is a multiple of 128, K = np is even
  if (np % 128 || ldx < nc) return cudaErrorInvalidValue;
  const int blocks = np / 8;
  if (nc <= 2) k_dgemv<2><<<blocks, 64, 0, s>>>(T, np, X, ldx, Y, ldy, np, np);
  else if (nc <= 4) k_dgemv<4><<<blocks, 64, 0, s>>>(T, np, X, ldx, Y, ldy, np, np);
  else if (nc <= 8) k_dgemv<8><<<blocks, 64, 0, s>>>(T, np, X, ldx, Y, ldy, np, np);
  else return cudaErrorInvalidValue;
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_sgemm(const float* T, int np, const float* X, int ldx, float* Y, int ldy,
                         int ncols, cudaStream_t s, long long* nl) {
  dim3 grd(ncols / 128, np / 128);
  k_sgemm<<<grd, 256, 0, s>>>(T, np, X, ldx, Y, ldy, np);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_dgemm(const double* T, int np, const double* X, int ldx, double* Y, int ldy,
                         int ncols, cudaStream_t s, long long* nl) {
  dim3 grd(ncols / 64, np / 64);
  k_dgemm<<<grd, 256, 0, s>>>(T, np, X, ldx, Y, ldy, np, 0);
  ++*nl;
  return cudaGetLastError();
}

namespace {
// Y[i][c] = sum_z P[z][i][c], z in order (deterministic), c < ncols
__global__ void k_sum_parts(const double* __restrict__ P, int nz, size_t zstride, int np,
                            int ncols, int ldp, double* __restrict__ Y, int ldy) {
  const size_t n = (size_t)np * ncols;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / ncols), c = (int)(t % ncols);
    double v = 0.0;
    for (int z = 0; z < nz; ++z) v += P[z * zstride + (size_t)i * ldp + c];
    Y[(size_t)i * ldy + c] = v;
  }
}
}  // namespace

int dgemm_splits(int np, int ncols) {
  const int tiles = (ncols / 64) * (np / 64);
  const int nk = np / 16;
  int nz = (2 * 152 + tiles - 1) / tiles;   // about two waves of blocks
  return std::max(1, std::min(std::min(nz, 16), nk));
}

cudaError_t launch_dgemm_splitk(const double* T, int np, const double* X, int ldx, double* Y,
                                int ldy, int ncols, double* part, size_t part_elems, cudaStream_t s,
                                long long* nl) {
  const int nz = dgemm_splits(np, ncols);
  const size_t zstride = (size_t)np * ncols;
  if (nz == 1 || part == nullptr || part_elems < nz * zstride)
    return launch_dgemm(T, np, X, ldx, Y, ldy, ncols, s, nl);
  dim3 grd(ncols / 64, np / 64, nz);
  k_dgemm<<<grd, 256, 0, s>>>(T, np, X, ldx, part, ncols, np, zstride);
  k_sum_parts<<<152 * 8, 256, 0, s>>>(part, nz, zstride, np, ncols, ncols, Y, ldy);
  *nl += 2;
  return cudaGetLastError();
}

}  // namespace px
