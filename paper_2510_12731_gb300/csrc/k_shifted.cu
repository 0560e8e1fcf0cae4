// Shifted Krylov solve of a wFQ frequency sweep (Sec. 2.1, Eq. 1 with the shift of Eq. 6).
//
// In Eq. 1 the frequency enters only through the scalar shift z_q(w) I, and the
// right-hand side -Kbar V does not depend on w.  A Krylov space of Kbar T - z I
// started from b is therefore the same space for every z: one Arnoldi process on the
// real matrix A0 = Kbar T per field direction,
//     A0 V_m = V_{m+1} Hbar_m,
// serves every frequency, and GMRES for the shift z picks
//     y_z = argmin || beta e_1 - (Hbar_m - z Ibar) y ||,   x_z = V_m y_z
// (Ibar: the m x m identity with a zero row appended).  The basis, the Hessenberg
// matrix and the matvec are real; only the per-shift least-squares problems are
// complex.  The matvec work drops from one column per (frequency, direction) to one
// per direction.
//
// Precision: the whole Arnoldi process runs in double-FP32 (T as two FP32 planes, the
// basis as hi/lo float pairs, TwoProduct / TwoSum arithmetic, ~48 bits), because all
// shifts share one basis: an operator error cannot be refined away per frequency
// inside the process.  Columns whose FP64-class true residual still misses the
// tolerance afterwards are handed to the batched refinement of the caller.
//
// Layouts (NP <= 4 real columns, one per field direction of the group):
//   basis V [m+1][n][NP] float2 (hi, lo), products U_k = T V_k [m][n][NP] float2,
//   work vector W [n][NP] float2, Hessenberg H [m][m+2][NP] double (column j holds
//   H[0..j+1][j]), projections h [2][m+1][NP] double.
//   Systems s = f * NP + pl of the group (frequency f, direction pl): Givens rotations
//   cs [m][Bg], sn [m][Bg], rotated right-hand side g [m+1][Bg], and the rotated
//   triangular factor R of each system packed by columns, R[s][j (j+1) / 2 + k].
#include "px_internal.cuh"
#include "px_ff.cuh"

#include <algorithm>
#include <mutex>
#include <set>
#include <type_traits>
#include <utility>

namespace px {

namespace {

constexpr int kDotsRows = 512;   // rows per projection block
constexpr int kUpdK = 32;        // basis vectors per update block

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------- matvec
// part[sg][i][p] = sum over the columns j of segment sg of (Th + Tl)[i][j] (vh + vl)[j][p],
// for the work items (32-row block, column segment) handed out in a strided loop over a
// persistent grid.  T tiles (32 rows x 128 columns of both planes, 32 KB) and the operand's
// planar chunks stream through a 3-stage shared-memory ring filled with 16-byte cp.async,
// so two chunks are always in flight while the third is consumed.  Each warp owns four
// rows; each lane takes 4 consecutive columns of a chunk; the 32 lanes' double-FP32
// partial sums are added with TwoSum shuffles at the end of the item.
constexpr int kMvCols = 128;     // columns per pipeline stage
constexpr int kMvStages = 3;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <int NP>
__host__ __device__ constexpr int mv_stage_floats() { return 2 * 32 * kMvCols + 2 * NP * kMvCols; }

template <int NP>
__global__ void __launch_bounds__(256, 2)
k_sk_matvec(const float* __restrict__ Th, const float* __restrict__ Tl, int np, int S,
            int seg_cols, const float* __restrict__ vp, float2* __restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  constexpr int kSt = mv_stage_floats<NP>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrb = np / 32;
  const int items = nrb * S;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int rb = item % nrb, sg = item / nrb;
    const int c_begin = sg * seg_cols;
    const int c_end = min(np, c_begin + seg_cols);
    const int nch = (c_end - c_begin) / kMvCols;
    auto issue = [&](int ch) {
      float* st = smem + (ch % kMvStages) * kSt;
      const int c0 = c_begin + ch * kMvCols;
      // T: 2 planes x 32 rows x 32 chunks of 16 bytes, 8 per thread
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int id = threadIdx.x + 256 * q;
        const int pl = id >> 10, row = (id >> 5) & 31, c16 = id & 31;
        const float* src = (pl ? Tl : Th) + (size_t)(rb * 32 + row) * np + c0 + c16 * 4;
        cp_async16(st + (pl * 32 + row) * kMvCols + c16 * 4, src);
      }
      // operand: 2 NP planes x 32 chunks
      if ((int)threadIdx.x < 2 * NP * 32) {
        const int pl = threadIdx.x >> 5, c16 = threadIdx.x & 31;
        cp_async16(st + 2 * 32 * kMvCols + pl * kMvCols + c16 * 4, vp + (size_t)pl * np + c0 + c16 * 4);
      }
    };
    float ah[4][NP], al[4][NP];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int p = 0; p < NP; ++p) ah[r][p] = al[r][p] = 0.f;
#pragma unroll
    for (int c = 0; c < kMvStages - 1; ++c) {
      if (c < nch) issue(c);
      cp_async_commit();
    }
    for (int c = 0; c < nch; ++c) {
      // chunk c + 2 goes into the stage that held chunk c - 1 (consumed: see the barrier
      // at the end of the previous iteration)
      if (c + kMvStages - 1 < nch) issue(c + kMvStages - 1);
      cp_async_commit();
      cp_async_wait<kMvStages - 1>();
      __syncthreads();
      const float* st = smem + (c % kMvStages) * kSt;
      float4 th[4], tl[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        th[r] = *reinterpret_cast<const float4*>(st + (warp * 4 + r) * kMvCols + lane * 4);
        tl[r] = *reinterpret_cast<const float4*>(st + (32 + warp * 4 + r) * kMvCols + lane * 4);
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float4 xh = *reinterpret_cast<const float4*>(st + 2 * 32 * kMvCols + (2 * p) * kMvCols + lane * 4);
        const float4 xl = *reinterpret_cast<const float4*>(st + 2 * 32 * kMvCols + (2 * p + 1) * kMvCols + lane * 4);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          ff::mac(ah[r][p], al[r][p], th[r].x, tl[r].x, xh.x, xl.x);
          ff::mac(ah[r][p], al[r][p], th[r].y, tl[r].y, xh.y, xl.y);
          ff::mac(ah[r][p], al[r][p], th[r].z, tl[r].z, xh.z, xl.z);
          ff::mac(ah[r][p], al[r][p], th[r].w, tl[r].w, xh.w, xl.w);
        }
      }
      if ((c & 7) == 7)   // keep the compensations below ulp of the sums
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int p = 0; p < NP; ++p) ff::renorm(ah[r][p], al[r][p]);
      __syncthreads();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float bh = __shfl_xor_sync(0xffffffffu, ah[r][p], o);
          const float bl = __shfl_xor_sync(0xffffffffu, al[r][p], o);
          ff::add(ah[r][p], al[r][p], bh, bl);
        }
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int p = 0; p < NP; ++p)
          part[((size_t)sg * np + rb * 32 + warp * 4 + r) * NP + p] = make_float2(ah[r][p], al[r][p]);
  }
}

// U[i][p] = sum over segments of part[sg][i][p]  (i < n)
__global__ void k_sk_combine(int n, int np, int NP, int S, const float2* __restrict__ part,
                             float2* __restrict__ U) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * NP) return;
  float h = 0.f, l = 0.f;
  for (int sg = 0; sg < S; ++sg) {
    const float2 a = part[(size_t)sg * np * NP + idx];
    ff::add(h, l, a.x, a.y);
  }
  U[idx] = make_float2(h, l);
}

// The same product for an operator stored transposed (planes hold S = T^T, so
// U[i][p] = sum_k S[k][i] v[k][p]): part[sg][i][p] sums the rows k of row segment sg, for
// work items (128-column block, row segment).  Each stage holds 32 rows x 128 columns of both
// planes and the operand's 32 rows; warp w takes rows 4w .. 4w+3 of the stage, lane l the
// columns 4l .. 4l+3 (coalesced along the stored rows); the eight warps' double-FP32 sums
// are added through shared memory at the end of the item.
template <int NP>
__global__ void __launch_bounds__(256, 2)
k_sk_matvec_t(const float* __restrict__ Th, const float* __restrict__ Tl, int np, int St,
              int seg_rows, const float* __restrict__ vp, float2* __restrict__ part) {
  extern __shared__ __align__(16) float smem[];
  constexpr int kSt = mv_stage_floats<NP>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncb = np / kMvCols;
  const int items = ncb * St;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int cb = item % ncb, sg = item / ncb;
    const int r_begin = sg * seg_rows;
    const int r_end = min(np, r_begin + seg_rows);
    const int nch = (r_end - r_begin) / 32;
    auto issue = [&](int ch) {
      float* st = smem + (ch % kMvStages) * kSt;
      const int r0 = r_begin + ch * 32;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int id = threadIdx.x + 256 * q;
        const int pl = id >> 10, row = (id >> 5) & 31, c16 = id & 31;
        const float* src = (pl ? Tl : Th) + (size_t)(r0 + row) * np + cb * kMvCols + c16 * 4;
        cp_async16(st + (pl * 32 + row) * kMvCols + c16 * 4, src);
      }
      // operand rows r0 .. r0+31: 2 NP planes x 8 chunks of 16 bytes
      if ((int)threadIdx.x < 2 * NP * 8) {
        const int pl = threadIdx.x >> 3, c16 = threadIdx.x & 7;
        cp_async16(st + 2 * 32 * kMvCols + pl * 32 + c16 * 4, vp + (size_t)pl * np + r0 + c16 * 4);
      }
    };
    float ah[4][NP], al[4][NP];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int p = 0; p < NP; ++p) ah[c][p] = al[c][p] = 0.f;
#pragma unroll
    for (int c = 0; c < kMvStages - 1; ++c) {
      if (c < nch) issue(c);
      cp_async_commit();
    }
    for (int c = 0; c < nch; ++c) {
      if (c + kMvStages - 1 < nch) issue(c + kMvStages - 1);
      cp_async_commit();
      cp_async_wait<kMvStages - 1>();
      __syncthreads();
      const float* st = smem + (c % kMvStages) * kSt;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int k = warp * 4 + rr;
        const float4 th = *reinterpret_cast<const float4*>(st + k * kMvCols + lane * 4);
        const float4 tl = *reinterpret_cast<const float4*>(st + (32 + k) * kMvCols + lane * 4);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float xh = st[2 * 32 * kMvCols + (2 * p) * 32 + k];
          const float xl = st[2 * 32 * kMvCols + (2 * p + 1) * 32 + k];
          ff::mac(ah[0][p], al[0][p], th.x, tl.x, xh, xl);
          ff::mac(ah[1][p], al[1][p], th.y, tl.y, xh, xl);
          ff::mac(ah[2][p], al[2][p], th.z, tl.z, xh, xl);
          ff::mac(ah[3][p], al[3][p], th.w, tl.w, xh, xl);
        }
      }
      if ((c & 7) == 7)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
#pragma unroll
          for (int p = 0; p < NP; ++p) ff::renorm(ah[cc][p], al[cc][p]);
      __syncthreads();
    }
    // add the eight warps' sums: red[w][column][p] (hi, lo) in the ring's space
    cp_async_wait<0>();
    __syncthreads();
    float2* red = reinterpret_cast<float2*>(smem);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
#pragma unroll
      for (int p = 0; p < NP; ++p)
        red[((size_t)warp * kMvCols + lane * 4 + cc) * NP + p] = make_float2(ah[cc][p], al[cc][p]);
    __syncthreads();
    for (int t = threadIdx.x; t < kMvCols * NP; t += blockDim.x) {
      float h = 0.f, l = 0.f;
      for (int w = 0; w < 8; ++w) {
        const float2 a = red[(size_t)w * kMvCols * NP + t];
        ff::add(h, l, a.x, a.y);
      }
      const int col = t / NP, p = t - col * NP;
      part[((size_t)sg * np + cb * kMvCols + col) * NP + p] = make_float2(h, l);
    }
    __syncthreads();
  }
}

// W[i][p] = (Kbar U)_i = sum_j K_ij (U_j - U_i)  (Eq. 2) in double-FP32: the differences by
// TwoSum, K_ij = val32 + its FP32 remainder, products by TwoProduct (the FP64 pipe is
// 1/64 of the FP32 rate).  Eight lanes share a row (each takes every eighth neighbour),
// so a row's gathers are in flight together; the partial sums meet by shuffles.
template <int NP>
__global__ void __launch_bounds__(256) k_sk_kbar(int n, const int* __restrict__ rowptr,
                                                 const int* __restrict__ col,
                                                 const double* __restrict__ val,
                                                 const float* __restrict__ val32,
                                                 const float2* __restrict__ U,
                                                 float2* __restrict__ W) {
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 3, sub = threadIdx.x & 7;
  const bool valid = g < n;
  const int i = valid ? g : n - 1;
  float2 ui[NP];
  float ah[NP], al[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    ui[p] = U[(size_t)i * NP + p];
    ah[p] = al[p] = 0.f;
  }
  if (valid)
    for (int e = rowptr[i] + sub; e < rowptr[i + 1]; e += 8) {
      const int j = col[e];
      const float kh = val32[e];
      const float kl = (float)(val[e] - (double)kh);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        float dh = U[(size_t)j * NP + p].x, dl = U[(size_t)j * NP + p].y;
        ff::add(dh, dl, -ui[p].x, -ui[p].y);
        ff::mac(ah[p], al[p], kh, kl, dh, dl);
      }
    }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      const float bh = __shfl_xor_sync(0xffffffffu, ah[p], o);
      const float bl = __shfl_xor_sync(0xffffffffu, al[p], o);
      ff::add(ah[p], al[p], bh, bl);
    }
    ff::renorm(ah[p], al[p]);
  }
  if (valid && sub == 0)
#pragma unroll
    for (int p = 0; p < NP; ++p) W[(size_t)i * NP + p] = make_float2(ah[p], al[p]);
}

// ---------------------------------------------------------------- Gram-Schmidt
// dpart[rb][k][p] = sum over the rows of block rb of V_k[i][p] W[i][p]: one basis vector k
// per block column (grid x = j + 1), rows in blocks of rows_per_blk (grid y).  Each thread
// keeps NP double-FP32 sums over many rows, so the block reduction is a small part of
// the work; W is re-read per basis vector from L2 (it is n NP 8 bytes).
template <int NP>
__global__ void __launch_bounds__(256)
k_sk_dots(const float2* __restrict__ V, const float2* __restrict__ W, int n, int j,
          int rows_per_blk, int m1, double* __restrict__ dpart) {
  const int k = blockIdx.x;
  const int r0 = blockIdx.y * rows_per_blk, r1 = min(n, r0 + rows_per_blk);
  const float2* Vk = V + (size_t)k * n * NP;
  float ah[NP], al[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) ah[p] = al[p] = 0.f;
  int nmac = 0;
#pragma unroll 4
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float2 v = __ldcs(Vk + (size_t)i * NP + p);   // streamed: W stays in L2
      const float2 w = W[(size_t)i * NP + p];
      ff::mac(ah[p], al[p], v.x, v.y, w.x, w.y);
    }
    if (++nmac == 32) {   // keep the compensation below ulp of the sum
      nmac = 0;
#pragma unroll
      for (int p = 0; p < NP; ++p) ff::renorm(ah[p], al[p]);
    }
  }
  __shared__ double sred[8][NP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    float h = ah[p], l = al[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float bh = __shfl_xor_sync(0xffffffffu, h, o);
      const float bl = __shfl_xor_sync(0xffffffffu, l, o);
      ff::add(h, l, bh, bl);
    }
    if (lane == 0) sred[warp][p] = ff::join(h, l);
  }
  __syncthreads();
  if ((int)threadIdx.x < NP) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sred[w][threadIdx.x];
    dpart[((size_t)blockIdx.y * m1 + k) * NP + threadIdx.x] = t;
  }
}

// h[k][p] = sum over row blocks of dpart[rb][k][p], k <= j
__global__ void k_sk_dots_reduce(int j, int NP, int nrb, int m1, const double* __restrict__ dpart,
                                 double* __restrict__ h) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (j + 1) * NP) return;
  double t = 0.0;
  for (int rb = 0; rb < nrb; ++rb) t += dpart[(size_t)rb * m1 * NP + idx];
  h[idx] = t;
}

// upart[kc][i][p] = sum over the block's kUpdK basis vectors k of V_k[i][p] h[k][p]
template <int NP>
__global__ void __launch_bounds__(256)
k_sk_update(const float2* __restrict__ V, int n, int j, const double* __restrict__ h,
            float2* __restrict__ upart) {
  const int k0 = blockIdx.x * kUpdK;
  if (k0 > j) return;
  const int kend = min(j + 1, k0 + kUpdK);
  __shared__ float2 sh[kUpdK * NP];
  for (int t = threadIdx.x; t < (kend - k0) * NP; t += blockDim.x) sh[t] = ff::split(h[(size_t)k0 * NP + t]);
  __syncthreads();
  const int i = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float ah[NP], al[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) ah[p] = al[p] = 0.f;
#pragma unroll 8
  for (int k = k0; k < kend; ++k)
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float2 vv = __ldcs(V + ((size_t)k * n + i) * NP + p);
      const float2 c = sh[(k - k0) * NP + p];
      ff::mac(ah[p], al[p], vv.x, vv.y, c.x, c.y);
    }
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    ff::renorm(ah[p], al[p]);
    upart[((size_t)blockIdx.x * n + i) * NP + p] = make_float2(ah[p], al[p]);
  }
}

// W[i][p] -= sum_kc upart[kc][i][p]; with `last`, per-block partial |W_p|^2 in npart[blk][p]
template <int NP>
__global__ void __launch_bounds__(256)
k_sk_update_fin(float2* __restrict__ W, int n, int nkc, const float2* __restrict__ upart, int last,
                double* __restrict__ npart) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double nr[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) nr[p] = 0.0;
  if (i < n) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      float h = 0.f, l = 0.f;
      for (int kc = 0; kc < nkc; ++kc) {
        const float2 a = upart[((size_t)kc * n + i) * NP + p];
        ff::add(h, l, a.x, a.y);
      }
      float2 w = W[(size_t)i * NP + p];
      ff::add(w.x, w.y, -h, -l);
      W[(size_t)i * NP + p] = w;
      const double d = ff::join(w);
      nr[p] = d * d;
    }
  }
  if (!last) return;
  __shared__ double sn[8][NP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    double t = nr[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sn[warp][p] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < NP) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sn[w][threadIdx.x];
    npart[(size_t)blockIdx.x * NP + threadIdx.x] = t;
  }
}

// ---------------------------------------------------------------- Hessenberg, Givens
// Column j of Hbar for every direction: H[j][k][p] = sum_pass h[pass][k][p] (k <= j),
// H[j][j+1][p] = ||W_p||, and the scale of the next basis vector (0 on breakdown, i.e.
// when the new direction is negligible against the column: an invariant subspace, in
// which every shift's least-squares residual is exact).  One block.
__global__ void __launch_bounds__(256) k_sk_hess(int j, int NP, int m1, int m2, int passes,
                                                 const double* __restrict__ h,
                                                 const double* __restrict__ npart, int nnb,
                                                 double* __restrict__ H, double* __restrict__ inv_h) {
  double* Hc = H + (size_t)j * m2 * NP;
  __shared__ double sc[8][4], sn2[8][4];
  double c2[4] = {0.0, 0.0, 0.0, 0.0}, n2[4] = {0.0, 0.0, 0.0, 0.0};
  for (int idx = threadIdx.x; idx < (j + 1) * NP; idx += blockDim.x) {
    double v = h[idx];
    if (passes > 1) v += h[(size_t)m1 * NP + idx];
    Hc[idx] = v;
    c2[idx % NP] += v * v;
  }
  for (int b = threadIdx.x; b < nnb * NP; b += blockDim.x) n2[b % NP] += npart[b];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int p = 0; p < NP; ++p) {
    double a = c2[p], q = n2[p];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if (lane == 0) {
      sc[warp][p] = a;
      sn2[warp][p] = q;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < NP) {
    const int p = threadIdx.x;
    double hn2 = 0.0, cc = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      hn2 += sn2[w][p];
      cc += sc[w][p];
    }
    const double hn = sqrt(hn2);
    Hc[(size_t)(j + 1) * NP + p] = hn;
    inv_h[p] = hn > 1e-14 * sqrt(cc + hn2) ? 1.0 / hn : 0.0;
  }
}

// One warp per system s = f * NP + pl: rotate column j of Hbar - z Ibar by the system's
// previous rotations, store the rotated column in R, form the new rotation, update the
// rotated right-hand side and stop the system once its least-squares residual |g_{j+1}|
// reaches its target (or the subspace is invariant, or the basis is full).  active[j]
// counts the systems still iterating after step j.
//
// Rotation k maps the carried entry x_k and the column entry h_{k+1} to
//   R_k = c_k x_k + s_k h_{k+1},   x_{k+1} = -conj(s_k) x_k + c_k h_{k+1},
// an affine recurrence x_{k+1} = A_k x_k + B_k.  Affine maps compose associatively, so
// the 32 lanes take 32 consecutive rotations and an inclusive shuffle scan gives each
// lane the composed map from the chunk's carried-in entry: the dependent FP64 chain is
// 5 scan steps per 32 rotations instead of 32 (GB300's FP64 pipe has a long latency).
__global__ void __launch_bounds__(128)
k_sk_givens(int j, int m, int NP, int P, int p0, int Bg, int m2, const double* __restrict__ H,
            const double* __restrict__ inv_h, const double2* __restrict__ zq,
            double* __restrict__ cs, double2* __restrict__ sn, double2* __restrict__ g,
            double2* __restrict__ R, size_t rstride, const double* __restrict__ target,
            int* __restrict__ jconv, int* __restrict__ active) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (s >= Bg || jconv[s] != 0) return;   // uniform over the warp
  const int f = s / NP, pl = s - f * NP;
  const double2 z = zq[(size_t)f * P + p0 + pl];
  const double* Hc = H + (size_t)j * m2 * NP;
  auto hcol = [&](int k) {
    const double v = Hc[(size_t)k * NP + pl];
    return k == j ? make_double2(v - z.x, -z.y) : make_double2(v, 0.0);
  };
  double2* Rs = R + (size_t)s * rstride + (size_t)j * (j + 1) / 2;
  double2 x = hcol(0);   // carried entry entering the chunk (the same on every lane)
  for (int k0 = 0; k0 < j; k0 += 32) {
    const int k = k0 + lane;
    const bool ok = k < j;
    const double c = ok ? cs[(size_t)k * Bg + s] : 1.0;
    const double2 sk = ok ? sn[(size_t)k * Bg + s] : make_double2(0.0, 0.0);
    const double2 h1 = ok ? hcol(k + 1) : make_double2(0.0, 0.0);
    // this lane's map: A = -conj(s), B = c h_{k+1}; identity beyond the last rotation
    double2 A = ok ? make_double2(-sk.x, sk.y) : make_double2(1.0, 0.0);
    double2 Bv = ok ? make_double2(c * h1.x, c * h1.y) : make_double2(0.0, 0.0);
    // inclusive scan: (A, B) <- (A, B) o (A', B') of the lane d below = (A A', A B' + B)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const double ar = __shfl_up_sync(0xffffffffu, A.x, d), ai = __shfl_up_sync(0xffffffffu, A.y, d);
      const double br = __shfl_up_sync(0xffffffffu, Bv.x, d), bi = __shfl_up_sync(0xffffffffu, Bv.y, d);
      if (lane >= d) {
        const double2 nb = make_double2(fma(A.x, br, fma(-A.y, bi, Bv.x)), fma(A.x, bi, fma(A.y, br, Bv.y)));
        A = cmul(A, make_double2(ar, ai));
        Bv = nb;
      }
    }
    // x_{k+1} from the composed map; x_k is the previous lane's (the carry for lane 0)
    const double2 xn = make_double2(fma(A.x, x.x, fma(-A.y, x.y, Bv.x)), fma(A.x, x.y, fma(A.y, x.x, Bv.y)));
    double2 xk = make_double2(__shfl_up_sync(0xffffffffu, xn.x, 1), __shfl_up_sync(0xffffffffu, xn.y, 1));
    if (lane == 0) xk = x;
    if (ok) {
      const double2 sh = cmul(sk, h1);
      Rs[k] = make_double2(fma(c, xk.x, sh.x), fma(c, xk.y, sh.y));
    }
    // carry: x after the chunk's last rotation
    const int last = min(31, j - 1 - k0);
    x = make_double2(__shfl_sync(0xffffffffu, xn.x, last), __shfl_sync(0xffffffffu, xn.y, last));
  }
  if (lane != 0) return;
  const double hn = Hc[(size_t)(j + 1) * NP + pl];
  const double aa = sqrt(x.x * x.x + x.y * x.y);
  const double rho = sqrt(aa * aa + hn * hn);
  double c;
  double2 sj, r;
  if (aa == 0.0) {
    c = 0.0;
    sj = make_double2(1.0, 0.0);
    r = make_double2(hn, 0.0);
  } else {
    const double2 ph = make_double2(x.x / aa, x.y / aa);
    c = aa / rho;
    sj = make_double2(ph.x * hn / rho, ph.y * hn / rho);
    r = make_double2(ph.x * rho, ph.y * rho);
  }
  cs[(size_t)j * Bg + s] = c;
  sn[(size_t)j * Bg + s] = sj;
  Rs[j] = r;
  const double2 gj = g[(size_t)j * Bg + s];
  g[(size_t)j * Bg + s] = make_double2(c * gj.x, c * gj.y);
  const double2 gn = make_double2(-(sj.x * gj.x + sj.y * gj.y), -(sj.x * gj.y - sj.y * gj.x));
  g[(size_t)(j + 1) * Bg + s] = gn;
  const double res = sqrt(gn.x * gn.x + gn.y * gn.y);
  if (res <= target[s] || inv_h[pl] == 0.0 || j + 1 == m) {
    jconv[s] = j + 1;
  } else {
    atomicAdd(&active[j], 1);
  }
}

// V[j+1][i][p] = W[i][p] * inv_h[p], and its planar copy vp[2p][i], vp[2p+1][i] (hi, lo:
// the matvec operand, rows n .. np-1 stay zero)
template <int NP>
__global__ void k_sk_normalize(int n, int np, int j, const float2* __restrict__ W,
                               const double* __restrict__ inv_h, float2* __restrict__ V,
                               float* __restrict__ vp) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * NP) return;
  const int i = idx / NP, p = idx - i * NP;
  const float2 sc = ff::split(inv_h[p]);
  const float2 w = W[idx];
  float h = 0.f, l = 0.f;
  ff::mac(h, l, w.x, w.y, sc.x, sc.y);
  ff::renorm(h, l);
  V[(size_t)(j + 1) * n * NP + idx] = make_float2(h, l);
  vp[(size_t)(2 * p) * np + i] = h;
  vp[(size_t)(2 * p + 1) * np + i] = l;
}

// Start: V_0 = b_p / beta_p, g_0 = beta_p for every system of direction p, targets,
// jconv = 0 (iterating) or -1 (zero right-hand side: x = 0 exactly).
__global__ void k_sk_start(int n, int np, int NP, int P, int p0, int Bg, const double* __restrict__ b,
                           const double* __restrict__ bnorm, double tol_abs_frac,
                           float2* __restrict__ V, float* __restrict__ vp, double2* __restrict__ g,
                           double* __restrict__ target, int* __restrict__ jconv) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n * NP) {
    const int i = idx / NP, p = idx - i * NP;
    const double bn = bnorm[p0 + p];
    const float2 v = ff::split(bn > 0.0 ? b[(size_t)i * P + p0 + p] / bn : 0.0);
    V[idx] = v;
    vp[(size_t)(2 * p) * np + i] = v.x;
    vp[(size_t)(2 * p + 1) * np + i] = v.y;
  }
  if (idx < Bg) {
    const int pl = idx % NP;
    const double bn = bnorm[p0 + pl];
    g[idx] = make_double2(bn, 0.0);
    target[idx] = tol_abs_frac * bn;
    jconv[idx] = bn > 0.0 ? 0 : -1;
  }
}

// ---------------------------------------------------------------- solution
// y = R^-1 g for one system per block (R packed by columns, upper triangular, size jc):
// column-oriented back substitution with g staged in shared memory.
__global__ void k_sk_backsolve(int Bg, int jend, const double2* __restrict__ R, size_t rstride,
                               const double2* __restrict__ g, const int* __restrict__ jconv,
                               int mstride, double2* __restrict__ y) {
  extern __shared__ double2 sg[];
  const int s = blockIdx.x;
  const int jcv = jconv[s];
  const int jc = jcv < 0 ? 0 : (jcv == 0 ? jend : jcv);
  for (int k = threadIdx.x; k < jc; k += blockDim.x) sg[k] = g[(size_t)k * Bg + s];
  __syncthreads();
  const double2* Rs = R + (size_t)s * rstride;
  __shared__ double2 yl_sh;
  for (int l = jc - 1; l >= 0; --l) {
    const double2* Rc = Rs + (size_t)l * (l + 1) / 2;
    if (threadIdx.x == 0) {
      const double2 d = Rc[l];
      const double den = d.x * d.x + d.y * d.y;
      const double2 t = sg[l];
      yl_sh = den > 0.0 ? make_double2((t.x * d.x + t.y * d.y) / den, (t.y * d.x - t.x * d.y) / den)
                        : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const double2 yl = yl_sh;
    for (int k = threadIdx.x; k < l; k += blockDim.x) {
      const double2 p = cmul(Rc[k], yl);
      sg[k].x -= p.x;
      sg[k].y -= p.y;
    }
    if (threadIdx.x == 0) y[(size_t)l * Bg + s] = yl;
    __syncthreads();
  }
  // y_k = 0 beyond the system's own basis size (the solution GEMM runs to the longest)
  for (int k = jc + threadIdx.x; k < mstride; k += blockDim.x) y[(size_t)k * Bg + s] = make_double2(0.0, 0.0);
}

// x[i][c] = sum_k V_k[i][pl] y_k,s and (T x)[i][c] = sum_k U_k[i][pl] y_k,s for the systems
// of the group (c = f P + p0 + pl), double-FP32 sums rounded to FP64; T x goes to the real
// operand layout Y[i][2c], Y[i][2c+1] of the residual kernel.  Tile: 64 rows x 32 systems,
// 4 rows x 2 systems per thread, 8 basis vectors per shared-memory stage.
constexpr int kSolRows = 64, kSolSys = 32, kSolK = 8;

template <int NP>
__global__ void __launch_bounds__(256, 1)
k_sk_solution(int n, int kmax, int Bg, int P, int p0, const float2* __restrict__ V,
              const float2* __restrict__ U, const double2* __restrict__ y, double2* __restrict__ x,
              int B, double* __restrict__ Y, int ldy) {
  __shared__ float2 sv[kSolK][kSolRows][NP], su[kSolK][kSolRows][NP];
  __shared__ float4 sy[kSolK][kSolSys];   // (re_hi, im_hi, re_lo, im_lo)
  const int tid = threadIdx.x;
  const int tr = tid & 15, ts = tid >> 4;   // rows tr*4 .. +3, systems ts*2 .. +1
  const int i0 = blockIdx.x * kSolRows, s0 = blockIdx.y * kSolSys;
  float xa[4][2][4], ta[4][2][4];   // [row][sys][re_h, re_l, im_h, im_l]
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) xa[r][q][e] = ta[r][q][e] = 0.f;
  int plq[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) plq[q] = (s0 + ts * 2 + q) % NP;
  for (int k0 = 0; k0 < kmax; k0 += kSolK) {
    __syncthreads();
    for (int t = tid; t < kSolK * kSolRows * NP; t += blockDim.x) {
      const int kk = t / (kSolRows * NP), rem = t - kk * kSolRows * NP;
      const int rr = rem / NP, p = rem - rr * NP;
      const int k = k0 + kk, i = i0 + rr;
      const bool ok = k < kmax && i < n;
      sv[kk][rr][p] = ok ? V[((size_t)k * n + i) * NP + p] : make_float2(0.f, 0.f);
      su[kk][rr][p] = ok ? U[((size_t)k * n + i) * NP + p] : make_float2(0.f, 0.f);
    }
    for (int t = tid; t < kSolK * kSolSys; t += blockDim.x) {
      const int kk = t / kSolSys, q = t - kk * kSolSys;
      const int k = k0 + kk, s = s0 + q;
      double2 yv = (k < kmax && s < Bg) ? y[(size_t)k * Bg + s] : make_double2(0.0, 0.0);
      const float2 re = ff::split(yv.x), im = ff::split(yv.y);
      sy[kk][q] = make_float4(re.x, im.x, re.y, im.y);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kSolK; ++kk) {
      float4 yq[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) yq[q] = sy[kk][ts * 2 + q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float2 vv = sv[kk][tr * 4 + r][plq[q]];
          const float2 uu = su[kk][tr * 4 + r][plq[q]];
          ff::mac(xa[r][q][0], xa[r][q][1], vv.x, vv.y, yq[q].x, yq[q].z);
          ff::mac(xa[r][q][2], xa[r][q][3], vv.x, vv.y, yq[q].y, yq[q].w);
          ff::mac(ta[r][q][0], ta[r][q][1], uu.x, uu.y, yq[q].x, yq[q].z);
          ff::mac(ta[r][q][2], ta[r][q][3], uu.x, uu.y, yq[q].y, yq[q].w);
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        ff::renorm(xa[r][q][0], xa[r][q][1]);
        ff::renorm(xa[r][q][2], xa[r][q][3]);
        ff::renorm(ta[r][q][0], ta[r][q][1]);
        ff::renorm(ta[r][q][2], ta[r][q][3]);
      }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + tr * 4 + r;
    if (i >= n) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int s = s0 + ts * 2 + q;
      if (s >= Bg) continue;
      const int c = (s / NP) * P + p0 + s % NP;
      x[(size_t)i * B + c] = make_double2(ff::join(xa[r][q][0], xa[r][q][1]),
                                          ff::join(xa[r][q][2], xa[r][q][3]));
      Y[(size_t)i * ldy + 2 * c] = ff::join(ta[r][q][0], ta[r][q][1]);
      Y[(size_t)i * ldy + 2 * c + 1] = ff::join(ta[r][q][2], ta[r][q][3]);
    }
  }
}

// iters[c] += basis size used by system s (c = f P + p0 + pl)
__global__ void k_sk_iters(int Bg, int NP, int P, int p0, int jend, const int* __restrict__ jconv,
                           int* __restrict__ iters) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Bg) return;
  const int jcv = jconv[s];
  const int jc = jcv < 0 ? 0 : (jcv == 0 ? jend : jcv);
  iters[(s / NP) * P + p0 + s % NP] += jc;
}

template <class F>
void with_np(int NP, F&& f) {
  switch (NP) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    default: f(std::integral_constant<int, 4>{}); break;
  }
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cached[dev] = v;
  }
  return cached[dev];
}

}  // namespace

// ---------------------------------------------------------------- launchers
SkMatvecPlan sk_matvec_plan(int np) {
  SkMatvecPlan pl;
  const int nrb = np / 32;
  pl.grid = 2 * sm_count();
  // enough (32-row block, column segment) items that the persistent grid's last round
  // is a small fraction: about 16 items per block; segments stay >= 256 columns
  int S = (16 * pl.grid + nrb - 1) / nrb;
  S = std::max(1, std::min(S, np / 256));
  const int tiles = np / 128;
  const int seg_tiles = (tiles + S - 1) / S;
  pl.seg_cols = seg_tiles * 128;
  pl.S = (tiles + seg_tiles - 1) / seg_tiles;
  // transposed operator: (128-column block, row segment) items, segments >= 128 rows
  const int ncb = np / 128;
  int St = (16 * pl.grid + ncb - 1) / ncb;
  St = std::max(1, std::min(St, np / 128));
  const int rblocks = np / 32;
  const int seg_rb = (rblocks + St - 1) / St;
  pl.seg_rows = seg_rb * 32;
  pl.St = (rblocks + seg_rb - 1) / seg_rb;
  return pl;
}

cudaError_t launch_sk_matvec(const float* Th, const float* Tl, int n, int np, int NP,
                             const SkMatvecPlan& pl, bool trans, const float* vp, float2* part,
                             float2* U, cudaStream_t s, long long* nl) {
  if (np % 128 || NP < 1 || NP > 4) return cudaErrorInvalidValue;
  cudaError_t err = cudaSuccess;
  with_np(NP, [&](auto c) {
    constexpr int K = decltype(c)::value;
    const int shm = kMvStages * mv_stage_floats<K>() * (int)sizeof(float);
    // the shared-memory opt-in, once per device and kernel (handles on several threads
    // may race here)
    static std::mutex mu;
    static std::set<std::pair<int, int>> done;
    int dev = 0;
    err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return;
    const int key = (trans ? 8 : 0) + K;
    {
      std::lock_guard<std::mutex> lock(mu);
      if (!done.count({dev, key})) {
        err = trans ? cudaFuncSetAttribute(k_sk_matvec_t<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm)
                    : cudaFuncSetAttribute(k_sk_matvec<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
        if (err == cudaSuccess) done.insert({dev, key});
      }
    }
    if (err != cudaSuccess) return;
    if (trans) k_sk_matvec_t<K><<<pl.grid, 256, shm, s>>>(Th, Tl, np, pl.St, pl.seg_rows, vp, part);
    else k_sk_matvec<K><<<pl.grid, 256, shm, s>>>(Th, Tl, np, pl.S, pl.seg_cols, vp, part);
  });
  if (err != cudaSuccess) return err;
  k_sk_combine<<<(n * NP + 255) / 256, 256, 0, s>>>(n, np, NP, trans ? pl.St : pl.S, part, U);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_sk_kbar(int n, int NP, const int* rowptr, const int* col, const double* val,
                           const float* val32, const float2* U, float2* W, cudaStream_t s,
                           long long* nl) {
  with_np(NP, [&](auto c) {
    constexpr int K = decltype(c)::value;
    k_sk_kbar<K><<<(unsigned)(((size_t)n * 8 + 255) / 256), 256, 0, s>>>(n, rowptr, col, val, val32,
                                                                         U, W);
  });
  ++*nl;
  return cudaGetLastError();
}

int sk_row_blocks(int n) { return (n + kDotsRows - 1) / kDotsRows; }
int sk_update_chunks(int m) { return (m + 1 + kUpdK - 1) / kUpdK; }

cudaError_t launch_sk_gs_pass(const float2* V, float2* W, int n, int NP, int j, int m1,
                              double* dpart, double* h, float2* upart, bool last, double* npart,
                              cudaStream_t s, long long* nl) {
  // row blocks of the projections: enough blocks (basis vectors x row blocks) to fill
  // the GPU twice, each thread summing at least 16 rows
  const int nrb = std::max(1, std::min(std::min(sk_row_blocks(n), (n + 4095) / 4096),
                                       (2 * sm_count() + j) / (j + 1)));
  const int rows_per_blk = (n + nrb - 1) / nrb;
  const int nkc = (j + 1 + kUpdK - 1) / kUpdK;
  with_np(NP, [&](auto c) {
    constexpr int K = decltype(c)::value;
    k_sk_dots<K><<<dim3(j + 1, nrb), 256, 0, s>>>(V, W, n, j, rows_per_blk, m1, dpart);
    k_sk_dots_reduce<<<((j + 1) * K + 255) / 256, 256, 0, s>>>(j, K, nrb, m1, dpart, h);
    k_sk_update<K><<<dim3(nkc, (n + 255) / 256), 256, 0, s>>>(V, n, j, h, upart);
    k_sk_update_fin<K><<<(n + 255) / 256, 256, 0, s>>>(W, n, nkc, upart, last ? 1 : 0, npart);
  });
  *nl += 4;
  return cudaGetLastError();
}

cudaError_t launch_sk_step_end(const SkGroup& G, int j, const double* h, int passes,
                               const double* npart, float2* V, const float2* W, cudaStream_t s,
                               long long* nl) {
  const int nnb = (G.n + 255) / 256;
  k_sk_hess<<<1, 256, 0, s>>>(j, G.NP, G.m + 1, G.m + 2, passes, h, npart, nnb, G.H, G.inv_h);
  // one warp per system, 4 systems per block
  k_sk_givens<<<(G.Bg + 3) / 4, 128, 0, s>>>(j, G.m, G.NP, G.P, G.p0, G.Bg, G.m + 2, G.H,
                                                 G.inv_h, G.zq, G.cs, G.sn, G.g, G.R, G.rstride,
                                                 G.target, G.jconv, G.active);
  with_np(G.NP, [&](auto c) {
    constexpr int K = decltype(c)::value;
    k_sk_normalize<K><<<(G.n * K + 255) / 256, 256, 0, s>>>(G.n, G.np, j, W, G.inv_h, V, G.vp);
  });
  *nl += 3;
  return cudaGetLastError();
}

cudaError_t launch_sk_start(const SkGroup& G, const double* b, const double* bnorm,
                            double tol_abs_frac, float2* V, cudaStream_t s, long long* nl) {
  const int n = std::max(G.n * G.NP, G.Bg);
  cudaError_t e = cudaMemsetAsync(G.vp, 0, sizeof(float) * 2 * G.NP * (size_t)G.np, s);
  if (e != cudaSuccess) return e;
  k_sk_start<<<(n + 255) / 256, 256, 0, s>>>(G.n, G.np, G.NP, G.P, G.p0, G.Bg, b, bnorm, tol_abs_frac,
                                             V, G.vp, G.g, G.target, G.jconv);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_sk_solution(const SkGroup& G, int jend, const float2* V, const float2* U,
                               double2* y, double2* x, int B, double* Y, int ldy, int* iters,
                               cudaStream_t s, long long* nl) {
  const size_t shm = sizeof(double2) * (size_t)std::max(jend, 1);
  if (shm > 200 * 1024) return cudaErrorInvalidValue;
  if (shm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_sk_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)shm);
    if (e != cudaSuccess) return e;
  }
  k_sk_backsolve<<<G.Bg, 256, shm, s>>>(G.Bg, jend, G.R, G.rstride, G.g, G.jconv, jend, y);
  with_np(G.NP, [&](auto c) {
    constexpr int K = decltype(c)::value;
    dim3 grd((G.n + kSolRows - 1) / kSolRows, (G.Bg + kSolSys - 1) / kSolSys);
    k_sk_solution<K><<<grd, 256, 0, s>>>(G.n, jend, G.Bg, G.P, G.p0, V, U, y, x, B, Y, ldy);
  });
  k_sk_iters<<<(G.Bg + 127) / 128, 128, 0, s>>>(G.Bg, G.NP, G.P, G.p0, jend, G.jconv, iters);
  *nl += 3;
  return cudaGetLastError();
}

}  // namespace px
