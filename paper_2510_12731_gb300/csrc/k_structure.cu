// Structure set-up kernels: neighbour list / CSR of K (Eqs. 2-4) and the dense
// Gaussian kernels T (Eq. 5 and its derivatives, Sec. 2.2).  Run once per structure.
#include "px_internal.cuh"

#include <cuda_fp16.h>

namespace px {

namespace {

constexpr double kTwoOverSqrtPi = 1.1283791670955126;   // 2 / sqrt(pi)
constexpr double kSqrt2OverPi = 0.7978845608028654;     // sqrt(2 / pi)

__device__ __forceinline__ double dist2(const double* pos, int i, int j) {
  double dx = pos[3 * i] - pos[3 * j];
  double dy = pos[3 * i + 1] - pos[3 * j + 1];
  double dz = pos[3 * i + 2] - pos[3 * j + 2];
  return dx * dx + dy * dy + dz * dz;
}

// One warp per row i; lanes sweep j.  A pair is kept when r_ij^2 <= rcut^2 of the
// two atoms' types (1 - f(r) >= kcut_eps, Eq. 4).
__global__ void k_neigh_count(const double* __restrict__ pos, int N, const int* __restrict__ type,
                              int ntypes, const double* __restrict__ rcut2, int* counts) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= N) return;
  int i = warp, ti = type[i];
  int cnt = 0;
  for (int j0 = 0; j0 < N; j0 += 32) {
    int j = j0 + lane;
    bool keep = false;
    if (j < N && j != i) keep = dist2(pos, i, j) <= rcut2[ti * ntypes + type[j]];
    cnt += __popc(__ballot_sync(0xffffffffu, keep));
  }
  if (lane == 0) counts[i] = cnt;
}

// Exclusive scan of counts into rowptr[0..N]; one block.
__global__ void k_scan(const int* __restrict__ counts, int N, int* rowptr) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < N; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = (i < N) ? counts[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int nw = blockDim.x >> 5;
      int w = (lane < nw) ? warp_sums[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    int prefix = carry + (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
    if (i < N) rowptr[i] = prefix;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = prefix + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) rowptr[N] = carry;
}

// Fill the CSR in increasing j order (deterministic): K_ij = [1 - f(r)] A_i / r (Eq. 3),
// 1 - f(r) = 1 / (1 + exp[d (r / (s r0) - 1)]) (Eq. 4).
__global__ void k_neigh_fill(const double* __restrict__ pos, int N, const int* __restrict__ type,
                             int ntypes, const double* __restrict__ rcut2,
                             const double* __restrict__ r0t, const double* __restrict__ dt,
                             const double* __restrict__ st, const double* __restrict__ area,
                             const int* __restrict__ rowptr, int* col, double* val64,
                             float* val32) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= N) return;
  int i = warp, ti = type[i];
  int base = rowptr[i];
  double Ai = area[i];
  for (int j0 = 0; j0 < N; j0 += 32) {
    int j = j0 + lane;
    bool keep = false;
    double r2 = 0.0;
    int tp = 0;
    if (j < N && j != i) {
      tp = ti * ntypes + type[j];
      r2 = dist2(pos, i, j);
      keep = r2 <= rcut2[tp];
    }
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      int off = __popc(m & ((1u << lane) - 1u));
      double r = sqrt(r2);
      double omf = 1.0 / (1.0 + exp(dt[tp] * (r / (st[tp] * r0t[tp]) - 1.0)));
      double k = omf * Ai / r;
      col[base + off] = j;
      val64[base + off] = k;
      val32[base + off] = (float)k;
    }
    base += __popc(m);
  }
}

// Eq. 10's nearest neighbours: nn[i][t] = atoms j of type t in row i of the CSR (so within
// r_cut) with r_ij <= s_ij r0_ij, the Fermi midpoint of the pair (f = 1/2, Eq. 4); the first
// shell of an fcc or bcc lattice for s = 1.1.  ident[i] = i.  One thread per atom.
__global__ void k_nn_counts(const double* __restrict__ pos, int N, const int* __restrict__ type,
                            int ntypes, const double* __restrict__ r0t, const double* __restrict__ st,
                            const int* __restrict__ rowptr, const int* __restrict__ col, int* nn,
                            int* ident) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  ident[i] = i;
  for (int t = 0; t < ntypes; ++t) nn[(size_t)i * ntypes + t] = 0;
  const int ti = type[i];
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int j = col[e];
    const int tp = ti * ntypes + type[j];
    const double rm = st[tp] * r0t[tp];
    if (dist2(pos, i, j) <= rm * rm) nn[(size_t)i * ntypes + type[j]] += 1;
  }
}

// T^qq (Eq. 5), symmetric: each 32 x 32 tile of the upper triangle (tile row <= tile
// column) is evaluated once, written in place and, through shared memory, to its mirror
// tile, so every pair costs one erf.  32 x 8 threads per tile, 4 rows each.
__global__ void __launch_bounds__(256) k_build_Tqq(const double* __restrict__ pos,
                                                   const double* __restrict__ Rq, int N, int ld,
                                                   double* T) {
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bi > bj) return;
  __shared__ double tile[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j = bj * 32 + tx;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int il = ty + 8 * q;
    const int i = bi * 32 + il;
    double v = 0.0;
    if (i < N && j < N) {
      if (i == j) {
        v = kSqrt2OverPi / Rq[i];
      } else {
        const double r = sqrt(dist2(pos, i, j));
        const double R = sqrt(Rq[i] * Rq[i] + Rq[j] * Rq[j]);
        v = erf(r / R) / r;
      }
      T[(size_t)i * ld + j] = v;
    }
    tile[il][tx] = v;
  }
  if (bi == bj) return;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jl = ty + 8 * q;
    const int jr = bj * 32 + jl, ic = bi * 32 + tx;
    if (jr < N && ic < N) T[(size_t)jr * ld + ic] = tile[tx][jl];
  }
}

struct Radial { double t0, t1, t2; };   // T, T', T'' of erf(r/R)/r at r
__device__ __forceinline__ Radial radial(double r, double R) {
  double x = r / R;
  double e = erf(x);
  double g = kTwoOverSqrtPi * exp(-x * x);
  double ir = 1.0 / r;
  Radial o;
  o.t0 = e * ir;
  o.t1 = (g * x - e) * ir * ir;
  o.t2 = (2.0 * e - 2.0 * g * x - 2.0 * g * x * x * x) * ir * ir * ir;
  return o;
}

// wFQFmu kernel blocks (Sec. 2.2), unknown order (q_1..q_N, mu_1x, mu_1y, mu_1z, ...):
//   T^qmu_ij  = -T'(r; R_q,i mu,j) rhat           (row i, cols N+3j+b)
//   T^muq_ij  = +T'(r; R_mu,i q,j) rhat           (rows N+3i+a, col j)
//   T^mumu_ij = -[T'' rhat rhat + (T'/r)(I - rhat rhat)]   (R_mu,i mu,j)
// with rhat = (r_i - r_j)/r.  Diagonals: T^qq self limit, T^qmu = T^muq = 0,
// T^mumu = 0 or the Gaussian self term 4/(3 sqrt(pi) R^3) I, R = sqrt(2) R_mu.
__global__ void k_build_T4(const double* __restrict__ pos, const double* __restrict__ Rq,
                           const double* __restrict__ Rmu, int N, int ld, int mu_self,
                           double* T) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= N || j >= N) return;
  size_t rq = (size_t)i * ld;
  if (i == j) {
    T[rq + j] = kSqrt2OverPi / Rq[i];
    double self = 0.0;
    if (mu_self) {
      double R = 1.4142135623730951 * Rmu[i];
      double sq_pi = 1.7724538509055159;
      self = 4.0 / (3.0 * sq_pi * R * R * R);
    }
    for (int a = 0; a < 3; ++a) {
      T[rq + N + 3 * j + a] = 0.0;
      size_t rm = (size_t)(N + 3 * i + a) * ld;
      T[rm + j] = 0.0;
      for (int b = 0; b < 3; ++b) T[rm + N + 3 * j + b] = (a == b) ? self : 0.0;
    }
    return;
  }
  double dx[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1],
                  pos[3 * i + 2] - pos[3 * j + 2]};
  double r = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
  double rh[3] = {dx[0] / r, dx[1] / r, dx[2] / r};
  double Rqq = sqrt(Rq[i] * Rq[i] + Rq[j] * Rq[j]);
  double Rqm = sqrt(Rq[i] * Rq[i] + Rmu[j] * Rmu[j]);
  double Rmq = sqrt(Rmu[i] * Rmu[i] + Rq[j] * Rq[j]);
  double Rmm = sqrt(Rmu[i] * Rmu[i] + Rmu[j] * Rmu[j]);
  T[rq + j] = erf(r / Rqq) / r;
  Radial qm = radial(r, Rqm);
  Radial mq = radial(r, Rmq);
  Radial mm = radial(r, Rmm);
  for (int b = 0; b < 3; ++b) T[rq + N + 3 * j + b] = -qm.t1 * rh[b];
  for (int a = 0; a < 3; ++a) {
    size_t rm = (size_t)(N + 3 * i + a) * ld;
    T[rm + j] = mq.t1 * rh[a];
    for (int b = 0; b < 3; ++b) {
      double rr = rh[a] * rh[b];
      double id = (a == b) ? 1.0 : 0.0;
      T[rm + N + 3 * j + b] = -(mm.t2 * rr + (mm.t1 / r) * (id - rr));
    }
  }
}

// T32 = float(T64)
__global__ void k_convert_T(const double* __restrict__ T64, size_t n, float* T32) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    T32[k] = (float)T64[k];
}

// One block per row i of M = diag(Kbar, I) T: charge rows apply the CSR of K (Eq. 2,
// Laplacian form) to the rows of T in FP64; other rows copy T.  Block max |M| goes to
// *absmax_bits with an integer atomicMax on the bits of the (non-negative) double.
__global__ void __launch_bounds__(256) k_build_M(const double* __restrict__ T, int np, int N,
                                                 const int* __restrict__ rowptr,
                                                 const int* __restrict__ col,
                                                 const double* __restrict__ val, double* M,
                                                 unsigned long long* absmax_bits) {
  const int i = blockIdx.x;
  const double* Ti = T + (size_t)i * np;
  double* Mi = M + (size_t)i * np;
  double amax = 0.0;
  if (i < N) {
    const int e0 = rowptr[i], e1 = rowptr[i + 1];
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
      const double ti = Ti[k];
      double acc = 0.0;
      for (int e = e0; e < e1; ++e) acc = fma(val[e], T[(size_t)col[e] * np + k] - ti, acc);
      Mi[k] = acc;
      amax = fmax(amax, fabs(acc));
    }
  } else {
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
      const double v = Ti[k];
      Mi[k] = v;
      amax = fmax(amax, fabs(v));
    }
  }
  __shared__ double sh[8];
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = amax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    atomicMax(absmax_bits, (unsigned long long)__double_as_longlong(m));
  }
}

// hi/lo 16-bit split of an FP64 operator (see launch_split_op)
__global__ void k_split_op(const double* __restrict__ A, size_t n, uint16_t* hi, uint16_t* lo,
                           int f16, double scale) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const double v = A[k];
    if (f16) {
      const double vs = v * scale;
      const __half h = __float2half_rn((float)vs);
      hi[k] = __half_as_ushort(h);
      lo[k] = __half_as_ushort(__float2half_rn((float)((vs - (double)__half2float(h)) * 2048.0)));
    } else {
      const __nv_bfloat16 h = __double2bfloat16(v);
      hi[k] = __bfloat16_as_ushort(h);
      lo[k] = __bfloat16_as_ushort(__double2bfloat16(v - (double)__bfloat162float(h)));
    }
  }
}

__global__ void k_stage_pos4(const double* __restrict__ pos, const double* __restrict__ Rq,
                             const double* __restrict__ Rmu, int N, float4* p4f, double* p4d,
                             float* rm2f, double* rm2d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (rm2f) {
    const double m2 = Rmu[i] * Rmu[i];
    rm2f[i] = (float)m2;
    rm2d[i] = m2;
  }
  const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], r2 = Rq[i] * Rq[i];
  p4f[i] = make_float4((float)x, (float)y, (float)z, (float)r2);
  p4d[4 * (size_t)i] = x;
  p4d[4 * (size_t)i + 1] = y;
  p4d[4 * (size_t)i + 2] = z;
  p4d[4 * (size_t)i + 3] = r2;
}

}  // namespace

cudaError_t launch_stage_pos4(const DevStructure& d, cudaStream_t s, long long* nl) {
  k_stage_pos4<<<(d.N + 255) / 256, 256, 0, s>>>(d.pos64, d.Rq, d.Rmu, d.N, d.pos4f, d.pos4d,
                                                  d.rm2f, d.rm2d);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_neigh_count(const double* pos, int N, const int* type, int ntypes,
                               const double* rcut2, int* counts, cudaStream_t s, long long* nl) {
  int threads = 256;
  int blocks = (int)((N * 32LL + threads - 1) / threads);
  k_neigh_count<<<blocks, threads, 0, s>>>(pos, N, type, ntypes, rcut2, counts);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_scan(const int* counts, int N, int* rowptr, cudaStream_t s, long long* nl) {
  k_scan<<<1, 1024, 0, s>>>(counts, N, rowptr);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_neigh_fill(const double* pos, int N, const int* type, int ntypes,
                              const double* rcut2, const double* r0, const double* dd,
                              const double* ss, const double* area, const int* rowptr,
                              int* col, double* val64, float* val32, cudaStream_t s,
                              long long* nl) {
  int threads = 256;
  int blocks = (int)((N * 32LL + threads - 1) / threads);
  k_neigh_fill<<<blocks, threads, 0, s>>>(pos, N, type, ntypes, rcut2, r0, dd, ss, area, rowptr,
                                          col, val64, val32);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_build_T64(const DevStructure& d, int mu_self_term, cudaStream_t s,
                             long long* nl) {
  cudaError_t e = cudaMemsetAsync(d.T64, 0, sizeof(double) * (size_t)d.np * d.np, s);
  if (e != cudaSuccess) return e;
  dim3 blk(32, 8);
  if (d.model == 0) {
    const int nt = (d.N + 31) / 32;
    k_build_Tqq<<<dim3(nt, nt), blk, 0, s>>>(d.pos64, d.Rq, d.N, d.np, d.T64);
  } else {
    dim3 grd((d.N + 31) / 32, (d.N + 7) / 8);
    k_build_T4<<<grd, blk, 0, s>>>(d.pos64, d.Rq, d.Rmu, d.N, d.np, mu_self_term, d.T64);
  }
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_convert_T(const DevStructure& d, cudaStream_t s, long long* nl) {
  const size_t n = (size_t)d.np * d.np;
  k_convert_T<<<152 * 16, 256, 0, s>>>(d.T64, n, d.T32);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_build_M64(const DevStructure& d, double* M64,
                             unsigned long long* absmax_bits, cudaStream_t s, long long* nl) {
  k_build_M<<<d.np, 256, 0, s>>>(d.T64, d.np, d.N, d.rowptr, d.col, d.val64, M64, absmax_bits);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_split_op(const double* A, size_t n, uint16_t* hi, uint16_t* lo, bool f16,
                            int scale_exp, cudaStream_t s, long long* nl) {
  k_split_op<<<152 * 16, 256, 0, s>>>(A, n, hi, lo, f16 ? 1 : 0, ldexp(1.0, scale_exp));
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_nn_counts(const double* pos, int N, const int* type, int ntypes,
                             const double* r0t, const double* st, const int* rowptr,
                             const int* col, int* nn, int* ident, cudaStream_t s, long long* nl) {
  k_nn_counts<<<(N + 127) / 128, 128, 0, s>>>(pos, N, type, ntypes, r0t, st, rowptr, col, nn, ident);
  ++*nl;
  return cudaGetLastError();
}

namespace {
// caller index of internal unknown u: charges follow perm, dipole component k of internal
// atom a goes to N + 3 perm[a] + k
__device__ __forceinline__ int caller_unknown(int u, int N, const int* perm) {
  if (u < N) return perm[u];
  const int a = (u - N) / 3;
  return N + 3 * perm[a] + (u - N - 3 * a);
}

__global__ void k_unpermute_op(const double* __restrict__ M, int np, int nu, int N,
                               const int* __restrict__ perm, double* A, size_t lda) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nu) return;
  const int cc = caller_unknown(c, N, perm);
  for (int r = blockIdx.y; r < nu; r += gridDim.y)
    A[(size_t)caller_unknown(r, N, perm) * lda + cc] = M[(size_t)r * np + c];
}

__global__ void k_unpermute_rows(const double* __restrict__ b, int nu, int N, int P,
                                 const int* __restrict__ perm, double* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nu * P) return;
  const int r = idx / P, p = idx - r * P;
  out[(size_t)caller_unknown(r, N, perm) * P + p] = b[idx];
}
}  // namespace

cudaError_t launch_unpermute_system(const double* M, int np, int nu, int N, const int* perm,
                                    double* A, size_t lda, const double* b, int P, double* bout,
                                    cudaStream_t s, long long* nl) {
  if (A) {
    k_unpermute_op<<<dim3((nu + 255) / 256, nu < 65535 ? nu : 65535), 256, 0, s>>>(M, np, nu, N, perm, A,
                                                                              lda);
    ++*nl;
  }
  if (bout) {
    k_unpermute_rows<<<(nu * P + 255) / 256, 256, 0, s>>>(b, nu, N, P, perm, bout);
    ++*nl;
  }
  return cudaGetLastError();
}

namespace {
// Boundary-element operators of a meshed surface (Sec. 2.3).  Ft is not symmetric, and
// the FP32 / FP64 / double-FP32 block matvecs read row k of the stored operator as column
// k of the applied one (exact for the symmetric T of Eqs. 1 and 7), so these operators are
// stored transposed: S[j][i] = Op[i][j].
//   DPCM (Eq. 11, normal-field form): Op_ij = A_j (s_i - s_j).n_i / |s_i - s_j|^3 (i != j),
//     Op_ii = +1.0694 sqrt(4 pi A_i) / (2R);
//   IEFPCM (Eq. 12): Op_ij = A_j (s_i - s_j).n_j / |s_i - s_j|^3 (i != j),
//     Op_ii = -1.0694 sqrt(4 pi A_i) / (2R)  (the sign of the off-diagonal double-layer sum).
__global__ void k_build_F(const double* __restrict__ pos, const double* __restrict__ nrm,
                          const double* __restrict__ area, double R, int n, int ld, int ief,
                          double* S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // row of Op, column of S
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  double v;
  if (i == j) {
    v = 1.0694 * sqrt(4.0 * 3.141592653589793 * area[i]) / (2.0 * R);
    if (ief) v = -v;
  } else {
    const double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                 dz = pos[3 * i + 2] - pos[3 * j + 2];
    const double r2 = dx * dx + dy * dy + dz * dz;
    const int t = ief ? j : i;
    const double dn = dx * nrm[3 * t] + dy * nrm[3 * t + 1] + dz * nrm[3 * t + 2];
    v = area[j] * dn / (r2 * sqrt(r2));
  }
  S[(size_t)j * ld + i] = v;
}

// S A^-1 of Eq. 12 (the Coulomb matrix of the tesserae, symmetric): 1/|s_i - s_j| off the
// diagonal, 1.0694 sqrt(4 pi / A_i) on it.
__global__ void k_build_G(const double* __restrict__ pos, const double* __restrict__ area, int n,
                          int ld, double* G) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  double v;
  if (i == j) {
    v = 1.0694 * sqrt(4.0 * 3.141592653589793 / area[i]);
  } else {
    const double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                 dz = pos[3 * i + 2] - pos[3 * j + 2];
    v = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
  }
  G[(size_t)i * ld + j] = v;
}

// M = S^T through 32 x 32 shared-memory tiles, and max |M| (integer atomicMax on the bits
// of the non-negative double).
__global__ void __launch_bounds__(256) k_transpose_absmax(const double* __restrict__ S, int np,
                                                          double* M, unsigned long long* absmax_bits) {
  __shared__ double tile[32][33];
  __shared__ double sh[8];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  double amax = 0.0;
  for (int r = ty; r < 32; r += 8) tile[r][tx] = S[(size_t)(by + r) * np + bx + tx];
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const double v = tile[tx][r];
    M[(size_t)(bx + r) * np + by + tx] = v;
    amax = fmax(amax, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if (tx == 0) sh[ty] = amax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < 8; ++w) m = fmax(m, sh[w]);
    atomicMax(absmax_bits, (unsigned long long)__double_as_longlong(m));
  }
}
}  // namespace

cudaError_t launch_build_F(const double* pos, const double* nrm, const double* area, double R,
                           int n, int np, bool ief, double* S, cudaStream_t s, long long* nl) {
  cudaError_t e = cudaMemsetAsync(S, 0, sizeof(double) * (size_t)np * np, s);
  if (e != cudaSuccess) return e;
  dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
  k_build_F<<<grd, blk, 0, s>>>(pos, nrm, area, R, n, np, ief ? 1 : 0, S);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_build_G(const double* pos, const double* area, int n, int np, double* G,
                           cudaStream_t s, long long* nl) {
  cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * (size_t)np * np, s);
  if (e != cudaSuccess) return e;
  dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
  k_build_G<<<grd, blk, 0, s>>>(pos, area, n, np, G);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_transpose_absmax(const double* S, int np, double* M,
                                    unsigned long long* absmax_bits, cudaStream_t s, long long* nl) {
  if (np % 32) return cudaErrorInvalidValue;
  k_transpose_absmax<<<dim3(np / 32, np / 32), 256, 0, s>>>(S, np, M, absmax_bits);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace px
