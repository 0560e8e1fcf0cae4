// Block matvec Y = T X on the 5th-generation tensor cores (tcgen05), split precision.
//
// BF16 split:  T = T_hi + T_lo, X = X_hi + X_lo (bf16; hi = RN(v), lo = RN(v - hi)),
//   Y = T_hi X_hi + T_hi X_lo + T_lo X_hi  in one FP32 TMEM accumulator
//   (~16 significant bits per product: the dropped T_lo X_lo is below 2^-16 relative).
// FP16 split:  T' = 2^12 T, X' = 2^8 X (X is a unit vector), hi = RN_fp16(v'),
//   lo = RN_fp16((v' - hi) 2^11), so that every part stays in fp16's normal range;
//   D1 = T_hi X_hi and D2 = T_hi X_lo + T_lo X_hi in two TMEM accumulators,
//   Y = (D1 + 2^-11 D2) 2^-20  (~22 significant bits per product; FP32 accumulation).
// One CTA computes a 128 x BN tile of Y (BN = 256 with a 2-stage ring, or BN = 128
// with a 3-stage ring; launch_tc_gemm's autotuner picks one per shape):
//   warp 0   TMA producer: per 64-wide K step, loads T_hi, T_lo (128 x 64) and
//            X_hi, X_lo (BN x 64, from the transposed operand Xt[c][k]) into a
//            ring of 128B-swizzled shared-memory tiles;
//   warp 1   one elected thread issues 4 x 3 tcgen05.mma (M = 128, N = BN, K = 16)
//            per K step into the TMEM accumulator(s) and releases the stage with
//            tcgen05.commit;
//   warps 4-7 epilogue: tcgen05.ld of the 128 x BN FP32 accumulator, row-major store.
// Every output element accumulates its K products in the same order for either tile
// shape, so the variants give bit-identical Y.
// Every mbarrier wait is bounded by a clock64 limit; on time-out the kernel sets an
// error flag, stops issuing work, waits (bounded) for its accumulator, frees its
// TMEM and returns.
#include "px_internal.cuh"

#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <set>
#include <tuple>

namespace px {

namespace {

constexpr int TC_BM = 128, TC_BK = 64;
constexpr int A_TILE = TC_BM * TC_BK * 2;                  // 16 KB
constexpr long long kWaitCycles = 4000000000LL;            // ~2 s at 2 GHz

// Tile configuration: BN operand columns per CTA, STAGES-deep ring.
template <int BN, int STAGES>
struct TcCfg {
  static constexpr int B_TILE = BN * TC_BK * 2;                     // 32 / 16 KB
  static constexpr int STAGE = 2 * A_TILE + 2 * B_TILE;              // 96 / 64 KB
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;           // + alignment, barriers
  static constexpr int TMEM_COLS = 2 * BN;   // two 128 x BN FP32 accumulators (BF16 uses one)
  static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
  static_assert(TMEM_COLS == 256 || TMEM_COLS == 512, "TMEM allocation is a power of two");
};

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; false (and *err set) when the limit ran out or
// another role of this kernel already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err,
                                          volatile int* cta_abort) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (*cta_abort) return false;
    if (clock64() - t0 > kWaitCycles) {
      *cta_abort = 1;
      atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), sm_100 descriptor version.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16 (format 1) or F16 (format 0),
// both K-major, M = 128, N = BN.
template <int BN>
__host__ __device__ constexpr uint32_t idesc(bool f16) {
  return (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24) |
         (f16 ? 0u : ((1u << 7) | (1u << 10)));
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                        uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}

#define TMEM_LD32(taddr, v)                                                                      \
  asm volatile(                                                                                  \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "    \
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "    \
      "%28, %29, %30, %31}, [%32];"                                                              \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),     \
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),               \
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),            \
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),            \
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),            \
        "=r"(v[31])                                                                              \
      : "r"(taddr))

template <int F16, int TC_BN, int TC_STAGES>
__global__ void __launch_bounds__(256, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap mTh, const __grid_constant__ CUtensorMap mTl,
          const __grid_constant__ CUtensorMap mXh, const __grid_constant__ CUtensorMap mXl,
          float* __restrict__ Y, int ldy, int K, int* err) {
  using Cfg = TcCfg<TC_BN, TC_STAGES>;
  constexpr int B_TILE = Cfg::B_TILE, STAGE = Cfg::STAGE, TC_TMEM_COLS = Cfg::TMEM_COLS;
  constexpr uint32_t kIdescF16 = idesc<TC_BN>(true), kIdescBF16 = idesc<TC_BN>(false);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + TC_STAGES * STAGE);
  uint64_t* full = bars;                    // [TC_STAGES]
  uint64_t* empty = bars + TC_STAGES;       // [TC_STAGES]
  uint64_t* accum = bars + 2 * TC_STAGES;   // [1]
  __shared__ uint32_t tmem_slot;
  __shared__ int cta_abort;
  __shared__ int n_issued, n_consumed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.y * TC_BM, c0 = blockIdx.x * TC_BN;
  const int nk = K / TC_BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    cta_abort = 0;
    n_issued = 0;
    n_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abort_flag = &cta_abort;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % TC_STAGES;
      const uint32_t ph = (uint32_t)(kt / TC_STAGES) & 1u;
      if (kt >= TC_STAGES && !mbar_wait(&empty[s], ph ^ 1u, err, abort_flag)) break;
      unsigned char* st = base + s * STAGE;
      mbar_expect_tx(&full[s], STAGE);
      const int kx = kt * TC_BK;
      tma_load_2d(st, &mTh, &full[s], kx, i0);
      tma_load_2d(st + A_TILE, &mTl, &full[s], kx, i0);
      tma_load_2d(st + 2 * A_TILE, &mXh, &full[s], kx, c0);
      tma_load_2d(st + 2 * A_TILE + B_TILE, &mXl, &full[s], kx, c0);
      n_issued = kt + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    bool ok = true;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % TC_STAGES;
      const uint32_t ph = (uint32_t)(kt / TC_STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, err, abort_flag)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = su32(base + s * STAGE);
      const uint64_t ah = sdesc(st), al = sdesc(st + A_TILE);
      const uint64_t bh = sdesc(st + 2 * A_TILE), bl = sdesc(st + 2 * A_TILE + B_TILE);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
        const uint64_t dk = (uint64_t)(kk * 32) >> 4;   // 16 elements = 32 bytes along K
        const uint32_t first = (kt | kk) ? 1u : 0u;
        if (F16) {
          mma_f16(tmem, ah + dk, bh + dk, kIdescF16, first);
          mma_f16(tmem + TC_BN, ah + dk, bl + dk, kIdescF16, first);
          mma_f16(tmem + TC_BN, al + dk, bh + dk, kIdescF16, 1u);
        } else {
          mma_f16(tmem, ah + dk, bh + dk, kIdescBF16, first);
          mma_f16(tmem, ah + dk, bl + dk, kIdescBF16, 1u);
          mma_f16(tmem, al + dk, bh + dk, kIdescBF16, 1u);
        }
      }
      mma_commit(&empty[s]);
      n_consumed = kt + 1;
    }
    (void)ok;
    mma_commit(accum);   // arrives once every MMA issued above has completed
  } else if (warp >= 4) {
    // ---------------- epilogue: TMEM -> registers -> Y
    const bool ok = mbar_wait(accum, 0, err, abort_flag);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int wq = warp & 3;                      // TMEM lanes 32*wq .. 32*wq+31
    const int row = i0 + wq * 32 + lane;
    if (ok && !*abort_flag) {
      float* yr = Y + (size_t)row * ldy + c0;
#pragma unroll 1
      for (int cc = 0; cc < TC_BN; cc += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)cc;
        TMEM_LD32(taddr, v);
        if (F16) {
          uint32_t v2[32];
          TMEM_LD32(taddr + TC_BN, v2);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          const float s1 = 1.0f / 1048576.0f;             // 2^-20
          const float s2 = 1.0f / 2147483648.0f;          // 2^-31
#pragma unroll
          for (int q = 0; q < 32; ++q)
            v[q] = __float_as_uint(fmaf(__uint_as_float(v2[q]), s2, __uint_as_float(v[q]) * s1));
        } else {
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(yr + cc + 4 * q) =
              make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                          __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
      }
    }
  }
  // every role is done with TMEM (the accumulator barrier was waited on by the epilogue)
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (cta_abort && threadIdx.x == 0) {
    // after a time-out: wait (bounded) for TMA loads that were issued but never consumed
    for (int kt = n_consumed; kt < n_issued; ++kt) {
      const long long t0 = clock64();
      while (!mbar_try(&full[kt % TC_STAGES], (uint32_t)(kt / TC_STAGES) & 1u) &&
             clock64() - t0 < kWaitCycles) {
      }
    }
  }
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TC_TMEM_COLS));
  }
}

// Xt_hi[c][k], Xt_lo[c][k] (K-major) from X[k][c] (FP32, row-major); 32 x 32 tiles.
// BF16: hi = RN(x), lo = RN(x - hi).  FP16: x' = 2^8 x, hi = RN(x'), lo = RN((x' - hi) 2^11).
// PERM (wFQFmu, N atoms): K index k is atom-blocked, groups of 16 atoms holding their 16
// charges then their 48 dipole components (atom by atom), read from the charges-first row
// of X; the unknowns of atoms beyond N are 0.
template <int F16, int PERM>
__global__ void k_split_xt(const float* __restrict__ X, int ldx, int K, int N,
                           uint16_t* __restrict__ Xh, uint16_t* __restrict__ Xl) {
  __shared__ float tile[32][33];
  const int k0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    int row = k0 + r;
    bool real = true;
    if (PERM) {
      const int g = row >> 6, w = row & 63, b0 = 16 * g;
      const int atom = w < 16 ? b0 + w : b0 + (w - 16) / 3;
      real = atom < N;
      row = w < 16 ? atom : N + 3 * b0 + (w - 16);
    }
    tile[r][threadIdx.x] = real ? X[(size_t)row * ldx + c0 + threadIdx.x] : 0.0f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const float v = tile[threadIdx.x][r];
    const size_t o = (size_t)(c0 + r) * K + k0 + threadIdx.x;
    if (F16) {
      const float vs = v * 256.0f;
      const __half h = __float2half_rn(vs);
      Xh[o] = __half_as_ushort(h);
      Xl[o] = __half_as_ushort(__float2half_rn((vs - __half2float(h)) * 2048.0f));
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      Xh[o] = __bfloat16_as_ushort(h);
      Xl[o] = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  // looked up once (thread-safe static initialisation); nullptr if the driver lacks it
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
  }();
  return fn;
}

// 2D 16-bit tensor [rows][cols] (cols contiguous), box = 64 x box_rows, 128B swizzle.
bool make_map(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols, uint32_t box_rows,
              bool f16) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(ptr), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_split_xt(const float* X, int ldx, int np, int ncols, uint16_t* Xh,
                            uint16_t* Xl, bool f16, cudaStream_t s, long long* nl) {
  if (np % 32 || ncols % 32) return cudaErrorInvalidValue;
  dim3 grd(np / 32, ncols / 32), blk(32, 8);
  if (f16) k_split_xt<1, 0><<<grd, blk, 0, s>>>(X, ldx, np, 0, Xh, Xl);
  else k_split_xt<0, 0><<<grd, blk, 0, s>>>(X, ldx, np, 0, Xh, Xl);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_split_xt_mu(const float* X, int ldx, int np, int ncols, int N, uint16_t* Xh,
                               uint16_t* Xl, bool f16, cudaStream_t s, long long* nl) {
  // every K index maps to a row below 4 N <= np
  if (np % 64 || ncols % 32 || N < 1 || 4 * (long long)N > np) return cudaErrorInvalidValue;
  dim3 grd(np / 32, ncols / 32), blk(32, 8);
  if (f16) k_split_xt<1, 1><<<grd, blk, 0, s>>>(X, ldx, np, N, Xh, Xl);
  else k_split_xt<0, 1><<<grd, blk, 0, s>>>(X, ldx, np, N, Xh, Xl);
  ++*nl;
  return cudaGetLastError();
}

namespace {

template <int F16, int BN, int ST>
cudaError_t launch_variant(const CUtensorMap& mTh, const CUtensorMap& mTl, const CUtensorMap& mXh,
                           const CUtensorMap& mXl, int np, int ncols, float* Y, int ldy, int* err,
                           cudaStream_t s) {
  dim3 grd(ncols / BN, np / TC_BM);
  k_tc_gemm<F16, BN, ST><<<grd, 256, TcCfg<BN, ST>::SMEM, s>>>(mTh, mTl, mXh, mXl, Y, ldy, np, err);
  return cudaGetLastError();
}

template <int F16>
cudaError_t set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<F16, 256, 2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TcCfg<256, 2>::SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_gemm<F16, 128, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcCfg<128, 3>::SMEM);
  return e;
}

// Tile variants: 0 = 128 x 256 tiles, 2-stage ring; 1 = 128 x 128 tiles, 3-stage ring.
constexpr int kTcVariants = 2;
constexpr int kTcBN[kTcVariants] = {256, 128};

cudaError_t launch_tc_variant(int v, bool f16, const CUtensorMap* m, int np, int ncols, float* Y,
                              int ldy, int* err, cudaStream_t s) {
  if (f16)
    return v == 0 ? launch_variant<1, 256, 2>(m[0], m[1], m[2], m[3], np, ncols, Y, ldy, err, s)
                  : launch_variant<1, 128, 3>(m[0], m[1], m[2], m[3], np, ncols, Y, ldy, err, s);
  return v == 0 ? launch_variant<0, 256, 2>(m[0], m[1], m[2], m[3], np, ncols, Y, ldy, err, s)
                : launch_variant<0, 128, 3>(m[0], m[1], m[2], m[3], np, ncols, Y, ldy, err, s);
}

// Autotuner cache: (device, np, ncols, f16) -> fastest variant, measured once per
// process on the first matvec of that shape.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune;

}  // namespace

cudaError_t launch_tc_gemm(const uint16_t* Th, const uint16_t* Tl, int np, const uint16_t* Xh,
                           const uint16_t* Xl, int ncols, float* Y, int ldy, bool f16, int* err,
                           cudaStream_t s, long long* nl, int variant, int* used) {
  // shape contract: M and K tiles of 128 / 64 rows of T, N tiles of 128 or 256 operand
  // columns, 16-byte aligned rows; every TMA x coordinate is a multiple of 64 elements
  // (128 bytes).  The 256-column tiles need ncols % 256 == 0; other column counts run
  // the 128-column tiles.
  if (np % TC_BM || ncols % 128 || ldy % 4 || ldy < ncols) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(Th) | reinterpret_cast<uintptr_t>(Tl) |
       reinterpret_cast<uintptr_t>(Xh) | reinterpret_cast<uintptr_t>(Xl)) & 15)
    return cudaErrorMisalignedAddress;
  if (variant < -1 || variant >= kTcVariants) return cudaErrorInvalidValue;
  auto fits = [&](int v) { return ncols % kTcBN[v] == 0; };
  if (variant >= 0 && !fits(variant)) variant = 1;   // 128-column tiles fit every shape
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    static std::mutex attr_mu;
    static std::set<int> attr_done;
    std::lock_guard<std::mutex> lock(attr_mu);
    if (!attr_done.count(dev)) {
      e = set_attrs<0>();
      if (e == cudaSuccess) e = set_attrs<1>();
      if (e != cudaSuccess) return e;
      attr_done.insert(dev);
    }
  }
  CUtensorMap maps[4];
  auto encode = [&](int bn) {
    return make_map(&maps[0], Th, np, np, TC_BM, f16) && make_map(&maps[1], Tl, np, np, TC_BM, f16) &&
           make_map(&maps[2], Xh, ncols, np, bn, f16) && make_map(&maps[3], Xl, ncols, np, bn, f16);
  };
  if (variant < 0) {
    const auto key = std::make_tuple(dev, np, ncols, f16 ? 1 : 0);
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) variant = it->second;
    }
    if (variant < 0) {
      // time every variant on these operands (each writes the same Y), twice each,
      // keep the faster; the stream is synchronised once per new shape
      cudaEvent_t ev[2 * kTcVariants + 1];
      for (auto& x : ev) {
        e = cudaEventCreate(&x);
        if (e != cudaSuccess) return e;
      }
      for (int v = 0; v < kTcVariants && e == cudaSuccess; ++v) {
        if (!fits(v)) continue;
        if (!encode(kTcBN[v])) e = cudaErrorInvalidValue;
        if (e == cudaSuccess) e = launch_tc_variant(v, f16, maps, np, ncols, Y, ldy, err, s);   // warm
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * v], s);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r)
          e = launch_tc_variant(v, f16, maps, np, ncols, Y, ldy, err, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * v + 1], s);
        *nl += 3;
      }
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[2 * kTcVariants - 1]);
      float best_ms = 0.f;
      variant = -1;
      for (int v = 0; v < kTcVariants && e == cudaSuccess; ++v) {
        if (!fits(v)) continue;
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ev[2 * v], ev[2 * v + 1]);
        if (e == cudaSuccess && (variant < 0 || ms < best_ms)) {
          best_ms = ms;
          variant = v;
        }
      }
      for (auto& x : ev) cudaEventDestroy(x);
      if (e != cudaSuccess) return e;
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune[key] = variant;
    }
  }
  if (!encode(kTcBN[variant])) return cudaErrorInvalidValue;
  e = launch_tc_variant(variant, f16, maps, np, ncols, Y, ldy, err, s);
  ++*nl;
  if (used) *used = variant;
  return e;
}

int tc_tuned_variant(int np, int ncols, bool f16) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(dev, np, ncols, f16 ? 1 : 0));
  return it == g_tune.end() ? -1 : it->second;
}

}  // namespace px

#include "px_radial.cuh"

namespace px {

// ---------------------------------------------------------------- on-the-fly pair kernel
// Matrix-free wFQ block matvec Y = T X on the tensor cores: the T tile of every 64-atom K
// step is generated from the atom positions (Eq. 5 in FP32) by sixteen generator warps
// straight into shared memory, as the hi / lo planes of the split (the layout a
// 128-byte-swizzled TMA load would produce), and contracted with the X tiles (TMA) by
// tcgen05.mma exactly as in k_tc_gemm; nothing of T is stored.
//   warp 0        TMA producer: the 64 atoms' positions of each K step (1 KB bulk copies,
//                 running ahead) and the X hi / lo tiles (BN x 64)
//   warp 1        MMA issuer (one elected thread, 4 x 3 MMAs per K step)
//   warp 2        TMEM allocation
//   warps 4-19    generators: warp w writes the 16-byte chunk c = w % 8 (atoms 8c .. 8c+7
//                 of the step) of 64 rows (lane, lane + 32 of its half), so the warp reads
//                 the same eight positions (a broadcast) and its stores cover eight swizzled
//                 chunk positions (no bank conflicts); then warps 4-7 run the epilogue
// Positions come pre-scaled by 2^-e (launch_tc_mf_positions), so 1/r and erf(r/R)/r are
// generated as 2^e T directly, and padded to np atoms with distinct far-away dummies
// (their columns meet zero operand rows; their rows are never read); they are stored as
// atom pairs with negated coordinates, so the differences and r^2 run as packed FP32x2
// operations (two pairs per instruction).  A pair costs one
// reciprocal square root while r >= 4 R (erf(r/R) = 1 in FP32); closer pairs take
// erf(r/R)/r, or sqrt(2/pi)/R_q on the diagonal, in a branch a warp enters only when one
// of its lanes has such a pair (atoms are in Morton order, so most tiles have none).
// Barriers: per position slot (a 4-slot ring the producer keeps 3 K steps ahead) pos_full
// (copy landed) and pos_empty (all generator warps finished the step that used it); per
// stage full (X bytes +
// sixteen generator arrivals, each after a proxy fence so the tensor core sees the
// generic-proxy stores) and empty (MMA commit; the generators wait for it before writing
// the stage's A tile again).  Close pairs use the branch-free erf of erf_as.
// FP16 split: hi = RN(2^e T), lo = RN((2^e T - hi) 2^11), Y = D1 2^-(e+8) + D2 2^-(e+19)
// (X' = 2^8 X).  BF16 split (e = 0): hi = RN(T), lo = RN(T - hi), one accumulator, Y = D.
// wFQFmu (MU = 1, Sec. 2.2): the unknowns are reordered atom-blocked, so that a 128-row tile
// holds those of 32 atoms (their 32 charges, then their dipoles x, y, z atom by atom) and a
// 64-unknown K step those of 16 atoms in the same order (launch_split_xt_mu permutes X
// alike; the epilogue writes each row back to its place in the charges-first vector).
// Generator thread (al, bl) evaluates the 4 x 4 block of T^qq / T^qmu / T^muq / T^mumu of
// row atom al and column atom bl of the step (512 blocks, one per generator thread), in
// FP32 from unscaled positions: the closed far-field forms (1/r, d/r^3, (I - 3 rhat rhat)/r^3)
// when every pair of the warp has r >= 5 R for all four widths (erf = 1 and the Gaussian
// terms below 1e-9 there), else the full radial functions; the block is multiplied by 2^e
// (tscale) before the split, and blocks with an atom beyond N are zero.
namespace {

constexpr int kMfGenWarps = 16;
constexpr int kMfThreads = 128 + 32 * kMfGenWarps;
constexpr int kMfPosBytes = TC_BK * 16;   // 64 float4 per K step
constexpr int kMfPosSlots = 4;            // position ring: copies run 3 K steps ahead

// erf for close pairs: Abramowitz & Stegun 7.1.26 (after Hastings), |error| <= 1.5e-7 for
// x >= 0, below the 2^-22 resolution of the fp16 split for the x >= ~1 of distinct atoms;
// branch-free: one reciprocal and one exponential on the SFU.
__device__ __forceinline__ float erf_as(float x) {
  const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
  float p = fmaf(1.061405429f, t, -1.453152027f);
  p = fmaf(p, t, 1.421413741f);
  p = fmaf(p, t, -0.284496736f);
  p = fmaf(p, t, 0.254829592f);
  p *= t;
  return fmaf(-p, __expf(-x * x), 1.0f);
}

template <int F16, int TC_BN, int TC_STAGES, int MU>
__global__ void __launch_bounds__(kMfThreads, 1)
k_tc_mf(const float4* __restrict__ pos, float wmax, float tscale, int N, int mu_self,
        const __grid_constant__ CUtensorMap mXh, const __grid_constant__ CUtensorMap mXl,
        float* __restrict__ Y, int ldy, int K, float s1, float s2, int* err) {
  using Cfg = TcCfg<TC_BN, TC_STAGES>;
  constexpr int B_TILE = Cfg::B_TILE, STAGE = Cfg::STAGE, TC_TMEM_COLS = Cfg::TMEM_COLS;
  constexpr uint32_t kIdescF16 = idesc<TC_BN>(true), kIdescBF16 = idesc<TC_BN>(false);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float4* spos = reinterpret_cast<float4*>(base + TC_STAGES * STAGE);   // [kMfPosSlots][64]
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + TC_STAGES * STAGE + kMfPosSlots * kMfPosBytes);
  uint64_t* full = bars;                      // [TC_STAGES]: X bytes + generator warps
  uint64_t* empty = bars + TC_STAGES;         // [TC_STAGES]: MMA commit
  uint64_t* pfull = bars + 2 * TC_STAGES;     // [kMfPosSlots]: positions landed
  uint64_t* pempty = pfull + kMfPosSlots;     // [kMfPosSlots]: generator warps read them
  uint64_t* accum = pempty + kMfPosSlots;     // [1]
  __shared__ uint32_t tmem_slot;
  __shared__ int cta_abort;
  __shared__ int n_issued, n_consumed, p_issued, p_consumed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.y * TC_BM, c0 = blockIdx.x * TC_BN;
  const int nk = K / TC_BK;

  if (threadIdx.x == 0) {
    p_issued = 0;
    p_consumed = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1 + kMfGenWarps);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < kMfPosSlots; ++s) {
      mbar_init(&pfull[s], 1);
      mbar_init(&pempty[s], kMfGenWarps);
    }
    mbar_init(accum, 1);
    cta_abort = 0;
    n_issued = 0;
    n_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abort_flag = &cta_abort;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: positions (a ring running ahead), operand tiles
    // one K step's positions: 64 atoms x 16 bytes (wFQ), 16 atoms x 32 bytes (wFQFmu)
    constexpr int kStepPos = MU ? 32 : TC_BK;   // float4 per K step
    constexpr int kStepBytes = kStepPos * 16;
    auto issue_pos = [&](int kp) {   // positions of K step kp into slot kp % kMfPosSlots
      const int ps = kp % kMfPosSlots;
      if (kp >= kMfPosSlots &&
          !mbar_wait(&pempty[ps], (uint32_t)((kp / kMfPosSlots) & 1) ^ 1u, err, abort_flag))
        return false;
      mbar_expect_tx(&pfull[ps], kStepBytes);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              su32(spos + ps * TC_BK)),
          "l"(reinterpret_cast<uint64_t>(pos + (size_t)kp * kStepPos)), "r"(kStepBytes), "r"(su32(&pfull[ps]))
          : "memory");
      p_issued = kp + 1;
      return true;
    };
    bool ok = true;
    for (int kp = 0; kp < kMfPosSlots - 1 && kp < nk && ok; ++kp) ok = issue_pos(kp);
    for (int kt = 0; kt < nk && ok; ++kt) {
      const int s = kt % TC_STAGES;
      const uint32_t ph = (uint32_t)(kt / TC_STAGES) & 1u;
      if (kt >= TC_STAGES && !mbar_wait(&empty[s], ph ^ 1u, err, abort_flag)) break;
      unsigned char* st = base + s * STAGE;
      mbar_expect_tx(&full[s], 2 * B_TILE);
      const int kx = kt * TC_BK;
      tma_load_2d(st + 2 * A_TILE, &mXh, &full[s], kx, c0);
      tma_load_2d(st + 2 * A_TILE + B_TILE, &mXl, &full[s], kx, c0);
      n_issued = kt + 1;
      // positions of step kt + 3 (their slot frees when the generators finish step kt - 1)
      if (kt + kMfPosSlots - 1 < nk && !issue_pos(kt + kMfPosSlots - 1)) break;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % TC_STAGES;
      const uint32_t ph = (uint32_t)(kt / TC_STAGES) & 1u;
      if (!mbar_wait(&full[s], ph, err, abort_flag)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = su32(base + s * STAGE);
      const uint64_t ah = sdesc(st), al = sdesc(st + A_TILE);
      const uint64_t bh = sdesc(st + 2 * A_TILE), bl = sdesc(st + 2 * A_TILE + B_TILE);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
        const uint64_t dk = (uint64_t)(kk * 32) >> 4;
        const uint32_t first = (kt | kk) ? 1u : 0u;
        if (F16) {
          mma_f16(tmem, ah + dk, bh + dk, kIdescF16, first);
          mma_f16(tmem + TC_BN, ah + dk, bl + dk, kIdescF16, first);
          mma_f16(tmem + TC_BN, al + dk, bh + dk, kIdescF16, 1u);
        } else {
          mma_f16(tmem, ah + dk, bh + dk, kIdescBF16, first);
          mma_f16(tmem, ah + dk, bl + dk, kIdescBF16, 1u);
          mma_f16(tmem, al + dk, bh + dk, kIdescBF16, 1u);
        }
      }
      mma_commit(&empty[s]);
      n_consumed = kt + 1;
    }
    mma_commit(accum);
  } else if (warp >= 4) {
    if constexpr (MU == 0) {
      // ---------------- generators: T tiles in the swizzled K-major layout
      // Positions arrive as atom pairs [-x0 -x1 -y0 -y1 -z0 -z1 w0 w1] (w = R_q^2), so that the
      // differences and r^2 of two atoms run as packed FP32x2 instructions.
      const int gw = warp - 4;                     // 0 .. 15
      const int c = gw & 7;                        // 16-byte chunk (atoms 8c .. 8c+7 of the step)
      const int r_lo = (gw >> 3) * 64 + lane;      // rows r_lo and r_lo + 32
      const float* posf = reinterpret_cast<const float*>(pos);
      float2 px[2], py[2], pz[2];
      float pw[2], thr[2];
  #pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int i = i0 + r_lo + 32 * u;
        const float* pp = posf + (size_t)(i >> 1) * 8 + (i & 1);
        const float x = -__ldg(pp), y = -__ldg(pp + 2), z = -__ldg(pp + 4);
        px[u] = make_float2(x, x);
        py[u] = make_float2(y, y);
        pz[u] = make_float2(z, z);
        pw[u] = __ldg(pp + 6);
        thr[u] = 16.0f * (pw[u] + wmax);           // r^2 below this: a close pair is possible
      }
      const uint32_t sw = (uint32_t)((c ^ (lane & 7)) << 4);   // row & 7 == lane & 7
      const float2 k2048 = make_float2(2048.0f, 2048.0f), km1 = make_float2(-1.0f, -1.0f);
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % TC_STAGES;
        const uint32_t ph = (uint32_t)(kt / TC_STAGES) & 1u;
        const int ps = kt % kMfPosSlots;
        // this step's positions (copied ahead), then release their slot
        if (!mbar_wait(&pfull[ps], (uint32_t)(kt / kMfPosSlots) & 1u, err, abort_flag)) break;
        // atoms 8c .. 8c+7 = pairs 4c .. 4c+3
        float2 kx[4], ky[4], kz[4], kw[4];
  #pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 a = spos[ps * TC_BK + (4 * c + q) * 2];
          const float4 b = spos[ps * TC_BK + (4 * c + q) * 2 + 1];
          kx[q] = make_float2(a.x, a.y);
          ky[q] = make_float2(a.z, a.w);
          kz[q] = make_float2(b.x, b.y);
          kw[q] = make_float2(b.z, b.w);
        }
        // the A stage is free once the MMA of step kt - TC_STAGES completed
        if (kt >= TC_STAGES && !mbar_wait(&empty[s], ph ^ 1u, err, abort_flag)) break;
        unsigned char* sth = base + s * STAGE;
        unsigned char* stl = sth + A_TILE;
        const int kb = kt * TC_BK + c * 8;
  #pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int r = r_lo + 32 * u;
          float2 r2[4];
          float t[8];
          float mn = 3.0e38f;
  #pragma unroll
          for (int q = 0; q < 4; ++q) {
            // (x_i - x_k) for two atoms k: the pair holds -x_k
            const float2 dx = __fadd2_rn(px[u], kx[q]), dy = __fadd2_rn(py[u], ky[q]),
                         dz = __fadd2_rn(pz[u], kz[q]);
            r2[q] = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
            t[2 * q] = rsqrtf(r2[q].x);
            t[2 * q + 1] = rsqrtf(r2[q].y);
            mn = fminf(mn, fminf(r2[q].x, r2[q].y));
          }
          if (__any_sync(0xffffffffu, mn < thr[u])) {
            const int i = i0 + r;
  #pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float rr = (e & 1) ? r2[e >> 1].y : r2[e >> 1].x;
              const float wk = (e & 1) ? kw[e >> 1].y : kw[e >> 1].x;
              const float R2 = pw[u] + wk;
              if (i == kb + e) t[e] = radial::kSqrt2OverPiF * rsqrtf(pw[u]);
              else if (rr < 16.0f * R2) t[e] = erf_as(rr * t[e] * rsqrtf(R2)) * t[e];
            }
          }
          uint32_t hw[4], lw[4];
  #pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 tv = make_float2(t[2 * q], t[2 * q + 1]);
            if (F16) {
              const __half2 h = __float22half2_rn(tv);
              const float2 hf = __half22float2(h);
              // lo = RN((t - hi) 2^11)
              const __half2 l = __float22half2_rn(__fmul2_rn(__ffma2_rn(hf, km1, tv), k2048));
              hw[q] = *reinterpret_cast<const uint32_t*>(&h);
              lw[q] = *reinterpret_cast<const uint32_t*>(&l);
            } else {
              const __nv_bfloat162 h = __float22bfloat162_rn(tv);
              const float2 hf = __bfloat1622float2(h);
              const __nv_bfloat162 l = __float22bfloat162_rn(__ffma2_rn(hf, km1, tv));
              hw[q] = *reinterpret_cast<const uint32_t*>(&h);
              lw[q] = *reinterpret_cast<const uint32_t*>(&l);
            }
          }
          const uint32_t off = (uint32_t)r * 128u + sw;
          *reinterpret_cast<uint4*>(sth + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(stl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        // make the generic-proxy stores visible to the tensor core, then one arrival per warp
        // on the stage (A tile written) and on the position slot (its values are consumed:
        // releasing the slot any earlier let its next copy race the loads)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&full[s])) : "memory");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&pempty[ps])) : "memory");
          if (gw == 0) p_consumed = kt + 1;
        }
      }
    } else {
      // ---------------- wFQFmu generators: rows of 4 x 4 blocks in the swizzled K-major layout
      // Warp gw = 8 hh + 4 o + u writes row component u (0: charge, 1-3: dipole x, y, z) of
      // the tile's 32 row atoms (one per lane) against column atoms kc .. kc + 3 of the step
      // (kc = 8 o + 4 hh): per plane one 8-byte store of their 4 charge columns and a 16- and
      // an 8-byte store of their 12 dipole columns.  Lanes of a warp differ in the row only,
      // whose swizzle spreads them over the banks.
      const int gw = warp - 4;                       // 0 .. 15
      const int u = gw & 3, o = (gw >> 2) & 1, hh = gw >> 3;
      const int kdir = u - 1;                        // dipole component of a dipole row
      const int a = blockIdx.y * 32 + lane;
      const float4 pa = __ldg(pos + 2 * a);
      const float wma = __ldg(pos + 2 * a + 1).x;
      const float wa = fmaxf(pa.w, wma);
      const int r = u == 0 ? lane : 32 + 3 * lane + kdir;
      const int kc = 8 * o + 4 * hh;                 // charge columns kc .. kc + 3
      const int kd = 16 + 24 * o + 12 * hh;          // dipole columns kd .. kd + 11
      auto soff = [&](int k) -> uint32_t {
        return (uint32_t)r * 128u + ((uint32_t)((k >> 3) ^ (r & 7)) << 4) + (uint32_t)(k & 7) * 2u;
      };
      // hh = 0: dipole columns as 8 + 4; hh = 1: as 4 + 8 (16-byte chunks start at kd + 4)
      const uint32_t oc = soff(kc), od1 = soff(kd), od2 = soff(kd + (hh ? 4 : 8));
      const float qself = radial::kSqrt2OverPiF * rsqrtf(pa.w);
      const float vself = mu_self ? 4.0f / (3.0f * 1.7724538509055159f) * rsqrtf(2.0f * wma) /
                                        (2.0f * wma)
                                  : 0.0f;
      const float2 k2048 = make_float2(2048.0f, 2048.0f), km1 = make_float2(-1.0f, -1.0f);
      auto split2 = [&](float v0, float v1, uint32_t& hw, uint32_t& lw) {
        const float2 tv = make_float2(v0, v1);
        if (F16) {
          const __half2 h = __float22half2_rn(tv);
          const float2 hf = __half22float2(h);
          const __half2 l = __float22half2_rn(__fmul2_rn(__ffma2_rn(hf, km1, tv), k2048));
          hw = *reinterpret_cast<const uint32_t*>(&h);
          lw = *reinterpret_cast<const uint32_t*>(&l);
        } else {
          const __nv_bfloat162 h = __float22bfloat162_rn(tv);
          const float2 hf = __bfloat1622float2(h);
          const __nv_bfloat162 l = __float22bfloat162_rn(__ffma2_rn(hf, km1, tv));
          hw = *reinterpret_cast<const uint32_t*>(&h);
          lw = *reinterpret_cast<const uint32_t*>(&l);
        }
      };
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % TC_STAGES;
        const uint32_t ph = (uint32_t)(kt / TC_STAGES) & 1u;
        const int ps = kt % kMfPosSlots;
        if (!mbar_wait(&pfull[ps], (uint32_t)(kt / kMfPosSlots) & 1u, err, abort_flag)) break;
        float4 pb[4];
        float wmb[4], d[4][3], r2[4];
        bool close = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          pb[j] = spos[ps * TC_BK + 2 * (kc + j)];
          wmb[j] = spos[ps * TC_BK + 2 * (kc + j) + 1].x;
          d[j][0] = pa.x - pb[j].x;
          d[j][1] = pa.y - pb[j].y;
          d[j][2] = pa.z - pb[j].z;
          r2[j] = fmaf(d[j][0], d[j][0], fmaf(d[j][1], d[j][1], d[j][2] * d[j][2]));
          close |= a == kt * 16 + kc + j || r2[j] < 25.0f * (wa + fmaxf(pb[j].w, wmb[j]));
        }
        float e[4][4];   // e[j][0]: charge column of atom kc + j; e[j][1 + l]: its dipole l
        if (__any_sync(0xffffffffu, close)) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (a == kt * 16 + kc + j) {
              // diagonal block: the T^qq self limit, the T^mumu self term
              e[j][0] = u == 0 ? qself : 0.0f;
#pragma unroll
              for (int l = 0; l < 3; ++l) e[j][1 + l] = (u != 0 && l == kdir) ? vself : 0.0f;
            } else {
              const float rj = sqrtf(r2[j]), ir = 1.0f / rj;
              float G, G1, G2, g, t0, t2;
              if (u == 0) {
                // T^qq (widths R_q,a R_q,b); T^qmu_l = -G'/r (R_q,a R_mu,b) d_l
                radial::eval_f(rj, sqrtf(pa.w + pb[j].w), G, G1, G2, g);
                if (pb[j].w != wmb[j]) radial::eval_f(rj, sqrtf(pa.w + wmb[j]), t0, G1, t2, g);
                e[j][0] = G;
#pragma unroll
                for (int l = 0; l < 3; ++l) e[j][1 + l] = -G1 * d[j][l];
              } else {
                // T^muq_k = G'/r (R_mu,a R_q,b) d_k; T^mumu_kl from G'/r and G'' (R_mu,a R_mu,b)
                radial::eval_f(rj, sqrtf(wma + wmb[j]), t0, G1, G2, g);
                float G1m = G1;
                if (pb[j].w != wmb[j]) radial::eval_f(rj, sqrtf(wma + pb[j].w), t0, G1m, t2, g);
                const float dk = kdir == 0 ? d[j][0] : (kdir == 1 ? d[j][1] : d[j][2]);
                e[j][0] = G1m * dk;
                const float rhk = dk * ir;
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                  const float rr = rhk * (d[j][l] * ir);
                  e[j][1 + l] = -(G2 * rr + G1 * ((l == kdir ? 1.0f : 0.0f) - rr));
                }
              }
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // r >= 5 R: G = 1/r, G'/r = -1/r^3, G'' = 2/r^3
            const float ir = rsqrtf(r2[j]), ir3 = ir * ir * ir;
            if (u == 0) {
              e[j][0] = ir;
#pragma unroll
              for (int l = 0; l < 3; ++l) e[j][1 + l] = ir3 * d[j][l];
            } else {
              const float dk = kdir == 0 ? d[j][0] : (kdir == 1 ? d[j][1] : d[j][2]);
              const float ir5 = ir3 * ir * ir;
              e[j][0] = -ir3 * dk;
#pragma unroll
              for (int l = 0; l < 3; ++l)
                e[j][1 + l] = (l == kdir ? ir3 : 0.0f) - 3.0f * ir5 * dk * d[j][l];
            }
          }
        }
        // blocks with a padding atom are zero; the rest scaled by 2^e
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool real = a < N && kt * 16 + kc + j < N;
#pragma unroll
          for (int c = 0; c < 4; ++c) e[j][c] = real ? e[j][c] * tscale : 0.0f;
        }
        // charge columns j = 0..3; dipole columns in the order (atom j, component l) = 3 j + l
        uint32_t ch[2], cl[2], dh[6], dl[6];
        split2(e[0][0], e[1][0], ch[0], cl[0]);
        split2(e[2][0], e[3][0], ch[1], cl[1]);
        split2(e[0][1], e[0][2], dh[0], dl[0]);
        split2(e[0][3], e[1][1], dh[1], dl[1]);
        split2(e[1][2], e[1][3], dh[2], dl[2]);
        split2(e[2][1], e[2][2], dh[3], dl[3]);
        split2(e[2][3], e[3][1], dh[4], dl[4]);
        split2(e[3][2], e[3][3], dh[5], dl[5]);
        // the A stage is free once the MMA of step kt - TC_STAGES completed
        if (kt >= TC_STAGES && !mbar_wait(&empty[s], ph ^ 1u, err, abort_flag)) break;
        unsigned char* sth = base + s * STAGE;
        unsigned char* stl = sth + A_TILE;
        *reinterpret_cast<uint2*>(sth + oc) = make_uint2(ch[0], ch[1]);
        *reinterpret_cast<uint2*>(stl + oc) = make_uint2(cl[0], cl[1]);
        if (hh == 0) {
          *reinterpret_cast<uint4*>(sth + od1) = make_uint4(dh[0], dh[1], dh[2], dh[3]);
          *reinterpret_cast<uint4*>(stl + od1) = make_uint4(dl[0], dl[1], dl[2], dl[3]);
          *reinterpret_cast<uint2*>(sth + od2) = make_uint2(dh[4], dh[5]);
          *reinterpret_cast<uint2*>(stl + od2) = make_uint2(dl[4], dl[5]);
        } else {
          *reinterpret_cast<uint2*>(sth + od1) = make_uint2(dh[0], dh[1]);
          *reinterpret_cast<uint2*>(stl + od1) = make_uint2(dl[0], dl[1]);
          *reinterpret_cast<uint4*>(sth + od2) = make_uint4(dh[2], dh[3], dh[4], dh[5]);
          *reinterpret_cast<uint4*>(stl + od2) = make_uint4(dl[2], dl[3], dl[4], dl[5]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&full[s])) : "memory");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&pempty[ps])) : "memory");
          if (gw == 0) p_consumed = kt + 1;
        }
      }
    }
    if (warp < 8) {
      // ---------------- epilogue: TMEM -> registers -> Y
      const bool ok = mbar_wait(accum, 0, err, abort_flag);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int wq = warp & 3;
      int row = i0 + wq * 32 + lane;
      bool store = true;
      if constexpr (MU == 1) {
        // atom-blocked tile row -> charges-first row (charge of atom a0 + u, or dipole
        // component (u - 32) % 3 of atom a0 + (u - 32) / 3); rows of padding atoms are skipped
        const int u = wq * 32 + lane, a0 = blockIdx.y * 32;
        const int atom = u < 32 ? a0 + u : a0 + (u - 32) / 3;
        row = u < 32 ? atom : N + 3 * a0 + (u - 32);
        store = atom < N;
      }
      if (ok && !*abort_flag) {
        float* yr = Y + (size_t)row * ldy + c0;
#pragma unroll 1
        for (int cc = 0; cc < TC_BN; cc += 32) {
          uint32_t v[32];
          const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)cc;
          TMEM_LD32(taddr, v);
          if (F16) {
            uint32_t v2[32];
            TMEM_LD32(taddr + TC_BN, v2);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 32; ++q)
              v[q] = __float_as_uint(fmaf(__uint_as_float(v2[q]), s2, __uint_as_float(v[q]) * s1));
          } else {
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          }
          if (store) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              *reinterpret_cast<float4*>(yr + cc + 4 * q) =
                  make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                              __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (cta_abort && threadIdx.x == 0) {
    // after a time-out: wait (bounded) for the copies that were issued but never consumed
    for (int kt = n_consumed; kt < n_issued; ++kt) {
      const long long t0 = clock64();
      while (!mbar_try(&full[kt % TC_STAGES], (uint32_t)(kt / TC_STAGES) & 1u) &&
             clock64() - t0 < kWaitCycles) {
      }
    }
    for (int kp = p_consumed; kp < p_issued; ++kp) {
      const long long t0 = clock64();
      while (!mbar_try(&pfull[kp % kMfPosSlots], (uint32_t)(kp / kMfPosSlots) & 1u) &&
             clock64() - t0 < kWaitCycles) {
      }
    }
  }
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TC_TMEM_COLS));
  }
}

// Positions for k_tc_mf, scaled by 2^-e (R_q^2 by 2^-2e), as atom pairs
// [-x0 -x1 -y0 -y1 -z0 -z1 w0 w1] (w = R_q^2); np atoms, those beyond n distinct dummies
// 3e4 + 64 (i - n) bohr away along x.
__global__ void k_tc_mf_positions(const double* __restrict__ pos, const double* __restrict__ Rq,
                                  int n, int np, double sc, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  double x, y, z, w;
  if (i < n) {
    x = pos[3 * i];
    y = pos[3 * i + 1];
    z = pos[3 * i + 2];
    w = Rq[i] * Rq[i];
  } else {
    x = 3.0e4 + 64.0 * (i - n);
    y = z = 0.0;
    w = 1.0;
  }
  float* o = out + (size_t)(i >> 1) * 8 + (i & 1);
  o[0] = (float)(-x * sc);
  o[2] = (float)(-y * sc);
  o[4] = (float)(-z * sc);
  o[6] = (float)(w * sc * sc);
}

// Positions for the wFQFmu pair kernel: per atom two float4 (x, y, z, R_q^2) and
// (R_mu^2, 0, 0, 0) in bohr, unscaled; na atoms, those beyond n distinct dummies 3e4 + 64 (i - n)
// bohr away along x (their blocks are zeroed by the kernel).
__global__ void k_tc_mf4_positions(const double* __restrict__ pos, const double* __restrict__ Rq,
                                   const double* __restrict__ Rmu, int n, int na, float4* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= na) return;
  if (i < n) {
    out[2 * i] = make_float4((float)pos[3 * i], (float)pos[3 * i + 1], (float)pos[3 * i + 2],
                             (float)(Rq[i] * Rq[i]));
    out[2 * i + 1] = make_float4((float)(Rmu[i] * Rmu[i]), 0.f, 0.f, 0.f);
  } else {
    out[2 * i] = make_float4((float)(3.0e4 + 64.0 * (i - n)), 0.f, 0.f, 1.f);
    out[2 * i + 1] = make_float4(1.f, 0.f, 0.f, 0.f);
  }
}

template <int F16, int BN, int ST, int MU>
cudaError_t launch_mf_variant(const float4* pos, float wmax, float tscale, int N, int mu_self,
                              const CUtensorMap& mXh, const CUtensorMap& mXl, int np, int ncols,
                              float* Y, int ldy, float s1, float s2, int* err, cudaStream_t s) {
  constexpr int smem = TcCfg<BN, ST>::SMEM + kMfPosSlots * kMfPosBytes;
  static_assert(smem <= 227 * 1024, "shared memory per CTA");
  {
    // the shared-memory opt-in, once per device (handles on several threads may race here)
    static std::mutex mu;
    static std::set<int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (!done.count(dev)) {
      e = cudaFuncSetAttribute(k_tc_mf<F16, BN, ST, MU>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      done.insert(dev);
    }
  }
  dim3 grd(ncols / BN, np / TC_BM);
  k_tc_mf<F16, BN, ST, MU><<<grd, kMfThreads, smem, s>>>(pos, wmax, tscale, N, mu_self, mXh, mXl,
                                                         Y, ldy, np, s1, s2, err);
  return cudaGetLastError();
}

// tile-width cache of the pair kernels: (device, np, ncols, f16, model) -> 256 or 128
std::mutex g_mf_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_mf_tune;

// Launch run(bn) at the cached tile width of the shape, or, on the first call of a shape
// outside a stream capture, time both widths (each writes the same Y) and keep the faster:
// 256-column tiles share each generated T tile between more columns, 128-column tiles give
// more CTAs (fewer idle SMs in the last wave).
template <class Run>
cudaError_t launch_tuned_width(int np, int ncols, bool f16, int mu, cudaStream_t s,
                               long long* nl, Run run) {
  int bn = tc_mf_tuned_width(np, ncols, f16, mu != 0);
  cudaError_t e = cudaSuccess;
  if (bn < 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    if (ncols % 256 != 0 || cs != cudaStreamCaptureStatusNone) {
      bn = ncols % 256 == 0 ? 256 : 128;
    } else {
      cudaEvent_t ev[4];
      for (auto& x : ev) {
        e = cudaEventCreate(&x);
        if (e != cudaSuccess) return e;
      }
      const int widths[2] = {256, 128};
      for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
        e = run(widths[v]);   // warm
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * v], s);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = run(widths[v]);
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * v + 1], s);
        *nl += 3;
      }
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
      float t[2] = {0.f, 0.f};
      for (int v = 0; v < 2 && e == cudaSuccess; ++v) e = cudaEventElapsedTime(&t[v], ev[2 * v], ev[2 * v + 1]);
      for (auto& x : ev) cudaEventDestroy(x);
      if (e != cudaSuccess) return e;
      bn = t[1] < t[0] ? 128 : 256;
      int dev = 0;
      e = cudaGetDevice(&dev);
      if (e != cudaSuccess) return e;
      std::lock_guard<std::mutex> lock(g_mf_mu);
      g_mf_tune[std::make_tuple(dev, np, ncols, f16 ? 1 : 0, mu)] = bn;
    }
  }
  e = run(bn);
  ++*nl;
  return e;
}

}  // namespace

cudaError_t launch_tc_mf_positions(const double* pos, const double* Rq, int n, int np,
                                   int scale_exp, float4* out, cudaStream_t s, long long* nl) {
  k_tc_mf_positions<<<(np + 255) / 256, 256, 0, s>>>(pos, Rq, n, np, std::ldexp(1.0, -scale_exp),
                                                    reinterpret_cast<float*>(out));
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_tc_mf4_positions(const double* pos, const double* Rq, const double* Rmu, int n,
                                    int np, float4* out, cudaStream_t s, long long* nl) {
  if (np % TC_BM || n > np / 4) return cudaErrorInvalidValue;
  const int na = np / 4;
  k_tc_mf4_positions<<<(na + 255) / 256, 256, 0, s>>>(pos, Rq, Rmu, n, na, out);
  ++*nl;
  return cudaGetLastError();
}

int tc_mf_tuned_width(int np, int ncols, bool f16, bool mu) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  std::lock_guard<std::mutex> lock(g_mf_mu);
  auto it = g_mf_tune.find(std::make_tuple(dev, np, ncols, f16 ? 1 : 0, mu ? 1 : 0));
  return it == g_mf_tune.end() ? -1 : it->second;
}

cudaError_t launch_tc_mf(const float4* pos, int np, float wmax, const uint16_t* Xh,
                         const uint16_t* Xl, int ncols, float* Y, int ldy, bool f16, int scale_exp,
                         int* err, cudaStream_t s, long long* nl) {
  // shape contract as launch_tc_gemm: 128-row output tiles and 64-atom K steps (np % 128),
  // 128- or 256-column operand tiles, 16-byte aligned operand rows and positions
  if (np % TC_BM || ncols % 128 || ldy % 4 || ldy < ncols) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(Xh) | reinterpret_cast<uintptr_t>(Xl) |
       reinterpret_cast<uintptr_t>(pos)) & 15)
    return cudaErrorMisalignedAddress;
  const float s1 = std::ldexp(1.0f, -(scale_exp + 8)), s2 = std::ldexp(1.0f, -(scale_exp + 19));
  auto run = [&](int bn) -> cudaError_t {
    CUtensorMap mXh, mXl;
    if (!make_map(&mXh, Xh, ncols, np, bn, f16) || !make_map(&mXl, Xl, ncols, np, bn, f16))
      return cudaErrorInvalidValue;
    if (f16)
      return bn == 256 ? launch_mf_variant<1, 256, 2, 0>(pos, wmax, 1.0f, 0, 0, mXh, mXl, np, ncols, Y, ldy, s1, s2, err, s)
                       : launch_mf_variant<1, 128, 3, 0>(pos, wmax, 1.0f, 0, 0, mXh, mXl, np, ncols, Y, ldy, s1, s2, err, s);
    return bn == 256 ? launch_mf_variant<0, 256, 2, 0>(pos, wmax, 1.0f, 0, 0, mXh, mXl, np, ncols, Y, ldy, 1.0f, 1.0f, err, s)
                     : launch_mf_variant<0, 128, 3, 0>(pos, wmax, 1.0f, 0, 0, mXh, mXl, np, ncols, Y, ldy, 1.0f, 1.0f, err, s);
  };
  return launch_tuned_width(np, ncols, f16, 0, s, nl, run);
}

cudaError_t launch_tc_mf4(const float4* pos, int np, int N, int mu_self, const uint16_t* Xh,
                          const uint16_t* Xl, int ncols, float* Y, int ldy, bool f16, int scale_exp,
                          int* err, cudaStream_t s, long long* nl) {
  // 128-row tiles of 32 atoms, K steps of 16 atoms: np % 128 == 0 and N <= np / 4
  if (np % TC_BM || N < 1 || N > np / 4 || ncols % 128 || ldy % 4 || ldy < ncols)
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(Xh) | reinterpret_cast<uintptr_t>(Xl) |
       reinterpret_cast<uintptr_t>(pos)) & 15)
    return cudaErrorMisalignedAddress;
  const float tscale = f16 ? std::ldexp(1.0f, scale_exp) : 1.0f;
  const float s1 = f16 ? std::ldexp(1.0f, -(scale_exp + 8)) : 1.0f;
  const float s2 = f16 ? std::ldexp(1.0f, -(scale_exp + 19)) : 1.0f;
  auto run = [&](int bn) -> cudaError_t {
    CUtensorMap mXh, mXl;
    if (!make_map(&mXh, Xh, ncols, np, bn, f16) || !make_map(&mXl, Xl, ncols, np, bn, f16))
      return cudaErrorInvalidValue;
    if (f16)
      return bn == 256 ? launch_mf_variant<1, 256, 2, 1>(pos, 0.f, tscale, N, mu_self, mXh, mXl, np, ncols, Y, ldy, s1, s2, err, s)
                       : launch_mf_variant<1, 128, 3, 1>(pos, 0.f, tscale, N, mu_self, mXh, mXl, np, ncols, Y, ldy, s1, s2, err, s);
    return bn == 256 ? launch_mf_variant<0, 256, 2, 1>(pos, 0.f, tscale, N, mu_self, mXh, mXl, np, ncols, Y, ldy, s1, s2, err, s)
                     : launch_mf_variant<0, 128, 3, 1>(pos, 0.f, tscale, N, mu_self, mXh, mXl, np, ncols, Y, ldy, s1, s2, err, s);
  };
  return launch_tuned_width(np, ncols, f16, 1, s, nl, run);
}

}  // namespace px
