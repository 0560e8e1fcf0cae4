// Structure staging on the device (Sec. "Specify the Nanostructure"): Angstrom ->
// bohr, atoms reordered along a Morton (Z-order) curve of their positions, per-atom
// parameters (R_q, R_mu of Secs. 2.1-2.2, the effective area A_i of Eq. 3) expanded
// from the type table.
//
// Sorting puts spatial neighbours at nearby indices, so the CSR rows of K (Eq. 3) and
// the operand rows the conductance apply gathers for them stay within a few cache
// lines, and tiles of the pair kernel hold compact groups of atoms.  The order is
// deterministic: the sort key is the 30-bit Morton code of the position quantised to
// a 1024^3 grid over the bounding box, ties kept in input order (stable radix sort).
// perm[i] is the caller's index of internal atom i; outputs per atom are written back
// through it.
#include "px_internal.cuh"

#include <cub/device/device_radix_sort.cuh>

namespace px {

namespace {

constexpr double kBohrAng = 0.529177210903;   // Angstrom per bohr, CODATA 2018

// bbox[0..2] = min, bbox[3..5] = max of the Angstrom coordinates (one block).
__global__ void __launch_bounds__(1024) k_bbox(const double* __restrict__ xyz, int N, double* bbox) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    for (int k = 0; k < 3; ++k) {
      const double v = xyz[3 * (size_t)i + k];
      lo[k] = fmin(lo[k], v);
      hi[k] = fmax(hi[k], v);
    }
  __shared__ double sh[6][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fmin(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmax(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
    if (lane == 0) {
      sh[k][warp] = lo[k];
      sh[3 + k][warp] = hi[k];
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int k = threadIdx.x;
    double l = INFINITY, h = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
      l = fmin(l, sh[k][w]);
      h = fmax(h, sh[3 + k][w]);
    }
    bbox[k] = l;
    bbox[3 + k] = h;
  }
}

// 10 low bits of v spread to every third bit (bit b -> bit 3b).
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void k_morton(const double* __restrict__ xyz, int N, const double* __restrict__ bbox,
                         uint32_t* code, int* idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  uint32_t c[3];
  for (int k = 0; k < 3; ++k) {
    const double ext = bbox[3 + k] - bbox[k];
    const double u = ext > 0.0 ? (xyz[3 * (size_t)i + k] - bbox[k]) / ext : 0.0;   // [0, 1]
    c[k] = (uint32_t)fmin(1023.0, fmax(0.0, floor(u * 1024.0)));
  }
  code[i] = spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
  idx[i] = i;
}

// Internal atom i takes the caller's atom perm[i]: position in bohr, type, and the
// type's Gaussian widths and effective area.
__global__ void k_gather_atoms(const double* __restrict__ xyz, const int* __restrict__ tidx,
                               const px_atom_type* __restrict__ types, const int* __restrict__ perm,
                               int N, double* pos, int* type, double* Rq, double* Rmu,
                               double* area) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int src = perm[i];
  for (int k = 0; k < 3; ++k) pos[3 * (size_t)i + k] = xyz[3 * (size_t)src + k] / kBohrAng;
  const int t = tidx[src];
  type[i] = t;
  Rq[i] = types[t].Rq_bohr;
  Rmu[i] = types[t].Rmu_bohr;
  area[i] = types[t].area_bohr2;
}

__global__ void k_iota_i(int* a, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

}  // namespace

size_t stage_scratch_bytes(int N) {
  size_t tb = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tb, (const uint32_t*)nullptr, (uint32_t*)nullptr,
                                  (const int*)nullptr, (int*)nullptr, N, 0, 30);
  // bbox, two code arrays, one index array, sort temporaries
  return 256 + 2 * round_up(sizeof(uint32_t) * N, 256) + round_up(sizeof(int) * N, 256) +
         round_up(tb, 256);
}

cudaError_t launch_stage_atoms(const double* xyz_ang, const int* tidx, const px_atom_type* types,
                               int N, bool sort, void* scratch, size_t scratch_bytes, int* perm,
                               double* pos, int* type, double* Rq, double* Rmu, double* area,
                               cudaStream_t s, long long* nl) {
  if (N < 1) return cudaErrorInvalidValue;
  const int blocks = (N + 255) / 256;
  if (sort) {
    if (scratch_bytes < stage_scratch_bytes(N)) return cudaErrorInvalidValue;
    unsigned char* p = static_cast<unsigned char*>(scratch);
    double* bbox = reinterpret_cast<double*>(p);
    p += 256;
    uint32_t* code_in = reinterpret_cast<uint32_t*>(p);
    p += round_up(sizeof(uint32_t) * N, 256);
    uint32_t* code_out = reinterpret_cast<uint32_t*>(p);
    p += round_up(sizeof(uint32_t) * N, 256);
    int* idx = reinterpret_cast<int*>(p);
    p += round_up(sizeof(int) * N, 256);
    size_t tb = scratch_bytes - (size_t)(p - static_cast<unsigned char*>(scratch));
    k_bbox<<<1, 1024, 0, s>>>(xyz_ang, N, bbox);
    k_morton<<<blocks, 256, 0, s>>>(xyz_ang, N, bbox, code_in, idx);
    *nl += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // library radix sort (its kernels are not counted in *nl)
    e = cub::DeviceRadixSort::SortPairs(p, tb, code_in, code_out, idx, perm, N, 0, 30, s);
    if (e != cudaSuccess) return e;
  } else {
    k_iota_i<<<blocks, 256, 0, s>>>(perm, N);
    ++*nl;
  }
  k_gather_atoms<<<blocks, 256, 0, s>>>(xyz_ang, tidx, types, perm, N, pos, type, Rq, Rmu, area);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace px
