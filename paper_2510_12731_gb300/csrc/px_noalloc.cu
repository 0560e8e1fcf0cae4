// px_relres_device_noalloc: the FP64 true-residual check of px_solve_device, for a
// solution the caller holds in device memory, running entirely in a fixed scratch
// array that is part of the library image -- the call allocates no device memory.
//
// Who needs this: callers that cannot allocate device memory at the point of the
// call -- callers whose memory pool owns all free device memory (a framework caching
// allocator, another library's arena), and latency-bound loops that must never enter
// the driver's allocator (an allocation can synchronise the device).  They keep their
// solutions in their own buffers and only need the residual norm.  The first call on
// a device looks up the scratch array's device address; make it before any stream
// capture (under a capture the address found by the device's last call outside one is
// used).
//
// The scratch is one file-scope device array of kNoAllocScratchBytes.  Every GPU
// that loads the library holds it until the process exits.  Every call shares it
// and it keeps the last call's contents, so two calls that overlap on the GPU (two
// host threads, or two streams) race; calls on one stream, one after the other,
// are safe.  What must start at zero (the padding of the matvec operand) is cleared
// by each call.
#include "px.h"
#include "px_internal.cuh"

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

// handle internals needed here: the loaded structure, its n and tau, the error slot
#include "px_handle.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

// Device address of g_scratch on the current device.  Outside a stream capture it is
// looked up on every call (a cheap host-side query), so a module reloaded at another
// address (after cudaDeviceReset, say) is never served a stale pointer; under a capture
// the address of the device's last uncaptured call is reused, because a first lookup
// may load the module, which a capture does not allow.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(cudaStream_t s, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  } else if (!g_scratch_ptr[dev]) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Solution layout of px_solve_device -> the FP64 residual layouts: the column-major
// block x[i][c] (complex) and the real matvec operand X[i][2c], X[i][2c+1].
__global__ void k_pack_solution(int N, int model, int B, const int* __restrict__ perm,
                                const double2* __restrict__ q, const double2* __restrict__ mu,
                                double2* x, double* X, int ldx) {
  const int c = blockIdx.x * 32 + threadIdx.x;
  if (c >= B) return;
  const int nu = model == 1 ? 4 * N : N;
  for (int i = blockIdx.y * 8 + threadIdx.y; i < nu; i += 8 * gridDim.y) {
    double2 v;
    // the caller's buffers are in the caller's atom order; internal atom a is perm[a]
    if (i < N) {
      v = q[(size_t)c * N + perm[i]];
    } else {
      const int a = (i - N) / 3, k = (i - N) % 3;
      v = mu[((size_t)c * N + perm[a]) * 3 + k];
    }
    x[(size_t)i * B + c] = v;
    X[(size_t)i * ldx + 2 * c] = v.x;
    X[(size_t)i * ldx + 2 * c + 1] = v.y;
  }
}

__global__ void k_iota(int* a, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

struct Carve {
  unsigned char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
};

px_status fail_h(px_handle* h, px_status st, const std::string& msg) {
  px_set_error(h, msg);
  return st;
}

}  // namespace

extern "C" px_status px_relres_device_noalloc(px_handle* h, int n_freq, const double* omega_ev,
                                              const double* alpha_ib, int n_pol,
                                              const double* pol_dir, double e0, const double* d_q,
                                              const double* d_mu, double* d_relres,
                                              void* cuda_stream) {
  if (!h) return PX_EINVAL;
  const px::DevStructure* dsp = px_structure(h);
  if (!dsp) return fail_h(h, PX_EINVAL, "no structure loaded");
  const px::DevStructure& d = *dsp;
  if (d.hetero)
    return fail_h(h, PX_ENOTIMPL, "px_relres_device_noalloc does not cover PX_WFQFMU_HETERO");
  if (d.bem) return fail_h(h, PX_ENOTIMPL, "px_relres_device_noalloc does not cover meshes");
  if (n_freq < 1 || n_pol < 1 || !omega_ev || !pol_dir || !d_q || !d_relres)
    return fail_h(h, PX_EINVAL, "need n_freq, n_pol >= 1, omega_ev, pol_dir, d_q and d_relres");
  if (d.model == PX_WFQFMU && (!alpha_ib || !d_mu))
    return fail_h(h, PX_EINVAL, "alpha_ib and d_mu are required for PX_WFQFMU");
  if (!std::isfinite(e0) || !(e0 > 0.0)) return fail_h(h, PX_EINVAL, "e0 must be finite and > 0");
  for (int f = 0; f < n_freq; ++f)
    if (!std::isfinite(omega_ev[f]) || !(omega_ev[f] > 0.0))
      return fail_h(h, PX_EINVAL, "frequencies must be finite and > 0");
  // the same input checks as px_solve_device, before any size is derived from them
  if ((long long)n_freq * n_pol > (1LL << 24)) return fail_h(h, PX_EINVAL, "too many columns");
  for (int p = 0; p < n_pol; ++p) {
    double n2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double v = pol_dir[3 * p + k];
      if (!std::isfinite(v)) return fail_h(h, PX_EINVAL, "non-finite polarisation");
      n2 += v * v;
    }
    if (std::fabs(std::sqrt(n2) - 1.0) > 1e-6)
      return fail_h(h, PX_EINVAL, "polarisation directions must be unit vectors");
  }
  if (d.model == PX_WFQFMU)
    for (size_t k = 0; k < 2 * (size_t)d.ntypes * n_freq; ++k)
      if (!std::isfinite(alpha_ib[k])) return fail_h(h, PX_EINVAL, "non-finite alpha_ib");
  const int F = n_freq, P = n_pol, B = F * P;
  const int N = d.N, nu = d.nu, np = d.np, ntypes = d.ntypes, model = d.model;
  const int ldx = (int)px::round_up(2 * (size_t)B, px::kTile);
  const int nblk = px::reduction_blocks(nu);

  // scratch layout (bytes, each piece 256-aligned)
  auto need = [&]() {
    size_t s = 0;
    auto add = [&](size_t bytes) { s = ((s + 255) & ~size_t(255)) + bytes; };
    add(sizeof(double) * ((size_t)F + 3 * P + 2 * (size_t)ntypes * F));   // inputs
    add(sizeof(double2) * B);                      // z_q
    add(sizeof(double2) * (size_t)ntypes * B);     // z_mu
    add(sizeof(double) * (size_t)nu * P);          // b
    add(sizeof(double) * P);                       // ||b||
    add(sizeof(int) * B);                          // column list
    add(sizeof(double2) * (size_t)nu * B);         // x
    add(sizeof(double2) * (size_t)nu * B);         // r
    add(sizeof(double) * (size_t)np * ldx);        // X
    add(sizeof(double) * (size_t)np * ldx);        // Y
    add(sizeof(double) * (size_t)nblk * B);        // partial norms
    add(sizeof(double) * 3 * (size_t)B);           // rnorm, beta, target
    return s;
  }();
  if (need > kNoAllocScratchBytes)
    return fail_h(h, PX_EINVAL,
                  "px_relres_device_noalloc needs " + std::to_string(need) +
                      " bytes of scratch; its fixed scratch array holds " +
                      std::to_string(kNoAllocScratchBytes));

  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : px_stream(h);
  void* sp = nullptr;
  cudaError_t e = scratch_for_current_device(s, &sp);
  if (e != cudaSuccess)
    return fail_h(h, PX_ECUDA, std::string("scratch address lookup: ") + cudaGetErrorString(e));
  Carve cv{static_cast<unsigned char*>(sp)};
  double* d_in = cv.take<double>((size_t)F + 3 * P + 2 * (size_t)ntypes * F);
  double* d_omega = d_in;
  double* d_pol = d_in + F;
  double* d_aib = d_pol + 3 * P;
  double2* zq = cv.take<double2>(B);
  double2* zmu = cv.take<double2>((size_t)ntypes * B);
  double* b = cv.take<double>((size_t)nu * P);
  double* bnorm = cv.take<double>(P);
  int* act = cv.take<int>(B);
  double2* x = cv.take<double2>((size_t)nu * B);
  double2* r = cv.take<double2>((size_t)nu * B);
  double* X = cv.take<double>((size_t)np * ldx);
  double* Y = cv.take<double>((size_t)np * ldx);
  double* normpart = cv.take<double>((size_t)nblk * B);
  double* rnorm = cv.take<double>(3 * (size_t)B);
  double* beta = rnorm + B;
  double* target = beta + B;

  long long nl = 0;
#define NA_CU(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return fail_h(h, PX_ECUDA, std::string(#call) + ": " +     \
                                                          cudaGetErrorString(e_));    \
  } while (0)
  NA_CU(cudaMemcpyAsync(d_omega, omega_ev, sizeof(double) * F, cudaMemcpyHostToDevice, s));
  NA_CU(cudaMemcpyAsync(d_pol, pol_dir, sizeof(double) * 3 * P, cudaMemcpyHostToDevice, s));
  if (model == PX_WFQFMU)
    NA_CU(cudaMemcpyAsync(d_aib, alpha_ib, sizeof(double) * 2 * ntypes * F, cudaMemcpyHostToDevice, s));
  NA_CU(px::launch_shifts(F, P, ntypes, model, d_omega, d_aib, px_drude_n(h), px_tau(h), zq, zmu, s, &nl));
  NA_CU(px::launch_rhs(nu, N, model, d.rowptr, d.col, d.val64, d.pos64, d_pol, P, e0, b, s, &nl));
  NA_CU(px::launch_col_norms(b, nu, P, bnorm, s, &nl));
  k_iota<<<(B + 255) / 256, 256, 0, s>>>(act, B);
  NA_CU(cudaGetLastError());
  // the matvec operand's padding rows and columns must be zero
  NA_CU(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)np * ldx, s));
  k_pack_solution<<<dim3((B + 31) / 32, nblk), dim3(32, 8), 0, s>>>(
      N, model, B, d.perm, reinterpret_cast<const double2*>(d_q), reinterpret_cast<const double2*>(d_mu), x,
      X, ldx);
  NA_CU(cudaGetLastError());
  if (d.matfree && model == PX_WFQFMU)
    NA_CU(px::launch_dgemm_mf4(d.pos4d, d.rm2d, N, d.mu_self, X, ldx, Y, ldx, ldx, s, &nl));
  else if (d.matfree) NA_CU(px::launch_dgemm_mf(d.pos4d, N, np, X, ldx, Y, ldx, ldx, s, &nl));
  else if (2 * B <= 8) NA_CU(px::launch_dgemv(d.T64, np, X, ldx, Y, ldx, 2 * B, s, &nl));
  else NA_CU(px::launch_dgemm(d.T64, np, X, ldx, Y, ldx, ldx, s, &nl));
  px::ResidArgs ra{};
  ra.nu = nu; ra.N = N; ra.model = model; ra.Bact = B; ra.P = P; ra.B = B; ra.nblk = nblk;
  ra.rowptr = d.rowptr; ra.col = d.col; ra.val64 = d.val64; ra.type = d.type;
  ra.Y = Y; ra.ldy = ldx; ra.x = x; ra.act = act; ra.b = b; ra.zq = zq; ra.zmu = zmu;
  ra.R = r; ra.normpart = normpart;
  NA_CU(px::launch_resid(ra, s, &nl));
  NA_CU(px::launch_norm_finish(normpart, nblk, B, act, P, bnorm, 0.0, 0.0, rnorm, beta, target, s, &nl));
  NA_CU(px::launch_relres(rnorm, bnorm, B, P, d_relres, s, &nl));
  NA_CU(cudaStreamSynchronize(s));
#undef NA_CU
  return PX_OK;
}
