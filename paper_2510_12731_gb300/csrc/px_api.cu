// C ABI of the px library (include/px.h): handle management, input validation,
// structure set-up and the restarted-GMRES / refinement driver that sequences
// the device kernels.  All arithmetic of the method runs in the kernels; the
// host code here only validates, allocates, launches and reads back per-column
// residual norms between restart cycles.
#include "px.h"
#include "px_internal.cuh"
#include "px_handle.cuh"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using px::round_up;

namespace {

constexpr double kBohrAng = 0.529177210903;     // CODATA 2018

thread_local std::string g_create_error;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t n) {
    if (n <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, n);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

struct PxError {
  px_status st;
  std::string msg;
};

// One restart cycle captured as a graph: a while-loop node whose body is one Krylov
// step.  key lists every value the captured launches depend on (sizes, buffers, the
// structure generation); body_kernels counts the kernels of one step.
struct CycleGraph {
  std::vector<uint64_t> key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long body_kernels = 0;
};
constexpr size_t kMaxCachedGraphs = 64;

}  // namespace

struct px_handle {
  px_options opt;
  cudaStream_t own_stream = nullptr;
  int device = 0;
  std::string err;
  px_stats stats;
  bool have_structure = false;
  px::DevStructure ds;
  // structure buffers
  DevBuf b_pos, b_Rq, b_Rmu, b_area, b_type, b_rowptr, b_col, b_val64, b_val32, b_counts;
  DevBuf b_pair;   // rcut2, r0, d, s tables
  DevBuf b_perm;   // [N] caller index of internal atom i
  DevBuf b_stage;  // staging inputs (caller order) and sort scratch
  DevBuf b_T64, b_T32, b_Thi, b_Tlo, b_pos4f, b_pos4d, b_Tffh, b_Tffl;
  DevBuf b_rm2;    // matrix-free wFQFmu: R_mu^2 in FP32 and FP64
  DevBuf b_pos4tc; // matrix-free split precisions: scaled, padded positions
  DevBuf b_mesh;   // boundary elements: normals [N][3], areas [N]
  // IEFPCM (Eq. 12): the operator S A^-1 of the second step and its planes, and the first
  // step's solution y (the second step's right-hand side)
  px::DevStructure ds_g;
  DevBuf g_T64, g_T32, g_Thi, g_Tlo, g_Tffh, g_Tffl, b_yief;
  DevBuf b_M64;    // FP64 M = diag(Kbar, I) T while its split planes are built
  // solve buffers
  DevBuf b_pol, b_b, b_x, b_r, b_rnorm, b_bnorm, b_iters, b_act, b_zq, b_zmu;
  DevBuf b_V, b_W, b_h, b_part, b_normpart, b_R, b_g, b_cs, b_sn, b_target, b_jconv, b_invh, b_y;
  DevBuf b_X32, b_Y32, b_X64, b_Y64, b_Xth, b_Xtl;
  DevBuf b_dpart;  // split-K partial products of the FP64 GEMM
  int* d_err = nullptr;         // device flag: a bounded pipeline wait ran out of time
  DevBuf b_alpha, b_q, b_mu;
  DevBuf b_sk;                  // shifted Krylov work space (carved per solve)
  DevBuf b_het;                 // heterogeneous wFQFmu: per-column tables and right-hand sides
  DevBuf b_hstruct;             // heterogeneous wFQFmu: type parameters, Eq. 10 counts, identity
  int* h_skact = nullptr;       // pinned host copy of the shifted solve's active counts
  size_t h_skact_n = 0;
  cudaEvent_t ev_sk[2] = {nullptr, nullptr};   // start / end of the shifted phase
  int* h_active = nullptr;      // pinned host copy of d_active [kMaxRestart]
  int* d_active = nullptr;      // device: unfrozen columns after each Krylov step
  std::vector<cudaEvent_t> ev_pool;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_iter[2] = {nullptr, nullptr};
  long long nl = 0;
  int* d_jstep = nullptr;       // device step index of a captured cycle (in d_active's block)
  int* h_jstep = nullptr;       // pinned host copy (in h_active's block)
  cudaStream_t cap_stream = nullptr;   // stream used only to capture cycle graphs
  std::vector<CycleGraph> graphs;      // instantiated cycle graphs, reused by equal keys
  double drude_n = 0.0, tau = 0.0;   // shared n, tau of the loaded structure (Eq. 6)
  bool verbose = false;              // PX_VERBOSE=1: one stderr line per restart cycle
};

namespace {

void drop_graphs(px_handle* h) {
  for (CycleGraph& c : h->graphs) {
    if (c.exec) cudaGraphExecDestroy(c.exec);
    if (c.graph) cudaGraphDestroy(c.graph);
  }
  h->graphs.clear();
}

void free_all(px_handle* h) {
  DevBuf* bufs[] = {&h->b_M64, &h->b_perm, &h->b_stage, &h->b_pos, &h->b_Rq, &h->b_Rmu, &h->b_area, &h->b_type, &h->b_rowptr,
                    &h->b_col, &h->b_val64, &h->b_val32, &h->b_counts, &h->b_pair, &h->b_T64,
                    &h->b_T32, &h->b_Thi, &h->b_Tlo, &h->b_pos4f, &h->b_pos4d, &h->b_rm2, &h->b_pos4tc, &h->b_mesh, &h->b_Tffh, &h->b_Tffl, &h->b_pol, &h->b_b, &h->b_x, &h->b_r,
                    &h->b_rnorm, &h->b_bnorm, &h->b_iters, &h->b_act, &h->b_zq, &h->b_zmu,
                    &h->b_V, &h->b_W, &h->b_h, &h->b_part, &h->b_normpart, &h->b_R, &h->b_g,
                    &h->b_cs, &h->b_sn, &h->b_target, &h->b_jconv, &h->b_invh, &h->b_y,
                    &h->b_X32, &h->b_Y32, &h->b_X64, &h->b_Y64, &h->b_Xth, &h->b_Xtl, &h->b_dpart,
                    &h->b_alpha, &h->b_q, &h->b_mu, &h->b_sk, &h->b_het, &h->b_hstruct,
                    &h->g_T64, &h->g_T32, &h->g_Thi, &h->g_Tlo, &h->g_Tffh, &h->g_Tffl, &h->b_yief};
  for (DevBuf* b : bufs) b->release();
}

px_status validate_options(const px_options* o, std::string* msg) {
  if (o->precision < PX_FP64 || o->precision > PX_FP16SPLIT) { *msg = "bad precision"; return PX_EINVAL; }
  if (o->mode < PX_MODE_AUTO || o->mode > PX_MODE_MATERIALISED) { *msg = "bad mode"; return PX_EINVAL; }
  if (o->restart_m < 0 || o->restart_m > px::kMaxRestart) { *msg = "restart_m must be in [0, 400]"; return PX_EINVAL; }
  if (o->max_iter < 1 || o->max_cycles < 1) { *msg = "max_iter and max_cycles must be >= 1"; return PX_EINVAL; }
  if (o->max_refine < 0) { *msg = "max_refine must be >= 0"; return PX_EINVAL; }
  if (o->gs_passes < 1 || o->gs_passes > 2) { *msg = "gs_passes must be 1 or 2"; return PX_EINVAL; }
  if (o->basis < PX_BASIS_AUTO || o->basis > PX_BASIS_FP32) { *msg = "bad basis"; return PX_EINVAL; }
  if (o->gemm_tiles < 0 || o->gemm_tiles > 2) { *msg = "gemm_tiles must be 0, 1 or 2"; return PX_EINVAL; }
  if (o->cycle_graphs < 0 || o->cycle_graphs > 1) { *msg = "cycle_graphs must be 0 or 1"; return PX_EINVAL; }
  if (o->sort_atoms < 0 || o->sort_atoms > 1) { *msg = "sort_atoms must be 0 or 1"; return PX_EINVAL; }
  if (o->precision == PX_FP64 && o->basis != PX_BASIS_AUTO && o->basis != PX_BASIS_FP64) {
    *msg = "PX_FP64 needs an FP64 Krylov basis (PX_BASIS_AUTO or PX_BASIS_FP64)";
    return PX_EINVAL;
  }
  if (!(o->tol_rel > 0.0) || !(o->tol_rel < 1.0)) { *msg = "tol_rel must be in (0, 1)"; return PX_EINVAL; }
  if (!(o->inner_tol > 0.0) || !(o->inner_tol < 1.0)) { *msg = "inner_tol must be in (0, 1)"; return PX_EINVAL; }
  if (!(o->kcut_eps >= 0.0) || !(o->kcut_eps < 0.5)) { *msg = "kcut_eps must be in [0, 0.5)"; return PX_EINVAL; }
  if (!(o->device_wait_limit_s > 0.0)) { *msg = "device_wait_limit_s must be > 0"; return PX_EINVAL; }
  if (o->solver < PX_SOLVER_BATCHED || o->solver > PX_SOLVER_SHIFTED) { *msg = "bad solver"; return PX_EINVAL; }
  if (o->shift_krylov_max < 0) { *msg = "shift_krylov_max must be >= 0"; return PX_EINVAL; }
  return PX_OK;
}

#define CU(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      throw PxError{e_ == cudaErrorMemoryAllocation ? PX_ENOMEM : PX_ECUDA,          \
                    std::string(#call) + ": " + cudaGetErrorString(e_)};             \
  } while (0)

px_status fail(px_handle* h, px_status st, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return st;
}

// Bounded wait for an event: poll with sleeps so a stuck device cannot hang the
// caller forever.
void wait_event(px_handle* h, cudaEvent_t ev) {
  double limit = h->opt.device_wait_limit_s;
  double waited = 0.0;
  while (true) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return;
    if (e != cudaErrorNotReady) CU(e);
    if (waited > limit) throw PxError{PX_ETIMEOUT, "device did not finish within device_wait_limit_s"};
    // short spin first, then back off
    struct timespec ts = {0, waited < 0.01 ? 20000 : 200000};
    nanosleep(&ts, nullptr);
    waited += ts.tv_nsec * 1e-9;
  }
}

void sync_stream(px_handle* h, cudaStream_t s) {
  cudaEvent_t ev = h->ev_iter[0];
  CU(cudaEventRecord(ev, s));
  wait_event(h, ev);
}

cudaEvent_t pool_event(px_handle* h, size_t k) {
  while (h->ev_pool.size() <= k) {
    cudaEvent_t e;
    CU(cudaEventCreate(&e));
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[k];
}

// ------------------------------------------------------------------ structure
void set_structure(px_handle* h, int model, int N, const double* xyz, const int* tidx,
                   const px_atom_type* types, int ntypes) {
  if (!xyz || !tidx || !types) throw PxError{PX_EINVAL, "NULL input"};
  if (N < 1) throw PxError{PX_EINVAL, "n_atoms must be >= 1"};
  if (ntypes < 1) throw PxError{PX_EINVAL, "n_types must be >= 1"};
  if (model != PX_WFQ && model != PX_WFQFMU && model != PX_WFQFMU_HETERO)
    throw PxError{PX_EINVAL, "bad model"};
  const bool hetero = model == PX_WFQFMU_HETERO;
  for (int t = 0; t < ntypes; ++t) {
    const px_atom_type& a = types[t];
    double v[] = {a.r0_ang, a.d, a.s, a.area_bohr2, a.Rq_bohr, a.Rmu_bohr, a.drude_n_au, a.tau_au};
    for (double x : v)
      if (!std::isfinite(x) || !(x > 0.0)) throw PxError{PX_EINVAL, "atom type parameters must be finite and > 0"};
    if (!hetero && (a.drude_n_au != types[0].drude_n_au || a.tau_au != types[0].tau_au))
      throw PxError{PX_EINVAL, "all atom types must share drude_n_au and tau_au (Eqs. 1 and 7 have "
                               "one z_q; use PX_WFQFMU_HETERO for Eq. 9)"};
  }
  if (hetero && (h->opt.precision == PX_BF16SPLIT || h->opt.precision == PX_FP16SPLIT))
    throw PxError{PX_ENOTIMPL, "PX_WFQFMU_HETERO runs PX_FP32 or PX_FP64 matvecs (its conductance "
                               "block depends on the frequency, Eq. 9)"};
  // internally the heterogeneous model is wFQFmu (4N unknowns) with per-type Drude data
  if (hetero) model = PX_WFQFMU;
  for (int i = 0; i < N; ++i) {
    if (tidx[i] < 0 || tidx[i] >= ntypes) throw PxError{PX_EINVAL, "type index out of range"};
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(xyz[3 * (size_t)i + k])) throw PxError{PX_EINVAL, "non-finite coordinate"};
  }
  // duplicate atoms: sort by x, compare within a 1e-6 Angstrom window
  {
    std::vector<int> ord(N);
    for (int i = 0; i < N; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return xyz[3 * (size_t)a] < xyz[3 * (size_t)b]; });
    const double eps = 1e-6;
    for (int u = 0; u < N; ++u) {
      const double* pa = xyz + 3 * (size_t)ord[u];
      for (int v = u + 1; v < N; ++v) {
        const double* pb = xyz + 3 * (size_t)ord[v];
        if (pb[0] - pa[0] > eps) break;
        double dx = pb[0] - pa[0], dy = pb[1] - pa[1], dz = pb[2] - pa[2];
        if (dx * dx + dy * dy + dz * dz < eps * eps) throw PxError{PX_EINVAL, "two atoms closer than 1e-6 Angstrom"};
      }
    }
  }
  // pair tables: arithmetic means of the two types' r0, d, s; squared cutoff radius
  // where 1 - f(r) = kcut_eps (infinite when kcut_eps == 0).
  std::vector<double> pair(4 * (size_t)ntypes * ntypes);
  double* rcut2 = pair.data();
  double* r0t = rcut2 + ntypes * ntypes;
  double* dt = r0t + ntypes * ntypes;
  double* st = dt + ntypes * ntypes;
  double eps = h->opt.kcut_eps;
  for (int a = 0; a < ntypes; ++a)
    for (int b = 0; b < ntypes; ++b) {
      int k = a * ntypes + b;
      r0t[k] = 0.5 * (types[a].r0_ang + types[b].r0_ang) / kBohrAng;
      dt[k] = 0.5 * (types[a].d + types[b].d);
      st[k] = 0.5 * (types[a].s + types[b].s);
      if (eps > 0.0) {
        double rc = st[k] * r0t[k] * (1.0 + std::log((1.0 - eps) / eps) / dt[k]);
        rcut2[k] = rc * rc;
      } else {
        rcut2[k] = INFINITY;
      }
    }

  cudaStream_t s = h->own_stream;
  px::DevStructure& d = h->ds;
  h->have_structure = false;
  d.model = model;
  d.hetero = hetero;
  d.bem = false;
  d.nrm = nullptr;
  d.tarea = nullptr;
  d.N = N;
  d.nu = model == PX_WFQ ? N : 4 * N;
  d.np = (int)round_up(d.nu, px::kTile);
  d.ntypes = ntypes;
  h->nl = 0;
  CU(cudaEventRecord(h->ev_a, s));
  CU(h->b_pos.ensure(sizeof(double) * 3 * N));
  CU(h->b_Rq.ensure(sizeof(double) * N));
  CU(h->b_Rmu.ensure(sizeof(double) * N));
  CU(h->b_area.ensure(sizeof(double) * N));
  CU(h->b_type.ensure(sizeof(int) * N));
  CU(h->b_rowptr.ensure(sizeof(int) * (N + 1)));
  CU(h->b_counts.ensure(sizeof(int) * N));
  CU(h->b_pair.ensure(sizeof(double) * pair.size()));
  CU(h->b_perm.ensure(sizeof(int) * N));
  d.pos64 = h->b_pos.as<double>();
  d.Rq = h->b_Rq.as<double>();
  d.Rmu = h->b_Rmu.as<double>();
  d.area = h->b_area.as<double>();
  d.type = h->b_type.as<int>();
  d.rowptr = h->b_rowptr.as<int>();
  d.perm = h->b_perm.as<int>();
  // ---- staging (Angstrom -> bohr, Morton order, per-atom parameters) on the device
  {
    const size_t in_bytes = round_up(sizeof(double) * 3 * N, 256) + round_up(sizeof(int) * N, 256) +
                            round_up(sizeof(px_atom_type) * ntypes, 256);
    const size_t tmp_bytes = h->opt.sort_atoms ? px::stage_scratch_bytes(N) : 0;
    CU(h->b_stage.ensure(in_bytes + tmp_bytes));
    unsigned char* sp = h->b_stage.as<unsigned char>();
    double* d_xyz = reinterpret_cast<double*>(sp);
    int* d_tidx = reinterpret_cast<int*>(sp + round_up(sizeof(double) * 3 * N, 256));
    px_atom_type* d_types = reinterpret_cast<px_atom_type*>(
        sp + round_up(sizeof(double) * 3 * N, 256) + round_up(sizeof(int) * N, 256));
    CU(cudaMemcpyAsync(d_xyz, xyz, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d_tidx, tidx, sizeof(int) * N, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(d_types, types, sizeof(px_atom_type) * ntypes, cudaMemcpyHostToDevice, s));
    CU(px::launch_stage_atoms(d_xyz, d_tidx, d_types, N, h->opt.sort_atoms != 0, sp + in_bytes,
                              tmp_bytes, d.perm, d.pos64, d.type, d.Rq, d.Rmu, d.area, s, &h->nl));
  }
  CU(cudaMemcpyAsync(h->b_pair.p, pair.data(), sizeof(double) * pair.size(), cudaMemcpyHostToDevice, s));
  const double* dpair = h->b_pair.as<double>();
  const double* d_rcut2 = dpair;
  const double* d_r0 = dpair + ntypes * ntypes;
  const double* d_d = d_r0 + ntypes * ntypes;
  const double* d_s = d_d + ntypes * ntypes;

  CU(px::launch_neigh_count(d.pos64, N, d.type, ntypes, d_rcut2, h->b_counts.as<int>(), s, &h->nl));
  CU(px::launch_scan(h->b_counts.as<int>(), N, d.rowptr, s, &h->nl));
  int nnz = 0;
  CU(cudaMemcpyAsync(&nnz, d.rowptr + N, sizeof(int), cudaMemcpyDeviceToHost, s));
  sync_stream(h, s);
  d.nnz = nnz;
  size_t nnz_alloc = std::max(nnz, 1);
  CU(h->b_col.ensure(sizeof(int) * nnz_alloc));
  CU(h->b_val64.ensure(sizeof(double) * nnz_alloc));
  CU(h->b_val32.ensure(sizeof(float) * nnz_alloc));
  d.col = h->b_col.as<int>();
  d.val64 = h->b_val64.as<double>();
  d.val32 = h->b_val32.as<float>();
  CU(px::launch_neigh_fill(d.pos64, N, d.type, ntypes, d_rcut2, d_r0, d_d, d_s, d.area, d.rowptr,
                           d.col, d.val64, d.val32, s, &h->nl));
  d.tpar = nullptr;
  d.nncnt = nullptr;
  d.ident = nullptr;
  if (hetero) {
    // per-type n, tau, area; Eq. 10's nearest-neighbour counts; the identity numbering
    std::vector<double> tp(3 * (size_t)ntypes);
    for (int t = 0; t < ntypes; ++t) {
      tp[3 * t] = types[t].drude_n_au;
      tp[3 * t + 1] = types[t].tau_au;
      tp[3 * t + 2] = types[t].area_bohr2;
    }
    const size_t o1 = round_up(sizeof(double) * tp.size(), 256);
    const size_t o2 = o1 + round_up(sizeof(int) * (size_t)N * ntypes, 256);
    CU(h->b_hstruct.ensure(o2 + sizeof(int) * (size_t)N));
    unsigned char* hb = h->b_hstruct.as<unsigned char>();
    d.tpar = reinterpret_cast<double*>(hb);
    d.nncnt = reinterpret_cast<int*>(hb + o1);
    d.ident = reinterpret_cast<int*>(hb + o2);
    CU(cudaMemcpyAsync(d.tpar, tp.data(), sizeof(double) * tp.size(), cudaMemcpyHostToDevice, s));
    CU(px::launch_nn_counts(d.pos64, N, d.type, ntypes, d_r0, d_s, d.rowptr, d.col, d.nncnt, d.ident,
                            s, &h->nl));
    sync_stream(h, s);   // tp is read by the copy
  }

  // T storage: materialised (FP64 for the true residual, plus the low-precision copy of the
  // matvec) when it fits the HBM budget, else generated on the fly inside the matvecs.
  const int prec = h->opt.precision;
  const bool split = prec == PX_BF16SPLIT || prec == PX_FP16SPLIT;
  size_t np2 = (size_t)d.np * d.np;
  size_t need = np2 * sizeof(double);
  const bool ff_planes = prec != PX_FP64 || (h->opt.solver == PX_SOLVER_SHIFTED && model == PX_WFQ);
  if (ff_planes) need += 2 * np2 * sizeof(float);   // double-FP32 planes (residual, shifted)
  if (prec == PX_FP32) need += np2 * sizeof(float);
  if (split) need += 2 * np2 * sizeof(uint16_t) + np2 * sizeof(double);   // + transient FP64 M
  size_t budget = h->opt.hbm_budget_bytes;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    CU(cudaMemGetInfo(&fr, &tot));
    budget = (size_t)(0.6 * (double)fr) + h->b_T64.bytes + h->b_T32.bytes + h->b_Thi.bytes +
             h->b_Tlo.bytes;
  }
  int mode = h->opt.mode;
  if (mode == PX_MODE_AUTO) mode = need <= budget ? PX_MODE_MATERIALISED : PX_MODE_MATFREE;
  if (mode == PX_MODE_MATERIALISED && need > budget)
    throw PxError{PX_ENOMEM, "materialised T does not fit the HBM budget"};
  d.matfree = mode == PX_MODE_MATFREE;
  d.T64 = nullptr;
  d.T32 = nullptr;
  d.Thi = d.Tlo = nullptr;
  d.Tffh = d.Tffl = nullptr;
  d.op_has_kbar = false;
  d.op_scale_exp = 12;
  d.t_f16 = prec == PX_FP16SPLIT;
  d.mu_self = h->opt.mu_self_term;
  d.rm2f = nullptr;
  d.rm2d = nullptr;
  d.pos4tc = nullptr;
  d.tc_wmax = 0.f;
  if (d.matfree) {
    // split precisions run the tensor-core pair kernels: T scaled by 2^e before the fp16
    // split, 2^e max|T| <= 2^14 with max|T| bounded from the smallest widths: T^qq by its
    // diagonal sqrt(2/pi) / R_q; wFQFmu also |T^qmu| <= 0.43 / R^2 (R^2 = R_q^2 + R_mu^2)
    // and |T^mumu| <= 0.76 / R^3 (R^2 = 2 R_mu^2; the self term 0.75 / R^3), both taken with
    // margin (0.5, 1.0)
    if (split) {
      double rq_min = types[0].Rq_bohr, rq_max = types[0].Rq_bohr, rm_min = types[0].Rmu_bohr;
      for (int t = 1; t < ntypes; ++t) {
        rq_min = std::min(rq_min, types[t].Rq_bohr);
        rq_max = std::max(rq_max, types[t].Rq_bohr);
        rm_min = std::min(rm_min, types[t].Rmu_bohr);
      }
      double tmax = 0.7978845608028654 / rq_min;
      if (model == PX_WFQFMU)
        tmax = std::max({tmax, 0.5 / (rq_min * rq_min + rm_min * rm_min),
                         1.0 / std::pow(2.0 * rm_min * rm_min, 1.5)});
      d.op_scale_exp = prec == PX_FP16SPLIT
                           ? std::max(-60, std::min(60, (int)std::floor(std::log2(16384.0 / tmax))))
                           : 0;
      d.tc_wmax = (float)(rq_max * rq_max * std::ldexp(1.0, -2 * d.op_scale_exp));
    }
    CU(h->b_pos4f.ensure(sizeof(float4) * N));
    CU(h->b_pos4d.ensure(sizeof(double) * 4 * N));
    d.pos4f = h->b_pos4f.as<float4>();
    d.pos4d = h->b_pos4d.as<double>();
    if (model == PX_WFQFMU) {
      CU(h->b_rm2.ensure(round_up(sizeof(float) * N, 256) + sizeof(double) * N));
      d.rm2f = h->b_rm2.as<float>();
      d.rm2d = reinterpret_cast<double*>(h->b_rm2.as<unsigned char>() + round_up(sizeof(float) * N, 256));
    }
    CU(px::launch_stage_pos4(d, s, &h->nl));
    if (split) {
      // wFQ: np atoms of one float4; wFQFmu: np / 4 atoms of two
      CU(h->b_pos4tc.ensure(sizeof(float4) * (size_t)d.np));
      d.pos4tc = h->b_pos4tc.as<float4>();
      if (model == PX_WFQFMU)
        CU(px::launch_tc_mf4_positions(d.pos64, d.Rq, d.Rmu, N, d.np, d.pos4tc, s, &h->nl));
      else
        CU(px::launch_tc_mf_positions(d.pos64, d.Rq, N, d.np, d.op_scale_exp, d.pos4tc, s, &h->nl));
    }
  } else {
    CU(h->b_T64.ensure(np2 * sizeof(double)));
    d.T64 = h->b_T64.as<double>();
    if (prec == PX_FP32) {
      CU(h->b_T32.ensure(np2 * sizeof(float)));
      d.T32 = h->b_T32.as<float>();
    }
    if (split) {
      CU(h->b_Thi.ensure(np2 * sizeof(uint16_t)));
      CU(h->b_Tlo.ensure(np2 * sizeof(uint16_t)));
      d.Thi = h->b_Thi.as<uint16_t>();
      d.Tlo = h->b_Tlo.as<uint16_t>();
    }
    CU(px::launch_build_T64(d, h->opt.mu_self_term, s, &h->nl));
    if (d.T32) CU(px::launch_convert_T(d, s, &h->nl));
    if (d.Thi) {
      // tensor-core operator M = diag(Kbar, I) T: the conductance gather leaves the
      // Krylov step and Kbar's differences are taken in FP64.  The fp16 parts are scaled
      // by 2^e with 2^e max|M| <= 2^14 (the shift kernel undoes the scale).
      CU(h->b_M64.ensure(np2 * sizeof(double) + 256));
      double* M64 = h->b_M64.as<double>();
      unsigned long long* d_amax = reinterpret_cast<unsigned long long*>(M64 + np2);
      CU(cudaMemsetAsync(d_amax, 0, sizeof(unsigned long long), s));
      CU(px::launch_build_M64(d, M64, d_amax, s, &h->nl));
      unsigned long long amax_bits = 0;
      CU(cudaMemcpyAsync(&amax_bits, d_amax, sizeof(amax_bits), cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      double amax = 0.0;
      std::memcpy(&amax, &amax_bits, sizeof(amax));
      if (!std::isfinite(amax)) throw PxError{PX_EINVAL, "non-finite operator entries"};
      int e = 12;
      if (amax > 0.0) e = std::max(-60, std::min(60, (int)std::floor(std::log2(16384.0 / amax))));
      d.op_scale_exp = e;
      d.op_has_kbar = true;
      CU(px::launch_split_op(M64, np2, d.Thi, d.Tlo, d.t_f16, e, s, &h->nl));
      CU(cudaStreamSynchronize(s));
      h->b_M64.release();   // only the split planes stay resident
    }
    if (ff_planes) {
      CU(h->b_Tffh.ensure(np2 * sizeof(float)));
      CU(h->b_Tffl.ensure(np2 * sizeof(float)));
      d.Tffh = h->b_Tffh.as<float>();
      d.Tffl = h->b_Tffl.as<float>();
      CU(px::launch_split_ff(d.T64, np2, d.Tffh, d.Tffl, s, &h->nl));
    }
  }
  CU(cudaEventRecord(h->ev_b, s));
  wait_event(h, h->ev_b);
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
  h->stats.setup_ms = ms;
  h->stats.setup_launches = h->nl;
  h->stats.n_unknowns = d.nu;
  h->stats.used_mode = d.matfree ? PX_MODE_MATFREE : PX_MODE_MATERIALISED;
  h->drude_n = types[0].drude_n_au;
  h->tau = types[0].tau_au;
  h->have_structure = true;
}


// ------------------------------------------------------------------ boundary elements
// The precision planes of a dense boundary-element operator whose FP64 form d.T64 holds it
// transposed (S = Op^T, see launch_build_F): FP32 and double-FP32 copies of S (the block
// matvecs and the shifted matvec read S as the transposed operator), and for the
// tensor-core modes hi/lo planes of Op itself (row-major, as that GEMM reads them).
void bem_planes(px_handle* h, px::DevStructure& d, DevBuf& bT32, DevBuf& bThi, DevBuf& bTlo,
                DevBuf& bTffh, DevBuf& bTffl, cudaStream_t s) {
  const int prec = h->opt.precision;
  const bool split = prec == PX_BF16SPLIT || prec == PX_FP16SPLIT;
  const size_t np2 = (size_t)d.np * d.np;
  d.op_has_kbar = split;
  d.op_scale_exp = 12;
  d.t_f16 = prec == PX_FP16SPLIT;
  if (prec == PX_FP32) {
    CU(bT32.ensure(np2 * sizeof(float)));
    d.T32 = bT32.as<float>();
    CU(px::launch_convert_T(d, s, &h->nl));
  }
  if (split) {
    CU(bThi.ensure(np2 * sizeof(uint16_t)));
    CU(bTlo.ensure(np2 * sizeof(uint16_t)));
    d.Thi = bThi.as<uint16_t>();
    d.Tlo = bTlo.as<uint16_t>();
    CU(h->b_M64.ensure(np2 * sizeof(double) + 256));
    double* M64 = h->b_M64.as<double>();
    unsigned long long* d_amax = reinterpret_cast<unsigned long long*>(M64 + np2);
    CU(cudaMemsetAsync(d_amax, 0, sizeof(unsigned long long), s));
    CU(px::launch_transpose_absmax(d.T64, d.np, M64, d_amax, s, &h->nl));
    unsigned long long amax_bits = 0;
    CU(cudaMemcpyAsync(&amax_bits, d_amax, sizeof(amax_bits), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    double amax = 0.0;
    std::memcpy(&amax, &amax_bits, sizeof(amax));
    if (!std::isfinite(amax)) throw PxError{PX_EINVAL, "non-finite operator entries"};
    int e = 12;
    if (amax > 0.0) e = std::max(-60, std::min(60, (int)std::floor(std::log2(16384.0 / amax))));
    d.op_scale_exp = e;
    CU(px::launch_split_op(M64, np2, d.Thi, d.Tlo, d.t_f16, e, s, &h->nl));
    CU(cudaStreamSynchronize(s));
    h->b_M64.release();
  }
  if (prec != PX_FP64 || h->opt.solver == PX_SOLVER_SHIFTED) {
    CU(bTffh.ensure(np2 * sizeof(float)));
    CU(bTffl.ensure(np2 * sizeof(float)));
    d.Tffh = bTffh.as<float>();
    d.Tffl = bTffl.as<float>();
    CU(px::launch_split_ff(d.T64, np2, d.Tffh, d.Tffl, s, &h->nl));
  }
}

// A meshed surface (Sec. 2.3): tesserae with barycentres, outward normals and areas.  DPCM
// (Eq. 11, normal-field form): one dense operator Ft in place of Kbar T, every frequency a
// column shift Lambda(w).  IEFPCM (Eq. 12): the operator F of the first step (column shift
// -Lambda(w)) and the Coulomb matrix S A^-1 of the second.
void set_mesh(px_handle* h, int n, const double* pos_ang, const double* nrm,
              const double* area_ang2, double radius_ang, int formulation) {
  if (!pos_ang || !nrm || !area_ang2) throw PxError{PX_EINVAL, "NULL input"};
  if (n < 1) throw PxError{PX_EINVAL, "n_tess must be >= 1"};
  if (formulation != PX_BEM_DPCM && formulation != PX_BEM_IEFPCM)
    throw PxError{PX_EINVAL, "formulation must be PX_BEM_DPCM or PX_BEM_IEFPCM"};
  if (!std::isfinite(radius_ang) || !(radius_ang > 0.0)) throw PxError{PX_EINVAL, "radius must be finite and > 0"};
  std::vector<double> pos(3 * (size_t)n), area(n);
  for (int i = 0; i < n; ++i) {
    double n2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double p = pos_ang[3 * (size_t)i + k], v = nrm[3 * (size_t)i + k];
      if (!std::isfinite(p) || !std::isfinite(v)) throw PxError{PX_EINVAL, "non-finite mesh data"};
      pos[3 * (size_t)i + k] = p / kBohrAng;
      n2 += v * v;
    }
    if (std::fabs(std::sqrt(n2) - 1.0) > 1e-6) throw PxError{PX_EINVAL, "normals must be unit vectors"};
    if (!std::isfinite(area_ang2[i]) || !(area_ang2[i] > 0.0)) throw PxError{PX_EINVAL, "areas must be > 0"};
    area[i] = area_ang2[i] / (kBohrAng * kBohrAng);
  }
  if (h->opt.mode == PX_MODE_MATFREE) throw PxError{PX_ENOTIMPL, "meshes need the materialised operator"};
  const bool ief = formulation == PX_BEM_IEFPCM;
  cudaStream_t s = h->own_stream;
  px::DevStructure& d = h->ds;
  h->have_structure = false;
  d = px::DevStructure{};
  h->ds_g = px::DevStructure{};
  d.model = PX_WFQ;   // one unknown per element, one scalar shift per column
  d.bem = true;
  d.bem_stage = ief ? 1 : 0;
  d.N = n;
  d.nu = n;
  d.np = (int)round_up(n, px::kTile);
  d.ntypes = 1;
  h->nl = 0;
  CU(cudaEventRecord(h->ev_a, s));
  CU(h->b_pos.ensure(sizeof(double) * 3 * n));
  CU(h->b_mesh.ensure(round_up(sizeof(double) * 3 * n, 256) + sizeof(double) * n));
  CU(h->b_perm.ensure(sizeof(int) * n));
  CU(h->b_type.ensure(sizeof(int) * n));
  d.pos64 = h->b_pos.as<double>();
  d.nrm = h->b_mesh.as<double>();
  d.tarea = reinterpret_cast<double*>(h->b_mesh.as<unsigned char>() + round_up(sizeof(double) * 3 * n, 256));
  d.perm = h->b_perm.as<int>();
  d.type = h->b_type.as<int>();
  std::vector<int> iota(n);
  for (int i = 0; i < n; ++i) iota[i] = i;
  CU(cudaMemcpyAsync(d.pos64, pos.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(d.nrm, nrm, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(d.tarea, area.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(d.perm, iota.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(d.type, 0, sizeof(int) * n, s));
  const size_t np2 = (size_t)d.np * d.np;
  CU(h->b_T64.ensure(np2 * sizeof(double)));
  d.T64 = h->b_T64.as<double>();
  CU(px::launch_build_F(d.pos64, d.nrm, d.tarea, radius_ang / kBohrAng, n, d.np, ief, d.T64, s, &h->nl));
  bem_planes(h, d, h->b_T32, h->b_Thi, h->b_Tlo, h->b_Tffh, h->b_Tffl, s);
  if (ief) {
    // second step: (S A^-1) q = y, a symmetric operator with charges as unknowns (no
    // area weight in the observables)
    px::DevStructure& g = h->ds_g;
    g = d;
    g.bem_stage = 2;
    g.tarea = nullptr;
    g.T32 = nullptr;
    g.Thi = g.Tlo = nullptr;
    g.Tffh = g.Tffl = nullptr;
    CU(h->g_T64.ensure(np2 * sizeof(double)));
    g.T64 = h->g_T64.as<double>();
    CU(px::launch_build_G(d.pos64, d.tarea, n, d.np, g.T64, s, &h->nl));
    bem_planes(h, g, h->g_T32, h->g_Thi, h->g_Tlo, h->g_Tffh, h->g_Tffl, s);
  }
  CU(cudaEventRecord(h->ev_b, s));
  wait_event(h, h->ev_b);
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
  h->stats.setup_ms = ms;
  h->stats.setup_launches = h->nl;
  h->stats.n_unknowns = n;
  h->stats.used_mode = PX_MODE_MATERIALISED;
  h->drude_n = h->tau = 1.0;   // unused: the column shifts come from the permittivities
  h->have_structure = true;
}

// ------------------------------------------------------------------ solve
struct SolveOut {
  double2* d_alpha = nullptr;  // device [F][3][P]
  double2* d_q = nullptr;      // device [F][P][N]
  double2* d_mu = nullptr;     // device [F][P][N][3]
  double* d_relres = nullptr;  // device [F][P]
  double* d_sigma_pol = nullptr;  // device [F][P]
  double* d_sigma = nullptr;      // device [F] (P == 3)
  bool sigma_required = false;    // the caller asked for sigma_abs (P == 3 needs an
                                  // invertible triple of field directions)
  std::vector<double> relres;  // [B]
  std::vector<int> iters;      // [B]
  std::vector<int> status;     // [B]
};

template <typename T>
T* grow(DevBuf& b, size_t n) {
  CU(b.ensure(std::max<size_t>(n, 1) * sizeof(T)));
  return b.as<T>();
}

px_status solve(px_handle* h, int F, const double* omega_ev, const double* alpha_ib, int P,
                const double* pol, double e0, SolveOut* so, cudaStream_t s,
                const double* eps = nullptr, const double2* rhs_c = nullptr) {
  if (!h->have_structure) throw PxError{PX_EINVAL, "no structure loaded"};
  if (F < 1 || P < 1 || !omega_ev || !pol)
    throw PxError{PX_EINVAL, "need n_freq >= 1, n_pol >= 1, omega_ev and pol_dir"};
  if (!std::isfinite(e0) || !(e0 > 0.0)) throw PxError{PX_EINVAL, "e0 must be finite and > 0"};
  const px::DevStructure& d = h->ds;
  const int model = d.model;
  if (model == PX_WFQFMU && !alpha_ib) throw PxError{PX_EINVAL, "alpha_ib is required for PX_WFQFMU"};
  if (d.bem && !eps) throw PxError{PX_EINVAL, "a mesh is solved with px_solve_bem"};
  if (!d.bem && eps) throw PxError{PX_EINVAL, "px_solve_bem needs a mesh loaded with px_set_mesh"};
  if (d.bem)
    for (size_t k = 0; k < 4 * (size_t)F; ++k)
      if (!std::isfinite(eps[k])) throw PxError{PX_EINVAL, "non-finite permittivity"};
  if (d.bem)
    for (int f = 0; f < F; ++f)
      if (eps[4 * f] == eps[4 * f + 2] && eps[4 * f + 1] == eps[4 * f + 3])
        throw PxError{PX_EINVAL, "e2 == e1: the particle does not polarise"};
  for (int f = 0; f < F; ++f)
    if (!std::isfinite(omega_ev[f]) || !(omega_ev[f] > 0.0))
      throw PxError{PX_EINVAL, "frequencies must be finite and > 0"};
  for (int p = 0; p < P; ++p) {
    double n2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      double v = pol[3 * p + k];
      if (!std::isfinite(v)) throw PxError{PX_EINVAL, "non-finite polarisation"};
      n2 += v * v;
    }
    if (std::fabs(std::sqrt(n2) - 1.0) > 1e-6) throw PxError{PX_EINVAL, "polarisation directions must be unit vectors"};
  }
  if (model == PX_WFQFMU)
    for (size_t k = 0; k < 2 * (size_t)d.ntypes * F; ++k)
      if (!std::isfinite(alpha_ib[k])) throw PxError{PX_EINVAL, "non-finite alpha_ib"};
  if ((long long)F * P > (1LL << 24)) throw PxError{PX_EINVAL, "too many columns"};
  // sigma_abs = 4 pi w/(3c) Tr Im alpha needs the full alpha tensor, which three linearly
  // independent field directions determine: alpha = A E^-1
  double pol_inv[9];
  const bool have_triple = P == 3 && px::pol_triple_inverse(pol, pol_inv);
  if (P == 3 && so->sigma_required && !have_triple)
    throw PxError{PX_EINVAL, "sigma_abs needs three linearly independent field directions"};

  const int B = F * P;
  const int nu = d.nu, np = d.np, N = d.N, ntypes = d.ntypes;
  const px_options& o = h->opt;
  // restart length: explicit, or automatic (0): a low-precision wFQ solve converges about
  // as fast with short restarts, whose Gram-Schmidt traffic is lower; wFQFmu, and FP64
  // solves (whose cost is the FP64 matvec, not the orthogonalisation), take longer ones
  const int m_req = o.restart_m > 0 ? o.restart_m
                                    : (model == PX_WFQ && o.precision != PX_FP64 ? 60 : 100);
  const int m = std::min(m_req, o.max_iter);
  const int passes = o.gs_passes;
  const bool lowp = o.precision != PX_FP64;
  const bool tc = o.precision == PX_BF16SPLIT || o.precision == PX_FP16SPLIT;
  const bool tc_f16 = o.precision == PX_FP16SPLIT;
  if (tc && d.Thi == nullptr && !d.matfree)
    throw PxError{PX_EINVAL, "precision changed since px_set_structure"};
  // operand column padding of every matvec kernel; the tensor-core pair kernel runs
  // 256-column tiles (each generated T tile then serves twice the columns)
  const size_t colpad = (d.matfree && tc) ? 2 * px::kTile : px::kTile;
  // stopping targets of the inner (low-precision) iteration:
  //   max(inner_tol * ||r_outer||, tol_frac * tol * ||b||)
  const double inner_tol = lowp ? o.inner_tol : 0.0;
  const double tol_abs_frac = (lowp ? 0.1 : 0.5) * o.tol_rel;
  const int max_inner = 50;   // inner cycles per refinement round
  // restart cycles as graph launches, unless every matvec is timed with events
  const bool use_graphs = o.cycle_graphs != 0 && !o.profile;
  const int nblk = px::reduction_blocks(nu);
  long long& nl = h->nl;
  nl = 0;
  px_stats& st = h->stats;
  st.matvec_ms = st.resid_ms = 0.0;
  st.matvec_launches = st.resid_launches = 0;
  st.matvec_flops = st.matvec_bytes = st.resid_flops = 0.0;
  st.cycles = 0;
  st.total_iters = 0;
  st.used_precision = o.precision;
  st.gemm_tiles_used = 0;
  st.graph_launches = 0;
  st.graphs_built = 0;
  // the shifted solver applies to Eq. 1 (one scalar shift); wFQFmu solves stay batched
  const bool shifted = o.solver == PX_SOLVER_SHIFTED && model == PX_WFQ && !rhs_c;
  st.solver_used = shifted ? PX_SOLVER_SHIFTED : PX_SOLVER_BATCHED;
  st.shift_steps = st.shift_matvec_launches = 0;
  st.shift_matvec_ms = st.shift_matvec_bytes = st.shift_ms = 0.0;
  if (shifted && (d.matfree || d.Tffh == nullptr))
    throw PxError{d.matfree ? PX_ENOTIMPL : PX_EINVAL,
                  d.matfree ? "the shifted solver needs the materialised T"
                            : "select the shifted solver before px_set_structure"};
  CU(cudaEventRecord(h->ev_a, s));

  // ---- inputs, shifts (Eq. 6, Eq. 8) and right-hand sides
  double* d_omega = grow<double>(h->b_pol, 3 * (size_t)P + F + 2 * (size_t)ntypes * F + 4 * (size_t)F);
  double* d_pol = d_omega + F;
  double* d_aib = d_pol + 3 * P;
  double* d_eps = d_aib + 2 * (size_t)ntypes * F;
  if (d.bem) CU(cudaMemcpyAsync(d_eps, eps, sizeof(double) * 4 * F, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(d_omega, omega_ev, sizeof(double) * F, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(d_pol, pol, sizeof(double) * 3 * P, cudaMemcpyHostToDevice, s));
  if (model == PX_WFQFMU)
    CU(cudaMemcpyAsync(d_aib, alpha_ib, sizeof(double) * 2 * ntypes * F, cudaMemcpyHostToDevice, s));
  double2* zq_all = grow<double2>(h->b_zq, 2 * (size_t)B);          // [B] all, then [B] active
  double2* zq_act = zq_all + B;
  double2* zmu_all = grow<double2>(h->b_zmu, 3 * (size_t)ntypes * B);
  double2* zmu_act = zmu_all + (size_t)ntypes * B;
  // wFQFmu right preconditioner diag(I, alpha^IB): alpha^IB of every active column
  double2* amu_act = model == PX_WFQFMU ? zmu_all + 2 * (size_t)ntypes * B : nullptr;
  CU(px::launch_shifts(F, P, ntypes, model, d_omega, d_aib, h->drude_n, h->tau, zq_all, zmu_all,
                       s, &nl));
  double* b = grow<double>(h->b_b, (size_t)nu * P);
  double* bnorm = grow<double>(h->b_bnorm, P + (size_t)B);
  double* bn = bnorm + P;                                   // [B] per-column ||b||
  double* colv = grow<double>(h->b_rnorm, 3 * (size_t)B);   // rnorm | beta | target_all
  double* rnorm = colv;
  double* beta = colv + B;
  double* target_all = colv + 2 * (size_t)B;
  double2* x = grow<double2>(h->b_x, (size_t)nu * B);
  double2* r = grow<double2>(h->b_r, (size_t)nu * B);
  int* iters = grow<int>(h->b_iters, B);
  int* act = grow<int>(h->b_act, B);
  CU(cudaMemsetAsync(x, 0, sizeof(double2) * (size_t)nu * B, s));
  CU(cudaMemsetAsync(iters, 0, sizeof(int) * B, s));
  // heterogeneous wFQFmu (Eq. 9): z_q per type, the per-atom z_mu of Eq. 10, complex bond
  // weights of 1/2 (Kbar + Hbar(w)) and a complex right-hand side per column
  const bool het = d.hetero;
  double2* zq_het = nullptr;       // [ntypes][B] | act [ntypes][B]
  double2* kap_all = nullptr;      // [ntypes^2][B] | act [ntypes^2][B]
  double2* kap_act = nullptr;
  double2* bc = nullptr;           // [nu][B]
  double2* zmu_het = nullptr;      // per-atom z_mu: [N][B] all | [N][B] active | alpha^IB [N][B]
  if (het) {
    const size_t nt2 = (size_t)ntypes * ntypes;
    double2* hb = grow<double2>(h->b_het, (2 * ntypes + 2 * nt2 + 3 * (size_t)N + nu) * (size_t)B);
    zq_het = hb;
    kap_all = zq_het + 2 * (size_t)ntypes * B;
    kap_act = kap_all + nt2 * B;
    zmu_het = kap_act + nt2 * B;
    bc = zmu_het + 3 * (size_t)N * B;
    CU(px::launch_hetero_tables(F, P, ntypes, N, d_omega, d.tpar, d.type, d.nncnt, zmu_all, zq_het,
                                kap_all, zmu_het, s, &nl));
    CU(px::launch_rhs_hetero(N, F, P, d.rowptr, d.col, d.val64, d.type, ntypes, kap_all, d.pos64,
                             d_pol, e0, bc, bn, s, &nl));
    CU(px::launch_init_residual_c(bc, nu, B, bn, inner_tol, tol_abs_frac, r, rnorm, beta, target_all,
                                  s, &nl));
  } else if (rhs_c) {
    // second IEFPCM step (Eq. 12): (S A^-1) q = y, one complex right-hand side per column
    CU(px::launch_bem_setup(F, P, nu, np, d.bem_stage, d_eps, d.nrm, d.T64, d.pos64, d_pol, e0,
                            zq_all, b, s, &nl));
    bc = const_cast<double2*>(rhs_c);
    CU(px::launch_col_norms_c(bc, nu, B, bn, s, &nl));
    CU(px::launch_init_residual_c(bc, nu, B, bn, inner_tol, tol_abs_frac, r, rnorm, beta, target_all,
                                  s, &nl));
  } else {
    if (d.bem)   // Eqs. 11, 12: the shift of every column (overwrites z_q) and b
      CU(px::launch_bem_setup(F, P, nu, np, d.bem_stage, d_eps, d.nrm, d.T64, d.pos64, d_pol, e0,
                              zq_all, b, s, &nl));
    else
      CU(px::launch_rhs(nu, N, model, d.rowptr, d.col, d.val64, d.pos64, d_pol, P, e0, b, s, &nl));
    CU(px::launch_col_norms(b, nu, P, bnorm, s, &nl));
    CU(px::launch_bnorm_cols(bnorm, P, B, bn, s, &nl));
    CU(px::launch_init_residual(b, nu, P, B, bnorm, inner_tol, tol_abs_frac, r, rnorm, beta,
                                target_all, s, &nl));
  }
  // the active columns' shifts: homogeneous z_q per column and z_mu per type; the
  // heterogeneous model indexes z_mu per atom (dipole "types" = atoms) and z_q per type
  const int* dip_type = het ? d.ident : d.type;
  const int n_dip_types = het ? N : ntypes;
  const double2* zmu_src = het ? zmu_het : zmu_all;
  double2* zmu_act_h = het ? zmu_het + (size_t)N * B : zmu_act;
  double2* amu_act_h = het ? zmu_het + 2 * (size_t)N * B : amu_act;
  double2* zq_act_h = het ? zq_het + (size_t)ntypes * B : zq_act;
  auto gather_active = [&](int Bact, bool with_amu) {
    CU(px::launch_gather_shifts(het ? zq_het : zq_all, zmu_src, n_dip_types, B, act, Bact, zq_act_h,
                                zmu_act_h, with_amu ? amu_act_h : nullptr, s, &nl));
    if (het) {
      CU(px::launch_gather_rows(zq_het, ntypes, B, act, Bact, zq_act_h, s, &nl));
      CU(px::launch_gather_rows(kap_all, ntypes * ntypes, B, act, Bact, kap_act, s, &nl));
    }
  };

  // ---- Krylov workspace for up to B active columns
  px::KrylovArgs A{};
  A.nu = nu;
  A.m = m;
  A.nblk = nblk;
  // basis element: FP64 for FP64 solves; FP32 (automatic) or as the options say for the
  // low-precision ones
  A.basis = px::basis_kind(o.precision, o.basis);
  const size_t esz_max = px::basis_bytes(A.basis);
  void* V = grow<unsigned char>(h->b_V, (size_t)(m + 1) * nu * B * esz_max);
  void* W = grow<unsigned char>(h->b_W, (size_t)nu * B * esz_max);
  double2* hh = grow<double2>(h->b_h, 2 * (size_t)(m + 1) * B);
  double2* part = grow<double2>(h->b_part, (size_t)nblk * (m + 1) * B);
  double* normpart = grow<double>(h->b_normpart, (size_t)nblk * B);
  // the rotated Hessenberg is sized for the longest restart a shrunken active set may use
  double2* Rm = grow<double2>(h->b_R, (size_t)std::max(m, px::kMaxRestart) * (m + 1) * B);
  double2* g = grow<double2>(h->b_g, (size_t)(m + 1) * B);
  double* cs = grow<double>(h->b_cs, (size_t)(m + 1) * B);
  double2* sn = grow<double2>(h->b_sn, (size_t)(m + 1) * B);
  double* target = grow<double>(h->b_target, B);
  int* jconv = grow<int>(h->b_jconv, B);
  double* invh = grow<double>(h->b_invh, B);
  double2* yv = grow<double2>(h->b_y, (size_t)(2 * m + 2) * B);   // y [m][B] | u [m+1][B]
  const int ldx = (int)round_up(2 * (size_t)B, colpad);
  float* X32 = nullptr;
  float* Y32 = nullptr;
  uint16_t* Xth = nullptr;
  uint16_t* Xtl = nullptr;
  if (lowp) {
    X32 = grow<float>(h->b_X32, (size_t)np * ldx);
    Y32 = grow<float>(h->b_Y32, (size_t)np * ldx);
  }
  if (tc) {
    Xth = grow<uint16_t>(h->b_Xth, (size_t)np * ldx);
    Xtl = grow<uint16_t>(h->b_Xtl, (size_t)np * ldx);
  }
  CU(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
  double* X64 = grow<double>(h->b_X64, (size_t)np * ldx);
  double* Y64 = grow<double>(h->b_Y64, (size_t)np * ldx);
  // split-K partial products of the FP64 GEMM (small N, FP64 solves): sized here for
  // every operand width a cycle can have, so no allocation happens inside a cycle
  double* dpart = nullptr;
  size_t dpart_elems = 0;
  if (!lowp && !d.matfree) {
    for (size_t w = colpad; w <= (size_t)ldx; w += colpad)
      dpart_elems = std::max(dpart_elems, (size_t)px::dgemm_splits(np, (int)w) * np * w);
    if (dpart_elems > (size_t)np * ldx) dpart = grow<double>(h->b_dpart, dpart_elems);
    else dpart_elems = 0;
  }
  A.V = V; A.W = W; A.h = hh; A.part = part; A.normpart = normpart; A.R = Rm; A.g = g;
  A.cs = cs; A.sn = sn; A.target = target; A.jconv = jconv; A.inv_h = invh;
  A.y = yv; A.u = yv + (size_t)m * B;
  A.active_count = h->d_active;
  A.N = N;
  A.type = dip_type;
  A.amu = amu_act ? amu_act_h : nullptr;

  std::vector<int> h_outer(B), h_inner(B), h_iters(B);
  std::vector<double> h_col(3 * (size_t)B), h_bn(B);
  CU(cudaMemcpyAsync(h_bn.data(), bn, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  sync_stream(h, s);
  // a column whose right-hand side is zero (e.g. no bond has a component along the
  // field) has the exact solution x = 0 and needs no iteration
  int Bout = 0;
  for (int c = 0; c < B; ++c)
    if (h_bn[c] > 0.0) h_outer[Bout++] = c;

  size_t prof_k = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> mv_events, rs_events, sk_events;
  int total_cycles = 0;
  int round0 = 0;
  if (shifted && Bout > 0) {
    // ---- shifted Krylov phase (Eq. 1 with the scalar shift of Eq. 6): x of every column
    // from one real Arnoldi process per field direction, then the FP64-class true
    // residual of every column; the columns that still miss tol_rel continue in the
    // refinement rounds below
    CU(cudaEventRecord(h->ev_sk[0], s));
    const int NPmax = std::min(P, 4);
    const size_t BgMax = (size_t)F * NPmax;
    const px::SkMatvecPlan plan = px::sk_matvec_plan(np);
    const int nrb = px::sk_row_blocks(nu);
    const int nnb = (nu + 255) / 256;
    auto carve_all = [&](size_t m, unsigned char* base, std::vector<void*>* ptrs) {
      size_t t = 0;
      const size_t sizes[] = {
          8 * (m + 1) * nu * NPmax,                          // V
          8 * m * nu * NPmax,                                // U = T V
          8 * (size_t)nu * NPmax,                            // W
          8 * (size_t)plan.parts() * np * NPmax,             // matvec partials
          8 * (size_t)nrb * (m + 1) * NPmax,                 // projection partials
          8 * 2 * (m + 1) * NPmax,                           // projections
          8 * (size_t)px::sk_update_chunks((int)m) * nu * NPmax,  // update partials
          8 * (size_t)nnb * NPmax,                           // norm partials
          8 * m * (m + 2) * NPmax,                           // Hessenberg
          8 * (size_t)NPmax,                                 // inv_h
          8 * m * BgMax,                                     // cs
          16 * m * BgMax,                                    // sn
          16 * (m + 1) * BgMax,                              // g
          16 * BgMax * (m * (m + 1) / 2),                    // R
          8 * BgMax,                                         // target
          4 * BgMax,                                         // jconv
          4 * m,                                             // active
          16 * m * BgMax,                                    // y
          4 * 2 * (size_t)NPmax * np};                       // planar matvec operand
      for (size_t b : sizes) {
        if (ptrs) ptrs->push_back(base + t);
        t += round_up(std::max<size_t>(b, 1), 256);
      }
      return t;
    };
    size_t m_sk = o.shift_krylov_max > 0 ? (size_t)o.shift_krylov_max : std::min<size_t>(nu, 2500);
    m_sk = std::max<size_t>(1, std::min<size_t>(m_sk, nu));
    if (o.shift_krylov_max == 0) {
      size_t fr = 0, tot = 0;
      CU(cudaMemGetInfo(&fr, &tot));
      const size_t budget = (size_t)(0.4 * (double)fr) + h->b_sk.bytes;
      while (m_sk > 16 && carve_all(m_sk, nullptr, nullptr) > budget) m_sk = m_sk * 7 / 8;
    }
    const int m = (int)m_sk;
    CU(h->b_sk.ensure(carve_all(m_sk, nullptr, nullptr)));
    std::vector<void*> pp;
    carve_all(m_sk, h->b_sk.as<unsigned char>(), &pp);
    float2* skV = static_cast<float2*>(pp[0]);
    float2* skU = static_cast<float2*>(pp[1]);
    float2* skW = static_cast<float2*>(pp[2]);
    float2* skPart = static_cast<float2*>(pp[3]);
    double* skDpart = static_cast<double*>(pp[4]);
    double* skProj = static_cast<double*>(pp[5]);
    float2* skUpart = static_cast<float2*>(pp[6]);
    double* skNpart = static_cast<double*>(pp[7]);
    double2* skY = static_cast<double2*>(pp[17]);
    if (h->h_skact_n < m_sk) {
      if (h->h_skact) cudaFreeHost(h->h_skact);
      h->h_skact = nullptr;
      h->h_skact_n = 0;
      CU(cudaHostAlloc((void**)&h->h_skact, sizeof(int) * m_sk, cudaHostAllocDefault));
      h->h_skact_n = m_sk;
    }
    for (int p0 = 0; p0 < P; p0 += 4) {
      px::SkGroup G;
      G.n = nu;
      G.NP = std::min(4, P - p0);
      G.P = P;
      G.p0 = p0;
      G.Bg = F * G.NP;
      G.m = m;
      G.H = static_cast<double*>(pp[8]);
      G.inv_h = static_cast<double*>(pp[9]);
      G.zq = zq_all;
      G.cs = static_cast<double*>(pp[10]);
      G.sn = static_cast<double2*>(pp[11]);
      G.g = static_cast<double2*>(pp[12]);
      G.R = static_cast<double2*>(pp[13]);
      G.rstride = m_sk * (m_sk + 1) / 2;
      G.target = static_cast<double*>(pp[14]);
      G.jconv = static_cast<int*>(pp[15]);
      G.active = static_cast<int*>(pp[16]);
      G.np = np;
      G.vp = static_cast<float*>(pp[18]);
      const int NP = G.NP;
      CU(cudaMemsetAsync(G.active, 0, sizeof(int) * m_sk, s));
      // the least-squares estimate stops a system at half the requested relative residual
      CU(px::launch_sk_start(G, b, bnorm, 0.5 * o.tol_rel, skV, s, &nl));
      int jend = 0;
      for (int j = 0; j < m; ++j) {
        float2* Uj = skU + (size_t)j * nu * NP;
        cudaEvent_t e0v = nullptr, e1v = nullptr;
        if (o.profile) {
          e0v = pool_event(h, prof_k++);
          e1v = pool_event(h, prof_k++);
          CU(cudaEventRecord(e0v, s));
        }
        // boundary-element operators are stored transposed
        CU(px::launch_sk_matvec(d.Tffh, d.Tffl, nu, np, NP, plan, d.bem, G.vp, skPart, Uj, s, &nl));
        if (o.profile) {
          CU(cudaEventRecord(e1v, s));
          sk_events.push_back({e0v, e1v});
        }
        if (d.bem)   // the operator Ft is complete: W = U
          CU(cudaMemcpyAsync(skW, Uj, sizeof(float2) * (size_t)nu * NP, cudaMemcpyDeviceToDevice, s));
        else
          CU(px::launch_sk_kbar(nu, NP, d.rowptr, d.col, d.val64, d.val32, Uj, skW, s, &nl));
        // two classical Gram-Schmidt passes (CGS2): every frequency shares this basis
        for (int pass = 0; pass < 2; ++pass)
          CU(px::launch_sk_gs_pass(skV, skW, nu, NP, j, m + 1, skDpart,
                                   skProj + (size_t)pass * (m + 1) * NP, skUpart, pass == 1,
                                   skNpart, s, &nl));
        CU(px::launch_sk_step_end(G, j, skProj, 2, skNpart, skV, skW, s, &nl));
        CU(cudaMemcpyAsync(h->h_skact + j, G.active + j, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaEventRecord(h->ev_iter[j & 1], s));
        jend = j + 1;
        // lagged poll: wait for step j-1, stop once every system of the group has stopped
        if (j >= 1) {
          wait_event(h, h->ev_iter[(j - 1) & 1]);
          if (reinterpret_cast<volatile int*>(h->h_skact)[j - 1] == 0) break;
        }
      }
      CU(px::launch_sk_solution(G, jend, skV, skU, skY, x, B, Y64, ldx, iters, s, &nl));
      st.shift_steps += jend;
      st.shift_matvec_launches += jend;
      st.shift_matvec_bytes += 8.0 * (double)nu * nu * jend;
      if (h->verbose)
        std::fprintf(stderr, "px: shifted group p0=%d directions %d systems %d steps %d (basis limit %d)\n",
                     p0, NP, G.Bg, jend, m);
    }
    // FP64-class true residual of every column: (T x) from the stored products T V
    {
      std::vector<int> all(B);
      for (int c = 0; c < B; ++c) all[c] = c;
      CU(cudaMemcpyAsync(act, all.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
      gather_active(B, false);
      px::ResidArgs ra{};
      ra.nu = nu; ra.N = N; ra.model = model; ra.Bact = B; ra.P = P; ra.B = B; ra.nblk = nblk;
      ra.rowptr = d.rowptr; ra.col = d.col; ra.val64 = d.val64; ra.type = d.type;
      ra.Y = Y64; ra.ldy = ldx; ra.x = x; ra.act = act; ra.b = b; ra.zq = zq_act; ra.zmu = zmu_act;
      ra.R = r; ra.normpart = normpart;
      ra.op_full = d.bem ? 1 : 0;
      CU(px::launch_resid(ra, s, &nl));
      CU(px::launch_norm_finish(normpart, nblk, B, act, B, bn, inner_tol, tol_abs_frac, rnorm,
                                beta, target_all, s, &nl));
      CU(cudaEventRecord(h->ev_sk[1], s));
      CU(cudaMemcpyAsync(h_col.data(), colv, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
      CU(cudaMemcpyAsync(h_iters.data(), iters, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
      sync_stream(h, s);
      float ms_sk = 0.f;
      CU(cudaEventElapsedTime(&ms_sk, h->ev_sk[0], h->ev_sk[1]));
      st.shift_ms = ms_sk;
      int nb = 0;
      double worst = 0.0;
      for (int k = 0; k < Bout; ++k) {
        const int c = h_outer[k];
        if (!std::isfinite(h_col[c])) throw PxError{PX_ECUDA, "non-finite residual after the shifted solve"};
        worst = std::max(worst, h_col[c] / h_bn[c]);
        if (h_col[c] > o.tol_rel * h_bn[c] && h_iters[c] < o.max_iter) h_outer[nb++] = c;
      }
      if (h->verbose)
        std::fprintf(stderr, "px: shifted phase true residual: max rel %.3e, %d of %d columns left\n",
                     worst, nb, Bout);
      Bout = nb;
      round0 = 1;
    }
  }
  // Refinement rounds: low-precision restarted GMRES on the current residual until every
  // column reached its inner target, then the FP64 true residual r = b - A x.
  for (int round = round0; Bout > 0 && total_cycles < o.max_cycles && round <= o.max_refine; ++round) {
    std::copy(h_outer.begin(), h_outer.begin() + Bout, h_inner.begin());
    int Bin = Bout;
    for (int inner = 0; inner < max_inner && Bin > 0 && total_cycles < o.max_cycles; ++inner) {
      ++total_cycles;
      const int Bact = Bin;
      CU(cudaMemcpyAsync(act, h_inner.data(), sizeof(int) * Bact, cudaMemcpyHostToDevice, s));
      gather_active(Bact, amu_act != nullptr);
      A.Bact = Bact;
      // restart length of this cycle: the work space holds (m+1) basis vectors of B
      // columns, so a shrunken active set runs a longer restart (up to kMaxRestart)
      const int mc = std::max(m, (int)std::min<long long>(px::kMaxRestart,
                                                          (long long)(m + 1) * B / Bact - 1));
      A.m = mc;
      const size_t esz = px::basis_bytes(A.basis);
      A.y = yv;
      A.u = yv + (size_t)mc * Bact;
      const int ldxa = (int)round_up(2 * (size_t)Bact, colpad);
      std::memset(h->h_active, 0xff, sizeof(int) * px::kMaxRestart);
      CU(cudaMemsetAsync(h->d_active, 0, sizeof(int) * px::kMaxRestart, s));
      if (lowp) CU(cudaMemsetAsync(X32, 0, sizeof(float) * (size_t)np * ldxa, s));
      else CU(cudaMemsetAsync(X64, 0, sizeof(double) * (size_t)np * ldxa, s));
      CU(px::launch_cycle_start(A, act, r, B, beta, target_all, lowp ? X32 : nullptr,
                                lowp ? nullptr : X64, ldxa, s, &nl));
      px::ShiftArgs sa{};
      sa.nu = nu; sa.N = N; sa.model = model; sa.Bact = Bact; sa.nblk = nblk; sa.basis = A.basis;
      sa.rowptr = d.rowptr; sa.col = d.col; sa.val64 = d.val64; sa.val32 = d.val32; sa.type = dip_type;
      sa.zq = zq_act_h; sa.zmu = zmu_act_h;
      sa.qtype = het ? d.type : nullptr; sa.ntypes = ntypes; sa.kappa = het ? kap_act : nullptr;
      sa.Y = lowp ? (const void*)Y32 : (const void*)Y64;
      sa.ldy = ldxa;
      sa.y_is_f32 = lowp;
      sa.jconv = jconv;
      sa.precond_mu = amu_act ? 1 : 0;
      // the tensor-core planes hold M = diag(Kbar, I) T, fp16 parts scaled by 2^e (the
      // epilogue undoes 2^12)
      sa.kbar_in_y = (tc && d.op_has_kbar) || d.bem ? 1 : 0;
      sa.yscale = tc_f16 && d.op_has_kbar ? std::ldexp(1.0f, 12 - d.op_scale_exp) : 1.0f;
      sa.W = W;
      // the tensor-core pair kernel's matvec Y = T X (split of X, then the kernel)
      auto tc_mf_matvec = [&](cudaStream_t q, long long* cnt) -> cudaError_t {
        cudaError_t e;
        if (model == PX_WFQFMU) {
          e = px::launch_split_xt_mu(X32, ldxa, np, ldxa, N, Xth, Xtl, tc_f16, q, cnt);
          if (e == cudaSuccess)
            e = px::launch_tc_mf4(d.pos4tc, np, N, d.mu_self, Xth, Xtl, ldxa, Y32, ldxa, tc_f16,
                                  d.op_scale_exp, h->d_err, q, cnt);
        } else {
          e = px::launch_split_xt(X32, ldxa, np, ldxa, Xth, Xtl, tc_f16, q, cnt);
          if (e == cudaSuccess)
            e = px::launch_tc_mf(d.pos4tc, np, d.tc_wmax, Xth, Xtl, ldxa, Y32, ldxa, tc_f16,
                                 d.op_scale_exp, h->d_err, q, cnt);
        }
        return e;
      };
      // one Krylov step: j >= 0 eagerly (host-side step index, per-step poll), or
      // j < 0 under capture (kernels read the step index from the device)
      auto enqueue_step = [&](int j, cudaStream_t q, long long* cnt) {
        const bool cap = j < 0;
        px::KrylovArgs Aj = A;
        Aj.jdev = cap ? h->d_jstep : nullptr;
        const int jj = cap ? 0 : j;
        // ---- block matvec Y = T X (the dominant kernel)
        cudaEvent_t e0v = nullptr, e1v = nullptr;
        if (o.profile && !cap) {
          e0v = pool_event(h, prof_k++);
          e1v = pool_event(h, prof_k++);
          CU(cudaEventRecord(e0v, q));
        }
        if (d.matfree && tc) {
          // tensor-core pair kernels: T tiles generated in shared memory as split planes
          CU(tc_mf_matvec(q, cnt));
        } else if (d.matfree && model == PX_WFQFMU) {
          if (lowp) CU(px::launch_sgemm_mf4(d.pos4f, d.rm2f, N, d.mu_self, X32, ldxa, Y32, ldxa, ldxa, q, cnt));
          else CU(px::launch_dgemm_mf4(d.pos4d, d.rm2d, N, d.mu_self, X64, ldxa, Y64, ldxa, ldxa, q, cnt));
        } else if (d.matfree) {
          if (lowp) CU(px::launch_sgemm_mf(d.pos4f, N, np, X32, ldxa, Y32, ldxa, ldxa, q, cnt));
          else CU(px::launch_dgemm_mf(d.pos4d, N, np, X64, ldxa, Y64, ldxa, ldxa, q, cnt));
        } else if (tc) {
          CU(px::launch_split_xt(X32, ldxa, np, ldxa, Xth, Xtl, tc_f16, q, cnt));
          int used = -1;
          CU(px::launch_tc_gemm(d.Thi, d.Tlo, np, Xth, Xtl, ldxa, Y32, ldxa, tc_f16, h->d_err, q,
                                cnt, o.gemm_tiles - 1, &used));
          if (st.gemm_tiles_used == 0) st.gemm_tiles_used = used + 1;
        } else if (lowp) {
          CU(px::launch_sgemm(d.T32, np, X32, ldxa, Y32, ldxa, ldxa, q, cnt));
        } else if (2 * Bact <= 8 && !d.bem) {   // the GEMV reads rows: symmetric T only
          CU(px::launch_dgemv(d.T64, np, X64, ldxa, Y64, ldxa, 2 * Bact, q, cnt));
        } else {
          CU(px::launch_dgemm_splitk(d.T64, np, X64, ldxa, Y64, ldxa, ldxa, dpart, dpart_elems, q,
                                     cnt));
        }
        if (o.profile && !cap) {
          CU(cudaEventRecord(e1v, q));
          mv_events.push_back({e0v, e1v});
        }
        // ---- conductance + shift: W = Kbar Y - z V_j
        px::ShiftArgs sj = sa;
        sj.jdev = Aj.jdev;
        sj.X = cap ? V : static_cast<const char*>(V) + (size_t)j * nu * Bact * esz;
        CU(px::launch_shift(sj, q, cnt));
        // ---- classical Gram-Schmidt, Givens, next basis vector
        for (int pass = 0; pass < passes; ++pass) {
          CU(px::launch_dots(Aj, jj, pass, q, cnt));
          CU(px::launch_update(Aj, jj, pass, pass == passes - 1, q, cnt));
        }
        CU(px::launch_givens(Aj, jj, passes, q, cnt));
        if (!cap)
          CU(cudaMemcpyAsync(h->h_active + j, h->d_active + j, sizeof(int), cudaMemcpyDeviceToHost, q));
        CU(px::launch_normalize(Aj, jj, lowp ? X32 : nullptr, lowp ? nullptr : X64, ldxa, q, cnt));
      };
      int jend = 0;
      if (use_graphs) {
        // the whole restart cycle is one graph launch: a device-side while loop runs
        // Krylov steps until every column stopped or the basis is full
        if (tc && !d.matfree && o.gemm_tiles == 0 && px::tc_tuned_variant(np, ldxa, tc_f16) < 0) {
          // tune the tensor-core tile shape on this cycle's operands before capture
          CU(px::launch_split_xt(X32, ldxa, np, ldxa, Xth, Xtl, tc_f16, s, &nl));
          CU(px::launch_tc_gemm(d.Thi, d.Tlo, np, Xth, Xtl, ldxa, Y32, ldxa, tc_f16, h->d_err, s,
                                &nl, -1, nullptr));
        }
        if (tc && d.matfree && px::tc_mf_tuned_width(np, ldxa, tc_f16, model == PX_WFQFMU) < 0) {
          // likewise the pair kernel's tile width
          CU(tc_mf_matvec(s, &nl));
        }
        uint32_t wmax_bits = 0;
        std::memcpy(&wmax_bits, &d.tc_wmax, sizeof(wmax_bits));
        const std::vector<uint64_t> key = {
            (uint64_t)Bact, (uint64_t)mc, (uint64_t)ldxa, (uint64_t)passes, (uint64_t)A.basis,
            (uint64_t)o.precision, (uint64_t)d.matfree, (uint64_t)o.gemm_tiles,
            (uint64_t)(uintptr_t)V, (uint64_t)(uintptr_t)W, (uint64_t)(uintptr_t)hh,
            (uint64_t)(uintptr_t)part, (uint64_t)(uintptr_t)Rm, (uint64_t)(uintptr_t)yv,
            (uint64_t)(uintptr_t)X32, (uint64_t)(uintptr_t)Y32, (uint64_t)(uintptr_t)X64,
            (uint64_t)(uintptr_t)Y64, (uint64_t)(uintptr_t)Xth, (uint64_t)(uintptr_t)zq_act,
            (uint64_t)(uintptr_t)zmu_act, (uint64_t)(uintptr_t)jconv, (uint64_t)(uintptr_t)normpart,
            (uint64_t)(uintptr_t)g, (uint64_t)(uintptr_t)cs, (uint64_t)(uintptr_t)sn,
            (uint64_t)(uintptr_t)target, (uint64_t)(uintptr_t)invh, (uint64_t)(uintptr_t)amu_act,
            (uint64_t)(uintptr_t)Xtl, (uint64_t)(uintptr_t)h->d_err,
            // the structure's operators: a graph stays valid for a new structure that
            // reuses the same buffers and sizes (it captured addresses, not contents)
            (uint64_t)model, (uint64_t)N, (uint64_t)nu, (uint64_t)np, (uint64_t)nblk,
            (uint64_t)(uintptr_t)d.T64, (uint64_t)(uintptr_t)d.T32, (uint64_t)(uintptr_t)d.Thi,
            (uint64_t)(uintptr_t)d.Tlo, (uint64_t)(uintptr_t)d.rowptr, (uint64_t)(uintptr_t)d.col,
            (uint64_t)(uintptr_t)d.val64, (uint64_t)(uintptr_t)d.val32, (uint64_t)(uintptr_t)d.type,
            (uint64_t)(uintptr_t)d.pos4f, (uint64_t)(uintptr_t)d.pos4d,
            (uint64_t)d.op_has_kbar, (uint64_t)(int64_t)d.op_scale_exp, (uint64_t)d.bem,
            (uint64_t)(uintptr_t)d.pos4tc, wmax_bits, (uint64_t)d.mu_self,
            (uint64_t)(uintptr_t)dpart, (uint64_t)dpart_elems};
        CycleGraph* cg = nullptr;
        for (size_t k = 0; k < h->graphs.size(); ++k) {
          if (h->graphs[k].key != key) continue;
          if (h->graphs[k].exec) {
            cg = &h->graphs[k];
          } else {   // left over from a capture that failed
            if (h->graphs[k].graph) cudaGraphDestroy(h->graphs[k].graph);
            h->graphs.erase(h->graphs.begin() + k);
          }
          break;
        }
        if (!cg) {
          if (h->graphs.size() >= kMaxCachedGraphs) drop_graphs(h);
          CycleGraph c;
          c.key = key;
          CU(cudaGraphCreate(&c.graph, 0));
          h->graphs.push_back(c);   // owned by the handle from here on (freed on error too)
          cg = &h->graphs.back();
          cudaGraphConditionalHandle loop;
          CU(cudaGraphConditionalHandleCreate(&loop, cg->graph, 1, cudaGraphCondAssignDefault));
          cudaGraphNodeParams cp = {};
          cp.type = cudaGraphNodeTypeConditional;
          cp.conditional.handle = loop;
          cp.conditional.type = cudaGraphCondTypeWhile;
          cp.conditional.size = 1;
          cudaGraphNode_t wn;
          CU(cudaGraphAddNode(&wn, cg->graph, nullptr, nullptr, 0, &cp));
          cudaGraph_t body = cp.conditional.phGraph_out[0];
          long long body_nl = 0;
          CU(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed));
          try {
            enqueue_step(-1, h->cap_stream, &body_nl);
            CU(px::launch_step_advance(h->d_jstep, h->d_active, mc, loop, h->cap_stream, &body_nl));
          } catch (...) {
            cudaGraph_t dummy = nullptr;
            cudaStreamEndCapture(h->cap_stream, &dummy);
            throw;
          }
          CU(cudaStreamEndCapture(h->cap_stream, &body));
          CU(cudaGraphInstantiate(&cg->exec, cg->graph, 0));
          cg->body_kernels = body_nl;
          st.graphs_built++;
        }
        CU(cudaMemsetAsync(h->d_jstep, 0, sizeof(int), s));
        CU(cudaGraphLaunch(cg->exec, s));
        CU(cudaMemcpyAsync(h->h_jstep, h->d_jstep, sizeof(int), cudaMemcpyDeviceToHost, s));
        sync_stream(h, s);
        jend = *h->h_jstep;
        if (jend < 1 || jend > mc) throw PxError{PX_ECUDA, "captured restart cycle ran no steps"};
        nl += cg->body_kernels * jend;
        st.graph_launches++;
      } else {
        for (int j = 0; j < mc; ++j) {
          enqueue_step(j, s, &nl);
          CU(cudaEventRecord(h->ev_iter[j & 1], s));
          jend = j + 1;
          // lagged poll: wait for step j-1 and stop once every column has stopped
          if (j >= 1) {
            wait_event(h, h->ev_iter[(j - 1) & 1]);
            if (reinterpret_cast<volatile int*>(h->h_active)[j - 1] == 0) break;
          }
        }
      }
      st.matvec_launches += jend;
      st.matvec_flops += 4.0 * (double)nu * nu * Bact * jend;
      st.matvec_bytes += ((double)nu * nu * (lowp ? 4.0 : 8.0) + 2.0 * nu * 2.0 * Bact * (lowp ? 4.0 : 8.0)) * jend;
      st.total_iters += jend;
      if (h->verbose)
        std::fprintf(stderr, "px: round %d inner %d columns %d steps %d (restart %d)\n", round, inner,
                     Bact, jend, mc);
      // x += V y, r = V u (inner residual), beta = |gamma|
      CU(px::launch_cycle_end(A, jend, act, x, r, B, beta, iters, s, &nl));
      CU(cudaMemcpyAsync(h_col.data(), colv, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, s));
      CU(cudaMemcpyAsync(h_iters.data(), iters, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
      sync_stream(h, s);
      int nb = 0;
      for (int k = 0; k < Bin; ++k) {
        const int c = h_inner[k];
        if (!std::isfinite(h_col[B + c])) throw PxError{PX_ECUDA, "non-finite inner residual"};
        if (h_col[B + c] > h_col[2 * (size_t)B + c] && h_iters[c] < o.max_iter) h_inner[nb++] = c;
      }
      Bin = nb;
    }

    // ---- FP64 true residual r = b - A x for the columns of this round
    const int Bact = Bout;
    const int ldxa = (int)round_up(2 * (size_t)Bact, colpad);
    CU(cudaMemcpyAsync(act, h_outer.data(), sizeof(int) * Bact, cudaMemcpyHostToDevice, s));
    gather_active(Bact, false);
    CU(cudaMemsetAsync(X64, 0, sizeof(double) * (size_t)np * ldxa, s));
    CU(px::launch_gather_x(x, B, act, Bact, nu, X64, ldxa, s, &nl));
    cudaEvent_t r0e = nullptr, r1e = nullptr;
    if (o.profile) {
      r0e = pool_event(h, prof_k++);
      r1e = pool_event(h, prof_k++);
      CU(cudaEventRecord(r0e, s));
    }
    if (d.matfree && model == PX_WFQFMU) {
      CU(px::launch_dgemm_mf4(d.pos4d, d.rm2d, N, d.mu_self, X64, ldxa, Y64, ldxa, ldxa, s, &nl));
    } else if (d.matfree && lowp) {
      // double-FP32 contraction of FP64 pair values; X32 / Y32 are free between cycles
      CU(px::launch_split_ff(X64, (size_t)np * ldxa, X32, Y32, s, &nl));
      CU(px::launch_ffgemm_mf(d.pos4d, N, np, X32, Y32, ldxa, Y64, ldxa, ldxa, s, &nl));
    } else if (d.matfree) {
      CU(px::launch_dgemm_mf(d.pos4d, N, np, X64, ldxa, Y64, ldxa, ldxa, s, &nl));
    } else if (2 * Bact <= 8 && !d.bem) {   // the GEMV reads rows: symmetric T only
      CU(px::launch_dgemv(d.T64, np, X64, ldxa, Y64, ldxa, 2 * Bact, s, &nl));
    } else if (d.Tffh) {
      // double-FP32 residual matvec; X32 / Y32 are free between cycles
      CU(px::launch_split_ff(X64, (size_t)np * ldxa, X32, Y32, s, &nl));
      CU(px::launch_ffgemm(d.Tffh, d.Tffl, np, X32, Y32, ldxa, Y64, ldxa, ldxa, s, &nl));
    } else {
      CU(px::launch_dgemm_splitk(d.T64, np, X64, ldxa, Y64, ldxa, ldxa, dpart, dpart_elems, s,
                                 &nl));
    }
    if (o.profile) {
      CU(cudaEventRecord(r1e, s));
      rs_events.push_back({r0e, r1e});
    }
    st.resid_launches++;
    st.resid_flops += 4.0 * (double)nu * nu * Bact;
    if (h->verbose) std::fprintf(stderr, "px: round %d true residual of %d columns\n", round, Bact);
    px::ResidArgs ra{};
    ra.nu = nu; ra.N = N; ra.model = model; ra.Bact = Bact; ra.P = P; ra.B = B; ra.nblk = nblk;
    ra.rowptr = d.rowptr; ra.col = d.col; ra.val64 = d.val64; ra.type = dip_type;
    ra.Y = Y64; ra.ldy = ldxa; ra.x = x; ra.act = act; ra.b = b; ra.zq = zq_act_h; ra.zmu = zmu_act_h;
    ra.R = r; ra.normpart = normpart;
    ra.qtype = het ? d.type : nullptr; ra.ntypes = ntypes; ra.kappa = het ? kap_act : nullptr;
    ra.bc = bc;
    ra.op_full = d.bem ? 1 : 0;
    CU(px::launch_resid(ra, s, &nl));
    // per-column norms: bn indexed as [c % B]
    CU(px::launch_norm_finish(normpart, nblk, Bact, act, B, bn, inner_tol, tol_abs_frac, rnorm,
                              beta, target_all, s, &nl));
    CU(cudaMemcpyAsync(h_col.data(), colv, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(h_iters.data(), iters, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
    sync_stream(h, s);
    int nb = 0;
    double worst = 0.0;
    for (int k = 0; k < Bout; ++k) {
      const int c = h_outer[k];
      if (!std::isfinite(h_col[c])) throw PxError{PX_ECUDA, "non-finite residual"};
      worst = std::max(worst, h_col[c] / h_bn[c]);
      if (h_col[c] > o.tol_rel * h_bn[c] && h_iters[c] < o.max_iter) h_outer[nb++] = c;
    }
    if (h->verbose)
      std::fprintf(stderr, "px: round %d true residual: max rel %.3e over %d columns, %d left\n",
                   round, worst, Bout, nb);
    Bout = nb;
  }
  st.cycles = total_cycles;

  // ---- observables (Sec. "Observables")
  CU(px::launch_observables(N, model, F, P, d.pos64, d.perm, x, e0, d_omega, d_pol, so->d_alpha, so->d_q,
                            so->d_mu, so->d_sigma_pol, so->d_sigma, have_triple ? pol_inv : nullptr,
                            d.bem ? d.tarea : nullptr, s, &nl));
  if (so->d_relres) CU(px::launch_relres(rnorm, bn, B, B, so->d_relres, s, &nl));
  std::vector<double> h_rnorm(B);
  int h_err = 0;
  CU(cudaMemcpyAsync(&h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(h_rnorm.data(), rnorm, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(h_iters.data(), iters, sizeof(int) * B, cudaMemcpyDeviceToHost, s));
  CU(cudaEventRecord(h->ev_b, s));
  wait_event(h, h->ev_b);
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, h->ev_a, h->ev_b));
  st.solve_ms = ms;
  for (auto& pr : mv_events) {
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, pr.first, pr.second));
    st.matvec_ms += t;
  }
  for (auto& pr : rs_events) {
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, pr.first, pr.second));
    st.resid_ms += t;
  }
  for (auto& pr : sk_events) {
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, pr.first, pr.second));
    st.shift_matvec_ms += t;
  }
  st.kernel_launches = nl;
  if (h_err) throw PxError{PX_ETIMEOUT, "a tensor-core pipeline wait ran out of time"};
  so->relres.resize(B);
  so->iters.resize(B);
  so->status.resize(B);
  px_status ret = PX_OK;
  for (int c = 0; c < B; ++c) {
    so->relres[c] = h_bn[c] > 0.0 ? h_rnorm[c] / h_bn[c] : 0.0;
    so->iters[c] = h_iters[c];
    so->status[c] = so->relres[c] <= o.tol_rel ? PX_OK : PX_ENOTCONV;
    if (so->status[c] != PX_OK) ret = PX_ENOTCONV;
  }
  if (ret != PX_OK) h->err = "some columns did not reach tol_rel; see status[]";
  return ret;
}

void default_options(px_options* o) {
  std::memset(o, 0, sizeof(*o));
  o->precision = PX_FP32;
  o->mode = PX_MODE_AUTO;
  o->restart_m = 0;
  o->max_iter = 20000;
  o->max_cycles = 200;
  o->max_refine = 20;
  o->gs_passes = 1;
  o->basis = PX_BASIS_AUTO;
  o->gemm_tiles = 0;
  o->cycle_graphs = 1;
  o->sort_atoms = 1;
  o->tol_rel = 1e-7;
  o->inner_tol = 1e-3;
  o->kcut_eps = 1e-6;
  o->mu_self_term = 0;
  o->profile = 0;
  o->hbm_budget_bytes = 0;
  o->device_wait_limit_s = 600.0;
  o->solver = PX_SOLVER_BATCHED;
  o->shift_krylov_max = 0;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

int px_abi_version(void) { return PX_ABI_VERSION; }

px_status px_options_default(px_options* opt) {
  if (!opt) return PX_EINVAL;
  default_options(opt);
  return PX_OK;
}

px_status px_create(px_handle** out, const px_options* opt) {
  if (!out) return fail(nullptr, PX_EINVAL, "NULL handle pointer");
  *out = nullptr;
  px_options o;
  if (opt) o = *opt;
  else default_options(&o);
  std::string msg;
  px_status vs = validate_options(&o, &msg);
  if (vs != PX_OK) return fail(nullptr, vs, msg);
  px_handle* h = new (std::nothrow) px_handle();
  if (!h) return fail(nullptr, PX_ENOMEM, "host allocation failed");
  h->opt = o;
  std::memset(&h->stats, 0, sizeof(h->stats));
  {
    const char* v = std::getenv("PX_VERBOSE");
    h->verbose = v && v[0] == '1';
  }
  try {
    CU(cudaGetDevice(&h->device));
    CU(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    CU(cudaEventCreate(&h->ev_a));
    CU(cudaEventCreate(&h->ev_b));
    CU(cudaEventCreateWithFlags(&h->ev_iter[0], cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&h->ev_iter[1], cudaEventDisableTiming));
    CU(cudaHostAlloc((void**)&h->h_active, sizeof(int) * (px::kMaxRestart + 1), cudaHostAllocDefault));
    CU(cudaMalloc((void**)&h->d_active, sizeof(int) * (px::kMaxRestart + 1)));
    h->h_jstep = h->h_active + px::kMaxRestart;
    h->d_jstep = h->d_active + px::kMaxRestart;
    CU(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    CU(cudaMalloc((void**)&h->d_err, sizeof(int)));
    CU(cudaEventCreate(&h->ev_sk[0]));
    CU(cudaEventCreate(&h->ev_sk[1]));
  } catch (const PxError& e) {
    g_create_error = e.msg;
    px_destroy(h);
    return e.st;
  }
  *out = h;
  return PX_OK;
}

px_status px_set_options(px_handle* h, const px_options* opt) {
  if (!h || !opt) return fail(h, PX_EINVAL, "NULL argument");
  std::string msg;
  px_status vs = validate_options(opt, &msg);
  if (vs != PX_OK) return fail(h, vs, msg);
  bool rebuild = h->have_structure && (opt->precision != h->opt.precision || opt->mode != h->opt.mode ||
                                       opt->kcut_eps != h->opt.kcut_eps ||
                                       opt->mu_self_term != h->opt.mu_self_term ||
                                       opt->sort_atoms != h->opt.sort_atoms);
  h->opt = *opt;
  if (rebuild) {
    h->have_structure = false;
    return fail(h, PX_EINVAL, "options that change the operators need px_set_structure again");
  }
  return PX_OK;
}

px_status px_set_structure(px_handle* h, px_model model, int n_atoms, const double* xyz_ang,
                           const int* type_idx, const px_atom_type* types, int n_types) {
  if (!h) return fail(nullptr, PX_EINVAL, "NULL handle");
  try {
    set_structure(h, (int)model, n_atoms, xyz_ang, type_idx, types, n_types);
  } catch (const PxError& e) {
    h->have_structure = false;
    return fail(h, e.st, e.msg);
  }
  return PX_OK;
}

px_status solve_host(px_handle* h, int n_freq, const double* omega_ev, const double* alpha_ib,
                     const double* eps, int n_pol, const double* pol_dir, double e0, px_result* out,
                     void* cuda_stream);

px_status px_solve(px_handle* h, int n_freq, const double* omega_ev, const double* alpha_ib,
                   int n_pol, const double* pol_dir, double e0, px_result* out,
                   void* cuda_stream) {
  return solve_host(h, n_freq, omega_ev, alpha_ib, nullptr, n_pol, pol_dir, e0, out, cuda_stream);
}

px_status px_set_mesh(px_handle* h, int n_tess, const double* pos_ang, const double* normals,
                      const double* area_ang2, double radius_ang, int formulation) {
  if (!h) return fail(nullptr, PX_EINVAL, "NULL handle");
  try {
    set_mesh(h, n_tess, pos_ang, normals, area_ang2, radius_ang, formulation);
  } catch (const PxError& e) {
    h->have_structure = false;
    return fail(h, e.st, e.msg);
  }
  return PX_OK;
}

px_status px_solve_bem(px_handle* h, int n_freq, const double* omega_ev, const double* eps,
                       int n_pol, const double* pol_dir, double e0, px_result* out,
                       void* cuda_stream) {
  if (!eps) return fail(h, PX_EINVAL, "NULL permittivities");
  return solve_host(h, n_freq, omega_ev, nullptr, eps, n_pol, pol_dir, e0, out, cuda_stream);
}

px_status solve_host(px_handle* h, int n_freq, const double* omega_ev, const double* alpha_ib,
                     const double* eps, int n_pol, const double* pol_dir, double e0, px_result* out,
                     void* cuda_stream) {
  if (!h) return fail(nullptr, PX_EINVAL, "NULL handle");
  if (!out) return fail(h, PX_EINVAL, "NULL result");
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
  try {
    if (!h->have_structure) throw PxError{PX_EINVAL, "no structure loaded"};
    if (n_freq < 1 || n_pol < 1) throw PxError{PX_EINVAL, "need n_freq >= 1 and n_pol >= 1"};
    const size_t F = n_freq, P = n_pol, N = h->ds.N, B = F * P;
    SolveOut so;
    double* obs = grow<double>(h->b_alpha, 2 * F * 3 * P + F * P + F + B);
    so.d_alpha = reinterpret_cast<double2*>(obs);
    so.d_sigma_pol = obs + 2 * F * 3 * P;
    so.d_sigma = so.d_sigma_pol + F * P;
    so.d_relres = so.d_sigma + F;
    if (out->q) so.d_q = grow<double2>(h->b_q, B * N);
    if (out->mu && h->ds.model == PX_WFQFMU) so.d_mu = grow<double2>(h->b_mu, B * N * 3);
    so.sigma_required = out->sigma_abs != nullptr;
    px_status r = PX_OK;
    SolveOut so1;
    const bool ief = h->ds.bem && h->ds.bem_stage == 1;
    if (ief) {
      // IEFPCM (Eq. 12): y from the shifted system of F, then q from (S A^-1) q = y
      so1 = so;
      so1.d_q = nullptr;
      so1.sigma_required = false;
      const px_status r1 = solve(h, n_freq, omega_ev, alpha_ib, n_pol, pol_dir, e0, &so1, s, eps);
      const px_stats st1 = h->stats;
      double2* y = grow<double2>(h->b_yief, (size_t)N * B);
      CU(cudaMemcpyAsync(y, h->b_x.as<double2>(), sizeof(double2) * N * B, cudaMemcpyDeviceToDevice, s));
      std::swap(h->ds, h->ds_g);
      try {
        r = solve(h, n_freq, omega_ev, alpha_ib, n_pol, pol_dir, e0, &so, s, eps, y);
      } catch (...) {
        std::swap(h->ds, h->ds_g);
        throw;
      }
      std::swap(h->ds, h->ds_g);
      px_stats& st = h->stats;
      st.solve_ms += st1.solve_ms;
      st.matvec_ms += st1.matvec_ms;
      st.matvec_launches += st1.matvec_launches;
      st.matvec_flops += st1.matvec_flops;
      st.matvec_bytes += st1.matvec_bytes;
      st.resid_ms += st1.resid_ms;
      st.resid_launches += st1.resid_launches;
      st.resid_flops += st1.resid_flops;
      st.kernel_launches += st1.kernel_launches;
      st.cycles += st1.cycles;
      st.total_iters += st1.total_iters;
      st.graph_launches += st1.graph_launches;
      st.graphs_built += st1.graphs_built;
      st.solver_used = st1.solver_used;
      st.shift_steps = st1.shift_steps;
      st.shift_matvec_launches = st1.shift_matvec_launches;
      st.shift_matvec_ms = st1.shift_matvec_ms;
      st.shift_matvec_bytes = st1.shift_matvec_bytes;
      st.shift_ms = st1.shift_ms;
      for (size_t c = 0; c < B; ++c) {
        so.relres[c] = std::max(so.relres[c], so1.relres[c]);
        so.iters[c] += so1.iters[c];
        if (so1.status[c] != PX_OK) so.status[c] = so1.status[c];
      }
      if (r1 != PX_OK && r == PX_OK) {
        r = r1;
        h->err = "some columns did not reach tol_rel; see status[]";
      }
    } else {
      r = solve(h, n_freq, omega_ev, alpha_ib, n_pol, pol_dir, e0, &so, s, eps);
    }
    if (out->alpha) CU(cudaMemcpyAsync(out->alpha, so.d_alpha, sizeof(double2) * F * 3 * P, cudaMemcpyDeviceToHost, s));
    if (out->sigma_abs_pol) CU(cudaMemcpyAsync(out->sigma_abs_pol, so.d_sigma_pol, sizeof(double) * F * P, cudaMemcpyDeviceToHost, s));
    if (out->sigma_abs && P == 3) CU(cudaMemcpyAsync(out->sigma_abs, so.d_sigma, sizeof(double) * F, cudaMemcpyDeviceToHost, s));
    if (out->rel_residual && !ief) CU(cudaMemcpyAsync(out->rel_residual, so.d_relres, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    if (so.d_q) CU(cudaMemcpyAsync(out->q, so.d_q, sizeof(double2) * B * N, cudaMemcpyDeviceToHost, s));
    if (so.d_mu) CU(cudaMemcpyAsync(out->mu, so.d_mu, sizeof(double2) * B * N * 3, cudaMemcpyDeviceToHost, s));
    sync_stream(h, s);
    for (size_t c = 0; c < B; ++c) {
      if (out->iters) out->iters[c] = so.iters[c];
      if (out->status) out->status[c] = so.status[c];
      if (out->rel_residual && ief) out->rel_residual[c] = so.relres[c];
    }
    return r == PX_OK ? PX_OK : fail(h, r, h->err);
  } catch (const PxError& e) {
    return fail(h, e.st, e.msg);
  }
}

px_status px_solve_device(px_handle* h, int n_freq, const double* omega_ev,
                          const double* alpha_ib, int n_pol, const double* pol_dir, double e0,
                          double* d_alpha, double* d_q, double* d_mu, double* d_relres,
                          void* cuda_stream) {
  if (!h) return fail(nullptr, PX_EINVAL, "NULL handle");
  cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
  try {
    if (!h->have_structure) throw PxError{PX_EINVAL, "no structure loaded"};
    if (n_freq < 1 || n_pol < 1) throw PxError{PX_EINVAL, "need n_freq >= 1 and n_pol >= 1"};
    SolveOut so;
    const size_t F = n_freq, P = n_pol;
    double* obs = grow<double>(h->b_alpha, 2 * F * 3 * P + F * P + F);
    so.d_alpha = d_alpha ? (double2*)d_alpha : reinterpret_cast<double2*>(obs);
    so.d_sigma_pol = obs + 2 * F * 3 * P;
    so.d_sigma = so.d_sigma_pol + F * P;
    so.d_q = (double2*)d_q;
    so.d_mu = h->ds.model == PX_WFQFMU ? (double2*)d_mu : nullptr;
    so.d_relres = d_relres;
    px_status r = solve(h, n_freq, omega_ev, alpha_ib, n_pol, pol_dir, e0, &so, s);
    sync_stream(h, s);
    return r == PX_OK ? PX_OK : fail(h, r, h->err);
  } catch (const PxError& e) {
    return fail(h, e.st, e.msg);
  }
}

px_status px_system_device(px_handle* h, int n_pol, const double* pol_dir, double e0, double* d_A0,
                           size_t ld_A0, double* d_b, void* cuda_stream) {
  if (!h) return fail(nullptr, PX_EINVAL, "NULL handle");
  try {
    if (!h->have_structure) throw PxError{PX_EINVAL, "no structure loaded"};
    const px::DevStructure& d = h->ds;
    if (d.hetero) throw PxError{PX_ENOTIMPL, "Eq. 9's conductance block depends on the frequency"};
    if (d.bem) throw PxError{PX_ENOTIMPL, "the mesh operator is not exported"};
    if (d.matfree || !d.T64) throw PxError{PX_EINVAL, "needs the materialised T (FP64)"};
    if (d_A0 && ld_A0 < (size_t)d.nu) throw PxError{PX_EINVAL, "ld_A0 must be >= n_u"};
    if (d_b && (n_pol < 1 || !pol_dir || !std::isfinite(e0) || !(e0 > 0.0)))
      throw PxError{PX_EINVAL, "need n_pol >= 1, pol_dir and a finite e0 > 0 for d_b"};
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
    long long nl = 0;
    // built in the library's internal (Morton) atom order, written in the caller's
    if (d_A0) {
      const size_t np2 = (size_t)d.np * d.np;
      CU(h->b_M64.ensure(np2 * sizeof(double) + 256));
      double* M64 = h->b_M64.as<double>();
      unsigned long long* d_amax = reinterpret_cast<unsigned long long*>(M64 + np2);
      CU(cudaMemsetAsync(d_amax, 0, sizeof(unsigned long long), s));
      CU(px::launch_build_M64(d, M64, d_amax, s, &nl));
      CU(px::launch_unpermute_system(M64, d.np, d.nu, d.N, d.perm, d_A0, ld_A0, nullptr, 0, nullptr,
                                     s, &nl));
    }
    if (d_b) {
      double* dp = grow<double>(h->b_pol, 3 * (size_t)n_pol);
      double* bi = grow<double>(h->b_b, (size_t)d.nu * n_pol);
      CU(cudaMemcpyAsync(dp, pol_dir, sizeof(double) * 3 * n_pol, cudaMemcpyHostToDevice, s));
      CU(px::launch_rhs(d.nu, d.N, d.model, d.rowptr, d.col, d.val64, d.pos64, dp, n_pol, e0, bi, s,
                        &nl));
      CU(px::launch_unpermute_system(nullptr, d.np, d.nu, d.N, d.perm, nullptr, 0, bi, n_pol, d_b, s,
                                     &nl));
    }
    sync_stream(h, s);
    h->b_M64.release();
  } catch (const PxError& e) {
    return fail(h, e.st, e.msg);
  }
  return PX_OK;
}

px_status px_get_stats(const px_handle* h, px_stats* st) {
  if (!h || !st) return PX_EINVAL;
  *st = h->stats;
  return PX_OK;
}

px_status px_destroy(px_handle* h) {
  if (!h) return PX_OK;
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  free_all(h);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->ev_a) cudaEventDestroy(h->ev_a);
  if (h->ev_b) cudaEventDestroy(h->ev_b);
  for (cudaEvent_t e : h->ev_iter)
    if (e) cudaEventDestroy(e);
  if (h->h_active) cudaFreeHost(h->h_active);
  if (h->h_skact) cudaFreeHost(h->h_skact);
  for (cudaEvent_t e : h->ev_sk)
    if (e) cudaEventDestroy(e);
  if (h->d_active) cudaFree(h->d_active);
  if (h->d_err) cudaFree(h->d_err);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
  return PX_OK;
}

const char* px_last_error(const px_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------- accessors (px_handle.cuh)
const px::DevStructure* px_structure(const px_handle* h) {
  return (h && h->have_structure) ? &h->ds : nullptr;
}
cudaStream_t px_stream(const px_handle* h) { return h->own_stream; }
double px_drude_n(const px_handle* h) { return h->drude_n; }
double px_tau(const px_handle* h) { return h->tau; }
void px_set_error(px_handle* h, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
}
