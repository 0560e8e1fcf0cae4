// Continuous-batching request loop (include/px_serve.h).
//
// Host-side scheduling only: every solve runs through px_set_structure / px_solve on
// the slot's own handle and stream.  Admission keeps the sum of the admitted requests'
// device footprints (and of the memory idle slots still hold) inside the budget.
#include "px_serve.h"
#include "px_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

struct Req {
  uint64_t id = 0;
  int model = 0, N = 0, ntypes = 0, F = 0, P = 0, mode = PX_MODE_MATERIALISED;
  double e0 = 1.0;
  std::vector<double> xyz, omega, aib, pol;
  std::vector<int> tidx;
  std::vector<px_atom_type> types;
  uint64_t key = 0;
  size_t footprint = 0;
  // results
  std::vector<double> alpha, sigma, sigma_pol, q, mu, relres;
  std::vector<int> iters, status;
  px_status st = PX_OK;
  int state = 0;   // 0 queued, 1 running, 2 done
  double t_submit = 0, t_start = 0, t_done = 0;
  // requests solved with this one as extra columns of its block (this one leads)
  std::vector<Req*> group;
};

struct Slot {
  px_handle* h = nullptr;
  uint64_t key = 0;      // structure whose operators the handle holds (0 = none)
  int mode = -1;
  size_t retained = 0;   // estimate of the device memory the handle keeps
  Req* req = nullptr;
  bool stop = false;
  std::condition_variable cv;
  std::thread th;
};

uint64_t fnv1a(uint64_t hsh, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    hsh ^= b[i];
    hsh *= 1099511628211ull;
  }
  return hsh;
}

size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

// Device bytes a solve of this request needs on a fresh handle (operators + Krylov
// work space), for materialised (mat) or on-the-fly operators.
size_t footprint(const px_options& o, int model, int N, int B, bool mat) {
  const size_t nu = model == PX_WFQ ? N : 4 * (size_t)N;   // wFQFmu and its heterogeneous form
  const size_t np = round_up(nu, 128);
  const size_t ldx = round_up(2 * (size_t)B, 256);
  const size_t m = o.restart_m > 0 ? o.restart_m
                                   : (model == PX_WFQ && o.precision != PX_FP64 ? 60 : 100);
  size_t t = 0;
  if (mat) {
    t += np * np * 8;
    if (o.precision != PX_FP64) t += np * np * 8;   // double-FP32 planes of T
    if (o.precision == PX_FP32) t += np * np * 4;
    // split planes, plus the FP64 M = diag(Kbar, I) T they are cut from (transient)
    if (o.precision == PX_BF16SPLIT || o.precision == PX_FP16SPLIT) t += np * np * (4 + 8);
  }
  const size_t esz = px::basis_bytes(px::basis_kind(o.precision, o.basis));
  t += (m + 1) * nu * B * esz;         // Krylov basis
  t += nu * B * esz + 2 * nu * B * 16; // W, x, r
  t += np * ldx * (8 + 8 + 4 + 4 + 4); // X64, Y64, X32, Y32, split operand
  t += 2 * (m + 1) * B * 16 * 4;       // projections, Hessenberg, partials (bound)
  t += (size_t)128 * (m + 1) * B * 16; // partial projections
  t += 64 << 20;                       // CSR, small arrays, slack
  if (o.solver == PX_SOLVER_SHIFTED && model == PX_WFQ && mat) {
    // shifted Krylov work space with the server's basis limit: double-FP32 planes of T
    // (FP64 handles), basis and products T V, the per-system rotated triangular factors
    const size_t ms = std::min<size_t>(nu, (size_t)o.shift_krylov_max);
    if (o.precision == PX_FP64) t += np * np * 8;
    t += 2 * (ms + 1) * nu * 4 * 8;                  // V, U (up to 4 directions)
    t += (size_t)B * (ms * (ms + 1) / 2) * 16;       // R
    t += ms * (ms + 2) * 4 * 8 + 5 * ms * (size_t)B * 16;   // Hessenberg, rotations, y
  }
  return t;
}

}  // namespace

struct px_server {
  px_options opt;
  int max_slots = 1;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_done;
  std::deque<Req*> queue;
  std::map<uint64_t, Req*> reqs;
  std::vector<Slot*> slots;
  uint64_t next_id = 1;
  size_t peak_reserved = 0;
  long long submitted = 0, completed = 0, failed = 0, reuses = 0, merged = 0;
  double points = 0.0;
  std::vector<double> latencies_ms;
  Clock::time_point t0 = Clock::now();
  int device = 0;
  bool stopping = false;
};

namespace {

// Largest block one merged solve takes: frequencies, and complex per-atom results
// (frequencies x directions x unknowns) held on the host while the solve runs.
constexpr int kMergeMaxFreq = 512;
constexpr size_t kMergeMaxEntries = size_t(1) << 26;

// Queued requests that can join r's solve as extra columns: the same structure, operator
// mode and model (so the same T, CSR and shifts' form), the same field directions and E0
// (so the same right-hand sides); their frequency lists are appended to r's.  The
// group's footprint must still fit beside the other slots (lock held).
void gather_group(px_server* s, Req* r, const Slot* pick) {
  size_t others = 0;
  for (const Slot* o : s->slots)
    if (o != pick) others += std::max(o->retained, o->req ? o->req->footprint : 0);
  int F = r->F;
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    Req* q = *it;
    const bool same = q != r && q->key == r->key && q->mode == r->mode && q->model == r->model &&
                      q->P == r->P && q->e0 == r->e0 && q->ntypes == r->ntypes &&
                      q->pol == r->pol && F + q->F <= kMergeMaxFreq &&
                      (size_t)(F + q->F) * r->P * (r->model == PX_WFQ ? 1 : 4) * r->N <= kMergeMaxEntries;
    if (!same) {
      ++it;
      continue;
    }
    const size_t fp = footprint(s->opt, r->model, r->N, (F + q->F) * r->P,
                                r->mode == PX_MODE_MATERIALISED);
    if (others + std::max(pick->retained, fp) > s->budget) break;
    F += q->F;
    r->footprint = std::max(r->footprint, fp);
    q->state = 1;
    q->t_start = r->t_start;
    r->group.push_back(q);
    ++s->merged;
    it = s->queue.erase(it);
  }
}

size_t reserved_bytes(const px_server* s) {
  size_t t = 0;
  for (const Slot* sl : s->slots) t += std::max(sl->retained, sl->req ? sl->req->footprint : 0);
  return t;
}

// Assign queued requests to free slots (lock held).  Arrival order, except that a
// request that does not fit may be passed by later ones while the head has waited
// less than 2 s.
void admit(px_server* s) {
  const double now = seconds_since(s->t0);
  // structure affinity: a free slot first takes a queued request (among the first 16)
  // for the structure it already holds, keeping its operators on the device
  for (Slot* sl : s->slots) {
    if (sl->req || !sl->h || sl->key == 0) continue;
    int look = 0;
    for (auto it = s->queue.begin(); it != s->queue.end() && look < 16; ++it, ++look) {
      Req* r = *it;
      if (r->key != sl->key || r->mode != sl->mode) continue;
      size_t others = 0;
      for (const Slot* o : s->slots)
        if (o != sl) others += std::max(o->retained, o->req ? o->req->footprint : 0);
      if (others + std::max(sl->retained, r->footprint) > s->budget) break;
      ++s->reuses;
      sl->req = r;
      r->state = 1;
      r->t_start = now;
      s->queue.erase(it);
      gather_group(s, r, sl);
      s->peak_reserved = std::max(s->peak_reserved, reserved_bytes(s));
      sl->cv.notify_one();
      break;
    }
  }
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    Req* r = *it;
    // free slot, preferring one that already holds this structure
    Slot* pick = nullptr;
    for (Slot* sl : s->slots)
      if (!sl->req && sl->key == r->key && sl->mode == r->mode) { pick = sl; break; }
    if (!pick)
      for (Slot* sl : s->slots)
        if (!sl->req && (!pick || sl->retained < pick->retained)) pick = sl;
    if (!pick) return;
    auto fits = [&]() {
      size_t others = 0;
      for (const Slot* sl : s->slots)
        if (sl != pick) others += std::max(sl->retained, sl->req ? sl->req->footprint : 0);
      return others + std::max(pick->retained, r->footprint) <= s->budget;
    };
    if (!fits()) {
      // release the memory idle slots still hold, then retry once
      for (Slot* sl : s->slots)
        if (!sl->req && sl != pick && sl->h) {
          px_destroy(sl->h);
          sl->h = nullptr;
          sl->key = 0;
          sl->retained = 0;
        }
    }
    if (!fits()) {
      if (it == s->queue.begin() && now - r->t_submit > 2.0) return;   // hold for the head
      ++it;
      continue;
    }
    if (pick->key == r->key && pick->mode == r->mode) ++s->reuses;
    pick->req = r;
    r->state = 1;
    r->t_start = now;
    s->queue.erase(it);
    gather_group(s, r, pick);
    s->peak_reserved = std::max(s->peak_reserved, reserved_bytes(s));
    pick->cv.notify_one();
    // erasing invalidated the iterators: continue from the front (earlier entries that
    // did not fit are checked again, as the next admission pass would)
    it = s->queue.begin();
  }
}

// One solve for a request and the requests merged into it: the frequency lists (and the
// alpha_ib rows, [n_types][F]) are concatenated, the results split back per request
// (every result array is frequency-major).  Each request's status is its own columns'.
px_status solve_group(px_handle* h, Req* r) {
  std::vector<Req*> all{r};
  all.insert(all.end(), r->group.begin(), r->group.end());
  int F = 0;
  for (const Req* q : all) F += q->F;
  const size_t P = r->P, N = r->N, nt = r->ntypes, B = (size_t)F * P;
  std::vector<double> omega, aib;
  for (const Req* q : all) omega.insert(omega.end(), q->omega.begin(), q->omega.end());
  if (!r->aib.empty()) {
    aib.reserve(2 * nt * F);
    for (size_t t = 0; t < nt; ++t)
      for (const Req* q : all)
        aib.insert(aib.end(), q->aib.begin() + 2 * t * q->F, q->aib.begin() + 2 * (t + 1) * q->F);
  }
  std::vector<double> alpha(2 * B * 3), sigma(F), sigma_pol(B), qv(2 * B * N), mu, relres(B);
  if (!r->mu.empty()) mu.resize(6 * B * N);
  std::vector<int> iters(B), status(B);
  px_result res;
  res.alpha = alpha.data();
  res.sigma_abs = sigma.data();
  res.sigma_abs_pol = sigma_pol.data();
  res.q = qv.data();
  res.mu = mu.empty() ? nullptr : mu.data();
  res.rel_residual = relres.data();
  res.iters = iters.data();
  res.status = status.data();
  const px_status st = px_solve(h, F, omega.data(), aib.empty() ? nullptr : aib.data(), (int)P,
                                r->pol.data(), r->e0, &res, nullptr);
  if (st != PX_OK && st != PX_ENOTCONV) return st;
  size_t f0 = 0;
  for (Req* q : all) {
    const size_t Fq = q->F, Bq = Fq * P, b0 = f0 * P;
    std::copy(alpha.begin() + 2 * 3 * b0, alpha.begin() + 2 * 3 * (b0 + Bq), q->alpha.begin());
    std::copy(sigma.begin() + f0, sigma.begin() + f0 + Fq, q->sigma.begin());
    std::copy(sigma_pol.begin() + b0, sigma_pol.begin() + b0 + Bq, q->sigma_pol.begin());
    std::copy(qv.begin() + 2 * N * b0, qv.begin() + 2 * N * (b0 + Bq), q->q.begin());
    if (!mu.empty())
      std::copy(mu.begin() + 6 * N * b0, mu.begin() + 6 * N * (b0 + Bq), q->mu.begin());
    std::copy(relres.begin() + b0, relres.begin() + b0 + Bq, q->relres.begin());
    std::copy(iters.begin() + b0, iters.begin() + b0 + Bq, q->iters.begin());
    std::copy(status.begin() + b0, status.begin() + b0 + Bq, q->status.begin());
    q->st = PX_OK;
    for (size_t c = 0; c < Bq; ++c)
      if (q->status[c] != PX_OK) q->st = PX_ENOTCONV;
    f0 += Fq;
  }
  return r->st;
}

void slot_main(px_server* s, Slot* sl) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    sl->cv.wait(lk, [&] { return sl->req != nullptr || sl->stop; });
    if (!sl->req) break;
    Req* r = sl->req;
    const bool reuse = sl->h && sl->key == r->key && sl->mode == r->mode;
    lk.unlock();
    px_status st = PX_OK;
    if (!sl->h) st = px_create(&sl->h, &s->opt);
    if (st == PX_OK && !reuse) {
      px_options o = s->opt;
      o.mode = r->mode;
      st = px_set_options(sl->h, &o);
      if (st == PX_OK || st == PX_EINVAL)
        st = px_set_structure(sl->h, (px_model)r->model, r->N, r->xyz.data(), r->tidx.data(),
                              r->types.data(), r->ntypes);
    }
    if (st == PX_OK && r->group.empty()) {
      px_result res;
      res.alpha = r->alpha.data();
      res.sigma_abs = r->sigma.data();
      res.sigma_abs_pol = r->sigma_pol.data();
      res.q = r->q.data();
      res.mu = r->mu.empty() ? nullptr : r->mu.data();
      res.rel_residual = r->relres.data();
      res.iters = r->iters.data();
      res.status = r->status.data();
      st = px_solve(sl->h, r->F, r->omega.data(), r->aib.empty() ? nullptr : r->aib.data(), r->P,
                    r->pol.data(), r->e0, &res, nullptr);
    } else if (st == PX_OK) {
      st = solve_group(sl->h, r);
    }
    lk.lock();
    r->st = st;
    r->state = 2;
    r->t_done = seconds_since(s->t0);
    for (Req* q : r->group) {
      q->state = 2;
      q->t_done = r->t_done;
      if (st == PX_OK || st == PX_ENOTCONV) {
        ++s->completed;
        for (int c : q->status) s->points += (c == PX_OK) ? 1.0 : 0.0;
      } else {
        q->st = st;
        ++s->failed;
      }
      s->latencies_ms.push_back((q->t_done - q->t_submit) * 1e3);
    }
    r->group.clear();
    if (st == PX_OK || st == PX_ENOTCONV) {
      sl->key = r->key;
      sl->mode = r->mode;
      sl->retained = std::max(sl->retained, r->footprint);
      ++s->completed;
      for (int c : r->status) s->points += (c == PX_OK) ? 1.0 : 0.0;
    } else {
      ++s->failed;
      if (sl->h) px_destroy(sl->h);
      sl->h = nullptr;
      sl->key = 0;
      sl->retained = 0;
    }
    s->latencies_ms.push_back((r->t_done - r->t_submit) * 1e3);
    sl->req = nullptr;
    admit(s);
    s->cv_done.notify_all();
  }
  if (sl->h) px_destroy(sl->h);
  sl->h = nullptr;
}

px_status copy_out(const Req* r, px_result* out) {
  if (!out) return r->st;
  const size_t F = r->F, P = r->P, N = r->N;
  auto cp = [](double* dst, const std::vector<double>& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(double));
  };
  cp(out->alpha, r->alpha);
  if (out->sigma_abs && P == 3) cp(out->sigma_abs, r->sigma);
  cp(out->sigma_abs_pol, r->sigma_pol);
  cp(out->q, r->q);
  if (out->mu && r->model != PX_WFQ) cp(out->mu, r->mu);
  cp(out->rel_residual, r->relres);
  if (out->iters) std::memcpy(out->iters, r->iters.data(), F * P * sizeof(int));
  if (out->status) std::memcpy(out->status, r->status.data(), F * P * sizeof(int));
  (void)N;
  return r->st;
}

}  // namespace

extern "C" {

px_status px_server_create(px_server** out, const px_options* opt, int max_slots,
                           size_t hbm_budget_bytes) {
  if (!out || max_slots < 1 || max_slots > 32) return PX_EINVAL;
  *out = nullptr;
  px_server* s = new (std::nothrow) px_server();
  if (!s) return PX_ENOMEM;
  if (opt) s->opt = *opt;
  else px_options_default(&s->opt);

  // the shifted solver's basis limit is fixed for served requests, so that admission can
  // account for its work space (a handle alone sizes it from the free memory)
  if (s->opt.solver == PX_SOLVER_SHIFTED && s->opt.shift_krylov_max == 0) s->opt.shift_krylov_max = 1500;
  s->max_slots = max_slots;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return PX_ECUDA;
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    delete s;
    return PX_ECUDA;
  }
  s->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)fr);
  // every slot shares the server's budget, which admission already enforces: a slot's
  // handle checks its operators against the whole budget, not against the memory that
  // happens to be free beside the other slots
  s->opt.hbm_budget_bytes = s->budget;
  for (int i = 0; i < max_slots; ++i) {
    Slot* sl = new Slot();
    s->slots.push_back(sl);
    sl->th = std::thread(slot_main, s, sl);
  }
  *out = s;
  return PX_OK;
}

px_status px_submit(px_server* s, const px_request* r, uint64_t* req_id) {
  if (!s || !r || !req_id) return PX_EINVAL;
  if (r->model != PX_WFQ && r->model != PX_WFQFMU && r->model != PX_WFQFMU_HETERO) return PX_EINVAL;
  if (r->n_atoms < 1 || r->n_types < 1 || r->n_freq < 1 || r->n_pol < 1) return PX_EINVAL;
  if (!r->xyz_ang || !r->type_idx || !r->types || !r->omega_ev || !r->pol_dir) return PX_EINVAL;
  if (r->model != PX_WFQ && !r->alpha_ib) return PX_EINVAL;
  Req* q = new (std::nothrow) Req();
  if (!q) return PX_ENOMEM;
  q->model = r->model;
  q->N = r->n_atoms;
  q->ntypes = r->n_types;
  q->F = r->n_freq;
  q->P = r->n_pol;
  q->e0 = r->e0;
  q->xyz.assign(r->xyz_ang, r->xyz_ang + 3 * (size_t)r->n_atoms);
  q->tidx.assign(r->type_idx, r->type_idx + r->n_atoms);
  q->types.assign(r->types, r->types + r->n_types);
  q->omega.assign(r->omega_ev, r->omega_ev + r->n_freq);
  q->pol.assign(r->pol_dir, r->pol_dir + 3 * (size_t)r->n_pol);
  if (r->model != PX_WFQ) q->aib.assign(r->alpha_ib, r->alpha_ib + 2 * (size_t)r->n_types * r->n_freq);
  const size_t B = (size_t)q->F * q->P, N = q->N;
  // materialised operators when they fit a share of the budget, else on the fly
  const size_t fmat = footprint(s->opt, q->model, q->N, (int)B, true);
  const size_t ffree = footprint(s->opt, q->model, q->N, (int)B, false);
  // (on the fly: every precision for wFQ and wFQFmu, FP32 / FP64 for its heterogeneous form)
  const bool split = s->opt.precision == PX_BF16SPLIT || s->opt.precision == PX_FP16SPLIT;
  if (s->opt.mode == PX_MODE_MATFREE || (s->opt.mode == PX_MODE_AUTO && fmat > s->budget / 2 &&
                                         (q->model != PX_WFQFMU_HETERO || !split))) {
    q->mode = PX_MODE_MATFREE;
    q->footprint = ffree;
  } else {
    q->mode = PX_MODE_MATERIALISED;
    q->footprint = fmat;
  }
  if (q->footprint > s->budget) {
    delete q;
    return PX_ENOMEM;
  }
  uint64_t k = 1469598103934665603ull;
  k = fnv1a(k, &q->model, sizeof(int));
  k = fnv1a(k, &q->mode, sizeof(int));
  k = fnv1a(k, q->xyz.data(), q->xyz.size() * sizeof(double));
  k = fnv1a(k, q->tidx.data(), q->tidx.size() * sizeof(int));
  k = fnv1a(k, q->types.data(), q->types.size() * sizeof(px_atom_type));
  q->key = k ? k : 1;
  q->alpha.resize(2 * (size_t)q->F * 3 * q->P);
  q->sigma.resize(q->F);
  q->sigma_pol.resize(B);
  q->q.resize(2 * B * N);
  if (q->model != PX_WFQ) q->mu.resize(6 * B * N);
  q->relres.resize(B);
  q->iters.resize(B);
  q->status.resize(B);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->queue.size() >= 100000) {
    delete q;
    return PX_EBUSY;
  }
  q->id = s->next_id++;
  q->t_submit = seconds_since(s->t0);
  s->reqs[q->id] = q;
  s->queue.push_back(q);
  ++s->submitted;
  *req_id = q->id;
  admit(s);
  return PX_OK;
}

px_status px_poll(px_server* s, uint64_t req_id, px_result* out, int* done) {
  if (!s || !done) return PX_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return PX_ENOTFOUND;
  Req* r = it->second;
  if (r->state != 2) {
    *done = 0;
    return PX_OK;
  }
  *done = 1;
  px_status st = copy_out(r, out);
  s->reqs.erase(it);
  delete r;
  return st;
}

px_status px_wait(px_server* s, uint64_t req_id, px_result* out, double timeout_s) {
  if (!s) return PX_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return PX_ENOTFOUND;
  Req* r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration<double>(std::max(0.0, timeout_s));
  if (!s->cv_done.wait_until(lk, deadline, [&] { return r->state == 2; })) return PX_ETIMEOUT;
  px_status st = copy_out(r, out);
  s->reqs.erase(req_id);
  delete r;
  return st;
}

px_status px_server_get_stats(px_server* s, px_server_stats* st) {
  if (!s || !st) return PX_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->queued = (long long)s->queue.size();
  for (const Slot* sl : s->slots) st->running += sl->req ? 1 : 0;
  std::vector<double> l = s->latencies_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
      size_t i = (size_t)std::ceil(p * l.size()) - 1;
      return l[std::min(i, l.size() - 1)];
    };
    st->p50_latency_ms = pct(0.50);
    st->p99_latency_ms = pct(0.99);
    st->max_latency_ms = l.back();
  }
  st->busy_points = s->points;
  st->wall_s = seconds_since(s->t0);
  st->structure_reuses = s->reuses;
  st->peak_reserved_bytes = s->peak_reserved;
  st->merged_requests = s->merged;
  return PX_OK;
}

px_status px_server_destroy(px_server* s) {
  if (!s) return PX_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->stopping = true;
    for (Req* r : s->queue) {
      s->reqs.erase(r->id);
      delete r;
    }
    s->queue.clear();
    s->cv_done.wait(lk, [&] {
      for (const Slot* sl : s->slots)
        if (sl->req) return false;
      return true;
    });
    for (Slot* sl : s->slots) {
      sl->stop = true;
      sl->cv.notify_one();
    }
  }
  for (Slot* sl : s->slots) {
    if (sl->th.joinable()) sl->th.join();
    delete sl;
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return PX_OK;
}

}  // extern "C"
