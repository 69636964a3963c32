// Request server (hgks_server_*): continuous batching of steady solves.
//
// Requests (a mesh, its parameters, an initial state, a drop tolerance and a
// step limit) are submitted at any time. A host thread builds each mesh's
// stencils and reconstruction matrices in submission order while the GPU
// works. Every call to hgks_server_step() is one scheduling round: requests
// whose build is done are admitted in submission order while the batch arena
// has a free slot and free cell and face ranges for them (the arena is sized
// from the HBM budget, so this is admission by device-memory footprint); then
// every running solve takes one step of Algorithm 1 together (one launch per
// phase, replayed from a CUDA graph), with its convergence test on the device;
// solves that converged or hit their step limit leave, their state is copied
// out and their ranges are freed for the next admissions.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>
#include "batch_impl.h"

using namespace hgks;

namespace {

enum { Q_WAIT = 0, Q_BUILT = 1, Q_RUN = 2, Q_DONE = 3, Q_FAIL = 4 };

struct Request {
  int64_t id = 0;
  std::vector<double> xyz, pshift;
  std::vector<int64_t> tet, bface;     // cells [n][nvc] and boundary faces
  int32_t nvc = 4;                     // vertices per cell: 4 tetrahedra, 8 hexahedra
  std::vector<int32_t> btag;
  int32_t nps = 0;
  hgks_params p{};
  double drop = 0.0;
  int max_steps = 0;
  std::vector<double> Q0, G0;          // caller order [n][5], [n][15]
  HostMesh hm;
  std::vector<int64_t> perm;           // internal -> caller
  std::string err;
  hgks_status status = HGKS_OK;
  int state = Q_WAIT;
  int slot = -1;
  bool cancel = false;                 // set by hgks_server_cancel while building, admitting or running
  bool admitting = false;              // at the head of `built`, being placed by the round's thread
  std::vector<double> Q, G;            // result, caller order
  hgks_solve_info info{};
  double t_submit = 0, t_built = 0, t_admit = 0, t_done = 0;
};

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct hgks_server_s {
  Batch *B = nullptr;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request *> to_build;
  int building = 0;                     // taken off to_build by the builder, not yet back (still waiting)
  std::deque<Request *> built;          // built, waiting for admission (submission order)
  std::map<int64_t, std::unique_ptr<Request>> all;
  std::vector<Request *> running;       // by slot
  std::thread builder;
  bool stop = false;
  int64_t next_id = 1;
  int use_graph = 1;
};

namespace {

void builder_loop(hgks_server_s *S) {
  const int mask = S->B->p0.scheme == HGKS_WENO ? 1 : 2;
  for (;;) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !S->to_build.empty(); });
      if (S->stop) return;
      r = S->to_build.front();
      S->to_build.pop_front();
      S->building++;
    }
    std::string err;
    hgks_status st;
    try {
      st = build_host_mesh(r->xyz.data(), (int64_t)r->xyz.size() / 3, r->tet.data(), r->nvc,
                           (int64_t)r->tet.size() / r->nvc,
                           r->bface.empty() ? nullptr : r->bface.data(), r->btag.empty() ? nullptr : r->btag.data(),
                           (int64_t)r->btag.size(), r->pshift.empty() ? nullptr : r->pshift.data(), r->nps, mask, r->hm,
                           err);
    } catch (const std::exception &e) {     // host memory exhausted while building: the request fails
      st = HGKS_ERR_OOM;
      err = std::string("mesh build: ") + e.what();
      r->hm = HostMesh{};
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->building--;
    r->t_built = now_s(S->t0);
    if (r->cancel) {
      r->status = HGKS_ERR_CANCELLED;
      r->state = Q_DONE;
      r->t_done = r->t_built;
      r->hm = HostMesh{};
    } else if (st) {
      r->status = st;
      r->err = err;
      r->state = Q_FAIL;
      r->t_done = r->t_built;
    } else {
      r->perm = r->hm.perm;
      r->xyz.clear(); r->xyz.shrink_to_fit();
      r->tet.clear(); r->tet.shrink_to_fit();
      r->state = Q_BUILT;
      S->built.push_back(r);
    }
  }
}

// caller order [n][k] -> internal component-major [k][n]
std::vector<double> to_internal(const std::vector<double> &a, const std::vector<int64_t> &perm, int k) {
  const size_t n = perm.size();
  std::vector<double> out((size_t)k * n);
  for (size_t i = 0; i < n; i++)
    for (int c = 0; c < k; c++) out[(size_t)c * n + i] = a[(size_t)perm[i] * k + c];
  return out;
}
void to_caller(const std::vector<double> &in, const std::vector<int64_t> &perm, int k, std::vector<double> &out) {
  const size_t n = perm.size();
  out.assign((size_t)k * n, 0.0);
  for (size_t i = 0; i < n; i++)
    for (int c = 0; c < k; c++) out[(size_t)perm[i] * k + c] = in[(size_t)c * n + i];
}

// admit built requests in submission order while the arena has room. The head
// request is marked `admitting` while it is placed outside the lock: a concurrent
// hgks_server_cancel then only flags it (it stays at the head of `built`, and its
// mesh and state stay valid) and this function finishes the cancellation.
hgks_status admit(hgks_server_s &S, bool &changed) {
  Batch &B = *S.B;
  // under S.mu: take the head request off `built` as cancelled
  auto cancel_head = [&](Request *r) {
    S.built.pop_front();
    r->admitting = false;
    r->hm = HostMesh{};
    r->status = HGKS_ERR_CANCELLED;
    r->state = Q_DONE;
    r->t_done = now_s(S.t0);
  };
  auto stop_admitting = [&](Request *r) {
    std::lock_guard<std::mutex> lk(S.mu);
    r->admitting = false;
  };
  for (;;) {
    Request *r = nullptr;
    {
      std::lock_guard<std::mutex> lk(S.mu);
      if (S.built.empty()) return HGKS_OK;
      r = S.built.front();
      if (r->cancel) {                     // flagged during an earlier attempt
        cancel_head(r);
        continue;
      }
      r->admitting = true;
    }
    std::vector<double> inv;
    int slot = -1;
    hgks_status st = batch_place(B, source_of(r->hm, inv), r->p, &slot);
    if (st) { stop_admitting(r); return st; }
    if (slot < 0) {
      bool empty = true;
      for (auto *q : S.running) empty = empty && q == nullptr;
      std::lock_guard<std::mutex> lk(S.mu);
      if (r->cancel) {
        cancel_head(r);
        continue;
      }
      if (!empty) {                        // the head of the queue waits for room
        r->admitting = false;
        return HGKS_OK;
      }
      // nothing runs and it still does not fit (its faces exceed the arena's): it never will
      S.built.pop_front();
      r->admitting = false;
      r->hm = HostMesh{};
      r->status = HGKS_ERR_OOM;
      r->err = "mesh does not fit the server's arena";
      r->state = Q_FAIL;
      r->t_done = now_s(S.t0);
      continue;
    }
    const bool cmp = compact(B);
    std::vector<double> Qi = to_internal(r->Q0, r->perm, 5), Gi;
    if (cmp) Gi = r->G0.empty() ? std::vector<double>((size_t)15 * r->perm.size(), 0.0) : to_internal(r->G0, r->perm, 15);
    if ((st = batch_set_state(B, slot, Qi.data(), cmp ? Gi.data() : nullptr)) ||
        (st = batch_arm(B, slot, r->drop, r->max_steps))) {
      stop_admitting(r);
      return st;
    }
    if (cudaStreamSynchronize(B.stream) != cudaSuccess) {
      stop_admitting(r);
      return cuda_error(cudaGetLastError(), "admission");
    }
    {
      // admitted; a cancel that came meanwhile retires it at the start of the next round
      std::lock_guard<std::mutex> lk(S.mu);
      S.built.pop_front();
      r->admitting = false;
      r->hm = HostMesh{};
      r->Q0.clear(); r->Q0.shrink_to_fit();
      r->G0.clear(); r->G0.shrink_to_fit();
      r->slot = slot;
      r->state = Q_RUN;
      r->t_admit = now_s(S.t0);
      S.running[slot] = r;
    }
    changed = true;
  }
}

// retire the running requests whose slot is no longer active (act[1 + k] == 0),
// or, with cancelled_only, those cancelled by the user
hgks_status retire(hgks_server_s &S, const std::vector<int> &act, int *n_finished, bool cancelled_only = false) {
  Batch &B = *S.B;
  for (int k = 0; k < B.nslot; k++) {
    Request *r = S.running[k];
    if (!r) continue;
    if (cancelled_only ? !r->cancel : act[1 + k] != 0) continue;
    int steps = 0, conv = 0, bad = 0;
    double ref = 0.0, res = 0.0;
    const size_t n = r->perm.size();
    std::vector<double> Qi(5 * n), Gi(compact(B) ? 15 * n : 0);
    cudaStream_t st = B.stream;
    cudaMemcpyAsync(&steps, B.bs.steps + k, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&conv, B.bs.conv + k, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&bad, B.bs.bad + k, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&ref, B.bs.ref + k, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&res, B.bs.res + k, sizeof(double), cudaMemcpyDeviceToHost, st);
    hgks_status s = batch_get_state(B, k, Qi.data(), Gi.empty() ? nullptr : Gi.data(), nullptr, nullptr);
    if (s) return s;
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_error(cudaGetLastError(), "retire");
    batch_release(B, k);
    to_caller(Qi, r->perm, 5, r->Q);
    if (!Gi.empty()) to_caller(Gi, r->perm, 15, r->G);
    std::lock_guard<std::mutex> lk(S.mu);
    r->info.steps = steps;
    r->info.converged = conv;
    r->info.res_ref = ref;
    r->info.res_final = res;
    r->status = cancelled_only ? HGKS_ERR_CANCELLED : bad ? HGKS_ERR_NONPHYSICAL : (conv ? HGKS_OK : HGKS_ERR_NOT_CONVERGED);
    r->state = Q_DONE;
    r->t_done = now_s(S.t0);
    S.running[k] = nullptr;
    (*n_finished)++;
  }
  return HGKS_OK;
}

hgks_status server_create(int32_t device, int64_t hbm_budget_bytes, int32_t max_inflight, const hgks_params *shared,
                          int32_t use_graph, bool hex, hgks_server *out) {
  if (!out || !shared) return fail_msg(HGKS_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (max_inflight < 1 || max_inflight > 32767) return fail_msg(HGKS_ERR_ARG, "max_inflight must be in 1..32767");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return fail_msg(HGKS_ERR_ARG, "no such device");
  const int schemes = shared->scheme == HGKS_WENO ? 1 : 2;
  // the largest arena within the budget (faces: 2.1 per cell for tetrahedra, 3.1 for
  // hexahedra, the interior ratios plus boundary)
  auto faces_for = [hex](int64_t n) { return n * (hex ? 31 : 21) / 10 + 4096; };
  int64_t lo = 0, hi = (int64_t)(INT32_MAX / 14);
  while (hi - lo > kBatchBlock) {
    const int64_t mid = (lo + hi) / 2;
    if (arena_bytes(mid, faces_for(mid), *shared, schemes, hex) <= hbm_budget_bytes) lo = mid; else hi = mid;
  }
  const int64_t ncap = lo / kBatchBlock * kBatchBlock;
  if (ncap < kBatchBlock) return fail_msg(HGKS_ERR_ARG, "HBM budget too small for any mesh");
  HGKS_ON_DEVICE(device);
  hgks_server_s *S = new (std::nothrow) hgks_server_s;
  if (!S) return fail_msg(HGKS_ERR_OOM, "host allocation");
  hgks_status st = batch_new(device, ncap, faces_for(ncap), max_inflight, *shared, schemes, &S->B, hex);
  if (st) { delete S; return st; }
  S->t0 = std::chrono::steady_clock::now();
  S->running.assign(max_inflight, nullptr);
  S->use_graph = use_graph;
  S->builder = std::thread(builder_loop, S);
  *out = S;
  return HGKS_OK;
}
}  // namespace

extern "C" {

hgks_status hgks_server_create(int32_t device, int64_t hbm_budget_bytes, int32_t max_inflight, const hgks_params *shared,
                               int32_t use_graph, hgks_server *out) {
  return server_create(device, hbm_budget_bytes, max_inflight, shared, use_graph, false, out);
}

hgks_status hgks_server_create_hex(int32_t device, int64_t hbm_budget_bytes, int32_t max_inflight,
                                   const hgks_params *shared, int32_t use_graph, hgks_server *out) {
  return server_create(device, hbm_budget_bytes, max_inflight, shared, use_graph, true, out);
}

hgks_status hgks_server_destroy(hgks_server S) {
  if (!S) return fail_msg(HGKS_ERR_ARG, "server is NULL");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->builder.joinable()) S->builder.join();
  batch_delete(S->B);
  delete S;
  return HGKS_OK;
}

}  // extern "C"

namespace {
hgks_status server_submit(hgks_server S, const double *xyz, int64_t n_vert, const int64_t *tet4, int32_t nvc,
                          int64_t n_tet, const int64_t *bface3, const int32_t *btag, int64_t n_bface,
                          const double *periodic_shift, int32_t n_periodic, const hgks_params *p, const double *Q0,
                          const double *G0, double drop_tol, int32_t max_steps, int64_t *id_out) {
  if (!S || !p || !xyz || !tet4 || !Q0 || !id_out) return fail_msg(HGKS_ERR_ARG, "NULL argument");
  if (n_tet <= 0 || n_vert <= 0 || n_bface < 0 || n_periodic < 0) return fail_msg(HGKS_ERR_ARG, "bad sizes");
  if (!(drop_tol > 0.0) || max_steps < 0) return fail_msg(HGKS_ERR_ARG, "drop_tol must be > 0 and max_steps >= 0");
  Batch &B = *S->B;
  if ((nvc == 8) != (B.m.d.hex != 0))
    return fail_msg(HGKS_ERR_ARG, "a server takes one cell kind: tetrahedra (hgks_server_create) or hexahedra "
                                  "(hgks_server_create_hex)");
  const int64_t nfv = nvc == 8 ? 4 : 3;
  Mesh probe;
  probe.schemes = B.m.schemes;
  hgks_params P;
  hgks_status st = take_params(probe, p, &P);
  if (st) return st;
  p = &P;
  if (!same_shared(B.p0, *p))
    return fail_msg(HGKS_ERR_ARG, "scheme, precision, jv_mode, krylov_dim, restarts, jacobi_sweeps must match the server's");
  if ((n_tet + kBatchBlock - 1) / kBatchBlock * kBatchBlock > B.m.N)
    return fail_msg(HGKS_ERR_ARG, "mesh larger than the server's arena (HBM budget)");
  auto r = std::make_unique<Request>();
  r->xyz.assign(xyz, xyz + 3 * n_vert);
  r->nvc = nvc;
  r->tet.assign(tet4, tet4 + (int64_t)nvc * n_tet);
  if (n_bface) {
    if (!bface3 || !btag) return fail_msg(HGKS_ERR_ARG, "boundary arrays are NULL");
    r->bface.assign(bface3, bface3 + nfv * n_bface);
    r->btag.assign(btag, btag + n_bface);
  }
  if (n_periodic) {
    if (!periodic_shift) return fail_msg(HGKS_ERR_ARG, "periodic_shift is NULL");
    r->pshift.assign(periodic_shift, periodic_shift + 3 * n_periodic);
  }
  r->nps = n_periodic;
  r->p = *p;
  r->drop = drop_tol;
  r->max_steps = max_steps;
  r->Q0.assign(Q0, Q0 + 5 * n_tet);
  if (G0) r->G0.assign(G0, G0 + 15 * n_tet);
  std::lock_guard<std::mutex> lk(S->mu);
  r->id = S->next_id++;
  r->t_submit = now_s(S->t0);
  *id_out = r->id;
  S->to_build.push_back(r.get());
  S->all[r->id] = std::move(r);
  S->cv.notify_all();
  return HGKS_OK;
}
}  // namespace

extern "C" {

hgks_status hgks_server_submit(hgks_server S, const double *xyz, int64_t n_vert, const int64_t *tet4, int64_t n_tet,
                               const int64_t *bface3, const int32_t *btag, int64_t n_bface, const double *periodic_shift,
                               int32_t n_periodic, const hgks_params *p, const double *Q0, const double *G0,
                               double drop_tol, int32_t max_steps, int64_t *id_out) {
  return server_submit(S, xyz, n_vert, tet4, 4, n_tet, bface3, btag, n_bface, periodic_shift, n_periodic, p, Q0, G0,
                       drop_tol, max_steps, id_out);
}

hgks_status hgks_server_submit_hex(hgks_server S, const double *xyz, int64_t n_vert, const int64_t *hex8, int64_t n_hex,
                                   const int64_t *bquad4, const int32_t *btag, int64_t n_bface,
                                   const double *periodic_shift, int32_t n_periodic, const hgks_params *p,
                                   const double *Q0, const double *G0, double drop_tol, int32_t max_steps,
                                   int64_t *id_out) {
  return server_submit(S, xyz, n_vert, hex8, 8, n_hex, bquad4, btag, n_bface, periodic_shift, n_periodic, p, Q0, G0,
                       drop_tol, max_steps, id_out);
}

hgks_status hgks_server_step(hgks_server S, int32_t *n_finished, int32_t *n_running, int32_t *n_waiting) {
  HGKS_RANGE("hgks server step");
  if (!S) return fail_msg(HGKS_ERR_ARG, "server is NULL");
  Batch &B = *S->B;
  int fin = 0;
  bool changed = false;
  hgks_status st;
  HGKS_ON_DEVICE(B.m.device);
  {
    bool any_cancel = false;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (auto *r : S->running) any_cancel = any_cancel || (r && r->cancel);
    }
    if (any_cancel) {
      std::vector<int> none(B.nslot + 1, 0);
      if ((st = retire(*S, none, &fin, true))) return st;
      changed = true;
    }
  }
  if ((st = admit(*S, changed))) return st;
  int run = 0;
  for (auto *r : S->running) run += r ? 1 : 0;
  if (run) {
    if (changed) {
      std::vector<int> mask(B.nslot);
      for (int k = 0; k < B.nslot; k++) mask[k] = S->running[k] ? 1 : 0;
      if ((st = batch_set_active(B, mask))) return st;
    }
    if ((st = batch_enqueue_step(B, true, S->use_graph != 0))) return st;
    std::vector<int> act(B.nslot + 1);
    cudaMemcpyAsync(act.data(), B.active_base, sizeof(int) * (B.nslot + 1), cudaMemcpyDeviceToHost, B.stream);
    if (cudaStreamSynchronize(B.stream) != cudaSuccess) return cuda_error(cudaGetLastError(), "server step");
    if ((st = retire(*S, act, &fin))) return st;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  run = 0;
  for (auto *r : S->running) run += r ? 1 : 0;
  if (n_finished) *n_finished = fin;
  if (n_running) *n_running = run;
  // a request under construction still waits: a caller that drains the server
  // until nothing runs or waits must not stop while the builder holds one
  if (n_waiting) *n_waiting = (int32_t)(S->to_build.size() + S->building + S->built.size());
  return HGKS_OK;
}

hgks_status hgks_server_status(hgks_server S, int64_t id, hgks_request_info *info) {
  if (!S || !info) return fail_msg(HGKS_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return fail_msg(HGKS_ERR_ARG, "unknown request id");
  const Request &r = *it->second;
  std::memset(info, 0, sizeof(*info));
  info->state = r.state;
  info->status = r.status;
  info->n_cells = (int64_t)(r.perm.empty() ? r.tet.size() / r.nvc : r.perm.size());
  info->solve = r.info;
  info->t_submit = r.t_submit;
  info->t_built = r.t_built;
  info->t_admit = r.t_admit;
  info->t_done = r.t_done;
  return HGKS_OK;
}

hgks_status hgks_server_cancel(hgks_server S, int64_t id) {
  if (!S) return fail_msg(HGKS_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return fail_msg(HGKS_ERR_ARG, "unknown request id");
  Request *r = it->second.get();
  auto drop = [&](std::deque<Request *> &q) {
    auto qi = std::find(q.begin(), q.end(), r);
    if (qi == q.end()) return false;
    q.erase(qi);
    r->status = HGKS_ERR_CANCELLED;
    r->state = Q_DONE;
    r->t_done = now_s(S->t0);
    r->hm = HostMesh{};
    return true;
  };
  if (r->state == Q_WAIT) {
    if (!drop(S->to_build)) r->cancel = true;          // being built now: the builder drops it
  } else if (r->state == Q_BUILT) {
    if (r->admitting) r->cancel = true;                // being placed now: admission finishes it
    else drop(S->built);
  } else if (r->state == Q_RUN) {
    r->cancel = true;                                  // leaves at the start of the next round
  }
  return HGKS_OK;
}

hgks_status hgks_server_collect(hgks_server S, int64_t id, double *Q, double *G) {
  if (!S) return fail_msg(HGKS_ERR_ARG, "server is NULL");
  std::unique_ptr<Request> r;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail_msg(HGKS_ERR_ARG, "unknown request id");
    if (it->second->state != Q_DONE && it->second->state != Q_FAIL) return fail_msg(HGKS_ERR_ARG, "request not finished");
    r = std::move(it->second);
    S->all.erase(it);
  }
  if (r->state == Q_FAIL) return fail_msg(r->status, r->err);
  if (r->status == HGKS_ERR_CANCELLED && r->Q.empty()) return fail_msg(HGKS_ERR_CANCELLED, "cancelled before it ran");
  if (Q) std::memcpy(Q, r->Q.data(), sizeof(double) * r->Q.size());
  if (G && !r->G.empty()) std::memcpy(G, r->G.data(), sizeof(double) * r->G.size());
  return HGKS_OK;
}

hgks_status hgks_server_info(hgks_server S, hgks_batch_info_t *info) {
  if (!S || !info) return fail_msg(HGKS_ERR_ARG, "NULL argument");
  const Batch &B = *S->B;
  info->n_cells = B.m.N;
  info->n_faces = B.m.F;
  info->device_bytes = (int64_t)B.m.bytes;
  info->n_meshes = 0;
  for (auto &s : B.slots) info->n_meshes += s.used ? 1 : 0;
  info->blk_recon = B.m.s.blk_recon;
  info->blk_flux = B.m.s.blk_flux;
  return HGKS_OK;
}

}  // extern "C"
