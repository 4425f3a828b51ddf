// Served form: continuous batching of wave solves on one GPU.
//
// States are held at the Gauss points while admitted (DG_BASIS_G batches;
// one change of basis on admission and one on completion).
//
// Two threads.  The admission thread takes queued requests in arrival order
// while they fit the HBM budget (a request that does not fit lets later,
// smaller ones in: first-fit backfill) and the active-DoF cap, and sets each
// one up on the device (geometry, coefficients, state) on its own stream
// while the GPU keeps stepping.  The stepping thread keeps every admitted
// solve device-resident and advances all of them together with dg_batch in
// rounds of at most chunk_steps steps; a round ends early when a solve
// reaches its step count, whose state is then copied to the caller's host
// buffer and its memory released.  Solves set up meanwhile join at the next
// round, so requests arriving while others run overlap with them on the
// device.
//
// Built only on the public C ABI (include/dg.h) and the CUDA runtime.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dg.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t ticket = 0;
  // owned copies of the request's inputs
  std::vector<double> nodes, rho, c;
  std::vector<int32_t> nbr;
  std::vector<int8_t> nbr_face, orient;
  std::vector<unsigned char> U0;
  int32_t n_elem = 0, q = 1, k = 1, nsteps = 0, method = 1, red = 2;
  double alpha = 1.0, dt = 0.0;
  void* U_out = nullptr;
  size_t state_bytes = 0, est_bytes = 0;
  // progress
  dg_ctx* ctx = nullptr;
  void* U = nullptr;
  int32_t done_steps = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int status = DG_EAGAIN;  // read and written under the server's lock only
  std::string err;
  // a failure the stepping thread has met; it becomes the status, under the
  // lock, together with t_done and the release of the budget
  int fail = DG_OK;
  std::string fail_err;
};

// Device bytes a solve holds while admitted: the context's allocations with
// all scratch present (three LSRK states, the LSRK register, the predictor),
// plus its state.
size_t estimate_bytes(int E, int k, int q, int prec) {
  const size_t n = k + 1, n3 = n * n * n, rs = prec == DG_FP64 ? 8 : 4, qc = q + 1;
  size_t tck = 0;
  for (size_t m = n; m >= 2; m -= 2) tck += 11 * m * m * m;
  const size_t state = (size_t)E * 4 * n3 * rs;
  size_t b = 0;
  b += (size_t)E * (4 * 6 + 6 + 6);                  // connectivity
  b += (size_t)E * 3 * qc * qc * qc * 8;             // geometry nodes
  b += (size_t)E * 2 * n3 * 8;                       // rho, c
  b += (size_t)E * (11 * n3 + 36 * n * n + 24 + tck) * rs;  // geometry and coefficients (padded)
  b += 5 * state;                                    // U2, U3, dU, Ubar and U
  return b + (1 << 20);
}

}  // namespace

struct dg_server {
  size_t budget = 0, used = 0;
  dg_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::condition_variable cv_step;
  std::deque<std::shared_ptr<Req>> queue;
  std::vector<std::shared_ptr<Req>> ready;   // set up, waiting for the next round
  std::vector<std::shared_ptr<Req>> active;
  double admitted_dof = 0.0;                  // DoFs of set-up-or-active solves
  int admitted_count = 0;
  std::map<uint64_t, std::shared_ptr<Req>> all;  // until polled
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker, admitter;
  std::string err;
  // statistics
  uint64_t rounds = 0, batches_built = 0, completed = 0;
  double dof_steps = 0.0, busy_s = 0.0;
  size_t peak_used = 0;
  int peak_active = 0;

  void run();
  void admit_loop();
  double dof_of(const Req& r) const { return (double)r.state_bytes / (opts.prec == DG_FP64 ? 8 : 4); }
  bool admissible(const Req& r) const {
    if (used + r.est_bytes > budget) return false;
    if (opts.max_active > 0 && admitted_count >= opts.max_active) return false;
    if (opts.max_active_dof > 0 && admitted_count > 0 && admitted_dof + dof_of(r) > opts.max_active_dof)
      return false;
    return true;
  }
};

namespace {

int admit(dg_server* s, const std::shared_ptr<Req>& r, cudaStream_t st) {
  dg_mesh_desc m;
  m.n_elem = r->n_elem;
  m.geom_degree = r->q;
  m.nodes = r->nodes.data();
  m.nbr = r->nbr.data();
  m.nbr_face = r->nbr_face.data();
  m.orient = r->orient.data();
  int rc = dg_mesh_setup_coef(&m, r->k, s->opts.prec, r->alpha, r->rho.data(), r->c.data(), (uintptr_t)st,
                              &r->ctx);
  if (rc) {
    r->err = dg_last_error(nullptr);
    return rc;
  }
  if (cudaMalloc(&r->U, r->state_bytes) != cudaSuccess) {
    cudaGetLastError();
    r->err = "cudaMalloc of the state failed";
    return DG_ENOMEM;
  }
  if (cudaMemcpyAsync(r->U, r->U0.data(), r->state_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    r->err = "upload of the initial state failed";
    return DG_ECUDA;
  }
  // the state stays at the Gauss points while admitted (one change of basis
  // on admission, one on completion, however the steps are split in rounds)
  if ((rc = dg_change_basis(r->ctx, r->U, 1, (uintptr_t)st))) {
    r->err = dg_last_error(r->ctx);
    return rc;
  }
  // the inputs are on the device now
  std::vector<double>().swap(r->nodes);
  std::vector<double>().swap(r->rho);
  std::vector<double>().swap(r->c);
  std::vector<unsigned char>().swap(r->U0);
  return DG_OK;
}

void release(dg_server* s, const std::shared_ptr<Req>& r) {
  if (r->ctx) dg_destroy(r->ctx);
  if (r->U) cudaFree(r->U);
  r->ctx = nullptr;
  r->U = nullptr;
}

}  // namespace

void dg_server::admit_loop() {
  cudaSetDevice(opts.device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    std::shared_ptr<Req> r;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] {
        if (stop) return true;
        for (auto& q : queue)
          if (admissible(*q)) return true;
        return false;
      });
      if (stop) break;
      for (auto it = queue.begin(); it != queue.end(); ++it)  // first fit, arrival order
        if (admissible(**it)) {
          r = *it;
          queue.erase(it);
          break;
        }
      used += r->est_bytes;
      admitted_dof += dof_of(*r);
      ++admitted_count;
      peak_used = std::max(peak_used, used);
    }
    const int rc = admit(this, r, st);
    cudaStreamSynchronize(st);
    std::lock_guard<std::mutex> lk(mu);
    r->t_admit = now_s();
    if (rc || r->nsteps == 0) {
      if (!rc) {
        dg_change_basis(r->ctx, r->U, 0, (uintptr_t)st);
        cudaStreamSynchronize(st);
        cudaMemcpy(r->U_out, r->U, r->state_bytes, cudaMemcpyDeviceToHost);
      }
      release(this, r);
      used -= r->est_bytes;
      admitted_dof -= dof_of(*r);
      --admitted_count;
      r->status = rc ? rc : DG_OK;
      if (!rc) ++completed;
      r->t_done = now_s();
      cv_done.notify_all();
      cv_work.notify_all();
    } else {
      ready.push_back(r);
      cv_step.notify_one();
    }
  }
  if (st) cudaStreamDestroy(st);
}

void dg_server::run() {
  cudaSetDevice(opts.device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  // one batch per (method, reduce_every) group of active solves
  struct Group {
    int method, red;
    std::vector<std::shared_ptr<Req>> members;
    dg_batch* batch = nullptr;
  };
  std::vector<Group> groups;
  bool dirty = true;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_step.wait(lk, [&] { return stop || !ready.empty() || !active.empty(); });
      if (stop) break;
      if (!ready.empty()) {
        for (auto& r : ready) active.push_back(r);
        ready.clear();
        dirty = true;
      }
      peak_active = std::max(peak_active, (int)active.size());
    }
    if (dirty) {
      for (auto& g : groups)
        if (g.batch) dg_batch_destroy(g.batch);
      groups.clear();
      for (auto& r : active) {
        const int red = r->method == 1 ? r->red : 0;
        auto it = std::find_if(groups.begin(), groups.end(),
                               [&](const Group& g) { return g.method == r->method && g.red == red; });
        if (it == groups.end()) {
          groups.push_back({r->method, red, {}, nullptr});
          it = groups.end() - 1;
        }
        it->members.push_back(r);
      }
      for (auto& g : groups) {
        std::vector<dg_ctx*> ctxs;
        std::vector<void*> us;
        std::vector<double> dts;
        for (auto& r : g.members) {
          ctxs.push_back(r->ctx);
          us.push_back(r->U);
          dts.push_back(r->dt);
        }
        if (dg_batch_create(ctxs.data(), us.data(), dts.data(), (int32_t)ctxs.size(), (uintptr_t)st,
                            &g.batch) != DG_OK ||
            dg_batch_set_basis(g.batch, DG_BASIS_G, 0) != DG_OK) {
          for (auto& r : g.members) {  // fail the group's solves
            r->fail = DG_ECUDA;
            r->fail_err = dg_last_error(nullptr);
            r->done_steps = r->nsteps;
          }
          g.batch = nullptr;
        }
      }
      ++batches_built;
      dirty = false;
    }
    // one round: as many steps as the nearest completion allows
    int round = opts.chunk_steps > 0 ? opts.chunk_steps : 16;
    for (auto& r : active) round = std::min(round, r->nsteps - r->done_steps);
    round = std::max(round, 0);
    const double t0 = now_s();
    for (auto& g : groups) {
      if (!g.batch || round == 0) continue;
      const int rc = g.method == 1 ? dg_batch_step_ader(g.batch, round, g.red, (uintptr_t)st)
                                   : dg_batch_step_lsrk(g.batch, round, (uintptr_t)st);
      if (rc) {
        for (auto& r : g.members) {
          r->fail = rc;
          r->fail_err = dg_batch_last_error(g.batch);
          r->done_steps = r->nsteps;
        }
      }
    }
    cudaStreamSynchronize(st);
    busy_s += now_s() - t0;
    ++rounds;
    std::vector<std::shared_ptr<Req>> finished;
    for (auto& r : active) {
      if (r->fail == DG_OK) {
        r->done_steps += round;
        dof_steps += (double)round * dof_of(*r);
      }
      if (r->done_steps >= r->nsteps) finished.push_back(r);
    }
    if (finished.empty()) continue;
    for (auto& r : finished)
      if (r->fail == DG_OK &&
          (dg_change_basis(r->ctx, r->U, 0, (uintptr_t)st) != DG_OK ||
           cudaMemcpyAsync(r->U_out, r->U, r->state_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)) {
        cudaGetLastError();
        r->fail = DG_ECUDA;
        r->fail_err = "copy of the final state failed";
      }
    cudaStreamSynchronize(st);
    for (auto& g : groups)
      if (g.batch) dg_batch_destroy(g.batch);
    groups.clear();
    dirty = true;
    for (auto& r : finished) release(this, r);
    std::lock_guard<std::mutex> lk(mu);
    for (auto& r : finished) {
      used -= r->est_bytes;
      admitted_dof -= dof_of(*r);
      --admitted_count;
      if (r->fail == DG_OK) {
        r->status = DG_OK;
        ++completed;
      } else {
        r->status = r->fail;
        r->err = r->fail_err;
      }
      r->t_done = now_s();
      active.erase(std::find(active.begin(), active.end(), r));
    }
    cv_done.notify_all();
    cv_work.notify_all();  // memory freed: the admission thread may take more
  }
  for (auto& g : groups)
    if (g.batch) dg_batch_destroy(g.batch);
  std::lock_guard<std::mutex> lk(mu);
  for (auto& r : active) release(this, r);
  for (auto& r : ready) release(this, r);
  active.clear();
  ready.clear();
  if (st) cudaStreamDestroy(st);
}

extern "C" {

size_t dg_request_bytes(int32_t n_elem, int32_t k, int32_t geom_degree, int32_t prec) {
  if (n_elem < 1 || k < 1 || k > DG_KMAX || geom_degree < 1 || (prec != DG_FP32 && prec != DG_FP64)) return 0;
  return estimate_bytes(n_elem, k, geom_degree, prec);
}

int dg_server_create(size_t hbm_budget, const dg_server_opts* opts, dg_server** out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  if (hbm_budget == 0) return DG_EINVAL;
  dg_server_opts o{};
  if (opts) o = *opts;
  if (o.prec != DG_FP32 && o.prec != DG_FP64) return DG_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) {
    cudaGetLastError();
    return DG_ECUDA;
  }
  dg_server* s = new (std::nothrow) dg_server();
  if (!s) return DG_ENOMEM;
  s->budget = hbm_budget;
  s->opts = o;
  s->worker = std::thread([s] { s->run(); });
  s->admitter = std::thread([s] { s->admit_loop(); });
  *out = s;
  return DG_OK;
}

int dg_submit(dg_server* s, const dg_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return DG_EINVAL;
  const dg_mesh_desc& m = r->mesh;
  if (!m.nodes || !m.nbr || !m.nbr_face || !m.orient || m.n_elem < 1 || m.geom_degree < 1 ||
      r->k < 1 || r->k > DG_KMAX || !r->rho || !r->c || !r->U0 || !r->U_out || !(r->dt > 0.0) ||
      r->nsteps < 0 || (r->method != 0 && r->method != 1) ||
      (r->method == 1 && r->reduce_every != 0 && r->reduce_every != 2))
    return DG_EINVAL;
  auto q = std::make_shared<Req>();
  const size_t E = m.n_elem, n = r->k + 1, n3 = n * n * n, qc = m.geom_degree + 1;
  const size_t rs = s->opts.prec == DG_FP64 ? 8 : 4;
  q->n_elem = m.n_elem;
  q->q = m.geom_degree;
  q->k = r->k;
  q->alpha = r->flux_alpha;
  q->dt = r->dt;
  q->nsteps = r->nsteps;
  q->method = r->method;
  q->red = r->reduce_every;
  q->U_out = r->U_out;
  q->state_bytes = E * 4 * n3 * rs;
  q->est_bytes = estimate_bytes(m.n_elem, r->k, m.geom_degree, s->opts.prec);
  if (q->est_bytes > s->budget) return DG_ENOMEM;  // can never fit
  q->nodes.assign(m.nodes, m.nodes + E * qc * qc * qc * 3);
  q->nbr.assign(m.nbr, m.nbr + 6 * E);
  q->nbr_face.assign(m.nbr_face, m.nbr_face + 6 * E);
  q->orient.assign(m.orient, m.orient + 6 * E);
  q->rho.assign(r->rho, r->rho + E * n3);
  q->c.assign(r->c, r->c + E * n3);
  const unsigned char* u0 = static_cast<const unsigned char*>(r->U0);
  q->U0.assign(u0, u0 + q->state_bytes);
  q->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->ticket = s->next_ticket++;
    s->all[q->ticket] = q;
    s->queue.push_back(q);
  }
  s->cv_work.notify_one();
  *ticket = q->ticket;
  return DG_OK;
}

int dg_poll(dg_server* s, uint64_t ticket, dg_result* out, int32_t timeout_ms) {
  if (!s || !out) return DG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return DG_EINVAL;
  auto r = it->second;
  auto finished = [&] { return r->status != DG_EAGAIN; };
  if (!finished() && timeout_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished);
  if (!finished()) return DG_EAGAIN;
  out->t_submit = r->t_submit;
  out->t_admit = r->t_admit;
  out->t_done = r->t_done;
  out->status = r->status;
  s->all.erase(it);
  return DG_OK;
}

int dg_server_stats(dg_server* s, dg_server_stats_t* st) {
  if (!s || !st) return DG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  st->queued = (int32_t)s->queue.size();
  st->active = (int32_t)(s->active.size() + s->ready.size());
  st->completed = s->completed;
  st->rounds = s->rounds;
  st->batches_built = s->batches_built;
  st->hbm_used = s->used;
  st->hbm_peak = s->peak_used;
  st->peak_active = s->peak_active;
  st->dof_steps = s->dof_steps;
  st->busy_s = s->busy_s;
  return DG_OK;
}

void dg_server_destroy(dg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_step.notify_all();
  if (s->admitter.joinable()) s->admitter.join();
  if (s->worker.joinable()) s->worker.join();
  delete s;
}

}  // extern "C"
