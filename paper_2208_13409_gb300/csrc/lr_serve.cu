// lr_serve.cu -- the C ABI of include/lr_serve.h: a request queue in front
// of a batch, driven by one worker thread (admission into free pool units,
// chunks of batched steps sized to the next completion, retirement with the
// result copied to host memory).
#include "../../include/lr_serve.h"
#include "lr_host.h"

#include <stdarg.h>
#include <stdio.h>
#include <string.h>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace {

const int KEEP_FIELDS[] = {LR_F_K, LR_F_RHO_MAT, LR_F_E_MAT, LR_F_P, LR_F_UX, LR_F_UY};
constexpr int NKEEP = sizeof(KEEP_FIELDS) / sizeof(KEEP_FIELDS[0]);

struct Req {
  long id = 0;
  lr_config cfg;
  std::vector<lr_material> mats;
  std::vector<double> k, rho, p, ux, uy;
  double t_end = 0.0;
  long max_steps = 0;
  double submit_s = 0.0, admit_s = -1.0, done_s = -1.0;
  int state = 0;        // 0 waiting or resident, 1 done, -1 failed
  int member = -1;
  int bypassed = 0;     // times a later request was admitted before it
  double t = 0.0;
  long steps = 0;
  std::map<int, std::vector<double>> out;
};

}  // namespace

struct lr_server {
  lr_server_config cfg;
  lr_batch* b = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<long> pending;
  std::map<long, std::unique_ptr<Req>> reqs;
  std::vector<long> slot_req;
  long next_id = 0;
  long resident = 0;
  bool stop = false;
  bool broken = false;
  std::chrono::steady_clock::time_point t0;
  lr_server_stats st;
  char msg[512];
};

namespace {

void setmsg(lr_server* s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(s->msg, sizeof(s->msg), fmt, ap);
  va_end(ap);
}

double now_s(const lr_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// Admit waiting requests in arrival order while they fit; a request that
// has been passed over max_bypass times blocks everything behind it.
void admit(lr_server* s) {
  std::vector<Req*> cand;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (long id : s->pending) cand.push_back(s->reqs[id].get());
  }
  std::vector<Req*> waiting;  // earlier requests that did not fit this round
  for (Req* r : cand) {
    bool blocked = false;
    for (Req* w : waiting) blocked |= w->bypassed >= s->cfg.max_bypass;
    if (blocked) break;
    int m = -1;
    lr_status rc = lr_batch_add(s->b, &r->cfg, r->mats.data(), r->k.data(), r->rho.data(), r->p.data(),
                                r->ux.data(), r->uy.data(), r->t_end, r->max_steps, &m);
    std::lock_guard<std::mutex> lk(s->mu);
    if (rc == LR_OK) {
      for (Req* w : waiting) w->bypassed += 1;
      r->member = m;
      r->admit_s = now_s(s);
      s->slot_req[m] = r->id;
      s->resident += 1;
      s->st.admitted += 1;
      for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
        if (*it == r->id) { s->pending.erase(it); break; }
      r->k.clear(); r->rho.clear(); r->p.clear(); r->ux.clear(); r->uy.clear();
      r->k.shrink_to_fit(); r->rho.shrink_to_fit(); r->p.shrink_to_fit(); r->ux.shrink_to_fit(); r->uy.shrink_to_fit();
    } else if (rc == LR_ERR_OOM) {
      waiting.push_back(r);
    } else {
      if (m >= 0) lr_batch_remove(s->b, m);
      r->state = -1;
      r->done_s = now_s(s);
      s->st.failed += 1;
      for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
        if (*it == r->id) { s->pending.erase(it); break; }
      s->cv_done.notify_all();
    }
  }
}

// Copy the results of finished members to the host and release them.
bool retire(lr_server* s) {
  int S = s->cfg.batch.capacity_members;
  std::vector<int> state(S);
  std::vector<long> steps(S);
  if (lr_batch_status_all(s->b, state.data(), steps.data(), S) != LR_OK) return false;
  for (int m = 0; m < S; ++m) {
    long id;
    Req* r;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      id = s->slot_req[m];
      if (id < 0) continue;
      r = s->reqs[id].get();
      r->steps = steps[m];
    }
    if (state[m] == 0) continue;
    std::map<int, std::vector<double>> out;
    double t = 0.0;
    lr_batch_status(s->b, m, &t, nullptr, nullptr);
    if (state[m] == 1) {
      for (int q = 0; q < NKEEP; ++q) {
        size_t n = lr_batch_field_size(s->b, m, KEEP_FIELDS[q]);
        std::vector<double> v(n);
        if (lr_batch_get_fields(s->b, m, KEEP_FIELDS[q], v.data(), n) != LR_OK) return false;
        out[KEEP_FIELDS[q]].swap(v);
      }
    }
    lr_batch_remove(s->b, m);
    std::lock_guard<std::mutex> lk(s->mu);
    r->out.swap(out);
    r->t = t;
    r->state = state[m] == 1 ? 1 : -1;
    r->done_s = now_s(s);
    s->slot_req[m] = -1;
    s->resident -= 1;
    if (r->state == 1) {
      s->st.completed += 1;
      s->st.cell_updates += (double)r->cfg.nx * r->cfg.ny * (double)r->steps;
    } else {
      s->st.failed += 1;
    }
    s->cv_done.notify_all();
  }
  return true;
}

void fail_all(lr_server* s, const char* why) {
  std::lock_guard<std::mutex> lk(s->mu);
  s->broken = true;
  setmsg(s, "server stopped: %s (%s)", why, lr_batch_last_error(s->b));
  for (auto& kv : s->reqs)
    if (kv.second->state == 0) { kv.second->state = -1; kv.second->done_s = now_s(s); s->st.failed += 1; }
  s->pending.clear();
  s->cv_done.notify_all();
}

void worker_main(lr_server* s) {
  cudaSetDevice(s->cfg.device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty() || s->resident > 0; });
      if (s->stop) return;
    }
    admit(s);
    int chunk = s->cfg.max_chunk_steps;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->resident == 0) continue;  // nothing fits yet (cannot happen with an empty pool)
      for (long id : s->slot_req) {
        if (id < 0) continue;
        const Req* r = s->reqs[id].get();
        if (r->max_steps > 0) {
          long rem = r->max_steps - r->steps;
          if (rem < 1) rem = 1;
          if (rem < chunk) chunk = (int)rem;
        }
      }
    }
    double a = now_s(s);
    if (lr_batch_step(s->b, chunk) != LR_OK) { fail_all(s, "step"); return; }
    if (!retire(s)) { fail_all(s, "retire"); return; }
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.steps_launched += chunk;
    s->st.busy_s += now_s(s) - a;
  }
}

Req* find(lr_server* s, long id) {
  auto it = s->reqs.find(id);
  return it == s->reqs.end() ? nullptr : it->second.get();
}

}  // namespace

extern "C" {

void lr_server_config_default(lr_server_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  lr_batch_config_default(&c->batch);
  c->max_chunk_steps = 64;
  c->max_bypass = 8;
  c->device = 0;
}

lr_status lr_server_create(const lr_server_config* cfg, lr_server** out) {
  if (!cfg || !out) return LR_ERR_ARG;
  *out = nullptr;
  if (cfg->max_chunk_steps < 1 || cfg->max_bypass < 0 || cfg->batch.cuda_stream) return LR_ERR_ARG;
  if (cudaSetDevice(cfg->device) != cudaSuccess) return LR_ERR_CUDA;
  lr_server* s = new lr_server();
  s->cfg = *cfg;
  memset(&s->st, 0, sizeof(s->st));
  s->msg[0] = 0;
  lr_status rc = lr_batch_create(&cfg->batch, &s->b);
  if (rc != LR_OK) { delete s; return rc; }
  s->slot_req.assign(cfg->batch.capacity_members, -1);
  s->t0 = std::chrono::steady_clock::now();
  s->worker = std::thread(worker_main, s);
  *out = s;
  return LR_OK;
}

void lr_server_destroy(lr_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  lr_batch_destroy(s->b);
  delete s;
}

const char* lr_server_last_error(const lr_server* s) { return s ? s->msg : "null server"; }

lr_status lr_server_submit(lr_server* s, const lr_config* cfg, const lr_material* mats, const double* k,
                           const double* rho, const double* p, const double* ux, const double* uy, double t_end,
                           long max_steps, long* id) {
  if (!s || !cfg || !mats || !k || !rho || !p || !ux || !uy || !id) return LR_ERR_ARG;
  *id = -1;
  char why[160];
  if (!lr_config_ok(cfg, why, sizeof(why))) { setmsg(s, "submit: %s", why); return LR_ERR_ARG; }
  const lr_batch_config& bc = s->cfg.batch;
  if (cfg->precision != bc.precision || cfg->nmat > bc.nmat_max || !(t_end >= 0.0)) {
    setmsg(s, "submit: precision, nmat or t_end outside what the server runs");
    return LR_ERR_ARG;
  }
  long units = (long)(cfg->nx + 2) * (cfg->ny + 2);
  if (units > bc.capacity_units || (long)cfg->nx * cfg->ny > bc.max_member_cells) {
    setmsg(s, "submit: a %d x %d grid can never fit this server's pool", cfg->nx, cfg->ny);
    return LR_ERR_OOM;
  }
  std::unique_ptr<Req> r(new Req());
  r->cfg = *cfg;
  r->cfg.cuda_stream = nullptr;
  r->mats.assign(mats, mats + cfg->nmat);
  size_t nc = (size_t)cfg->nx * cfg->ny * cfg->nmat, nn = (size_t)(cfg->nx + 1) * (cfg->ny + 1);
  r->k.assign(k, k + nc); r->rho.assign(rho, rho + nc); r->p.assign(p, p + nc);
  r->ux.assign(ux, ux + nn); r->uy.assign(uy, uy + nn);
  r->t_end = t_end;
  r->max_steps = max_steps;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->broken) return LR_ERR_STATE;
    r->id = s->next_id++;
    r->submit_s = now_s(s);
    *id = r->id;
    s->pending.push_back(r->id);
    s->reqs[r->id] = std::move(r);
    s->st.submitted += 1;
  }
  s->cv_work.notify_all();
  return LR_OK;
}

lr_status lr_server_wait(lr_server* s, long id, double timeout_s, int* state) {
  if (!s) return LR_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  Req* r = find(s, id);
  if (!r) return LR_ERR_ARG;
  auto done = [&] { return r->state != 0; };
  if (timeout_s < 0.0) s->cv_done.wait(lk, done);
  else s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
  if (state) *state = r->state;
  return r->state != 0 ? LR_OK : LR_ERR_TIMEOUT;
}

lr_status lr_server_drain(lr_server* s, double timeout_s) {
  if (!s) return LR_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto all = [&] {
    for (auto& kv : s->reqs)
      if (kv.second->state == 0) return false;
    return true;
  };
  if (timeout_s < 0.0) s->cv_done.wait(lk, all);
  else s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), all);
  return all() ? LR_OK : LR_ERR_TIMEOUT;
}

lr_status lr_server_info(lr_server* s, long id, double* submit_s, double* admit_s, double* done_s, double* t,
                         long* steps) {
  if (!s) return LR_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  Req* r = find(s, id);
  if (!r) return LR_ERR_ARG;
  if (submit_s) *submit_s = r->submit_s;
  if (admit_s) *admit_s = r->admit_s;
  if (done_s) *done_s = r->done_s;
  if (t) *t = r->t;
  if (steps) *steps = r->steps;
  return LR_OK;
}

size_t lr_server_result_size(lr_server* s, long id, int field) {
  if (!s) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  Req* r = find(s, id);
  if (!r || r->state != 1) return 0;
  auto it = r->out.find(field);
  return it == r->out.end() ? 0 : it->second.size();
}

lr_status lr_server_result(lr_server* s, long id, int field, double* out, size_t n) {
  if (!s || !out) return LR_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  Req* r = find(s, id);
  if (!r) return LR_ERR_ARG;
  if (r->state != 1) return LR_ERR_STATE;
  auto it = r->out.find(field);
  if (it == r->out.end() || n < it->second.size()) return LR_ERR_ARG;
  memcpy(out, it->second.data(), it->second.size() * sizeof(double));
  return LR_OK;
}

lr_status lr_server_release(lr_server* s, long id) {
  if (!s) return LR_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  Req* r = find(s, id);
  if (!r) return LR_ERR_ARG;
  if (r->state == 0) return LR_ERR_STATE;
  s->reqs.erase(id);
  return LR_OK;
}

lr_status lr_server_get_stats(lr_server* s, lr_server_stats* out) {
  if (!s || !out) return LR_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->pending = (long)s->pending.size();
  out->resident = s->resident;
  return LR_OK;
}

double lr_server_clock(const lr_server* s) { return s ? now_s(s) : 0.0; }

}  // extern "C"
