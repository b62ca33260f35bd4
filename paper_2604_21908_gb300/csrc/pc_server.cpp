// Request loop (continuous batching) over the library's public C ABI.
//
// Circuits arrive at any time (pc_server_submit).  An admission thread takes them in
// arrival order and admits the head of the queue as soon as a slot is free and its
// projected device footprint (the MPO store at its chi_max, see pc_projected_bytes) fits in
// the memory budget next to the circuits already resident.  Each admitted circuit gets a
// worker thread that loads it (its MPO store stays resident on the device until it is
// done), attaches it to the server's batch launcher and runs Algorithm 1 (pc_contract), then
// extracts the peak and draws its samples on the circuit's own stream.  While circuits
// contract, the launcher merges the waves they post into combined launches, so the
// factorisations of every resident circuit run interleaved in the same kernels; requests
// that arrive later join the next launches as they are admitted.
//
// Timing: every request records submit, admission and completion on the server clock
// (seconds since pc_server_create); time-to-peak is completion - submit.
#include "../../include/peaked_mpo.h"

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

namespace {

struct Request {
  int64_t ticket = 0;
  pc_config cfg{};
  int32_t n = 0;
  std::vector<int32_t> pairs;
  std::vector<double> mats;
  int64_t split = -1;
  std::vector<int32_t> oneq_q;
  std::vector<double> oneq_m;
  int64_t n_samples = 0;
  uint64_t seed = 0;
  int64_t bytes = 0;
  pc_result res{};
  std::vector<uint8_t> bits, samples;
  bool done = false;
};

double since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct pc_server {
  pc_server_config cfg{};
  pc_ctx* ctx = nullptr;          // device and batch owner
  pc_batch* batch = nullptr;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> queue;
  std::map<int64_t, Request*> all;
  int64_t next_ticket = 1;
  int resident = 0;
  int64_t bytes = 0;
  bool stop = false;
  std::thread admitter;
  std::vector<std::thread> workers;
  // statistics
  int64_t submitted = 0, admitted = 0, completed = 0, failed = 0;
  int max_resident_seen = 0;
  int64_t max_bytes_seen = 0;
  double first_submit = -1.0, last_done = 0.0;
};

namespace {

void serve_one(pc_server* s, Request* r) {
  pc_result& res = r->res;
  pc_config cfg = r->cfg;
  cfg.device = s->cfg.device;
  pc_ctx* ctx = nullptr;
  pc_circuit* c = nullptr;
  pc_status st = pc_create(&cfg, &ctx);
  if (st == PC_OK)
    st = pc_load_gates(ctx, r->n, (int64_t)r->pairs.size() / 2, r->pairs.data(), r->mats.data(), r->split,
                       (int64_t)r->oneq_q.size(), r->oneq_q.data(), r->oneq_m.data(), &c);
  if (st == PC_OK) st = pc_batch_attach(s->batch, c);
  pc_stats stats{};
  if (st == PC_OK) {
    st = pc_contract(c, &stats);
    pc_batch_detach(s->batch, c);
    if (st > 0) st = PC_OK;   // a stalled contraction still yields its MPO
  }
  r->bits.assign(r->n, 0);
  if (st == PC_OK) st = pc_extract_peak(c, 0, r->bits.data(), &res.p_peak, &res.norm2);
  if (st == PC_OK && r->n_samples > 0) {
    r->samples.assign((size_t)r->n_samples * r->n, 0);
    st = pc_sample(c, r->n_samples, r->seed, r->samples.data());
  }
  if (c) {
    int32_t mc = 1;
    std::vector<int32_t> chi(r->n - 1);
    if (pc_get_bond_dims(c, chi.data()) == PC_OK)
      for (int32_t v : chi) mc = std::max(mc, v);
    res.max_chi = std::max(mc, stats.max_chi);
    pc_destroy_circuit(c);
  }
  if (ctx) pc_destroy(ctx);
  res.status = st;
  res.n_updates = stats.n_updates;
  res.n_trials = stats.n_trials;
  res.n_accepted = stats.n_accepted;
  std::lock_guard<std::mutex> lk(s->mu);
  res.t_done = since(s->t0);
  r->done = true;
  s->resident -= 1;
  s->bytes -= r->bytes;
  if (st == PC_OK) s->completed += 1;
  else s->failed += 1;
  s->last_done = std::max(s->last_done, res.t_done);
  s->cv.notify_all();
}

void admit_loop(pc_server* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv.wait(lk, [&] {
      if (s->stop) return true;
      if (s->queue.empty() || s->resident >= s->cfg.max_resident) return false;
      const Request* h = s->queue.front();
      return s->resident == 0 || s->bytes + h->bytes <= s->cfg.memory_budget;
    });
    if (s->stop) break;
    Request* r = s->queue.front();
    s->queue.pop_front();
    if (r->bytes > s->cfg.memory_budget) {
      // would never fit, even alone
      r->res.status = PC_ERR_OOM;
      r->res.t_admit = r->res.t_done = since(s->t0);
      r->done = true;
      s->failed += 1;
      s->cv.notify_all();
      continue;
    }
    s->resident += 1;
    s->bytes += r->bytes;
    s->admitted += 1;
    s->max_resident_seen = std::max(s->max_resident_seen, s->resident);
    s->max_bytes_seen = std::max(s->max_bytes_seen, s->bytes);
    r->res.t_admit = since(s->t0);
    s->workers.emplace_back(serve_one, s, r);
  }
}

}  // namespace

extern "C" {

pc_status pc_server_create(const pc_server_config* cfg, pc_server** out) {
  if (!cfg || !out || cfg->max_resident < 1 || cfg->memory_budget <= 0 || cfg->max_tasks < 1 ||
      cfg->max_tasks > 256 || cfg->arena_bytes < 0)
    return PC_ERR_INVALID_ARG;
  *out = nullptr;
  pc_config base;
  pc_default_config(&base);
  base.device = cfg->device;
  auto* s = new pc_server();
  s->cfg = *cfg;
  pc_status st = pc_create(&base, &s->ctx);
  if (st == PC_OK) st = pc_batch_create(s->ctx, cfg->max_tasks, cfg->arena_bytes, &s->batch);
  if (st != PC_OK) {
    if (s->ctx) pc_destroy(s->ctx);
    delete s;
    return st;
  }
  s->t0 = std::chrono::steady_clock::now();
  s->admitter = std::thread(admit_loop, s);
  *out = s;
  return PC_OK;
}

pc_status pc_server_submit(pc_server* s, const pc_request* q, int64_t* ticket) {
  if (!s || !q || !ticket || q->n_qubits < 2 || q->n_gates < 0 || (q->n_gates > 0 && (!q->pairs || !q->mats)) ||
      q->n_oneq < 0 || (q->n_oneq > 0 && (!q->oneq_qubits || !q->oneq_mats)) || q->n_samples < 0 ||
      q->cfg.chi_max < 1)
    return PC_ERR_INVALID_ARG;
  auto* r = new Request();
  r->cfg = q->cfg;
  r->n = q->n_qubits;
  r->pairs.assign(q->pairs, q->pairs + 2 * q->n_gates);
  r->mats.assign(q->mats, q->mats + 32 * q->n_gates);
  r->split = q->split_index;
  r->oneq_q.assign(q->oneq_qubits, q->oneq_qubits + q->n_oneq);
  r->oneq_m.assign(q->oneq_mats, q->oneq_mats + 8 * q->n_oneq);
  r->n_samples = q->n_samples;
  r->seed = q->seed;
  r->bytes = pc_projected_bytes(q->n_qubits, q->cfg.chi_max, q->n_samples);
  r->res.n_qubits = q->n_qubits;
  r->res.store_bytes = r->bytes;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete r;
    return PC_ERR_STATE;
  }
  r->ticket = s->next_ticket++;
  r->res.t_submit = since(s->t0);
  if (s->first_submit < 0) s->first_submit = r->res.t_submit;
  s->submitted += 1;
  s->all[r->ticket] = r;
  s->queue.push_back(r);
  *ticket = r->ticket;
  s->cv.notify_all();
  return PC_OK;
}

pc_status pc_server_wait(pc_server* s, int64_t ticket, double timeout_s, pc_result* res, uint8_t* bits,
                         uint8_t* samples) {
  if (!s || !res) return PC_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return PC_ERR_INVALID_ARG;
  Request* r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_s < 0) {
    s->cv.wait(lk, ready);
  } else if (!s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return PC_ERR_TIMEOUT;
  }
  *res = r->res;
  if (bits && !r->bits.empty()) std::memcpy(bits, r->bits.data(), r->bits.size());
  if (samples && !r->samples.empty()) std::memcpy(samples, r->samples.data(), r->samples.size());
  return PC_OK;
}

double pc_server_clock(pc_server* s) { return s ? since(s->t0) : -1.0; }

pc_status pc_server_get_stats(pc_server* s, pc_server_stats* out) {
  if (!s || !out) return PC_ERR_INVALID_ARG;
  pc_server_stats st{};
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    st.submitted = s->submitted;
    st.admitted = s->admitted;
    st.completed = s->completed;
    st.failed = s->failed;
    st.resident = s->resident;
    st.max_resident_seen = s->max_resident_seen;
    st.bytes_resident = s->bytes;
    st.max_bytes_seen = s->max_bytes_seen;
    for (auto& kv : s->all)
      if (kv.second->done && kv.second->res.status == PC_OK)
        lat.push_back(kv.second->res.t_done - kv.second->res.t_submit);
    if (s->completed > 0 && s->last_done > s->first_submit)
      st.circuits_per_hour = 3600.0 * (double)s->completed / (s->last_done - s->first_submit);
  }
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    // nearest-rank percentiles
    auto pct = [&](double p) {
      size_t k = (size_t)std::ceil(p / 100.0 * lat.size());
      if (k < 1) k = 1;
      return lat[std::min(k, lat.size()) - 1];
    };
    st.p50_s = pct(50.0);
    st.p99_s = pct(99.0);
    double sum = 0.0;
    for (double v : lat) sum += v;
    st.mean_s = sum / lat.size();
  }
  int32_t mt = 0;
  pc_batch_counters(s->batch, &st.launches, &st.tasks, &mt, nullptr, nullptr);
  st.max_tasks_per_launch = mt;
  *out = st;
  return PC_OK;
}

pc_status pc_server_destroy(pc_server* s) {
  if (!s) return PC_ERR_INVALID_ARG;
  // every submitted request is admitted and finished first
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.wait(lk, [&] { return s->queue.empty(); });
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->admitter.joinable()) s->admitter.join();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  pc_batch_destroy(s->batch);
  pc_destroy(s->ctx);
  for (auto& kv : s->all) delete kv.second;
  delete s;
  return PC_OK;
}

}  // extern "C"
