// serve.cu -- the serving loop: frame requests of mixed size and effect, admitted as
// slots free up, grouped into batched launches, with per-request latency records.
//
// A slot is the device state one batch needs: per_effect contexts per effect (level
// pyramids, work lists, sub-images -- resident for the server's lifetime), a stream and a
// batch object.  The number of slots is bounded by the configuration and by free device
// memory (slots are created until the next one would eat into the reserve).  A scheduler
// thread takes pending requests in arrival order, packs up to per_effect requests of each
// effect into a batch (one persistent shading launch for all of them), orders the batch's
// contexts by effect and index so that a given set of contexts always forms the same
// topology, enqueues it on a free slot's stream as a graph keyed on that topology (see
// mrr_batch_enqueue_graph) and records an event; it polls the events of busy slots and
// completes their requests.  Requests that arrive while others run are dispatched as
// soon as a slot frees, so work of different requests overlaps on the device.
// mrr_submit / mrr_poll / mrr_wait are thread-safe.  Test mode (mock_device_us > 0)
// runs the same scheduler without a GPU: a batch "completes" after that many
// microseconds of host time.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mrr_internal.cuh"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Req {
  uint64_t ticket;
  mrr_request r;
  mrr_status result = MRR_OK;
  bool done = false;
  int64_t submit_ns = 0, start_ns = 0, done_ns = 0;
  float device_ms = 0.f;
};

constexpr int MAX_PER_EFFECT = 8;

struct Slot {
  mrr_ctx* ctx[3][MAX_PER_EFFECT] = {};
  cudaStream_t stream = nullptr;
  mrr_batch* batch = nullptr;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  bool busy = false;
  std::vector<uint64_t> tickets;
  int64_t mock_done_ns = 0;
};

}  // namespace

struct mrr_server {
  mrr_server_config cfg;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending;
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  int device = 0;
  uint64_t batches = 0, completed = 0;
};

namespace {

bool mock(const mrr_server* s) { return s->cfg.mock_device_us > 0; }

void destroy_slot(Slot& sl) {
  for (auto& row : sl.ctx)
    for (auto& c : row) mrr_destroy(c);
  if (sl.batch) mrr_batch_destroy(sl.batch);
  if (sl.ev_start) cudaEventDestroy(sl.ev_start);
  if (sl.ev_done) cudaEventDestroy(sl.ev_done);
  if (sl.stream) cudaStreamDestroy(sl.stream);
  sl = Slot();
}

mrr_status create_slot(const mrr_server_config& cfg, Slot& sl) {
  for (int e = 0; e < 3; ++e) {
    if (!cfg.effect_enabled[e]) continue;
    mrr_config c = cfg.effect_cfg[e];
    c.effect = (mrr_effect)e;
    c.no_graph = 1;
    for (int k = 0; k < cfg.per_effect; ++k) {
      mrr_status st = mrr_create(&c, &sl.ctx[e][k]);
      if (st != MRR_OK) return st;
    }
  }
  if (mrr_batch_create(&sl.batch) != MRR_OK) return MRR_ENOMEM;
  if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) return MRR_ECUDA;
  if (cudaEventCreate(&sl.ev_start) != cudaSuccess || cudaEventCreate(&sl.ev_done) != cudaSuccess) return MRR_ECUDA;
  return MRR_OK;
}

// Complete the requests of a slot whose batch has finished.  Caller holds the lock.
void finish_slot(mrr_server* s, Slot& sl, mrr_status st) {
  float ms = 0.f;
  if (!mock(s) && st == MRR_OK) cudaEventElapsedTime(&ms, sl.ev_start, sl.ev_done);
  const int64_t t = now_ns();
  for (uint64_t tk : sl.tickets) {
    auto it = s->reqs.find(tk);
    if (it == s->reqs.end()) continue;
    it->second.done = true;
    it->second.result = st;
    it->second.done_ns = t;
    it->second.device_ms = ms;
    ++s->completed;
  }
  sl.tickets.clear();
  sl.busy = false;
  s->cv_done.notify_all();
}

// Pack pending requests into a batch for slot `sl` (at most per_effect of each effect, in
// arrival order, skipping requests whose effect is full) and enqueue it.  The batch lists
// its contexts by effect, then index.  Caller holds the lock.
void dispatch(mrr_server* s, Slot& sl) {
  const int per = s->cfg.per_effect;
  uint64_t chosen[3][MAX_PER_EFFECT];
  int count[3] = {0, 0, 0};
  int n = 0;
  const int64_t t_dispatch = now_ns();  // one dispatch time for the whole batch
  for (auto it = s->pending.begin(); it != s->pending.end() && n < mrr::MAX_BATCH;) {
    Req& q = s->reqs[*it];
    const int e = (int)q.r.effect;
    if (count[e] >= per) {
      ++it;
      continue;
    }
    chosen[e][count[e]++] = q.ticket;
    q.start_ns = t_dispatch;
    sl.tickets.push_back(q.ticket);
    ++n;
    it = s->pending.erase(it);
  }
  if (n == 0) return;
  mrr_ctx* ctxs[mrr::MAX_BATCH];
  mrr_gbuffer frames[mrr::MAX_BATCH];
  float* outs[mrr::MAX_BATCH];
  int k = 0;
  for (int e = 0; e < 3; ++e)
    for (int j = 0; j < count[e]; ++j) {
      const Req& q = s->reqs[chosen[e][j]];
      ctxs[k] = sl.ctx[e][j];
      frames[k] = q.r.frame;
      outs[k] = q.r.out_dev;
      ++k;
    }
  sl.busy = true;
  ++s->batches;
  if (mock(s)) {
    sl.mock_done_ns = now_ns() + (int64_t)s->cfg.mock_device_us * 1000;
    return;
  }
  cudaEventRecord(sl.ev_start, sl.stream);
  mrr_status st = s->cfg.direct_launches ? mrr_batch_enqueue_direct(sl.batch, ctxs, frames, outs, n, sl.stream)
                                         : mrr_batch_enqueue_graph(sl.batch, ctxs, frames, outs, n, sl.stream);
  cudaEventRecord(sl.ev_done, sl.stream);
  if (st != MRR_OK) finish_slot(s, sl, st);
}

void worker_loop(mrr_server* s) {
  if (!mock(s)) cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (!s->stop) {
    bool any_busy = false;
    for (Slot& sl : s->slots) {
      if (!sl.busy) continue;
      bool fin;
      if (mock(s)) fin = now_ns() >= sl.mock_done_ns;
      else fin = cudaEventQuery(sl.ev_done) != cudaErrorNotReady;
      if (fin) finish_slot(s, sl, MRR_OK);
      else any_busy = true;
    }
    for (Slot& sl : s->slots)
      if (!sl.busy && !s->pending.empty()) dispatch(s, sl);
    for (Slot& sl : s->slots) any_busy = any_busy || sl.busy;
    if (any_busy) {
      // poll completions at fine granularity while the device works
      s->cv_work.wait_for(lock, std::chrono::microseconds(20));
    } else {
      s->cv_work.wait(lock, [s] { return s->stop || !s->pending.empty(); });
    }
  }
}

}  // namespace

extern "C" {

mrr_status mrr_server_create(const mrr_server_config* cfg, mrr_server** out) {
  if (!out) return MRR_EINVAL;
  *out = nullptr;
  if (!cfg) return MRR_EINVAL;
  int enabled = 0;
  for (int e = 0; e < 3; ++e) enabled += cfg->effect_enabled[e] ? 1 : 0;
  if (!enabled || cfg->slots < 0 || cfg->max_queue < 0 || cfg->per_effect < 0) return MRR_EINVAL;
  const int per = cfg->per_effect ? cfg->per_effect : 2;
  if (per > MAX_PER_EFFECT || per * enabled > mrr::MAX_BATCH) return MRR_EINVAL;
  for (int e = 0; e < 3; ++e)  // requests are served in batches, which take no pyramid gathers
    if (cfg->effect_enabled[e] && (cfg->effect_cfg[e].pyramid_gathers || cfg->effect_cfg[e].disjoint))
      return MRR_EUNSUPPORTED;
  mrr_server* s = new (std::nothrow) mrr_server();
  if (!s) return MRR_ENOMEM;
  s->cfg = *cfg;
  if (s->cfg.slots == 0) s->cfg.slots = 4;
  if (s->cfg.max_queue == 0) s->cfg.max_queue = 1024;
  s->cfg.per_effect = per;
  if (mock(s)) {
    s->slots.resize(s->cfg.slots);
  } else {
    cudaGetDevice(&s->device);
    // create slots while free device memory stays above the reserve
    for (int k = 0; k < s->cfg.slots; ++k) {
      size_t free0 = 0, total = 0;
      if (cudaMemGetInfo(&free0, &total) != cudaSuccess) break;
      Slot sl;
      mrr_status st = create_slot(s->cfg, sl);
      size_t free1 = 0;
      cudaMemGetInfo(&free1, &total);
      if (st != MRR_OK || free1 < s->cfg.hbm_reserve) {
        destroy_slot(sl);
        if (k == 0) {
          delete s;
          return st != MRR_OK ? st : MRR_ENOMEM;
        }
        break;
      }
      s->slots.push_back(sl);
      const size_t cost = free0 > free1 ? free0 - free1 : 0;
      if (free1 < s->cfg.hbm_reserve + cost) break;  // the next slot would not fit
    }
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return MRR_OK;
}

void mrr_server_destroy(mrr_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (!mock(s)) {
    for (Slot& sl : s->slots)
      if (sl.stream) cudaStreamSynchronize(sl.stream);
    for (Slot& sl : s->slots) destroy_slot(sl);
  }
  delete s;
}

int mrr_server_slots(mrr_server* s) { return s ? (int)s->slots.size() : 0; }

mrr_status mrr_submit(mrr_server* s, const mrr_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return MRR_EINVAL;
  const int e = (int)r->effect;
  if (e < 0 || e > 2 || !s->cfg.effect_enabled[e]) return MRR_EINVAL;
  const mrr_config& c = s->cfg.effect_cfg[e];
  if (r->frame.width < 1 || r->frame.height < 1 || r->frame.width > c.max_width || r->frame.height > c.max_height)
    return MRR_EINVAL;
  if (!mock(s) && (!r->out_dev || !r->frame.depth || !r->frame.normal)) return MRR_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if ((int)s->pending.size() >= s->cfg.max_queue) return MRR_EBUSY;
  const uint64_t t = s->next_ticket++;
  Req q;
  q.ticket = t;
  q.r = *r;
  q.submit_ns = now_ns();
  s->reqs.emplace(t, q);
  s->pending.push_back(t);
  *ticket = t;
  s->cv_work.notify_one();
  return MRR_OK;
}

mrr_status mrr_poll(mrr_server* s, uint64_t ticket, int* done, mrr_status* result) {
  if (!s || !done) return MRR_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return MRR_EINVAL;
  *done = it->second.done ? 1 : 0;
  if (result) *result = it->second.result;
  return MRR_OK;
}

mrr_status mrr_wait(mrr_server* s, uint64_t ticket, int64_t timeout_ns) {
  if (!s) return MRR_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return MRR_EINVAL;
  const auto pred = [&] { return s->reqs[ticket].done; };
  if (timeout_ns < 0) {
    s->cv_done.wait(lock, pred);
  } else if (!s->cv_done.wait_for(lock, std::chrono::nanoseconds(timeout_ns), pred)) {
    return MRR_ETIMEDOUT;
  }
  return s->reqs[ticket].result;
}

mrr_status mrr_request_info(mrr_server* s, uint64_t ticket, mrr_request_info_t* out) {
  if (!s || !out) return MRR_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return MRR_EINVAL;
  const Req& q = it->second;
  out->done = q.done ? 1 : 0;
  out->result = q.result;
  out->submit_ns = q.submit_ns;
  out->start_ns = q.start_ns;
  out->done_ns = q.done_ns;
  out->device_ms = q.device_ms;
  return MRR_OK;
}

mrr_status mrr_server_stats(mrr_server* s, mrr_server_stats_t* out) {
  if (!s || !out) return MRR_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  out->batches = s->batches;
  out->completed = s->completed;
  out->graph_instantiations = out->graph_updates = 0;
  for (const Slot& sl : s->slots) {
    uint64_t inst = 0, upd = 0;
    if (sl.batch) mrr_batch_graph_counts(sl.batch, &inst, &upd);
    out->graph_instantiations += inst;
    out->graph_updates += upd;
  }
  return MRR_OK;
}

mrr_status mrr_release(mrr_server* s, uint64_t ticket) {
  if (!s) return MRR_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end() || !it->second.done) return MRR_EINVAL;
  s->reqs.erase(it);
  return MRR_OK;
}

}  // extern "C"
