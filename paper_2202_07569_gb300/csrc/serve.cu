// serve.cu -- online serving of PIR queries over resident databases.
//
// Requests for registered targets (a context, one of its databases and the
// query compression factor) are queued on the host and answered by worker
// lanes.  Every target has lanes_per_target lanes; a lane is a host thread
// with its own stream, its own scratch slot on the target's context
// (cwpir_slot_create) and its own staging buffers, so the lanes of all
// targets run at the same time and their kernels overlap on the device.
// Continuous batching: whenever a lane is free it takes the waiting
// requests of its target, up to the largest power of two that is at most
// the configured maximum and whose answer plan fits in free device memory
// (the target's cached plans are released when nothing fits), and answers
// them in one batched call replayed from a CUDA graph.  A request that
// arrives while a lane is busy starts at once on an idle lane of its target
// or, when all of them are busy, with the next batch of the first lane to
// finish.  Every response is the response of cwpir_answer for the same
// query; after each batch the lane reads its slot's device check flag, and
// a failed check fails the batch's requests with CWPIR_EINTERNAL.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cwpir.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct SrvRequest {
  uint64_t ticket = 0;
  uint32_t target = 0;
  std::vector<uint64_t> query, resp;
  int status = 0;  // 0 waiting or running, 1 done, < 0 error code
  double t_submit = 0, t_done = 0;
};

struct SrvTarget {
  cwpir_target t;
  int device = 0;
  uint64_t q_words = 0, r_words = 0;
  std::deque<SrvRequest *> waiting;
};

struct SrvLane {
  uint32_t target = 0, slot = 0;
  cudaStream_t st = nullptr;
  std::thread th;
  uint64_t *d_q = nullptr, *d_r = nullptr, *h_q = nullptr, *h_r = nullptr;
};

}  // namespace

struct cwpir_server {
  std::vector<SrvTarget> targets;
  std::vector<std::unique_ptr<SrvLane>> lanes;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::unordered_map<uint64_t, std::unique_ptr<SrvRequest>> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  cwpir_server_config cfg{};
  uint32_t n_pending = 0, running = 0;
  cwpir_server_stats stats{};
};

namespace {

uint32_t pow2_floor(uint32_t x) {
  uint32_t p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

// Largest power-of-two batch <= want whose plan on the lane's slot fits in
// free device memory minus the reserve; 0 if none does, even after the
// target's cached plans were released.
uint32_t admit(cwpir_server *s, const SrvTarget &tg, const SrvLane &ln, uint32_t want) {
  for (int pass = 0; pass < 2; ++pass) {
    for (uint32_t b = pow2_floor(want); b >= 1; b /= 2) {
      uint64_t need = 0;
      if (cwpir_plan_bytes_slot(tg.t.ctx, ln.slot, tg.t.db_id, b, tg.t.c, &need) != CWPIR_OK)
        continue;
      if (need == 0) return b;
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
      if (need + s->cfg.hbm_reserve_bytes <= free_b) return b;
    }
    cwpir_release_plans(tg.t.ctx, tg.t.db_id);
  }
  return 0;
}

// One batch of b requests on a lane: staging, the batched answer on the
// lane's slot, the response copy and the slot's device check.
int run_batch(SrvLane &ln, const SrvTarget &tg, const std::vector<SrvRequest *> &batch) {
  const uint32_t b = (uint32_t)batch.size();
  for (uint32_t i = 0; i < b; ++i)
    memcpy(ln.h_q + i * tg.q_words, batch[i]->query.data(), tg.q_words * sizeof(uint64_t));
  if (cudaMemcpyAsync(ln.d_q, ln.h_q, b * tg.q_words * sizeof(uint64_t), cudaMemcpyHostToDevice,
                      ln.st) != cudaSuccess)
    return CWPIR_ECUDA;
  int rc = cwpir_answer_batch_slot(tg.t.ctx, ln.slot, tg.t.db_id, tg.t.c, b, ln.d_q, ln.d_r,
                                   ln.st);
  if (rc == CWPIR_OK &&
      cudaMemcpyAsync(ln.h_r, ln.d_r, b * tg.r_words * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                      ln.st) != cudaSuccess)
    rc = CWPIR_ECUDA;
  // waits for the lane's stream and reads (and clears) the slot's flag, so
  // that a failed check fails this batch and no later one
  const int st = cwpir_device_status(tg.t.ctx, ln.slot, ln.st);
  return rc != CWPIR_OK ? rc : st;
}

void lane_loop(cwpir_server *s, uint32_t lane_id) {
  SrvLane &ln = *s->lanes[lane_id];
  SrvTarget &tg = s->targets[ln.target];
  cudaSetDevice(tg.device);
  for (;;) {
    uint32_t want;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !tg.waiting.empty(); });
      if (tg.waiting.empty()) return;  // stopping with nothing left
      want = (uint32_t)std::min<size_t>(tg.waiting.size(), s->cfg.max_batch);
    }
    // admission by free device memory (outside the lock: may wait for the GPU)
    uint32_t b = admit(s, tg, ln, want);
    if (b == 0) b = 1;  // nothing else can free memory for this lane: try alone
    std::vector<SrvRequest *> batch;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      b = std::min<uint32_t>(b, (uint32_t)tg.waiting.size());
      for (uint32_t i = 0; i < b; ++i) {
        batch.push_back(tg.waiting.front());
        tg.waiting.pop_front();
      }
      if (!batch.empty()) {
        s->running += 1;
        s->stats.max_concurrent = std::max<uint64_t>(s->stats.max_concurrent, s->running);
      }
    }
    if (batch.empty()) continue;  // another lane of the target took them
    const double t0 = now_s();
    const int rc = run_batch(ln, tg, batch);
    const double t1 = now_s();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (uint32_t i = 0; i < batch.size(); ++i) {
        SrvRequest *r = batch[i];
        if (rc == CWPIR_OK) {
          r->resp.assign(ln.h_r + i * tg.r_words, ln.h_r + (i + 1) * tg.r_words);
          r->status = 1;
        } else {
          r->status = rc;
        }
        r->t_done = t1;
      }
      s->running -= 1;
      s->n_pending -= (uint32_t)batch.size();
      s->stats.completed += batch.size();
      s->stats.batches += 1;
      s->stats.max_batch_seen = std::max<uint64_t>(s->stats.max_batch_seen, batch.size());
      s->stats.busy_s += t1 - t0;
      if (rc != CWPIR_OK) s->stats.failed += batch.size();
    }
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

int cwpir_server_create(const cwpir_target *targets, uint32_t n_targets,
                        const cwpir_server_config *cfg, cwpir_server **out) {
  if (!targets || !n_targets || !cfg || !out || cfg->max_batch < 1 ||
      cfg->lanes_per_target < 1 || cfg->lanes_per_target > 16 || cfg->max_pending < 1)
    return CWPIR_EINVAL;
  std::unique_ptr<cwpir_server> s(new cwpir_server());
  s->cfg = *cfg;
  for (uint32_t i = 0; i < n_targets; ++i) {
    SrvTarget tg;
    tg.t = targets[i];
    uint32_t N = 0, L = 0, m = 0, sp = 1, h = 0;
    if (!tg.t.ctx || cwpir_db_shape(tg.t.ctx, tg.t.db_id, &N, &L, &m) != CWPIR_OK ||
        cwpir_db_plaintexts(tg.t.ctx, tg.t.db_id, &sp) != CWPIR_OK ||
        cwpir_query_cts(tg.t.ctx, tg.t.db_id, tg.t.c, &h) != CWPIR_OK ||
        cwpir_ctx_device(tg.t.ctx, &tg.device) != CWPIR_OK)
      return CWPIR_EINVAL;
    tg.q_words = (uint64_t)h * 2ull * L * N;
    tg.r_words = (uint64_t)sp * 2ull * L * N;
    s->targets.push_back(tg);
  }
  for (uint32_t i = 0; i < n_targets; ++i) {
    const SrvTarget &tg = s->targets[i];
    cwpir_set_option(tg.t.ctx, CWPIR_OPT_USE_GRAPH, 1);
    for (uint32_t k = 0; k < cfg->lanes_per_target; ++k) {
      std::unique_ptr<SrvLane> ln(new SrvLane());
      ln->target = i;
      cudaSetDevice(tg.device);
      const uint64_t qb = tg.q_words * cfg->max_batch * sizeof(uint64_t);
      const uint64_t rb = tg.r_words * cfg->max_batch * sizeof(uint64_t);
      int rc = cwpir_slot_create(tg.t.ctx, &ln->slot);
      if (rc != CWPIR_OK) return rc;
      const bool ok = cudaStreamCreateWithFlags(&ln->st, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaMalloc(&ln->d_q, qb) == cudaSuccess &&
                      cudaMalloc(&ln->d_r, rb) == cudaSuccess &&
                      cudaMallocHost(&ln->h_q, qb) == cudaSuccess &&
                      cudaMallocHost(&ln->h_r, rb) == cudaSuccess;
      s->lanes.push_back(std::move(ln));
      if (!ok) {
        cwpir_server_destroy(s.release());
        return CWPIR_ENOMEM;
      }
    }
  }
  for (uint32_t i = 0; i < s->lanes.size(); ++i)
    s->lanes[i]->th = std::thread(lane_loop, s.get(), i);
  *out = s.release();
  return CWPIR_OK;
}

int cwpir_submit(cwpir_server *s, uint32_t target, const uint64_t *query, uint64_t *ticket) {
  if (!s || !query || !ticket || target >= s->targets.size()) return CWPIR_EINVAL;
  std::unique_ptr<SrvRequest> r(new SrvRequest());
  r->target = target;
  r->query.assign(query, query + s->targets[target].q_words);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return CWPIR_EINVAL;
    if (s->n_pending >= s->cfg.max_pending) {
      s->stats.rejected_busy += 1;
      return CWPIR_EBUSY;
    }
    r->ticket = s->next_ticket++;
    r->t_submit = now_s();
    *ticket = r->ticket;
    s->targets[target].waiting.push_back(r.get());
    s->n_pending += 1;
    s->stats.submitted += 1;
    s->reqs.emplace(r->ticket, std::move(r));
  }
  s->cv_work.notify_all();
  return CWPIR_OK;
}

static int take_result(cwpir_server *s,
                       std::unordered_map<uint64_t, std::unique_ptr<SrvRequest>>::iterator it,
                       uint64_t *response, int32_t *status, double *latency_s) {
  SrvRequest *r = it->second.get();
  *status = r->status;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  if (r->status == 1 && response)
    memcpy(response, r->resp.data(), r->resp.size() * sizeof(uint64_t));
  s->reqs.erase(it);
  return CWPIR_OK;
}

int cwpir_poll(cwpir_server *s, uint64_t ticket, uint64_t *response, int32_t *status,
               double *latency_s) {
  if (!s || !status) return CWPIR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return CWPIR_EINVAL;
  if (it->second->status == 0) {
    *status = 0;
    return CWPIR_OK;
  }
  return take_result(s, it, response, status, latency_s);
}

int cwpir_wait(cwpir_server *s, uint64_t ticket, uint64_t *response, int32_t *status,
               double *latency_s, double timeout_s) {
  if (!s || !status) return CWPIR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return CWPIR_EINVAL;
  SrvRequest *r = it->second.get();
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [&] { return r->status != 0; });
  if (!ok) {
    *status = 0;
    return CWPIR_ETIMEDOUT;
  }
  return take_result(s, s->reqs.find(ticket), response, status, latency_s);
}

int cwpir_server_get_stats(cwpir_server *s, cwpir_server_stats *out) {
  if (!s || !out) return CWPIR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return CWPIR_OK;
}

void cwpir_server_destroy(cwpir_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &lp : s->lanes)
    if (lp->th.joinable()) lp->th.join();
  for (auto &lp : s->lanes) {
    SrvLane &ln = *lp;
    cudaSetDevice(s->targets[ln.target].device);
    if (ln.st) cudaStreamSynchronize(ln.st);
    if (ln.d_q) cudaFree(ln.d_q);
    if (ln.d_r) cudaFree(ln.d_r);
    if (ln.h_q) cudaFreeHost(ln.h_q);
    if (ln.h_r) cudaFreeHost(ln.h_r);
    if (ln.st) cudaStreamDestroy(ln.st);
    if (ln.slot) cwpir_slot_release(s->targets[ln.target].t.ctx, ln.slot);
  }
  delete s;
}

}  // extern "C"
