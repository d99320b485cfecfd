// serve.cu -- online serving of PIR queries over resident databases.
//
// Requests for registered targets (a context, one of its databases and the
// query compression factor) are queued on the host and answered by one
// worker thread per context ("lane").  Continuous batching: whenever a lane
// is free it takes the waiting requests of the target whose oldest request
// has waited longest, up to the largest power of two that is at most the
// configured maximum and whose answer plan fits in free device memory
// (cached plans of the context are released when nothing fits), and
// answers them in one batched call replayed from a CUDA graph; requests
// that arrive meanwhile wait for the next batch.  Lanes of different
// contexts run concurrently on their own streams.  Every response is the
// response of cwpir_answer for the same query.
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
  uint32_t lane = 0;
  uint64_t q_words = 0, r_words = 0;
  std::deque<SrvRequest *> waiting;
};

struct SrvLane {
  cwpir_ctx *ctx = nullptr;
  int device = 0;
  cudaStream_t st = nullptr;
  std::thread th;
  uint64_t *d_q = nullptr, *d_r = nullptr, *h_q = nullptr, *h_r = nullptr;
  uint64_t q_cap = 0, r_cap = 0;  // words
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
  uint32_t max_batch = 16, max_pending = 1024, n_pending = 0;
  uint64_t reserve = 0;
  cwpir_server_stats stats{};
};

namespace {

uint32_t pow2_floor(uint32_t x) {
  uint32_t p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

// Largest power-of-two batch <= want whose plan fits in free memory.
uint32_t admit(cwpir_server *s, const SrvTarget &tg, uint32_t want) {
  for (int pass = 0; pass < 2; ++pass) {
    for (uint32_t b = pow2_floor(want); b >= 1; b /= 2) {
      uint64_t need = 0;
      if (cwpir_plan_bytes(tg.t.ctx, tg.t.db_id, b, tg.t.c, &need) != CWPIR_OK) continue;
      if (need == 0) return b;
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
      if (need + s->reserve <= free_b) return b;
    }
    // nothing fits: drop this context's cached plans and retry once
    cwpir_release_plans(tg.t.ctx, -1);
  }
  return 0;
}

void lane_loop(cwpir_server *s, uint32_t lane_id) {
  SrvLane &ln = *s->lanes[lane_id];
  cudaSetDevice(ln.device);
  for (;;) {
    std::vector<SrvRequest *> batch;
    uint32_t ti = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto has_work = [&] {
        for (const auto &t : s->targets)
          if (t.lane == lane_id && !t.waiting.empty()) return true;
        return false;
      };
      s->cv_work.wait(lk, [&] { return s->stop || has_work(); });
      if (s->stop && !has_work()) return;
      double oldest = 1e300;
      for (uint32_t i = 0; i < s->targets.size(); ++i) {
        const auto &t = s->targets[i];
        if (t.lane == lane_id && !t.waiting.empty() && t.waiting.front()->t_submit < oldest) {
          oldest = t.waiting.front()->t_submit;
          ti = i;
        }
      }
    }
    SrvTarget &tg = s->targets[ti];
    uint32_t want;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      want = (uint32_t)std::min<size_t>(tg.waiting.size(), s->max_batch);
    }
    // admission by free device memory (outside the lock: may wait for the GPU)
    uint32_t b = admit(s, tg, want);
    if (b == 0) b = 1;  // nothing else can free memory for this lane: try alone
    {
      std::lock_guard<std::mutex> lk(s->mu);
      b = std::min<uint32_t>(b, (uint32_t)tg.waiting.size());
      for (uint32_t i = 0; i < b; ++i) {
        batch.push_back(tg.waiting.front());
        tg.waiting.pop_front();
      }
    }
    if (batch.empty()) continue;
    for (uint32_t i = 0; i < b; ++i)
      memcpy(ln.h_q + i * tg.q_words, batch[i]->query.data(), tg.q_words * sizeof(uint64_t));
    double t0 = now_s();
    int rc = CWPIR_OK;
    cudaError_t e = cudaMemcpyAsync(ln.d_q, ln.h_q, b * tg.q_words * sizeof(uint64_t),
                                    cudaMemcpyHostToDevice, ln.st);
    if (e != cudaSuccess) rc = CWPIR_ECUDA;
    if (rc == CWPIR_OK)
      rc = cwpir_answer_batch_device(ln.ctx, tg.t.db_id, tg.t.c, b, ln.d_q, ln.d_r, ln.st);
    if (rc == CWPIR_OK &&
        cudaMemcpyAsync(ln.h_r, ln.d_r, b * tg.r_words * sizeof(uint64_t),
                        cudaMemcpyDeviceToHost, ln.st) != cudaSuccess)
      rc = CWPIR_ECUDA;
    if (cudaStreamSynchronize(ln.st) != cudaSuccess && rc == CWPIR_OK) rc = CWPIR_ECUDA;
    double t1 = now_s();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (uint32_t i = 0; i < b; ++i) {
        SrvRequest *r = batch[i];
        if (rc == CWPIR_OK) {
          r->resp.assign(ln.h_r + i * tg.r_words, ln.h_r + (i + 1) * tg.r_words);
          r->status = 1;
        } else {
          r->status = rc;
        }
        r->t_done = t1;
      }
      s->n_pending -= b;
      s->stats.completed += b;
      s->stats.batches += 1;
      s->stats.max_batch_seen = std::max<uint64_t>(s->stats.max_batch_seen, b);
      s->stats.busy_s += t1 - t0;
    }
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

int cwpir_server_create(const cwpir_target *targets, uint32_t n_targets, uint32_t max_batch,
                        uint64_t hbm_reserve_bytes, uint32_t max_pending, cwpir_server **out) {
  if (!targets || !n_targets || !out || max_batch < 1 || max_pending < 1) return CWPIR_EINVAL;
  std::unique_ptr<cwpir_server> s(new cwpir_server());
  s->max_batch = max_batch;
  s->max_pending = max_pending;
  s->reserve = hbm_reserve_bytes;
  std::map<cwpir_ctx *, uint32_t> lane_of;
  for (uint32_t i = 0; i < n_targets; ++i) {
    SrvTarget tg;
    tg.t = targets[i];
    uint32_t N = 0, L = 0, m = 0, sp = 1, h = 0;
    if (!tg.t.ctx || cwpir_db_shape(tg.t.ctx, tg.t.db_id, &N, &L, &m) != CWPIR_OK ||
        cwpir_db_plaintexts(tg.t.ctx, tg.t.db_id, &sp) != CWPIR_OK ||
        cwpir_query_cts(tg.t.ctx, tg.t.db_id, tg.t.c, &h) != CWPIR_OK)
      return CWPIR_EINVAL;
    tg.q_words = (uint64_t)h * 2ull * L * N;
    tg.r_words = (uint64_t)sp * 2ull * L * N;
    auto it = lane_of.find(tg.t.ctx);
    if (it == lane_of.end()) {
      it = lane_of.emplace(tg.t.ctx, (uint32_t)s->lanes.size()).first;
      s->lanes.emplace_back(new SrvLane());
      s->lanes.back()->ctx = tg.t.ctx;
    }
    tg.lane = it->second;
    SrvLane &ln = *s->lanes[tg.lane];
    ln.q_cap = std::max<uint64_t>(ln.q_cap, tg.q_words * max_batch);
    ln.r_cap = std::max<uint64_t>(ln.r_cap, tg.r_words * max_batch);
    s->targets.push_back(tg);
  }
  for (auto &lp : s->lanes) {
    SrvLane &ln = *lp;
    if (cwpir_ctx_device(ln.ctx, &ln.device) != CWPIR_OK) return CWPIR_EINVAL;
    cudaSetDevice(ln.device);
    cwpir_set_option(ln.ctx, CWPIR_OPT_USE_GRAPH, 1);
    if (cudaStreamCreateWithFlags(&ln.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&ln.d_q, ln.q_cap * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&ln.d_r, ln.r_cap * sizeof(uint64_t)) != cudaSuccess ||
        cudaMallocHost(&ln.h_q, ln.q_cap * sizeof(uint64_t)) != cudaSuccess ||
        cudaMallocHost(&ln.h_r, ln.r_cap * sizeof(uint64_t)) != cudaSuccess) {
      cwpir_server_destroy(s.release());
      return CWPIR_ENOMEM;
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
    if (s->n_pending >= s->max_pending) {
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

static int take_result(cwpir_server *s, std::unordered_map<uint64_t, std::unique_ptr<SrvRequest>>::iterator it,
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
    cudaSetDevice(ln.device);
    if (ln.st) cudaStreamSynchronize(ln.st);
    if (ln.d_q) cudaFree(ln.d_q);
    if (ln.d_r) cudaFree(ln.d_r);
    if (ln.h_q) cudaFreeHost(ln.h_q);
    if (ln.h_r) cudaFreeHost(ln.h_r);
    if (ln.st) cudaStreamDestroy(ln.st);
  }
  delete s;
}

}  // extern "C"
