// cwpir.cu -- host side of the C ABI (include/cwpir.h): parameter tables,
// contexts, database plans and the launch sequence of the answer path
// (arXiv 2202.07569, Sec. 3.3).  All arithmetic of the path runs in the
// kernels of kernels.cu; this file validates, plans and enqueues.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <memory>
#include <new>
#include <tuple>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/cwpir.h"
#include "host_tables.hpp"
#include "kernels.cuh"

using cw::u32;
using cw::u64;
using namespace cw::host;

namespace {

thread_local std::string g_setup_error;

}  // namespace

// ---------------------------------------------------------------------
// Context and database state
// ---------------------------------------------------------------------
// Device bytes a context holds in its buffers and the cap set by
// CWPIR_OPT_MEM_LIMIT (0: none).  A buffer that would pass the cap is
// refused as cudaErrorMemoryAllocation, i.e. CWPIR_ENOMEM, before any
// cudaMalloc.
struct MemAcct {
  u64 used = 0, limit = 0;
};

struct DevBuf {
  u64 *p = nullptr;
  size_t n = 0;  // u64 count
  MemAcct *acct = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      if (acct) acct->used -= n * sizeof(u64);
    }
    p = nullptr;
    n = 0;
  }
  cudaError_t ensure(size_t count, MemAcct *a) {
    if (count <= n) return cudaSuccess;
    release();
    acct = a;
    if (a && a->limit && a->used + count * sizeof(u64) > a->limit)
      return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&p, count * sizeof(u64));
    if (e == cudaSuccess) {
      n = count;
      if (a) a->used += count * sizeof(u64);
    } else {
      p = nullptr;
    }
    return e;
  }
};

struct Chunk {
  u64 off;    // offset into the plan's job array
  u32 count;  // jobs in the launch
  int mode;   // cw::RootMode
  u32 segs;   // ROOT_PM: queries in the launch, count / segs jobs each
};

// One expansion round: `count` substitution jobs (all queries) at `off`.
struct ExpRound {
  u64 off;
  u32 count;
};

// The launch sequence of an answer for nq queries (slots) against one
// database: leaves, shared first-level products, the batches of tree
// levels, accumulators, and for compressed queries the expansion rounds.
// All device job lists are uploaded when the plan is built, so the
// sequence itself contains only kernel launches and device copies and can
// be captured into a CUDA graph.
struct Plan {
  u32 nq = 1, cfac = 0, k = 0, top = 0, m = 0, h_in = 0, sp = 1;
  bool memo = false, leaf_root = false;
  bool rows_db = false;  // the database is held in the row basis
  u64 n_memo = 0, mults = 0;
  std::vector<Chunk> memo_chunks;
  std::vector<std::vector<Chunk>> batches;  // per row batch, levels bottom-up
  std::vector<cw::MulJob> host_jobs;
  cw::MulJob *d_jobs = nullptr;
  DevBuf memo_buf, level_buf;
  DevBuf leaves;     // [nq][m] QP-NTT cts
  DevBuf acc;        // [nq][sp][2][L][N] NTT-form accumulators
  DevBuf q_in, resp; // graph staging: [nq][h_in] cts and [nq][sp][2][L][N]
  DevBuf exp_a, exp_b, exp_tau, exp_S, exp_DN, exp_O, leaves_coef;
  std::vector<ExpRound> exp_rounds;
  cw::SubJob *d_subjobs = nullptr;
  u64 *exp_final = nullptr;
  cudaGraphExec_t graph = nullptr;
  cwpir_stats graph_stats{};
  ~Plan() {
    if (graph) cudaGraphExecDestroy(graph);
    if (d_jobs) cudaFree(d_jobs);
    if (d_subjobs) cudaFree(d_subjobs);
  }
};

struct Db {
  u64 n = 0, n_pairs = 0;  // rows, distinct first-level position pairs
  u32 plen = 0, k = 0, m = 0;
  u32 sp = 1;                 // plaintexts per row (Sec. 3.3.1): ceil(plen / N)
  bool folklore = false;      // rows indexed by the plain folklore operator
  // One plaintext per row and k >= 2: the rows are held in the row basis
  // ([n][4][N] u32, NTT form modulo the first four extension primes; the
  // last tree level multiplies them exactly as integers).  Otherwise
  // [n][sp][L][N] u64, NTT form modulo the ciphertext primes.
  bool rows = false;
  DevBuf db;
  std::vector<uint16_t> cw;   // [n][k]
  // answer plans over all rows, by (queries per call, compression factor,
  // scratch slot)
  std::map<std::tuple<u32, u32, u32>, std::unique_ptr<Plan>> plans;
};

// Scratch of the multiplication kernels for one stream of answers at a
// time ("slot"): answers on different slots of one context may run
// concurrently on different streams.  Sized for c->jmax multiplications per
// launch, the same for every slot of a context.
struct Scratch {
  DevBuf Tbuf, E, CP, DN;  // tensor, scaled tensor, partial products, digit transforms
  DevBuf RS, DNQ;          // row-basis row sums and their Q-basis forms
  DevBuf SEL;  // NTT-form selection entries [jmax][2][L][N] (rows of several plaintexts)
  int *d_err = nullptr;    // device consistency flag of the slot's kernels
  bool in_use = true;      // false once released (slot 0 never is)
  ~Scratch() {
    if (d_err) cudaFree(d_err);
  }
  void release() {
    Tbuf.release();
    E.release();
    CP.release();
    DN.release();
    RS.release();
    DNQ.release();
    SEL.release();
  }
};

struct cwpir_ctx {
  MemAcct acct;  // first member: destroyed after every buffer that counts in it
  int device = 0;
  u32 N = 0, logN = 0, L = 0, K = 0;
  u64 t = 0;
  std::vector<u64> q, p;
  cw::DevTables h;          // host copy (device pointers inside)
  cw::DevTables *d_tab = nullptr;
  DevBuf twiddles;    // ciphertext primes: [L][4N] (value, Shoup) pairs
  DevBuf twiddles32;  // extension primes: [K][4N] 32-bit pairs
  DevBuf rlk, rlk_s;        // [L][2][L][N] NTT form and Shoup companions
  std::map<u32, std::pair<std::shared_ptr<DevBuf>, std::shared_ptr<DevBuf>>> gal;
  std::map<int32_t, std::unique_ptr<Db>> dbs;
  int32_t next_db = 1;
  std::string err;
  int opt_share = 1, opt_graph = 0;
  // internal tree nodes switch keys in the key-switch basis (DevTables ksr)
  // with the relinearisation key in that basis: [L][2][L][5][N] u32
  bool ksr = false;
  DevBuf ksr_key;
  u32 opt_batch_rows = 0;
  u32 opt_max_jobs = 0;
  int opt_row_basis = 1;
  cudaStream_t stream = nullptr;
  // scratch: jmax multiplications per launch (0: not sized yet), one
  // Scratch per slot (slot 0 serves every call without a slot argument);
  // scratch_gen counts re-sizings, so that objects holding captured graphs
  // over a slot's buffers notice them
  u32 jmax = 0;
  u64 scratch_gen = 0;
  std::vector<std::unique_ptr<Scratch>> slots;
  // buffers of the single-step host calls
  DevBuf exp_tau, exp_DN, exp_O, tmp_ct, io_in, io_out, one_job;
  // the arithmetic operator's operands, intermediates and plans, kept for
  // the next call with the same (m, k); dropped with the answer plans
  struct ArithCache {
    u32 m = 0, k = 0;
    DevBuf leaves, prods, fac, flag;
    Db d1, d2;
    std::unique_ptr<Plan> p1, p2;
    void clear() {
      p1.reset();
      p2.reset();
      m = k = 0;
    }
  } arith;
  bool capturing = false;
  // serialises the slot calls, which several threads may make on one context
  std::recursive_mutex mu;
  cw::SubJob *d_subjobs = nullptr;
  size_t n_subjobs = 0;
  cwpir_stats stats{};
  // kernel timing (CWPIR_OPT_KERNEL_TIMING)
  int opt_timing = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<size_t, size_t>>> ev_marks;
  size_t ev_used = 0;
  double kt_ms[CWPIR_K_CLASSES] = {};
  uint64_t kt_n[CWPIR_K_CLASSES] = {};
  ~cwpir_ctx() {
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    if (d_tab) cudaFree(d_tab);
    if (d_subjobs) cudaFree(d_subjobs);
    if (stream) cudaStreamDestroy(stream);
  }
  // u64 words of a QP-layout polynomial (L u64 limbs, K u32 limbs) and of a
  // QP-NTT ciphertext
  u64 qp_poly() const { return cw::qp_poly_words(L, K, N); }
  u64 qp_ct() const { return 2 * qp_poly(); }
  u64 ct() const { return 2ull * L * N; }
};

namespace {

int fail(cwpir_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_setup_error = buf;
  return code;
}

// Runs `launch` (returning cudaError_t); with kernel timing on, brackets it
// with two events on `st` and files the pair under `cls`.
template <typename F>
cudaError_t timed(cwpir_ctx *c, int cls, cudaStream_t st, F launch) {
  if (!c->opt_timing || c->capturing) return launch();
  while (c->ev_pool.size() < c->ev_used + 2) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    c->ev_pool.push_back(e);
  }
  size_t a = c->ev_used, b = c->ev_used + 1;
  c->ev_used += 2;
  cudaError_t r = cudaEventRecord(c->ev_pool[a], st);
  if (r == cudaSuccess) r = launch();
  if (r == cudaSuccess) r = cudaEventRecord(c->ev_pool[b], st);
  c->ev_marks.push_back({cls, {a, b}});
  return r;
}

#define CUDA_TRY(ctx, expr)                                                          \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? CWPIR_ENOMEM : CWPIR_ECUDA, \
                  "%s: %s", #expr, cudaGetErrorString(e_));                        \
  } while (0)

int build_tables(cwpir_ctx *c) {
  cw::DevTables &h = c->h;
  memset(&h, 0, sizeof h);
  h.N = c->N;
  h.logN = c->logN;
  h.L = c->L;
  h.K = c->K;
  h.t = c->t;
  {
    int sms = 0, thr = 0;
    CUDA_TRY(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    CUDA_TRY(c, cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, c->device));
    h.sms = (u32)sms;
    h.sm_threads = (u32)thr;
    h.row_waves = cw::kDefaultRowWaves;
  }
  {  // Delta = (Q - r) / t with r = Q mod t, so Delta = -r t^-1 (mod q_j)
    u64 r = 1;
    for (u64 qj : c->q) r = (u64)((u128)r * (qj % c->t) % c->t);
    for (u32 j = 0; j < c->L; ++j) {
      const u64 qj = c->q[j], v = cw::host::hmul(r % qj, cw::host::hinv(c->t % qj, qj), qj);
      h.delta[j] = v ? qj - v : 0;
    }
  }
  const u32 L = c->L, K = c->K, N = c->N;
  std::vector<u64> host(4ull * L * N);
  CUDA_TRY(c, c->twiddles.ensure(4ull * L * N, &c->acct));
  for (u32 l = 0; l < L; ++l) {
    u64 q = c->q[l];
    u64 *tw = host.data() + 4ull * l * N;
    if (!make_twiddles(q, N, c->logN, tw))
      return fail(c, CWPIR_EINTERNAL, "no 2N-th root of unity mod %llu", (unsigned long long)q);
    cw::NttPrime &pr = h.prime[l];
    pr.q = q;
    pr.mu = (u64)(((u128)1 << 116) / q);
    pr.ninv = hinv(N % q, q);
    pr.ninv_s = shoup_of(pr.ninv, q);
    u64 *d = c->twiddles.p + 4ull * l * N;
    pr.psi2 = d;
    pr.ipsi2 = d + 2 * N;
  }
  CUDA_TRY(c, cudaMemcpy(c->twiddles.p, host.data(), host.size() * sizeof(u64),
                         cudaMemcpyHostToDevice));
  std::vector<u32> host32(4ull * K * N);
  CUDA_TRY(c, c->twiddles32.ensure(2ull * K * N, &c->acct));  // 4KN 32-bit words
  u32 *d32 = reinterpret_cast<u32 *>(c->twiddles32.p);
  for (u32 k = 0; k < K; ++k) {
    const u64 p = c->p[k];
    if (!cw::host::make_twiddles32(p, N, c->logN, host32.data() + 4ull * k * N))
      return fail(c, CWPIR_EINTERNAL, "no 2N-th root of unity mod %llu", (unsigned long long)p);
    cw::ExtNtt &e = h.ext[k];
    e.e = cw::host::ext_prime(p);
    e.psi2 = d32 + 4ull * k * N;
    e.ipsi2 = d32 + 4ull * k * N + 2 * N;
  }
  CUDA_TRY(c, cudaMemcpy(d32, host32.data(), host32.size() * sizeof(u32),
                         cudaMemcpyHostToDevice));
  fill_lift(h.lift, c->q, c->p);
  fill_scale(h.scale, c->q, c->p, c->t, N);
  fill_scale_p(h.scalep, c->q, c->p, c->t, N);
  // row basis: three primes when a group of 32 rows or more fits, else four
  const u64 lim3 = row_group_limit(c->q, c->p, 3, N, c->t);
  const u32 nr = lim3 >= 32 ? 3 : 4;
  fill_rows(h.rows, c->q, c->p, N, nr);
  h.rows.rmax = (u32)std::min<u64>(row_group_limit(c->q, c->p, nr, N, c->t), 2048);
  if (h.rows.rmax < 32) return fail(c, CWPIR_EINTERNAL, "row basis too small");
  // key-switch basis: the first five extension primes, when there are five
  // and their product R holds |sum_i D_i key_ij| < L N q_max^2 with the
  // row-digit margin (|x| < (1 - 2^-23) R / 2)
  if (K >= cw::kKsrPrimes) {
    long double lr = 0;
    for (u32 k = 0; k < cw::kKsrPrimes; ++k) lr += log2l((long double)c->p[k]);
    const long double need = log2l((long double)L) + log2l((long double)N) +
                             2 * log2l((long double)*std::max_element(c->q.begin(), c->q.end()));
    if (lr - 1 + log2l(1.0L - 1.0L / (1 << 23)) > need) {
      fill_rows(h.ksr, c->q, c->p, N, cw::kKsrPrimes);
      c->ksr = true;
    }
  }
  CUDA_TRY(c, cudaMalloc(&c->d_tab, sizeof(cw::DevTables)));
  CUDA_TRY(c, cudaMemcpy(c->d_tab, &h, sizeof h, cudaMemcpyHostToDevice));
  return CWPIR_OK;
}

bool valid_residues(const u64 *v, u32 L, u32 N, const std::vector<u64> &q, u64 count) {
  for (u64 u = 0; u < count; ++u)
    for (u32 j = 0; j < L; ++j) {
      const u64 *x = v + (u * L + j) * N;
      for (u32 i = 0; i < N; ++i)
        if (x[i] >= q[j]) return false;
    }
  return true;
}

// A switching key to the device: NTT form modulo each q_j with Shoup
// companions (kb, ks) and, with ksr_out, also in the key-switch basis.
int upload_key(cwpir_ctx *c, const u64 *key, DevBuf &kb, DevBuf &ks, DevBuf *ksr_out) {
  const u64 words = 2ull * c->L * c->L * c->N;
  if (!valid_residues(key, c->L, c->N, c->q, 2ull * c->L))
    return fail(c, CWPIR_EINVAL, "switching key residue out of range");
  CUDA_TRY(c, kb.ensure(words, &c->acct));
  CUDA_TRY(c, ks.ensure(words, &c->acct));
  CUDA_TRY(c, cudaMemcpy(kb.p, key, words * sizeof(u64), cudaMemcpyHostToDevice));
  if (ksr_out) {  // from the coefficient form, before kb is transformed
    CUDA_TRY(c, ksr_out->ensure(words * cw::kKsrPrimes / 2, &c->acct));
    CUDA_TRY(c, cw::launch_ksr_key(c->d_tab, c->h, kb.p, reinterpret_cast<u32 *>(ksr_out->p),
                                   c->stream));
  }
  CUDA_TRY(c, cw::launch_key_prep(c->d_tab, c->h, kb.p, ks.p, 1, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return CWPIR_OK;
}

// ---- scratch ----
// Multiplications per launch: as many as kScratchBytes of per-job scratch
// allows, between 32 and kMaxJobs (larger launches measured faster: 96,
// 256, ~940 and ~1800 jobs per launch for the configuration-2 answer).
constexpr u64 kMaxJobs = 2048;
constexpr u64 kScratchBytes = 8ull << 30;
// Row groups finished at a time on row-basis databases.
constexpr u32 kRowGroups = 64;

// u64 words per job of the digit transforms: (L+2) L N for the ciphertext
// basis, 3L x nr x N u32 for the row basis of nr <= 4 primes
u64 dn_words(u64 L, u64 N) { return std::max<u64>((L + 2) * L, 6 * L) * N; }
// u64 words of the row-basis group buffers: row sums [kRowGroups][3L][nr][N]
// u32 and their Q-basis forms [kRowGroups][L+2][L][N]
u64 rs_words(u64 L, u64 N) { return (u64)kRowGroups * 6 * L * N; }
u64 dnq_words(u64 L, u64 N) { return (u64)kRowGroups * (L + 2) * L * N; }

// Multiplications per launch of a context: as many as kScratchBytes of
// per-job scratch allows, between 32 and kMaxJobs, at most
// CWPIR_OPT_MAX_JOBS when set.
u32 jobs_per_launch(const cwpir_ctx *c) {
  const u64 N = c->N, L = c->L;
  const u64 per_job =
      (3 * cw::tensor_poly_words(c->K, c->N) + (3 * L + 2 * L) * N + dn_words(L, N)) * sizeof(u64);
  u64 j = kScratchBytes / per_job;
  j = std::max<u64>(32, std::min<u64>(kMaxJobs, j));
  if (c->opt_max_jobs) j = std::min<u64>(j, c->opt_max_jobs);
  return (u32)j;
}

// A new slot (or a released one again) with its device flag cleared; its
// buffers come with the first ensure_scratch on it.
int add_slot(cwpir_ctx *c, u32 *id) {
  for (u32 i = 1; i < c->slots.size(); ++i)
    if (!c->slots[i]->in_use) {
      CUDA_TRY(c, cudaMemset(c->slots[i]->d_err, 0, sizeof(int)));
      c->slots[i]->in_use = true;
      *id = i;
      return CWPIR_OK;
    }
  std::unique_ptr<Scratch> S(new (std::nothrow) Scratch());
  if (!S) return fail(c, CWPIR_ENOMEM, "host allocation");
  CUDA_TRY(c, cudaMalloc(&S->d_err, sizeof(int)));
  CUDA_TRY(c, cudaMemset(S->d_err, 0, sizeof(int)));
  *id = (u32)c->slots.size();
  c->slots.push_back(std::move(S));
  return CWPIR_OK;
}

bool slot_ok(const cwpir_ctx *c, u32 slot) {
  return slot < c->slots.size() && c->slots[slot]->in_use;
}

// The buffers of slot `slot` for c->jmax multiplications per launch.
int ensure_scratch(cwpir_ctx *c, u32 slot = 0) {
  if (!slot_ok(c, slot)) return fail(c, CWPIR_EINVAL, "unknown slot %u", slot);
  Scratch &S = *c->slots[slot];
  if (!c->jmax) c->jmax = jobs_per_launch(c);
  const u64 N = c->N, L = c->L, j = c->jmax;
  CUDA_TRY(c, S.Tbuf.ensure(j * 3 * cw::tensor_poly_words(c->K, c->N), &c->acct));
  CUDA_TRY(c, S.E.ensure(j * 3 * L * N, &c->acct));
  CUDA_TRY(c, S.CP.ensure(j * 2 * L * N, &c->acct));
  CUDA_TRY(c, S.DN.ensure(j * dn_words(L, N), &c->acct));
  CUDA_TRY(c, S.RS.ensure(rs_words(L, N), &c->acct));
  CUDA_TRY(c, S.DNQ.ensure(dnq_words(L, N), &c->acct));
  return CWPIR_OK;
}

// ---- plans: the product tree of every row (Alg. Selection Vector) ----
// Node (l, r) of a row covers positions [r 2^l, min((r+1) 2^l, k)) of its
// ascending codeword positions; a node with one position is a leaf and a
// node whose right half is empty carries its left child up unchanged.
// Every query slot s has its own leaves, shared pair products and tree
// levels; the jobs of all slots share launches.
struct PlanBuilder {
  const uint16_t *cw;
  u32 k, m, nq;
  u64 qp, rows_per_batch = 0;
  const u64 *leaves;
  bool memo;
  std::unordered_map<u32, u64> memo_id;
  u64 n_memo = 0;
  const u64 *memo_base = nullptr;
  std::vector<u64> level_off;  // offset (cts) of level l inside level_buf
  std::vector<u32> level_nodes;
  u64 *level_base = nullptr;

  u64 *level_slot(u32 s, u64 lr, u32 l, u32 r) const {
    return level_base + (level_off[l] + (s * rows_per_batch + lr) * level_nodes[l] + r) * qp;
  }
  const u64 *ptr(u32 s, u64 row, u64 lr, u32 l, u32 r) const {
    const uint16_t *pos = cw + row * k;
    u32 lo = r << l, hi = std::min<u32>(lo + (1u << l), k);
    if (hi - lo == 1) return leaves + ((u64)s * m + pos[lo]) * qp;
    u32 mid = lo + (1u << (l - 1));
    if (mid >= hi) return ptr(s, row, lr, l - 1, 2 * r);
    if (l == 1 && memo)
      return memo_base + ((u64)s * n_memo + memo_id.at(((u32)pos[lo] << 16) | pos[lo + 1])) * qp;
    return level_slot(s, lr, l, r);
  }
};

u32 ceil_log2(u32 k) {
  u32 l = 0;
  while ((1u << l) < k) ++l;
  return l;
}

// Buffers and substitution job lists of Alg. Query Expansion for the
// plan's nq * h_in inputs of 2^c entries each (uploaded once).
int setup_expand(cwpir_ctx *c, Plan *P) {
  const u64 ctw = c->ct();
  const u64 B = 1ull << P->cfac, inputs = (u64)P->nq * P->h_in;
  CUDA_TRY(c, P->exp_a.ensure(inputs * B * ctw, &c->acct));
  CUDA_TRY(c, P->exp_b.ensure(inputs * B * ctw, &c->acct));
  CUDA_TRY(c, P->exp_tau.ensure(inputs * (B / 2) * ctw, &c->acct));
  CUDA_TRY(c, P->exp_S.ensure(inputs * (B / 2) * ctw, &c->acct));
  CUDA_TRY(c, P->exp_O.ensure(inputs * (B / 2) * ctw, &c->acct));
  CUDA_TRY(c, P->exp_DN.ensure(inputs * (B / 2) * (c->L + 1) * c->L * c->N, &c->acct));
  CUDA_TRY(c, P->leaves_coef.ensure((u64)P->nq * P->m * ctw, &c->acct));
  std::vector<cw::SubJob> sj;
  u64 *cur = P->exp_a.p, *nxt = P->exp_b.p;
  for (u32 a = 0; a < P->cfac; ++a) {
    P->exp_rounds.push_back(ExpRound{sj.size(), (u32)(inputs << a)});
    for (u64 ja = 0; ja < inputs; ++ja)
      for (u64 b = 0; b < (1ull << a); ++b)
        sj.push_back(cw::SubJob{cur + (ja * B + b) * ctw, P->exp_S.p + ((ja << a) + b) * ctw});
    std::swap(cur, nxt);
  }
  P->exp_final = cur;
  CUDA_TRY(c, cudaMalloc(&P->d_subjobs, sj.size() * sizeof(cw::SubJob)));
  CUDA_TRY(c, cudaMemcpy(P->d_subjobs, sj.data(), sj.size() * sizeof(cw::SubJob),
                         cudaMemcpyHostToDevice));
  return CWPIR_OK;
}

// Plan over `rows` for nq query slots with compression factor cfac.
// root_mode ROOT_PM (answers into the plan's accumulators) or ROOT_SEL
// (nq = 1; selection entries in coefficient form to sel_out, [rows][2][L][N]).
int build_plan(cwpir_ctx *c, u32 slot, Db *db, const std::vector<u64> &rows, u32 nq, u32 cfac,
               int root_mode, u64 *sel_out, bool memo_opt, std::unique_ptr<Plan> &out) {
  std::unique_ptr<Plan> P(new Plan());
  const u32 k = db->k, m = db->m;
  const u64 qp = c->qp_ct(), ctw = c->ct();
  P->nq = nq;
  P->cfac = cfac;
  P->k = k;
  P->m = m;
  P->top = ceil_log2(k);
  P->memo = memo_opt && P->top >= 2;
  P->h_in = db->folklore ? m / 2 : cfac ? (m + (1u << cfac) - 1) >> cfac : m;
  P->sp = db->sp;
  P->rows_db = db->rows;
  if (db->folklore) CUDA_TRY(c, P->leaves_coef.ensure((u64)nq * m * ctw, &c->acct));
  const u32 J = c->jmax;
  if (root_mode == cw::ROOT_PM && (u64)nq * db->sp > J)
    return fail(c, CWPIR_EINVAL, "%u queries x %u plaintexts per row need more than %u partial "
                "sums per launch (raise CWPIR_OPT_MAX_JOBS)", nq, db->sp, J);
  if (db->sp > 1 && k > 1) CUDA_TRY(c, c->slots[slot]->SEL.ensure((u64)J * ctw, &c->acct));
  CUDA_TRY(c, P->leaves.ensure((u64)nq * m * qp, &c->acct));
  CUDA_TRY(c, P->acc.ensure((u64)nq * db->sp * ctw, &c->acct));
  CUDA_TRY(c, P->q_in.ensure((u64)nq * P->h_in * ctw, &c->acct));
  CUDA_TRY(c, P->resp.ensure((u64)nq * db->sp * ctw, &c->acct));

  if (cfac) {
    int rc = setup_expand(c, P.get());
    if (rc) return rc;
  }

  PlanBuilder Bd;
  Bd.cw = db->cw.data();
  Bd.k = k;
  Bd.m = m;
  Bd.nq = nq;
  Bd.qp = qp;
  Bd.leaves = P->leaves.p;
  Bd.memo = P->memo;
  auto &jobs = P->host_jobs;

  if (k == 1) {
    P->leaf_root = true;
    const u64 per = std::max<u64>(1, J / ((u64)nq * db->sp));  // partials [job][sp] fit J
    for (u64 x = 0; x < rows.size(); x += per) {
      u32 cnt = (u32)std::min<u64>(per, rows.size() - x);
      P->batches.push_back({Chunk{jobs.size(), cnt * nq, cw::ROOT_PM, nq}});
      for (u32 s = 0; s < nq; ++s)
        for (u32 i = 0; i < cnt; ++i) {
          u64 row = rows[x + i];
          jobs.push_back(cw::MulJob{Bd.leaves + ((u64)s * m + db->cw[row]) * qp, nullptr, nullptr, row});
        }
    }
  } else {
    if (P->memo) {
      std::vector<std::pair<u32, u32>> pairs;
      for (u64 row : rows) {
        const uint16_t *pos = db->cw.data() + row * k;
        for (u32 r = 0; 2 * r + 1 < k; ++r) {
          u32 key = ((u32)pos[2 * r] << 16) | pos[2 * r + 1];
          if (Bd.memo_id.emplace(key, pairs.size()).second) pairs.push_back({pos[2 * r], pos[2 * r + 1]});
        }
      }
      P->n_memo = Bd.n_memo = pairs.size();
      CUDA_TRY(c, P->memo_buf.ensure(std::max<u64>(1, (u64)nq * P->n_memo) * qp, &c->acct));
      Bd.memo_base = P->memo_buf.p;
      std::vector<cw::MulJob> mj;
      for (u32 s = 0; s < nq; ++s)
        for (u64 i = 0; i < pairs.size(); ++i)
          mj.push_back(cw::MulJob{Bd.leaves + ((u64)s * m + pairs[i].first) * qp,
                                  Bd.leaves + ((u64)s * m + pairs[i].second) * qp,
                                  P->memo_buf.p + ((u64)s * P->n_memo + i) * qp, 0});
      for (u64 x = 0; x < mj.size(); x += J) {
        u32 cnt = (u32)std::min<u64>(J, mj.size() - x);
        P->memo_chunks.push_back(Chunk{jobs.size(), cnt, cw::INTERNAL, 1});
        jobs.insert(jobs.end(), mj.begin() + x, mj.begin() + x + cnt);
      }
      P->mults += mj.size();
    }
    const u32 l0 = P->memo ? 2 : 1;
    u32 max_nodes = 1;
    Bd.level_off.assign(P->top + 1, 0);
    Bd.level_nodes.assign(P->top + 1, 0);
    for (u32 l = l0; l <= P->top; ++l) {
      u32 nodes = (k + (1u << l) - 1) >> l;
      Bd.level_nodes[l] = nodes;
      max_nodes = std::max(max_nodes, nodes);
    }
    if ((u64)nq * max_nodes > J)
      return fail(c, CWPIR_EINVAL, "%u queries per call need more than %u multiplications per "
                  "launch (raise CWPIR_OPT_MAX_JOBS)", nq, J);
    u64 rpb = std::max<u64>(1, J / ((u64)nq * max_nodes));
    if (c->opt_batch_rows) rpb = std::min<u64>(rpb, c->opt_batch_rows);
    Bd.rows_per_batch = rpb;
    u64 lvl_cts = 0;
    for (u32 l = l0; l < P->top; ++l) {
      Bd.level_off[l] = lvl_cts;
      lvl_cts += (u64)nq * rpb * Bd.level_nodes[l];
    }
    CUDA_TRY(c, P->level_buf.ensure(std::max<u64>(1, lvl_cts) * qp, &c->acct));
    Bd.level_base = P->level_buf.p;
    for (u64 x = 0; x < rows.size(); x += rpb) {
      u64 cnt = std::min<u64>(rpb, rows.size() - x);
      std::vector<Chunk> levels;
      for (u32 l = l0; l <= P->top; ++l) {
        const bool root = l == P->top;
        Chunk ch{jobs.size(), 0, root ? root_mode : (int)cw::INTERNAL, root ? nq : 1};
        for (u32 s = 0; s < nq; ++s)
          for (u64 lr = 0; lr < cnt; ++lr) {
            u64 row = rows[x + lr];
            for (u32 r = 0; r < Bd.level_nodes[l]; ++r) {
              u32 lo = r << l, mid = lo + (1u << (l - 1));
              if (mid >= std::min<u32>(lo + (1u << l), k)) continue;
              cw::MulJob mj;
              mj.a = Bd.ptr(s, row, lr, l - 1, 2 * r);
              mj.b = Bd.ptr(s, row, lr, l - 1, 2 * r + 1);
              mj.row = row;
              if (root) mj.dst = sel_out ? sel_out + (x + lr) * ctw : nullptr;
              else mj.dst = Bd.level_slot(s, lr, l, r);
              jobs.push_back(mj);
              ++ch.count;
            }
          }
        P->mults += ch.count;
        if (ch.count) levels.push_back(ch);
      }
      P->batches.push_back(levels);
    }
  }
  CUDA_TRY(c, cudaMalloc(&P->d_jobs, std::max<size_t>(1, jobs.size()) * sizeof(cw::MulJob)));
  CUDA_TRY(c, cudaMemcpy(P->d_jobs, jobs.data(), jobs.size() * sizeof(cw::MulJob),
                         cudaMemcpyHostToDevice));
  out = std::move(P);
  return CWPIR_OK;
}

// One chunk of multiplications: tensor, scale-down, relinearisation and
// the consumer of the result.
int run_chunk(cwpir_ctx *c, Scratch &S, Plan *P, const Chunk &ch, const u64 *dbp,
              cudaStream_t st) {
  const cw::MulJob *jobs = P->d_jobs + ch.off;
  if (P->leaf_root) {
    CUDA_TRY(c, timed(c, CWPIR_K_RELIN, st, [&] { return cw::launch_pm_leaf(c->d_tab, c->h, jobs, ch.count, P->sp, dbp, S.CP.p, st); }));
    CUDA_TRY(c, timed(c, CWPIR_K_ACC, st, [&] { return cw::launch_accumulate(c->h, c->d_tab, S.CP.p, ch.segs, ch.count / ch.segs, P->sp, P->acc.p, st); }));
    c->stats.kernel_launches += 2;
    c->stats.db_bytes_read += (u64)ch.count * P->sp * c->L * c->N * sizeof(u64);
    return CWPIR_OK;
  }
  CUDA_TRY(c, timed(c, CWPIR_K_TENSOR, st, [&] { return cw::launch_tensor(c->d_tab, c->h, jobs, ch.count, S.Tbuf.p, st); }));
  CUDA_TRY(c, timed(c, CWPIR_K_SCALE, st, [&] { return cw::launch_scale(c->d_tab, c->h, S.Tbuf.p, ch.count, S.E.p, S.d_err, st); }));
  const bool rows = ch.mode == cw::ROOT_PM && P->rows_db;
  if (ch.mode == cw::INTERNAL && c->ksr) {
    // key switch in the key-switch basis (digits in the dead tensor buffer,
    // the basis sums in the digit-transform buffer), the result in
    // coefficient form to CP, then the extension limbs of the QP-NTT
    // destination: the tensor of the next level reads nothing else
    CUDA_TRY(c, timed(c, CWPIR_K_RELIN, st, [&] {
      return cw::launch_relin_ksr(c->d_tab, c->h, S.E.p, ch.count,
                                  reinterpret_cast<const u32 *>(c->ksr_key.p),
                                  reinterpret_cast<u32 *>(S.Tbuf.p), reinterpret_cast<u32 *>(S.DN.p),
                                  S.d_err, S.CP.p, st);
    }));
    CUDA_TRY(c, timed(c, CWPIR_K_LIFT, st, [&] { return cw::launch_lift_jobs(c->d_tab, c->h, S.CP.p, jobs, ch.count, st); }));
    CUDA_TRY(c, timed(c, CWPIR_K_NTT, st, [&] { return cw::launch_ntt_jobs_p(c->d_tab, c->h, jobs, ch.count, st); }));
    c->stats.kernel_launches += 2 + 4 + 2;  // tensor, scale; key switch; lift, NTT
    c->stats.mults += ch.count;
    c->stats.ntt_polys += (u64)ch.count * (3 * c->K + 3 * c->L * cw::kKsrPrimes + 2 * c->K);
    return CWPIR_OK;
  }
  if (rows)
    CUDA_TRY(c, timed(c, CWPIR_K_ROWS, st, [&] {
      return cw::launch_rows_transforms(c->d_tab, c->h, S.E.p, ch.count,
                                        reinterpret_cast<u32 *>(S.DN.p), st);
    }));
  CUDA_TRY(c, timed(c, CWPIR_K_RELIN, st, [&] {
    if (rows)
      return cw::launch_relin_rows(c->d_tab, c->h, S.E.p, ch.count, ch.segs, jobs, c->rlk.p,
                                   c->rlk_s.p, reinterpret_cast<const u32 *>(dbp), kRowGroups,
                                   reinterpret_cast<u32 *>(S.DN.p),
                                   reinterpret_cast<u32 *>(S.RS.p), S.DNQ.p, S.d_err,
                                   S.CP.p, st);
    return cw::launch_relin(c->d_tab, c->h, S.E.p, ch.count, ch.segs, jobs, ch.mode, c->rlk.p,
                            c->rlk_s.p, dbp, P->sp, c->jmax, S.DN.p, S.SEL.p, S.CP.p, st);
  }));
  c->stats.kernel_launches += 2;  // tensor, scale-down
  c->stats.mults += ch.count;
  c->stats.ntt_polys += (u64)ch.count * 3 * c->K;
  if (rows) {
    const u32 seg_len = ch.count / ch.segs;
    const u32 G = cw::relin_rows_groups(c->h, ch.segs, seg_len, kRowGroups);
    const u32 spp = G >= kRowGroups ? 1 : kRowGroups / G, passes = (ch.segs + spp - 1) / spp;
    // row transforms; per pass: row sums, inverse NTT, CRT, NTT, key products
    c->stats.kernel_launches += 1 + 5ull * passes;
    c->stats.ntt_polys += (u64)ch.count * 3 * c->L * c->h.rows.nr;
  } else {
    // digit NTTs, key multiply-accumulate (and, for rows of several
    // plaintexts, their products)
    c->stats.kernel_launches += (ch.mode == cw::ROOT_PM && P->sp > 1) ? 3 : 2;
    c->stats.ntt_polys += (u64)ch.count * c->L * (c->L + 2);
  }
  if (ch.mode == cw::INTERNAL) {
    CUDA_TRY(c, timed(c, CWPIR_K_LIFT, st, [&] { return cw::launch_lift_jobs(c->d_tab, c->h, S.CP.p, jobs, ch.count, st); }));
    CUDA_TRY(c, timed(c, CWPIR_K_NTT, st, [&] { return cw::launch_ntt_jobs_p(c->d_tab, c->h, jobs, ch.count, st); }));
    c->stats.kernel_launches += 3;  // inverse NTT, lift, P-limb NTT
    c->stats.ntt_polys += (u64)ch.count * (2 * c->L + 2 * c->K);
  } else if (ch.mode == cw::ROOT_PM) {
    const u32 seg_len = ch.count / ch.segs;
    const u32 groups = rows ? cw::relin_rows_groups(c->h, ch.segs, seg_len, kRowGroups)
                            : cw::relin_pm_groups(c->h, ch.segs, seg_len, P->sp, c->jmax);
    CUDA_TRY(c, timed(c, CWPIR_K_ACC, st, [&] { return cw::launch_accumulate(c->h, c->d_tab, S.CP.p, ch.segs, groups, P->sp, P->acc.p, st); }));
    c->stats.kernel_launches += 1;
    c->stats.db_bytes_read += rows ? (u64)ch.count * c->h.rows.nr * c->N * sizeof(u32)
                                   : (u64)ch.count * P->sp * c->L * c->N * sizeof(u64);
  } else {
    c->stats.kernel_launches += 1;  // inverse NTT
    c->stats.ntt_polys += (u64)ch.count * 2 * c->L;
  }
  return CWPIR_OK;
}

int ensure_subjobs(cwpir_ctx *c, size_t n) {
  if (n <= c->n_subjobs) return CWPIR_OK;
  if (c->d_subjobs) cudaFree(c->d_subjobs);
  c->d_subjobs = nullptr;
  c->n_subjobs = 0;
  CUDA_TRY(c, cudaMalloc(&c->d_subjobs, n * sizeof(cw::SubJob)));
  c->n_subjobs = n;
  return CWPIR_OK;
}

const std::pair<std::shared_ptr<DevBuf>, std::shared_ptr<DevBuf>> *find_gal(cwpir_ctx *c, u32 g) {
  auto it = c->gal.find(g);
  return it == c->gal.end() ? nullptr : &it->second;
}

int check_keys(cwpir_ctx *c, u32 cfac) {
  for (u32 a = 0; a < cfac; ++a)
    if (!find_gal(c, c->N / (1u << a) + 1))
      return fail(c, CWPIR_ENOKEY, "no Galois key for element %u", c->N / (1u << a) + 1);
  return CWPIR_OK;
}

// Alg. Query Expansion for the plan's nq * h_in inputs (d_query, [nq][h_in]
// cts): rounds of substitutions shared by all queries; the first m entries
// of every query end up in P->leaves_coef ([nq][m] cts).  Capturable.
int enqueue_expand(cwpir_ctx *c, Plan *P, const u64 *d_query, cudaStream_t st) {
  const u64 B = 1ull << P->cfac, ctw = c->ct(), inputs = (u64)P->nq * P->h_in;
  CUDA_TRY(c, cudaMemcpy2DAsync(P->exp_a.p, B * ctw * sizeof(u64), d_query, ctw * sizeof(u64),
                                ctw * sizeof(u64), inputs, cudaMemcpyDeviceToDevice, st));
  u64 *cur = P->exp_a.p, *nxt = P->exp_b.p;
  for (u32 a = 0; a < P->cfac; ++a) {
    const u32 g = c->N / (1u << a) + 1;
    const u32 nj = P->exp_rounds[a].count;
    const auto *key = find_gal(c, g);
    const cw::SubJob *jobs = P->d_subjobs + P->exp_rounds[a].off;
    CUDA_TRY(c, timed(c, CWPIR_K_EXPAND, st, [&] { return cw::launch_automorph(c->d_tab, c->h, jobs, nj, g, P->exp_tau.p, st); }));
    CUDA_TRY(c, timed(c, CWPIR_K_EXPAND, st, [&] {
      return cw::launch_sub_keyswitch(c->d_tab, c->h, P->exp_tau.p, nj, jobs, key->first->p,
                                      key->second->p, P->exp_DN.p, P->exp_O.p, st);
    }));
    CUDA_TRY(c, timed(c, CWPIR_K_EXPAND, st, [&] { return cw::launch_expand_combine(c->d_tab, c->h, cur, P->exp_S.p, nxt, (u32)inputs, P->cfac, a, st); }));
    c->stats.kernel_launches += 5;
    c->stats.substitutions += nj;
    c->stats.ntt_polys += (u64)nj * c->L * (c->L + 3);
    std::swap(cur, nxt);
  }
  // entry j * 2^c + b of input j encrypts query bit j * 2^c + b: the first
  // m entries of each query's h_in * 2^c are its expanded ciphertexts
  CUDA_TRY(c, cudaMemcpy2DAsync(P->leaves_coef.p, (u64)P->m * ctw * sizeof(u64), P->exp_final,
                                (u64)P->h_in * B * ctw * sizeof(u64), (u64)P->m * ctw * sizeof(u64),
                                P->nq, cudaMemcpyDeviceToDevice, st));
  return CWPIR_OK;
}

// Leaves: coefficient-form cts -> QP-NTT form.
int prep_leaves(cwpir_ctx *c, const u64 *coef, u32 count, u64 *dst, cudaStream_t st) {
  const u64 LK = c->L + c->K;
  CUDA_TRY(c, timed(c, CWPIR_K_LIFT, st, [&] {
    return cw::launch_lift(c->d_tab, c->h, coef, (u64)c->L * c->N, dst, c->qp_poly(),
                           2 * count, true, st);
  }));
  CUDA_TRY(c, timed(c, CWPIR_K_NTT, st, [&] {
    return cw::launch_ntt(c->d_tab, c->h, dst, 2 * count, c->qp_poly(), 0, (u32)LK, false,
                          nullptr, 0, st);
  }));
  c->stats.kernel_launches += 2;
  c->stats.ntt_polys += 2ull * count * LK;
  return CWPIR_OK;
}

// Reads and clears the device consistency flag of a slot (after the work
// that sets it is complete): CWPIR_EINTERNAL if a check failed.
int check_err_flag(cwpir_ctx *c, u32 slot = 0) {
  if (!slot_ok(c, slot)) return fail(c, CWPIR_EINVAL, "unknown slot %u", slot);
  int *flag = c->slots[slot]->d_err;
  int h = 0;
  CUDA_TRY(c, cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    CUDA_TRY(c, cudaMemset(flag, 0, sizeof(int)));
    return fail(c, CWPIR_EINTERNAL,
                "device consistency check failed (scale-down or row-basis rounding)");
  }
  return CWPIR_OK;
}

Db *get_db(cwpir_ctx *c, int32_t id) {
  auto it = c->dbs.find(id);
  return it == c->dbs.end() ? nullptr : it->second.get();
}

// Coefficient-form leaves of a plan's queries: the query itself, its
// expansion (c > 0) or, for a folklore database, (1 - x[i], x[i]) per bit.
int leaf_coefs(cwpir_ctx *c, Db *db, Plan *P, const u64 *d_query, cudaStream_t st,
               const u64 **coef) {
  int rc;
  *coef = d_query;
  if (P->cfac) {
    if ((rc = enqueue_expand(c, P, d_query, st))) return rc;
    *coef = P->leaves_coef.p;
  } else if (db->folklore) {
    CUDA_TRY(c, cw::launch_folklore_leaves(c->d_tab, c->h, d_query, P->nq * P->h_in,
                                           P->leaves_coef.p, st));
    c->stats.kernel_launches += 1;
    *coef = P->leaves_coef.p;
  }
  return CWPIR_OK;
}

// The whole answer of a plan: expansion, leaves, tree, accumulation and the
// final inverse transform into d_resp ([nq][sp][2][L][N]).  Capturable.
int enqueue_answer(cwpir_ctx *c, Scratch &S, Db *db, Plan *P, const u64 *d_query, u64 *d_resp,
                   cudaStream_t st) {
  int rc;
  const u64 *coef;
  if ((rc = leaf_coefs(c, db, P, d_query, st, &coef))) return rc;
  if ((rc = prep_leaves(c, coef, P->nq * P->m, P->leaves.p, st))) return rc;
  CUDA_TRY(c, cudaMemsetAsync(P->acc.p, 0, (u64)P->nq * P->sp * c->ct() * sizeof(u64), st));
  for (const Chunk &ch : P->memo_chunks)
    if ((rc = run_chunk(c, S, P, ch, db->db.p, st))) return rc;
  for (const auto &batch : P->batches)
    for (const Chunk &ch : batch)
      if ((rc = run_chunk(c, S, P, ch, db->db.p, st))) return rc;
  CUDA_TRY(c, timed(c, CWPIR_K_NTT, st, [&] {
    return cw::launch_ntt(c->d_tab, c->h, d_resp, 2 * P->nq * P->sp, (u64)c->L * c->N, 0, c->L,
                          true, P->acc.p, (u64)c->L * c->N, st);
  }));
  c->stats.kernel_launches += 1;
  c->stats.ntt_polys += 2ull * P->nq * P->sp * c->L;
  c->stats.rows = db->n * P->nq;
  return CWPIR_OK;
}

// The cached all-rows plan of a database for (nq, cfac) on a slot.
int get_plan(cwpir_ctx *c, u32 slot, Db *db, u32 nq, u32 cfac, Plan **out) {
  int rc = ensure_scratch(c, slot);
  if (rc) return rc;
  auto key = std::make_tuple(nq, cfac, slot);
  auto it = db->plans.find(key);
  if (it == db->plans.end()) {
    std::vector<u64> rows(db->n);
    for (u64 i = 0; i < db->n; ++i) rows[i] = i;
    std::unique_ptr<Plan> P;
    if ((rc = build_plan(c, slot, db, rows, nq, cfac, cw::ROOT_PM, nullptr, c->opt_share != 0,
                         P)))
      return rc;
    it = db->plans.emplace(key, std::move(P)).first;
  }
  *out = it->second.get();
  return CWPIR_OK;
}

// Captures a plan's whole answer (from its staging buffers q_in to resp)
// into a CUDA graph on the context's stream.
int capture_plan(cwpir_ctx *c, Scratch &S, Db *db, Plan *P) {
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  cudaGraph_t g = nullptr;
  c->capturing = true;
  int rc = CWPIR_OK;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = enqueue_answer(c, S, db, P, P->q_in.p, P->resp.p, c->stream);
    e = cudaStreamEndCapture(c->stream, &g);
  }
  c->capturing = false;
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&P->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, CWPIR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  P->graph_stats = c->stats;
  return CWPIR_OK;
}

// Answers nq queries (d_query: [nq][h_in] cts) into d_resp ([nq][sp][2][L][N])
// with the scratch of `slot`.  With CWPIR_OPT_USE_GRAPH the plan's sequence
// is captured once into a CUDA graph (on the context's stream) and replayed
// on `st`, staging the queries and responses through the plan's fixed
// buffers.
int answer_batch_enqueue(cwpir_ctx *c, u32 slot, Db *db, u32 cfac, u32 nq, const u64 *d_query,
                         u64 *d_resp, cudaStream_t st) {
  Plan *P;
  int rc = get_plan(c, slot, db, nq, cfac, &P);
  if (rc) return rc;
  Scratch &S = *c->slots[slot];
  c->stats = cwpir_stats{};
  if (!c->opt_graph) return enqueue_answer(c, S, db, P, d_query, d_resp, st);
  const u64 ctw = c->ct();
  if (!P->graph && (rc = capture_plan(c, S, db, P))) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(P->q_in.p, d_query, (u64)nq * P->h_in * ctw * sizeof(u64),
                              cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(c, cudaGraphLaunch(P->graph, st));
  CUDA_TRY(c, cudaMemcpyAsync(d_resp, P->resp.p, (u64)nq * P->sp * ctw * sizeof(u64),
                              cudaMemcpyDeviceToDevice, st));
  c->stats = P->graph_stats;
  return CWPIR_OK;
}

}  // namespace

// ---------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------
extern "C" {

int cwpir_abi_version(void) { return CWPIR_ABI_VERSION; }

const char *cwpir_strerror(int code) {
  switch (code) {
    case CWPIR_OK: return "ok";
    case CWPIR_EINVAL: return "invalid argument";
    case CWPIR_ENOMEM: return "out of memory";
    case CWPIR_ENODB: return "unknown database";
    case CWPIR_ECUDA: return "CUDA error";
    case CWPIR_ETIMEDOUT: return "device wait timed out";
    case CWPIR_EBUSY: return "busy";
    case CWPIR_ENOKEY: return "missing Galois key";
    case CWPIR_EINTERNAL: return "internal consistency check failed";
    default: return "unknown error";
  }
}

const char *cwpir_last_error(const cwpir_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_setup_error.c_str();
}

int cwpir_default_primes(uint32_t N, uint32_t L, uint64_t *q_out) {
  if (N < 2 || (N & (N - 1)) || N > (1u << 20) || L == 0 || !q_out) return CWPIR_EINVAL;
  std::vector<u64> p = ntt_primes(N, L, {});
  if (p.size() != L) return CWPIR_EINVAL;
  for (u32 i = 0; i < L; ++i) q_out[i] = p[i];
  return CWPIR_OK;
}

static u128 binom_sat(u64 n, u64 r) {
  if (r > n) return 0;
  if (r > n - r) r = n - r;
  const u128 lim = (u128)1 << 126;
  u128 v = 1;
  for (u64 i = 1; i <= r; ++i) {
    u64 f = n - r + i;
    if (v > lim / f) return lim;
    v = v * f / i;
  }
  return v;
}

int cwpir_map_perfect(uint64_t x, uint32_t m, uint32_t k, uint16_t *pos_out) {
  if (!pos_out || k == 0 || k > m || m > 65535) return CWPIR_EINVAL;
  if ((u128)x >= binom_sat(m, k)) return CWPIR_EINVAL;
  // Alg. Perfect Mapping: scan m' = m-1 .. 0, take m' when the remainder is
  // at least C(m', h); positions come out in descending order.
  u128 rem = x;
  u32 h = k;
  for (int64_t mp = (int64_t)m - 1; mp >= 0 && h; --mp) {
    u128 b = binom_sat((u64)mp, h);
    if (rem >= b) {
      pos_out[--h] = (uint16_t)mp;
      rem -= b;
    }
  }
  return h == 0 ? CWPIR_OK : CWPIR_EINVAL;
}

// Alg. Lossy Mapping (App. A): draw positions H_1(x), H_2(x), ... and keep
// each new one until k are set.  H_i(x) = (i-th output of SplitMix64 seeded
// with x) mod m, i.e. mix64(x + i * 0x9E3779B97F4A7C15) mod m with the
// SplitMix64 output mixer.
static u64 splitmix64_output(u64 z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int cwpir_map_lossy(uint64_t x, uint32_t m, uint32_t k, uint16_t *pos_out) {
  if (!pos_out || k == 0 || k > m || m > 65535) return CWPIR_EINVAL;
  std::vector<char> set(m, 0);
  u32 cnt = 0;
  // a bound on the draws: reached with probability below 2^-60 for any k <= m
  const u64 limit = 64ull * m + 1024;
  for (u64 i = 1; cnt < k && i <= limit; ++i) {
    const u32 mp = (u32)(splitmix64_output(x + i * 0x9E3779B97F4A7C15ull) % m);
    if (!set[mp]) {
      set[mp] = 1;
      ++cnt;
    }
  }
  if (cnt < k) return CWPIR_EINVAL;
  u32 h = 0;
  for (u32 mp = 0; mp < m; ++mp)
    if (set[mp]) pos_out[h++] = (uint16_t)mp;
  return CWPIR_OK;
}

int cwpir_code_length(uint64_t n, uint32_t k, uint32_t *m_out) {
  if (!m_out || k == 0 || k > 64) return CWPIR_EINVAL;
  for (u64 m = k; m <= 65535; ++m)
    if (binom_sat(m, k) >= (u128)n) {
      *m_out = (uint32_t)m;
      return CWPIR_OK;
    }
  return CWPIR_EINVAL;
}

int cwpir_setup(const cwpir_params *params, const cwpir_keys *keys, cwpir_ctx **out) {
  g_setup_error.clear();
  if (!params || !keys || !out || !params->q || !keys->relin)
    return fail(nullptr, CWPIR_EINVAL, "null argument");
  const u32 N = params->N, L = params->L;
  if (N < 1024 || N > 16384 || (N & (N - 1)))
    return fail(nullptr, CWPIR_EINVAL, "N must be a power of two in [1024, 16384]");
  if (L < 1 || L > (u32)cw::kMaxL) return fail(nullptr, CWPIR_EINVAL, "L must be in [1, 8]");
  if (params->t < 3 || params->t >= (1ull << 20) || !miller_rabin(params->t))
    return fail(nullptr, CWPIR_EINVAL, "t must be a prime in [3, 2^20)");
  std::vector<u64> q(params->q, params->q + L);
  for (u32 j = 0; j < L; ++j) {
    if (q[j] <= (1ull << 53) || q[j] >= (1ull << 54) || !miller_rabin(q[j]) ||
        (q[j] - 1) % (2ull * N))
      return fail(nullptr, CWPIR_EINVAL, "q[%u] must be a prime in (2^53, 2^54), = 1 mod 2N", j);
    for (u32 l = 0; l < j; ++l)
      if (q[l] == q[j]) return fail(nullptr, CWPIR_EINVAL, "primes must be distinct");
  }
  std::unique_ptr<cwpir_ctx> c(new (std::nothrow) cwpir_ctx());
  if (!c) return fail(nullptr, CWPIR_ENOMEM, "host allocation");
  cudaGetDevice(&c->device);
  c->N = N;
  c->logN = 0;
  while ((1u << c->logN) < N) ++c->logN;
  c->L = L;
  c->t = params->t;
  c->q = q;
  // Extension basis P: 30-bit primes with P >= 2 N Q^2 (the tensor alone)
  // and P > 2^17 t N Q (the exact scale-down), checked below.
  c->K = (u32)cw::ext_count((int)L);
  c->p = cw::host::ext_primes(N, c->K);
  if (c->p.size() != c->K) return fail(nullptr, CWPIR_EINVAL, "not enough extension primes");
  long double lq = 0, lp = 0;
  for (u64 v : q) lq += log2l((long double)v);
  for (u64 v : c->p) lp += log2l((long double)v);
  if (lp < lq + log2l((long double)N) + log2l((long double)params->t) + 17 ||
      lp < 2 * lq + log2l((long double)N) + 1)
    return fail(nullptr, CWPIR_EINVAL, "extension basis too small");
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(nullptr, CWPIR_ECUDA, "stream: %s", cudaGetErrorString(e));
  int rc = build_tables(c.get());
  u32 slot0 = 0;
  if (!rc) rc = add_slot(c.get(), &slot0);
  if (rc) {
    g_setup_error = c->err;
    return rc;
  }
  rc = upload_key(c.get(), keys->relin, c->rlk, c->rlk_s, c->ksr ? &c->ksr_key : nullptr);
  if (rc) {
    g_setup_error = c->err;
    return rc;
  }
  for (u32 i = 0; i < keys->n_galois; ++i) {
    u32 g = keys->galois_elts[i];
    if (!(g & 1) || g >= 2 * N) return fail(nullptr, CWPIR_EINVAL, "bad Galois element %u", g);
    auto kb = std::make_shared<DevBuf>(), ks = std::make_shared<DevBuf>();
    rc = upload_key(c.get(), keys->galois + (u64)i * 2 * L * L * N, *kb, *ks, nullptr);
    if (rc) {
      g_setup_error = c->err;
      return rc;
    }
    c->gal[g] = {kb, ks};
  }
  *out = c.release();
  return CWPIR_OK;
}

void cwpir_destroy(cwpir_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  delete ctx;
}

static int load_db_impl(cwpir_ctx *c, uint64_t n, uint32_t plen, uint32_t k, uint32_t m,
                        const uint32_t *items, const uint16_t *codewords, bool folklore,
                        int32_t *db_id) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  cudaSetDevice(c->device);
  if (!items || !codewords || !db_id) return fail(c, CWPIR_EINVAL, "null argument");
  if (n < 1 || n > (1ull << 24)) return fail(c, CWPIR_EINVAL, "n must be in [1, 2^24]");
  if (plen > (u64)CWPIR_MAX_PLAINTEXTS * c->N)
    return fail(c, CWPIR_EINVAL, "payload_len > %u N", CWPIR_MAX_PLAINTEXTS);
  if (k < 1 || k > 16 || k > m || m > 16384)
    return fail(c, CWPIR_EINVAL, "need 1 <= k <= 16, k <= m <= 16384");
  for (u64 i = 0; i < n * plen; ++i)
    if (items[i] >= c->t) return fail(c, CWPIR_EINVAL, "item coefficient >= t at %llu", (unsigned long long)i);
  for (u64 i = 0; i < n; ++i)
    for (u32 u = 0; u < k; ++u) {
      uint16_t p = codewords[i * k + u];
      if (p >= m || (u && p <= codewords[i * k + u - 1]))
        return fail(c, CWPIR_EINVAL, "codeword of row %llu is not ascending positions < m",
                    (unsigned long long)i);
    }
  std::unique_ptr<Db> db(new Db());
  db->n = n;
  db->plen = plen;
  db->k = k;
  db->m = m;
  db->sp = plen ? (plen + c->N - 1) / c->N : 1;
  db->folklore = folklore;
  db->cw.assign(codewords, codewords + n * k);
  {
    std::unordered_map<u32, char> seen;
    for (u64 i = 0; i < n; ++i)
      for (u32 r = 0; 2 * r + 1 < k; ++r)
        seen.emplace(((u32)codewords[i * k + 2 * r] << 16) | codewords[i * k + 2 * r + 1], 0);
    db->n_pairs = seen.size();
  }
  db->rows = c->opt_row_basis && db->sp == 1 && k >= 2;
  // u64 words per row: [4][N] u32 in the row basis, [sp][L][N] otherwise
  const u64 row_words = db->rows ? (u64)c->h.rows.nr * c->N / 2 : (u64)db->sp * c->L * c->N;
  CUDA_TRY(c, db->db.ensure(n * row_words, &c->acct));
  // upload rows in chunks and transform
  const u64 chunk_rows = std::max<u64>(1, (256ull << 20) / (std::max<u32>(plen, 1) * 4ull));
  uint32_t *d_items = nullptr;
  if (plen) {
    CUDA_TRY(c, cudaMalloc(&d_items, std::min(chunk_rows, n) * plen * sizeof(uint32_t)));
  }
  for (u64 r0 = 0; r0 < n; r0 += chunk_rows) {
    u64 nr = std::min(chunk_rows, n - r0);
    if (plen) {
      cudaError_t e = cudaMemcpyAsync(d_items, items + r0 * plen, nr * plen * sizeof(uint32_t),
                                      cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess)
        e = db->rows ? cw::launch_db_load_rows(c->d_tab, c->h, d_items, nr, plen,
                                               reinterpret_cast<u32 *>(db->db.p + r0 * row_words),
                                               c->stream)
                     : cw::launch_db_load(c->d_tab, c->h, d_items, nr, plen, db->sp,
                                          db->db.p + r0 * row_words, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) {
        cudaFree(d_items);
        return fail(c, CWPIR_ECUDA, "database upload: %s", cudaGetErrorString(e));
      }
    }
  }
  if (d_items) cudaFree(d_items);
  if (!plen) CUDA_TRY(c, cudaMemset(db->db.p, 0, n * row_words * sizeof(u64)));
  int32_t id = c->next_db++;
  c->dbs[id] = std::move(db);
  *db_id = id;
  return CWPIR_OK;
}

int cwpir_load_db(cwpir_ctx *c, uint64_t n, uint32_t plen, uint32_t k, uint32_t m,
                  const uint32_t *items, const uint16_t *codewords, int32_t *db_id) {
  return load_db_impl(c, n, plen, k, m, items, codewords, false, db_id);
}

int cwpir_map_folklore(uint64_t y, uint32_t ell, uint16_t *pos_out) {
  if (!pos_out || ell == 0 || ell > 16 || (y >> ell)) return CWPIR_EINVAL;
  for (u32 i = 0; i < ell; ++i) pos_out[i] = (uint16_t)(2 * i + ((y >> i) & 1));
  return CWPIR_OK;
}

int cwpir_load_db_folklore(cwpir_ctx *c, uint64_t n, uint32_t plen, uint32_t ell,
                           const uint32_t *items, int32_t *db_id) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  if (ell < 1 || ell > 16 || n < 1 || n > (1ull << ell))
    return fail(c, CWPIR_EINVAL, "folklore needs 1 <= ell <= 16 and 1 <= n <= 2^ell");
  std::vector<uint16_t> cw(n * ell);
  for (u64 i = 0; i < n; ++i) cwpir_map_folklore(i, ell, cw.data() + i * ell);
  return load_db_impl(c, n, plen, ell, 2 * ell, items, cw.data(), true, db_id);
}

int cwpir_free_db(cwpir_ctx *c, int32_t id) {
  if (!c) return CWPIR_EINVAL;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (!c->dbs.erase(id)) return fail(c, CWPIR_ENODB, "unknown database %d", id);
  return CWPIR_OK;
}

static int query_shape(cwpir_ctx *c, Db *db, u32 cfac, u64 *h) {
  if (cfac > c->logN) return fail(c, CWPIR_EINVAL, "c > log2 N");
  if (db->folklore) {
    if (cfac) return fail(c, CWPIR_EINVAL, "folklore queries are ell bit ciphertexts (c = 0)");
    *h = db->m / 2;
    return CWPIR_OK;
  }
  *h = cfac == 0 ? db->m : (db->m + (1u << cfac) - 1) >> cfac;
  return CWPIR_OK;
}

int cwpir_query_cts(cwpir_ctx *c, int32_t db_id, uint32_t cfac, uint32_t *h) {
  if (!c || !h) return CWPIR_EINVAL;
  Db *db = get_db(c, db_id);
  if (!db) return fail(c, CWPIR_ENODB, "unknown database %d", db_id);
  u64 hh;
  int rc = query_shape(c, db, cfac, &hh);
  if (rc) return rc;
  *h = (uint32_t)hh;
  return CWPIR_OK;
}

int cwpir_answer_batch_slot(cwpir_ctx *c, uint32_t slot, int32_t db_id, uint32_t cfac,
                            uint32_t nq, const uint64_t *d_queries, uint64_t *d_responses,
                            void *stream) {
  if (!c) return CWPIR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  c->err.clear();
  cudaSetDevice(c->device);
  if (!slot_ok(c, slot)) return fail(c, CWPIR_EINVAL, "unknown slot %u", slot);
  Db *db = get_db(c, db_id);
  if (!db) return fail(c, CWPIR_ENODB, "unknown database %d", db_id);
  if (!d_queries || !d_responses || nq == 0) return fail(c, CWPIR_EINVAL, "null buffer or nq = 0");
  u64 h;
  int rc = query_shape(c, db, cfac, &h);
  if (rc || (rc = check_keys(c, cfac))) return rc;
  return answer_batch_enqueue(c, slot, db, cfac, nq, d_queries, d_responses,
                              (cudaStream_t)stream);
}

int cwpir_answer_batch_device(cwpir_ctx *c, int32_t db_id, uint32_t cfac, uint32_t nq,
                              const uint64_t *d_queries, uint64_t *d_responses, void *stream) {
  return cwpir_answer_batch_slot(c, 0, db_id, cfac, nq, d_queries, d_responses, stream);
}

int cwpir_slot_create(cwpir_ctx *c, uint32_t *slot) {
  if (!c || !slot) return CWPIR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  c->err.clear();
  cudaSetDevice(c->device);
  return add_slot(c, slot);
}

int cwpir_slot_release(cwpir_ctx *c, uint32_t slot) {
  if (!c) return CWPIR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  c->err.clear();
  if (slot == 0 || !slot_ok(c, slot)) return fail(c, CWPIR_EINVAL, "slot %u cannot be released", slot);
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaDeviceSynchronize());
  for (auto &kv : c->dbs)
    for (auto it = kv.second->plans.begin(); it != kv.second->plans.end();)
      it = std::get<2>(it->first) == slot ? kv.second->plans.erase(it) : std::next(it);
  c->slots[slot]->release();
  c->slots[slot]->in_use = false;
  return CWPIR_OK;
}

int cwpir_device_status(cwpir_ctx *c, uint32_t slot, void *stream) {
  if (!c) return CWPIR_EINVAL;
  cudaSetDevice(c->device);
  // the wait comes before the context lock, so that other threads keep
  // enqueueing on their slots meanwhile
  const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  c->err.clear();
  if (e != cudaSuccess) return fail(c, CWPIR_ECUDA, "stream: %s", cudaGetErrorString(e));
  if (!slot_ok(c, slot)) return fail(c, CWPIR_EINVAL, "unknown slot %u", slot);
  return check_err_flag(c, slot);
}

int cwpir_inject_status(cwpir_ctx *c, uint32_t slot) {
  if (!c) return CWPIR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (!slot_ok(c, slot)) return fail(c, CWPIR_EINVAL, "unknown slot %u", slot);
  const int one = 1;
  CUDA_TRY(c, cudaMemcpy(c->slots[slot]->d_err, &one, sizeof one, cudaMemcpyHostToDevice));
  return CWPIR_OK;
}

int cwpir_answer_device(cwpir_ctx *c, int32_t db_id, uint32_t cfac, const uint64_t *d_query,
                        uint64_t *d_resp, void *stream) {
  return cwpir_answer_batch_device(c, db_id, cfac, 1, d_query, d_resp, stream);
}

int cwpir_answer_batch(cwpir_ctx *c, int32_t db_id, uint32_t cfac, uint32_t nq,
                       const uint64_t *queries, uint64_t *responses) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  cudaSetDevice(c->device);
  Db *db = get_db(c, db_id);
  if (!db) return fail(c, CWPIR_ENODB, "unknown database %d", db_id);
  if (!queries || !responses || nq == 0) return fail(c, CWPIR_EINVAL, "null buffer or nq = 0");
  u64 h;
  int rc = query_shape(c, db, cfac, &h);
  if (rc || (rc = check_keys(c, cfac))) return rc;
  if (!valid_residues(queries, c->L, c->N, c->q, 2 * h * nq))
    return fail(c, CWPIR_EINVAL, "query residue out of range");
  const u64 ctw = c->ct();
  CUDA_TRY(c, c->io_in.ensure(h * nq * ctw, &c->acct));
  CUDA_TRY(c, c->io_out.ensure((u64)nq * db->sp * ctw, &c->acct));
  CUDA_TRY(c, cudaMemcpyAsync(c->io_in.p, queries, h * nq * ctw * sizeof(u64),
                              cudaMemcpyHostToDevice, c->stream));
  rc = answer_batch_enqueue(c, 0, db, cfac, nq, c->io_in.p, c->io_out.p, c->stream);
  if (rc) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(responses, c->io_out.p, (u64)nq * db->sp * ctw * sizeof(u64),
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return check_err_flag(c);
}

int cwpir_answer(cwpir_ctx *c, int32_t db_id, uint32_t cfac, const uint64_t *query,
                 uint64_t *response) {
  return cwpir_answer_batch(c, db_id, cfac, 1, query, response);
}

int cwpir_sum_responses_device(cwpir_ctx *c, uint32_t count, uint32_t s,
                               const uint64_t *d_parts, uint64_t *d_out, void *stream) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  cudaSetDevice(c->device);
  if (!d_parts || !d_out) return fail(c, CWPIR_EINVAL, "null buffer");
  if (count == 0 || s == 0 || s > CWPIR_MAX_PLAINTEXTS)
    return fail(c, CWPIR_EINVAL, "need count >= 1 and 1 <= s <= %d", CWPIR_MAX_PLAINTEXTS);
  const u64 ctw = c->ct();
  for (u32 p = 0; p < s; ++p)
    CUDA_TRY(c, cw::launch_ct_sum(c->d_tab, c->h, d_parts + p * ctw, count, (u64)s * ctw,
                                  d_out + p * ctw, (cudaStream_t)stream));
  return 0;
}

int cwpir_reduce_responses_device(cwpir_ctx *c, uint32_t s, const uint64_t *d_sums,
                                  uint64_t *d_out, void *stream) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  cudaSetDevice(c->device);
  if (!d_sums || !d_out) return fail(c, CWPIR_EINVAL, "null buffer");
  if (s == 0 || s > CWPIR_MAX_PLAINTEXTS)
    return fail(c, CWPIR_EINVAL, "need 1 <= s <= %d", CWPIR_MAX_PLAINTEXTS);
  CUDA_TRY(c, cw::launch_ct_reduce(c->d_tab, c->h, d_sums, s, d_out, (cudaStream_t)stream));
  return CWPIR_OK;
}

int cwpir_autotune_grid(cwpir_ctx *c, int32_t db_id, uint32_t cfac, uint32_t nq,
                        const uint64_t *d_queries, uint64_t *d_responses, const int64_t *jobs,
                        uint32_t n_jobs, const int64_t *waves, uint32_t n_waves,
                        int64_t *best_jobs, int64_t *best_waves, double *best_ms) {
  if (!c) return CWPIR_EINVAL;
  if (!jobs || !n_jobs || !best_jobs || !best_ms || (n_waves && !waves))
    return fail(c, CWPIR_EINVAL, "null argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaSetDevice(c->device);
  cudaEvent_t e0, e1;
  CUDA_TRY(c, cudaEventCreate(&e0));
  CUDA_TRY(c, cudaEventCreate(&e1));
  const int64_t no_wave = 0;
  const int64_t *wv = n_waves ? waves : &no_wave;
  const uint32_t nw = n_waves ? n_waves : 1;
  double best_t = 1e300;
  int64_t bj = -1, bw = 0;
  int rc = CWPIR_OK;
  for (uint32_t i = 0; i < n_jobs && rc == CWPIR_OK; ++i)
    for (uint32_t w = 0; w < nw && rc == CWPIR_OK; ++w) {
      if ((rc = cwpir_set_option(c, CWPIR_OPT_MAX_JOBS, jobs[i]))) break;
      if ((rc = cwpir_set_option(c, CWPIR_OPT_ROW_GROUP_WAVES, wv[w]))) break;
      // the first call builds the plan (and the graph when enabled)
      rc = cwpir_answer_batch_device(c, db_id, cfac, nq, d_queries, d_responses, c->stream);
      if (rc == CWPIR_EINVAL) {  // this size cannot hold nq queries: skip it
        rc = CWPIR_OK;
        continue;
      }
      if (rc) break;
      cudaEventRecord(e0, c->stream);
      for (int r = 0; r < 2 && rc == CWPIR_OK; ++r)
        rc = cwpir_answer_batch_device(c, db_id, cfac, nq, d_queries, d_responses, c->stream);
      cudaEventRecord(e1, c->stream);
      if (rc) break;
      cudaError_t e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        rc = fail(c, CWPIR_ECUDA, "autotune timing: %s", cudaGetErrorString(e));
        break;
      }
      if (ms / 2 < best_t) {
        best_t = ms / 2;
        bj = jobs[i];
        bw = wv[w];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (bj < 0) return fail(c, CWPIR_EINVAL, "no candidate could hold %u queries", nq);
  if ((rc = cwpir_set_option(c, CWPIR_OPT_MAX_JOBS, bj))) return rc;
  if ((rc = cwpir_set_option(c, CWPIR_OPT_ROW_GROUP_WAVES, bw))) return rc;
  if ((rc = check_err_flag(c, 0))) return rc;
  *best_jobs = bj;
  if (best_waves) *best_waves = bw;
  *best_ms = best_t;
  return CWPIR_OK;
}

int cwpir_autotune(cwpir_ctx *c, int32_t db_id, uint32_t cfac, uint32_t nq,
                   const uint64_t *d_queries, uint64_t *d_responses, const int64_t *cand,
                   uint32_t count, int64_t *best, double *best_ms) {
  return cwpir_autotune_grid(c, db_id, cfac, nq, d_queries, d_responses, cand, count, nullptr, 0,
                             best, nullptr, best_ms);
}

int cwpir_mul(cwpir_ctx *c, const uint64_t *a, const uint64_t *b, uint64_t *out) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  cudaSetDevice(c->device);
  if (!a || !b || !out) return fail(c, CWPIR_EINVAL, "null buffer");
  if (!valid_residues(a, c->L, c->N, c->q, 2) || !valid_residues(b, c->L, c->N, c->q, 2))
    return fail(c, CWPIR_EINVAL, "residue out of range");
  int rc = ensure_scratch(c);
  if (rc) return rc;
  const u64 ctw = c->ct(), qp = c->qp_ct();
  CUDA_TRY(c, c->io_in.ensure(2 * ctw, &c->acct));
  CUDA_TRY(c, c->io_out.ensure(ctw, &c->acct));
  CUDA_TRY(c, c->tmp_ct.ensure(2 * qp, &c->acct));
  CUDA_TRY(c, cudaMemcpyAsync(c->io_in.p, a, ctw * sizeof(u64), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->io_in.p + ctw, b, ctw * sizeof(u64), cudaMemcpyHostToDevice,
                              c->stream));
  if ((rc = prep_leaves(c, c->io_in.p, 2, c->tmp_ct.p, c->stream))) return rc;
  Plan P;
  cw::MulJob job{c->tmp_ct.p, c->tmp_ct.p + qp, c->io_out.p, 0};
  CUDA_TRY(c, cudaMalloc(&P.d_jobs, sizeof job));
  CUDA_TRY(c, cudaMemcpy(P.d_jobs, &job, sizeof job, cudaMemcpyHostToDevice));
  if ((rc = run_chunk(c, *c->slots[0], &P, Chunk{0, 1, cw::ROOT_SEL, 1}, nullptr, c->stream)))
    return rc;
  CUDA_TRY(c, cudaMemcpyAsync(out, c->io_out.p, ctw * sizeof(u64), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return check_err_flag(c);
}

int cwpir_substitute(cwpir_ctx *c, uint32_t g, const uint64_t *ct, uint64_t *out) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  cudaSetDevice(c->device);
  if (!ct || !out) return fail(c, CWPIR_EINVAL, "null buffer");
  const auto *key = find_gal(c, g);
  if (!key) return fail(c, CWPIR_ENOKEY, "no Galois key for element %u", g);
  if (!valid_residues(ct, c->L, c->N, c->q, 2)) return fail(c, CWPIR_EINVAL, "residue out of range");
  const u64 ctw = c->ct();
  CUDA_TRY(c, c->io_in.ensure(ctw, &c->acct));
  CUDA_TRY(c, c->io_out.ensure(ctw, &c->acct));
  CUDA_TRY(c, c->exp_tau.ensure(ctw, &c->acct));
  CUDA_TRY(c, c->exp_DN.ensure((u64)(c->L + 1) * c->L * c->N, &c->acct));
  CUDA_TRY(c, c->exp_O.ensure(ctw, &c->acct));
  int rc = ensure_subjobs(c, 1);
  if (rc) return rc;
  cw::SubJob sj{c->io_in.p, c->io_out.p};
  CUDA_TRY(c, cudaMemcpyAsync(c->io_in.p, ct, ctw * sizeof(u64), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_subjobs, &sj, sizeof sj, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cw::launch_automorph(c->d_tab, c->h, c->d_subjobs, 1, g, c->exp_tau.p, c->stream));
  CUDA_TRY(c, cw::launch_sub_keyswitch(c->d_tab, c->h, c->exp_tau.p, 1, c->d_subjobs,
                                       key->first->p, key->second->p, c->exp_DN.p, c->exp_O.p,
                                       c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(out, c->io_out.p, ctw * sizeof(u64), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return CWPIR_OK;
}

int cwpir_expand(cwpir_ctx *c, uint32_t cfac, uint32_t m, const uint64_t *query, uint64_t *out) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  cudaSetDevice(c->device);
  if (!query || !out) return fail(c, CWPIR_EINVAL, "null buffer");
  if (cfac < 1 || cfac > c->logN || m < 1 || m > 16384)
    return fail(c, CWPIR_EINVAL, "need 1 <= c <= log2 N and 1 <= m <= 16384");
  const u64 h = (m + (1u << cfac) - 1) >> cfac, ctw = c->ct();
  if (!valid_residues(query, c->L, c->N, c->q, 2 * h)) return fail(c, CWPIR_EINVAL, "residue out of range");
  CUDA_TRY(c, c->io_in.ensure(h * ctw, &c->acct));
  CUDA_TRY(c, c->io_out.ensure((u64)m * ctw, &c->acct));
  CUDA_TRY(c, cudaMemcpyAsync(c->io_in.p, query, h * ctw * sizeof(u64), cudaMemcpyHostToDevice,
                              c->stream));
  int rc = check_keys(c, cfac);
  if (rc) return rc;
  Plan P;
  P.nq = 1;
  P.cfac = cfac;
  P.m = m;
  P.h_in = (u32)h;
  if ((rc = setup_expand(c, &P))) return rc;
  if ((rc = enqueue_expand(c, &P, c->io_in.p, c->stream))) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(out, P.leaves_coef.p, (u64)m * ctw * sizeof(u64),
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return CWPIR_OK;
}

int cwpir_selection(cwpir_ctx *c, int32_t db_id, uint32_t cfac, const uint64_t *query,
                    uint64_t count, const uint64_t *rows, uint64_t *out) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  cudaSetDevice(c->device);
  Db *db = get_db(c, db_id);
  if (!db) return fail(c, CWPIR_ENODB, "unknown database %d", db_id);
  if (!query || !rows || !out || count == 0) return fail(c, CWPIR_EINVAL, "null buffer or empty");
  for (u64 i = 0; i < count; ++i)
    if (rows[i] >= db->n) return fail(c, CWPIR_EINVAL, "row out of range");
  u64 h;
  int rc = query_shape(c, db, cfac, &h);
  if (rc) return rc;
  if (!valid_residues(query, c->L, c->N, c->q, 2 * h)) return fail(c, CWPIR_EINVAL, "residue out of range");
  if ((rc = ensure_scratch(c))) return rc;
  const u64 ctw = c->ct();
  CUDA_TRY(c, c->io_in.ensure(h * ctw, &c->acct));
  CUDA_TRY(c, c->io_out.ensure(count * ctw, &c->acct));
  CUDA_TRY(c, cudaMemcpyAsync(c->io_in.p, query, h * ctw * sizeof(u64), cudaMemcpyHostToDevice,
                              c->stream));
  if ((rc = check_keys(c, cfac))) return rc;
  std::vector<u64> rv(rows, rows + count);
  std::unique_ptr<Plan> P;
  if ((rc = build_plan(c, 0, db, rv, 1, cfac, cw::ROOT_SEL, c->io_out.p, c->opt_share != 0, P)))
    return rc;
  const u64 *coef;
  if ((rc = leaf_coefs(c, db, P.get(), c->io_in.p, c->stream, &coef))) return rc;
  if (db->k == 1) {
    // the selection entry is the (expanded) query ciphertext itself
    for (u64 i = 0; i < count; ++i)
      CUDA_TRY(c, cudaMemcpyAsync(out + i * ctw, coef + db->cw[rows[i]] * ctw, ctw * sizeof(u64),
                                  cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return CWPIR_OK;
  }
  if ((rc = prep_leaves(c, coef, db->m, P->leaves.p, c->stream))) return rc;
  for (const Chunk &ch : P->memo_chunks)
    if ((rc = run_chunk(c, *c->slots[0], P.get(), ch, nullptr, c->stream))) return rc;
  for (const auto &batch : P->batches)
    for (const Chunk &ch : batch)
      if ((rc = run_chunk(c, *c->slots[0], P.get(), ch, nullptr, c->stream))) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(out, c->io_out.p, count * ctw * sizeof(u64), cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return check_err_flag(c);
}

// The plan of the selection entries (coefficient form, [rows][2][L][N] at
// out) of every row of a database description d, kept by the caller: its
// jobs point into its own buffers and at out.
static int rows_plan(cwpir_ctx *c, Db &d, u64 *out, std::unique_ptr<Plan> &P) {
  std::vector<u64> rv(d.n);
  for (u64 i = 0; i < d.n; ++i) rv[i] = i;
  return build_plan(c, 0, &d, rv, 1, 0, cw::ROOT_SEL, out, false, P);
}

// Enqueues the plan's products over the coefficient-form leaves `coef`
// ([d.m][2][L][N]).
static int run_rows_plan(cwpir_ctx *c, Db &d, Plan *P, const u64 *coef) {
  int rc = prep_leaves(c, coef, d.m, P->leaves.p, c->stream);
  if (rc) return rc;
  for (const auto &batch : P->batches)
    for (const Chunk &ch : batch)
      if ((rc = run_chunk(c, *c->slots[0], P, ch, nullptr, c->stream))) return rc;
  return CWPIR_OK;
}

int cwpir_arith_cw_eq(cwpir_ctx *c, uint32_t m, uint32_t k, const uint64_t *x,
                      const uint64_t *y, uint64_t *out) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  cudaSetDevice(c->device);
  if (!x || !y || !out) return fail(c, CWPIR_EINVAL, "null buffer");
  if (k < 1 || k > 16 || k > m || m > 8192)
    return fail(c, CWPIR_EINVAL, "need 1 <= k <= 16, k <= m <= 8192");
  int rc = ensure_scratch(c);
  if (rc) return rc;
  const u64 ctw = c->ct();
  // leaves x_0 .. x_{m-1}, y_0 .. y_{m-1}; then m products, their sum, the
  // k factors and their product
  auto &A = c->arith;
  if (A.m != m || A.k != k) {
    A.clear();
    CUDA_TRY(c, A.leaves.ensure(2ull * m * ctw, &c->acct));
    CUDA_TRY(c, A.prods.ensure((u64)m * ctw, &c->acct));
    CUDA_TRY(c, A.fac.ensure((u64)(k + 2) * ctw, &c->acct));
    CUDA_TRY(c, A.flag.ensure(1, &c->acct));
    // k' = sum_i x_i y_i: rows i with codewords {i, m + i}
    A.d1.n = m;
    A.d1.k = 2;
    A.d1.m = 2 * m;
    A.d1.cw.resize(2ull * m);
    for (u32 i = 0; i < m; ++i) {
      A.d1.cw[2 * i] = (uint16_t)i;
      A.d1.cw[2 * i + 1] = (uint16_t)(m + i);
    }
    if ((rc = rows_plan(c, A.d1, A.prods.p, A.p1))) return rc;
    if (k > 1) {  // the product of the k factors by the balanced tree
      A.d2.n = 1;
      A.d2.k = k;
      A.d2.m = k;
      A.d2.cw.resize(k);
      for (u32 i = 0; i < k; ++i) A.d2.cw[i] = (uint16_t)i;
      if ((rc = rows_plan(c, A.d2, A.fac.p + (u64)(k + 1) * ctw, A.p2))) return rc;
    }
    A.m = m;
    A.k = k;
  }
  CUDA_TRY(c, cudaMemcpyAsync(A.leaves.p, x, (u64)m * ctw * sizeof(u64), cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(A.leaves.p + (u64)m * ctw, y, (u64)m * ctw * sizeof(u64),
                              cudaMemcpyHostToDevice, c->stream));
  // the residue check runs on the device (the operands are large); its flag
  // is read once the call has finished
  int *flag = reinterpret_cast<int *>(A.flag.p);
  CUDA_TRY(c, cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  CUDA_TRY(c, cw::launch_check_residues(c->d_tab, c->h, A.leaves.p, 2ull * m, flag, c->stream));
  if ((rc = run_rows_plan(c, A.d1, A.p1.get(), A.leaves.p))) return rc;
  u64 *kp = A.fac.p + (u64)k * ctw, *res = A.fac.p + (u64)(k + 1) * ctw;
  CUDA_TRY(c, cw::launch_ct_sum(c->d_tab, c->h, A.prods.p, m, c->ct(), kp, c->stream));
  // factors k' - i, i < k, and their product
  CUDA_TRY(c, cw::launch_minus_consts(c->d_tab, c->h, kp, k, A.fac.p, c->stream));
  const u64 *prod = A.fac.p;
  if (k > 1) {
    if ((rc = run_rows_plan(c, A.d2, A.p2.get(), A.fac.p))) return rc;
    prod = res;
  }
  // times (k!)^-1 mod t
  u64 kf = 1;
  for (u32 i = 2; i <= k; ++i) kf = kf * i % c->t;
  const u64 s = hpow(kf, c->t - 2, c->t);
  CUDA_TRY(c, cw::launch_ct_scalar(c->d_tab, c->h, prod, s, kp, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(out, kp, ctw * sizeof(u64), cudaMemcpyDeviceToHost, c->stream));
  int bad = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (bad) return fail(c, CWPIR_EINVAL, "residue out of range");
  return check_err_flag(c);
}

int cwpir_plain_mul(cwpir_ctx *c, int32_t db_id, uint64_t row, const uint64_t *ct, uint64_t *out) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  cudaSetDevice(c->device);
  Db *db = get_db(c, db_id);
  if (!db) return fail(c, CWPIR_ENODB, "unknown database %d", db_id);
  if (!ct || !out || row >= db->n) return fail(c, CWPIR_EINVAL, "null buffer or row out of range");
  if (!valid_residues(ct, c->L, c->N, c->q, 2)) return fail(c, CWPIR_EINVAL, "residue out of range");
  const u64 ctw = c->ct(), LN = (u64)c->L * c->N, sp = db->sp;
  CUDA_TRY(c, c->io_in.ensure(sp * ctw, &c->acct));
  CUDA_TRY(c, c->io_out.ensure(sp * ctw, &c->acct));
  CUDA_TRY(c, c->tmp_ct.ensure(ctw, &c->acct));
  CUDA_TRY(c, cudaMemcpyAsync(c->io_in.p, ct, ctw * sizeof(u64), cudaMemcpyHostToDevice, c->stream));
  if (db->rows) {  // the exact integer product in the row basis, back to each q_j
    int rc = ensure_scratch(c);
    if (rc) return rc;
    Scratch &S = *c->slots[0];
    CUDA_TRY(c, c->one_job.ensure((sizeof(cw::MulJob) + 7) / 8, &c->acct));
    const cw::MulJob job{nullptr, nullptr, nullptr, row};
    CUDA_TRY(c, cudaMemcpyAsync(c->one_job.p, &job, sizeof job, cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cw::launch_plain_mul_rows(
                    c->d_tab, c->h, c->io_in.p, reinterpret_cast<const cw::MulJob *>(c->one_job.p),
                    reinterpret_cast<const u32 *>(db->db.p), reinterpret_cast<u32 *>(S.DN.p),
                    reinterpret_cast<u32 *>(S.RS.p), S.d_err, c->io_out.p, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(out, c->io_out.p, ctw * sizeof(u64), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return check_err_flag(c);
  }
  CUDA_TRY(c, cw::launch_ntt(c->d_tab, c->h, c->tmp_ct.p, 2, LN, 0, c->L, false, c->io_in.p, LN,
                             c->stream));
  for (u64 p = 0; p < sp; ++p)
    CUDA_TRY(c, cw::launch_pm_ntt(c->d_tab, c->h, c->tmp_ct.p, db->db.p + (row * sp + p) * LN,
                                  c->io_in.p + p * ctw, c->stream));
  CUDA_TRY(c, cw::launch_ntt(c->d_tab, c->h, c->io_out.p, 2 * (u32)sp, LN, 0, c->L, true,
                             c->io_in.p, LN, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(out, c->io_out.p, sp * ctw * sizeof(u64), cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return CWPIR_OK;
}

int cwpir_db_shape(const cwpir_ctx *c, int32_t db_id, uint32_t *N, uint32_t *L, uint32_t *m) {
  if (!c || !N || !L || !m) return CWPIR_EINVAL;
  auto it = c->dbs.find(db_id);
  if (it == c->dbs.end()) return CWPIR_ENODB;
  *N = c->N;
  *L = c->L;
  *m = it->second->m;
  return CWPIR_OK;
}

int cwpir_db_plaintexts(const cwpir_ctx *c, int32_t db_id, uint32_t *sp) {
  if (!c || !sp) return CWPIR_EINVAL;
  auto it = c->dbs.find(db_id);
  if (it == c->dbs.end()) return CWPIR_ENODB;
  *sp = it->second->sp;
  return CWPIR_OK;
}

int cwpir_ctx_device(const cwpir_ctx *c, int *device) {
  if (!c || !device) return CWPIR_EINVAL;
  *device = c->device;
  return CWPIR_OK;
}

int cwpir_plan_bytes_slot(cwpir_ctx *c, uint32_t slot, int32_t db_id, uint32_t nq,
                          uint32_t cfac, uint64_t *bytes) {
  if (!c || !bytes || !nq) return CWPIR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  if (!slot_ok(c, slot)) return fail(c, CWPIR_EINVAL, "unknown slot %u", slot);
  Db *db = get_db(c, db_id);
  if (!db) return fail(c, CWPIR_ENODB, "unknown database %d", db_id);
  if (db->plans.count(std::make_tuple(nq, cfac, slot))) {
    *bytes = 0;
    return CWPIR_OK;
  }
  const u64 N = c->N, L = c->L, qp = c->qp_ct(), ctw = c->ct();
  const u64 J = c->jmax ? c->jmax : jobs_per_launch(c);
  const Scratch &S = *c->slots[slot];
  u64 w = 0;
  if (!S.Tbuf.n) {  // the slot's scratch comes first
    const u64 per_job = 3 * cw::tensor_poly_words(c->K, c->N) + (3 * L + 2 * L) * N + dn_words(L, N);
    w += J * per_job + rs_words(L, N) + dnq_words(L, N);
  }
  const u32 top = [&] { u32 l = 0; while ((1u << l) < db->k) ++l; return l; }();
  const bool memo = c->opt_share && top >= 2;
  const u64 h = db->folklore ? db->m / 2 : cfac ? (db->m + (1u << cfac) - 1) >> cfac : db->m;
  w += (u64)nq * db->m * qp + 2ull * nq * db->sp * ctw + (u64)nq * h * ctw;
  if (db->folklore) w += (u64)nq * db->m * ctw;
  if (db->sp > 1 && db->k > 1 && S.SEL.n < J * ctw) w += J * ctw;
  if (memo) w += (u64)nq * db->n_pairs * qp;
  u64 widest = 1, internal_nodes = 0;
  for (u32 l = memo ? 2 : 1; l <= top; ++l) {
    u64 nodes = (db->k + (1u << l) - 1) >> l;
    widest = std::max(widest, nodes);
    if (l < top) internal_nodes += nodes;
  }
  const u64 rpb = std::max<u64>(1, J / (nq * widest));
  w += (u64)nq * rpb * internal_nodes * qp;
  if (cfac) {
    const u64 B = 1ull << cfac, in = (u64)nq * h;
    w += 2 * in * B * ctw + 3 * in * (B / 2) * ctw + in * (B / 2) * (L + 1) * L * N +
         (u64)nq * db->m * ctw;
  }
  *bytes = w * sizeof(u64) + (u64)nq * (db->n + db->n_pairs) * db->k * sizeof(cw::MulJob);
  return CWPIR_OK;
}

int cwpir_plan_bytes(cwpir_ctx *c, int32_t db_id, uint32_t nq, uint32_t cfac,
                     uint64_t *bytes) {
  return cwpir_plan_bytes_slot(c, 0, db_id, nq, cfac, bytes);
}

int cwpir_release_plans(cwpir_ctx *c, int32_t db_id) {
  if (!c) return CWPIR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  cudaDeviceSynchronize();
  if (db_id < 0) {
    for (auto &kv : c->dbs) kv.second->plans.clear();
    c->arith.clear();
    return CWPIR_OK;
  }
  Db *db = get_db(c, db_id);
  if (!db) return fail(c, CWPIR_ENODB, "unknown database %d", db_id);
  db->plans.clear();
  return CWPIR_OK;
}

// Waits for the device and drops every cached plan (their graphs and job
// lists depend on the option being changed).
static void drop_plans(cwpir_ctx *c) {
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  cudaDeviceSynchronize();
  for (auto &kv : c->dbs) kv.second->plans.clear();
  c->arith.clear();
}

int cwpir_set_option(cwpir_ctx *c, int option, int64_t value) {
  if (!c) return CWPIR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  switch (option) {
    case CWPIR_OPT_SHARE_LEVEL1:
      drop_plans(c);
      c->opt_share = value ? 1 : 0;
      return CWPIR_OK;
    case CWPIR_OPT_BATCH_ROWS:
      if (value < 0 || value > 0xffffffffll)
        return fail(c, CWPIR_EINVAL, "batch rows must be in [0, 2^32)");
      drop_plans(c);
      c->opt_batch_rows = (u32)value;
      return CWPIR_OK;
    case CWPIR_OPT_USE_GRAPH:
      c->opt_graph = value ? 1 : 0;
      return CWPIR_OK;
    case CWPIR_OPT_KERNEL_TIMING: c->opt_timing = value ? 1 : 0; return CWPIR_OK;
    case CWPIR_OPT_ROW_BASIS: c->opt_row_basis = value ? 1 : 0; return CWPIR_OK;
    case CWPIR_OPT_MAX_JOBS:
      if (value < 0 || value > (int64_t)kMaxJobs)
        return fail(c, CWPIR_EINVAL, "max jobs must be in [0, %llu]", (unsigned long long)kMaxJobs);
      drop_plans(c);
      c->opt_max_jobs = (u32)value;
      c->jmax = 0;  // scratch is re-sized on the next call that needs it
      for (auto &S : c->slots) S->release();
      c->scratch_gen += 1;
      return CWPIR_OK;
    case CWPIR_OPT_MEM_LIMIT:
      if (value < 0) return fail(c, CWPIR_EINVAL, "memory limit must be >= 0");
      c->acct.limit = (u64)value;
      return CWPIR_OK;
    case CWPIR_OPT_ROW_GROUP_WAVES:
      if (value < 0 || value > 64) return fail(c, CWPIR_EINVAL, "row-group waves must be in [0, 64]");
      drop_plans(c);
      c->h.row_waves = value ? (u32)value : cw::kDefaultRowWaves;
      return CWPIR_OK;
    case CWPIR_OPT_SCALE_EXACT:
      if (value < 0 || value > 1) return fail(c, CWPIR_EINVAL, "scale-exact must be 0 or 1");
      drop_plans(c);
      c->h.scalep.exact_all = (u32)value;  // read from the launch parameters
      return CWPIR_OK;
    default: return fail(c, CWPIR_EINVAL, "unknown option %d", option);
  }
}

int cwpir_get_option(cwpir_ctx *c, int option, int64_t *value) {
  if (!c || !value) return CWPIR_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  switch (option) {
    case CWPIR_OPT_SHARE_LEVEL1: *value = c->opt_share; return CWPIR_OK;
    case CWPIR_OPT_BATCH_ROWS: *value = c->opt_batch_rows; return CWPIR_OK;
    case CWPIR_OPT_USE_GRAPH: *value = c->opt_graph; return CWPIR_OK;
    case CWPIR_OPT_KERNEL_TIMING: *value = c->opt_timing; return CWPIR_OK;
    case CWPIR_OPT_MAX_JOBS: *value = c->opt_max_jobs; return CWPIR_OK;
    case CWPIR_OPT_ROW_BASIS: *value = c->opt_row_basis; return CWPIR_OK;
    case CWPIR_OPT_MEM_LIMIT: *value = (int64_t)c->acct.limit; return CWPIR_OK;
    case CWPIR_OPT_ROW_GROUP_WAVES: *value = c->h.row_waves; return CWPIR_OK;
    case CWPIR_OPT_SCALE_EXACT: *value = c->h.scalep.exact_all; return CWPIR_OK;
    default: return fail(c, CWPIR_EINVAL, "unknown option %d", option);
  }
}

int cwpir_mem_used(const cwpir_ctx *c, uint64_t *bytes) {
  if (!c || !bytes) return CWPIR_EINVAL;
  *bytes = c->acct.used;
  return CWPIR_OK;
}

int cwpir_kernel_times(cwpir_ctx *c, double *ms, uint64_t *launches) {
  if (!c || !ms || !launches) return CWPIR_EINVAL;
  cudaSetDevice(c->device);
  for (const auto &mk : c->ev_marks) {
    CUDA_TRY(c, cudaEventSynchronize(c->ev_pool[mk.second.second]));
    float t = 0;
    CUDA_TRY(c, cudaEventElapsedTime(&t, c->ev_pool[mk.second.first], c->ev_pool[mk.second.second]));
    c->kt_ms[mk.first] += t;
    c->kt_n[mk.first] += 1;
  }
  c->ev_marks.clear();
  c->ev_used = 0;
  for (int i = 0; i < CWPIR_K_CLASSES; ++i) {
    ms[i] = c->kt_ms[i];
    launches[i] = c->kt_n[i];
    c->kt_ms[i] = 0;
    c->kt_n[i] = 0;
  }
  return CWPIR_OK;
}

const char *cwpir_kernel_class_name(int cls) {
  static const char *names[CWPIR_K_CLASSES] = {"tensor", "scale", "relin_pm", "lift",
                                                "ntt", "accumulate", "expand", "row_ntt"};
  return (cls >= 0 && cls < CWPIR_K_CLASSES) ? names[cls] : "unknown";
}

int cwpir_last_stats(const cwpir_ctx *c, cwpir_stats *out) {
  if (!c || !out) return CWPIR_EINVAL;
  *out = c->stats;
  return CWPIR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------
// Batched answering across databases (configuration 4): one launch
// sequence for the queries of several resident databases, one branch per
// database on its own stream and scratch slot, forked from and joined into
// the caller's stream, captured once into a single CUDA graph.
// ---------------------------------------------------------------------
struct MultiItem {
  cwpir_ctx *c = nullptr;
  int32_t db_id = 0;
  Db *db = nullptr;
  u32 cfac = 0, nq = 0, nq_call = 0, slot = 0;
  u64 qw = 0, rw = 0;  // u64 words of one query and of one response
  u64 gen = 0;         // the context's scratch_gen when the plan was built
  std::unique_ptr<Plan> plan;
  DevBuf qstage, rstage;  // [nq][h][2][L][N] and [nq][s][2][L][N]
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
};

struct cwpir_multi {
  std::vector<std::unique_ptr<MultiItem>> items;
  int device = 0;
  cudaStream_t main = nullptr;
  cudaEvent_t fork = nullptr, sync = nullptr;
  cudaGraphExec_t graph = nullptr;
  cwpir_stats stats{};
  std::string err;
  ~cwpir_multi() {
    if (graph) cudaGraphExecDestroy(graph);
    for (auto &ip : items) {
      MultiItem &it = *ip;
      if (it.st) cudaStreamDestroy(it.st);
      if (it.done) cudaEventDestroy(it.done);
      it.plan.reset();
      if (it.slot) cwpir_slot_release(it.c, it.slot);
    }
    if (fork) cudaEventDestroy(fork);
    if (sync) cudaEventDestroy(sync);
    if (main) cudaStreamDestroy(main);
  }
};

namespace {

// Locks the contexts of a multi object in address order.
struct MultiLock {
  std::vector<std::unique_lock<std::recursive_mutex>> locks;
  explicit MultiLock(const cwpir_multi *mb) {
    std::vector<cwpir_ctx *> cs;
    for (const auto &it : mb->items) cs.push_back(it->c);
    std::sort(cs.begin(), cs.end());
    cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
    for (cwpir_ctx *c : cs) locks.emplace_back(c->mu);
  }
};

int multi_fail(cwpir_multi *mb, int code, const cwpir_ctx *c) {
  mb->err = c ? c->err : std::string("invalid argument");
  return code;
}

// (Re)builds an item's plan when it has none or its context's scratch was
// re-sized since.
int multi_plan(MultiItem &it, bool *rebuilt) {
  cwpir_ctx *c = it.c;
  if (get_db(c, it.db_id) != it.db) return fail(c, CWPIR_ENODB, "database %d was freed", it.db_id);
  int rc = ensure_scratch(c, it.slot);
  if (rc) return rc;
  if (it.plan && it.gen == c->scratch_gen) return CWPIR_OK;
  std::vector<u64> rows(it.db->n);
  for (u64 i = 0; i < it.db->n; ++i) rows[i] = i;
  it.plan.reset();
  if ((rc = build_plan(c, it.slot, it.db, rows, it.nq_call, it.cfac, cw::ROOT_PM, nullptr,
                       c->opt_share != 0, it.plan)))
    return rc;
  it.gen = c->scratch_gen;
  *rebuilt = true;
  return CWPIR_OK;
}

// Every item's branch: fork from `main`, the item's sub-batches of nq_call
// queries from qstage to rstage on the item's stream, join into `main`.
int multi_enqueue(cwpir_multi *mb) {
  CUDA_TRY(mb->items[0]->c, cudaEventRecord(mb->fork, mb->main));
  mb->stats = cwpir_stats{};
  for (auto &ip : mb->items) {
    MultiItem &it = *ip;
    cwpir_ctx *c = it.c;
    CUDA_TRY(c, cudaStreamWaitEvent(it.st, mb->fork, 0));
    Scratch &S = *c->slots[it.slot];
    for (u32 j = 0; j < it.nq / it.nq_call; ++j) {
      c->stats = cwpir_stats{};
      int rc = enqueue_answer(c, S, it.db, it.plan.get(), it.qstage.p + (u64)j * it.nq_call * it.qw,
                              it.rstage.p + (u64)j * it.nq_call * it.rw, it.st);
      if (rc) return rc;
      mb->stats.rows += c->stats.rows;
      mb->stats.mults += c->stats.mults;
      mb->stats.substitutions += c->stats.substitutions;
      mb->stats.ntt_polys += c->stats.ntt_polys;
      mb->stats.kernel_launches += c->stats.kernel_launches;
      mb->stats.db_bytes_read += c->stats.db_bytes_read;
    }
    CUDA_TRY(c, cudaEventRecord(it.done, it.st));
    CUDA_TRY(c, cudaStreamWaitEvent(mb->main, it.done, 0));
  }
  return CWPIR_OK;
}

}  // namespace

extern "C" {

int cwpir_multi_create(const cwpir_multi_item *items, uint32_t count, cwpir_multi **out) {
  if (!items || !count || !out) return CWPIR_EINVAL;
  std::unique_ptr<cwpir_multi> mb(new (std::nothrow) cwpir_multi());
  if (!mb) return CWPIR_ENOMEM;
  for (uint32_t i = 0; i < count; ++i) {
    cwpir_ctx *c = items[i].ctx;
    if (!c) return CWPIR_EINVAL;
    if (i == 0) mb->device = c->device;
    if (c->device != mb->device) return fail(c, CWPIR_EINVAL, "items on different devices");
  }
  cudaSetDevice(mb->device);
  for (uint32_t i = 0; i < count; ++i) {
    cwpir_ctx *c = items[i].ctx;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    c->err.clear();
    mb->items.emplace_back(new MultiItem());
    MultiItem &it = *mb->items.back();
    it.c = c;
    it.db_id = items[i].db_id;
    it.cfac = items[i].c;
    it.nq = items[i].nq;
    it.nq_call = items[i].nq_call ? items[i].nq_call : items[i].nq;
    if (!(it.db = get_db(c, it.db_id))) return fail(c, CWPIR_ENODB, "unknown database %d", it.db_id);
    if (!it.nq || it.nq % it.nq_call)
      return fail(c, CWPIR_EINVAL, "nq must be a positive multiple of nq_call");
    u64 h;
    int rc = query_shape(c, it.db, it.cfac, &h);
    if (rc || (rc = check_keys(c, it.cfac))) return rc;
    it.qw = h * c->ct();
    it.rw = (u64)it.db->sp * c->ct();
    if ((rc = add_slot(c, &it.slot))) return rc;
    CUDA_TRY(c, it.qstage.ensure((u64)it.nq * it.qw, &c->acct));
    CUDA_TRY(c, it.rstage.ensure((u64)it.nq * it.rw, &c->acct));
    CUDA_TRY(c, cudaStreamCreateWithFlags(&it.st, cudaStreamNonBlocking));
    CUDA_TRY(c, cudaEventCreateWithFlags(&it.done, cudaEventDisableTiming));
    bool rebuilt = false;
    if ((rc = multi_plan(it, &rebuilt))) return rc;
  }
  if (cudaStreamCreateWithFlags(&mb->main, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&mb->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&mb->sync, cudaEventDisableTiming) != cudaSuccess)
    return CWPIR_ECUDA;
  *out = mb.release();
  return CWPIR_OK;
}

int cwpir_multi_answer_device(cwpir_multi *mb, const uint64_t *const *d_queries,
                              uint64_t *const *d_responses, int use_graph, void *stream) {
  if (!mb || !d_queries || !d_responses) return CWPIR_EINVAL;
  MultiLock lk(mb);
  cudaSetDevice(mb->device);
  mb->err.clear();
  const cudaStream_t st = (cudaStream_t)stream;
  const size_t n = mb->items.size();
  cwpir_ctx *c0 = mb->items[0]->c;
  bool rebuilt = false;
  for (size_t i = 0; i < n; ++i) {
    MultiItem &it = *mb->items[i];
    it.c->err.clear();
    if (!d_queries[i] || !d_responses[i]) return CWPIR_EINVAL;
    int rc = multi_plan(it, &rebuilt);
    if (rc) return multi_fail(mb, rc, it.c);
  }
  if (rebuilt && mb->graph) {
    cudaGraphExecDestroy(mb->graph);
    mb->graph = nullptr;
  }
  // queries in on the caller's stream, which `main` then follows
  for (size_t i = 0; i < n; ++i) {
    MultiItem &it = *mb->items[i];
    CUDA_TRY(it.c, cudaMemcpyAsync(it.qstage.p, d_queries[i], it.nq * it.qw * sizeof(u64),
                                   cudaMemcpyDeviceToDevice, st));
  }
  CUDA_TRY(c0, cudaEventRecord(mb->sync, st));
  CUDA_TRY(c0, cudaStreamWaitEvent(mb->main, mb->sync, 0));
  int rc = CWPIR_OK;
  if (!use_graph) {
    rc = multi_enqueue(mb);
    if (rc) return multi_fail(mb, rc, c0);
  } else {
    if (!mb->graph) {
      for (auto &ip : mb->items) ip->c->capturing = true;
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(mb->main, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        rc = multi_enqueue(mb);
        e = cudaStreamEndCapture(mb->main, &g);
      }
      for (auto &ip : mb->items) ip->c->capturing = false;
      if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(&mb->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (rc) return multi_fail(mb, rc, c0);
      if (e != cudaSuccess) {
        mb->err = std::string("graph capture: ") + cudaGetErrorString(e);
        return CWPIR_ECUDA;
      }
    }
    const cudaError_t e = cudaGraphLaunch(mb->graph, mb->main);
    if (e != cudaSuccess) {
      mb->err = std::string("graph launch: ") + cudaGetErrorString(e);
      return CWPIR_ECUDA;
    }
  }
  // responses out on the caller's stream, after `main`
  CUDA_TRY(c0, cudaEventRecord(mb->sync, mb->main));
  CUDA_TRY(c0, cudaStreamWaitEvent(st, mb->sync, 0));
  for (size_t i = 0; i < n; ++i) {
    MultiItem &it = *mb->items[i];
    CUDA_TRY(it.c, cudaMemcpyAsync(d_responses[i], it.rstage.p, it.nq * it.rw * sizeof(u64),
                                   cudaMemcpyDeviceToDevice, st));
  }
  return CWPIR_OK;
}

int cwpir_multi_status(cwpir_multi *mb, void *stream) {
  if (!mb) return CWPIR_EINVAL;
  int worst = CWPIR_OK;
  for (auto &ip : mb->items) {
    const int rc = cwpir_device_status(ip->c, ip->slot, stream);
    if (rc && !worst) {
      worst = rc;
      mb->err = ip->c->err;
    }
  }
  return worst;
}

int cwpir_multi_stats(const cwpir_multi *mb, cwpir_stats *out) {
  if (!mb || !out) return CWPIR_EINVAL;
  *out = mb->stats;
  return CWPIR_OK;
}

const char *cwpir_multi_last_error(const cwpir_multi *mb) { return mb ? mb->err.c_str() : ""; }

void cwpir_multi_destroy(cwpir_multi *mb) {
  if (!mb) return;
  cudaSetDevice(mb->device);
  if (mb->main) cudaStreamSynchronize(mb->main);
  delete mb;
}

}  // extern "C"

// ---------------------------------------------------------------------
// Multiplication that allocates nothing.
//
// For callers that cannot allocate device memory on the answer path (a
// process whose memory pool is fixed at start-up, a caller inside a
// section where cudaMalloc is forbidden or would stall other work, a host
// runtime that pre-partitions HBM): the intermediates of one homomorphic
// multiplication live in this file-scope device array instead of
// context-owned buffers.  Every GPU that loads the library holds the array
// until the process exits.
// ---------------------------------------------------------------------
namespace {

// 2^20 words (8 MiB) of intermediates plus a 64-word header (error flag at
// word 0, the job descriptor at words 8..11).
constexpr size_t kNoAllocWords = size_t(1) << 20;
constexpr size_t kNoAllocHeader = 64;
static __device__ __align__(256) u64 g_noalloc_scratch[kNoAllocHeader + kNoAllocWords];

std::mutex g_noalloc_mu;
u64 *g_noalloc_addr[256] = {};

// Address of the array on the current device; resolved once per device.
int noalloc_scratch(cwpir_ctx *c, u64 **out) {
  if (c->device < 0 || c->device >= 256) return fail(c, CWPIR_EINVAL, "device index");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[c->device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(c, CWPIR_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_noalloc_addr[c->device] = (u64 *)p;
  }
  *out = g_noalloc_addr[c->device];
  return CWPIR_OK;
}

}  // namespace

extern "C" int cwpir_mul_noalloc(cwpir_ctx *c, const uint64_t *d_a, const uint64_t *d_b,
                                 uint64_t *d_out, void *stream) {
  if (!c) return CWPIR_EINVAL;
  c->err.clear();
  if (!d_a || !d_b || !d_out) return fail(c, CWPIR_EINVAL, "null buffer");
  const u64 LK = c->L + c->K, N = c->N, L = c->L;
  const u64 pw = c->qp_poly(), qp = 2 * pw;
  const u64 need = 2 * qp + 3 * pw + 3 * L * N + (L + 2) * L * N + 2 * L * N;
  if (need > kNoAllocWords)
    return fail(c, CWPIR_EINVAL,
                "N=%u, L=%u needs (L^2 + 14L + 7K/2)N = %llu scratch words (K = %u extension "
                "primes); the static array holds %llu (N = 4096 allows L <= 7, N = 8192 "
                "allows L <= 4, N = 16384 allows L <= 2)",
                c->N, c->L, (unsigned long long)need, c->K,
                (unsigned long long)kNoAllocWords);
  cudaSetDevice(c->device);
  u64 *base = nullptr;
  int rc = noalloc_scratch(c, &base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int *err = (int *)base;
  cw::MulJob *job_dev = (cw::MulJob *)(base + 8);
  u64 *qa = base + kNoAllocHeader, *qb = qa + qp, *tb = qb + qp, *eb = tb + 3 * pw;
  u64 *dn = eb + 3 * L * N, *ob = dn + (L + 2) * L * N;
  cw::MulJob job{qa, qb, d_out, 0};
  // the array keeps the previous call's contents: clear the error flag
  CUDA_TRY(c, cudaMemsetAsync(err, 0, sizeof(int), st));
  CUDA_TRY(c, cudaMemcpyAsync(job_dev, &job, sizeof job, cudaMemcpyHostToDevice, st));
  CUDA_TRY(c, cw::launch_lift(c->d_tab, c->h, d_a, (u64)c->L * N, qa, pw, 2, true, st));
  CUDA_TRY(c, cw::launch_lift(c->d_tab, c->h, d_b, (u64)c->L * N, qb, pw, 2, true, st));
  CUDA_TRY(c, cw::launch_ntt(c->d_tab, c->h, qa, 4, pw, 0, (u32)LK, false, nullptr, 0, st));
  CUDA_TRY(c, cw::launch_tensor(c->d_tab, c->h, job_dev, 1, tb, st));
  CUDA_TRY(c, cw::launch_scale(c->d_tab, c->h, tb, 1, eb, err, st));
  CUDA_TRY(c, cw::launch_relin(c->d_tab, c->h, eb, 1, 1, job_dev, cw::ROOT_SEL, c->rlk.p,
                               c->rlk_s.p, nullptr, 1, 1, dn, nullptr, ob, st));
  int h_err = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if (h_err) return fail(c, CWPIR_EINTERNAL, "device consistency check failed (scale-down)");
  return CWPIR_OK;
}
