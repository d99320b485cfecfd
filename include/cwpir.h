/*
 * cwpir.h -- C ABI of the GB300 (sm_103a) server answer path of
 * constant-weight PIR (Mahdavi & Kerschbaum, arXiv 2202.07569).
 *
 * The calls follow the paper's protocol stages (Sec. 3.3, Table "Stages of
 * PIR using constant-weight codewords"): Setup (parameters and evaluation
 * keys, then the database in plaintext form) and Process (query expansion,
 * selection vector, inner product).  Query construction and Extract are
 * client-side and not part of this library.
 *
 * Conventions shared by every call
 *  - Ring: R_Q = Z_Q[x]/(x^N + 1) with Q = q_0 * ... * q_{L-1}; plaintexts in
 *    R_t (Sec. 2.1.1).  N is a power of two in [1024, 16384], 1 <= L <= 8,
 *    every q_j is a prime with 2^53 < q_j < 2^54 and q_j = 1 (mod 2N), all
 *    distinct; t is a prime in [3, 2^20).
 *  - Polynomials cross the ABI in RNS coefficient form: u64 residues,
 *    limb-major, [L][N], limb j holding the residues mod q_j, each < q_j.
 *    A ciphertext is [2][L][N] (c0, c1), decrypting as c0 + c1*s.
 *    The NTT form used inside the library is never observable.
 *  - Switching keys are [L][2][L][N]: digit i, component (0: b_i, 1: a_i),
 *    limb j, with b_i = -a_i*s + e_i + g_i*w (mod Q) where g_i is the CRT
 *    idempotent of q_i (g_i = 1 mod q_i, 0 mod q_l for l != i) and w = s^2
 *    (relinearisation) or s(x^g) (substitution by g).  Key switching of z
 *    uses the digits D_i = [z]_{q_i} in [0, q_i): sum_i D_i * (b_i, a_i).
 *  - Multiplication M (Sec. 2.1.1): lift both ciphertexts to centered
 *    integers, multiply exactly, e_l = round(t * d_l / Q) for the three
 *    products, then relinearise e_2.  Results are exact integer functions of
 *    the inputs: identical bits for identical inputs, on any launch shape.
 *  - Host pointers are caller-owned and only read (or written for outputs)
 *    during the call; nothing is retained.  Device pointers (the *_device
 *    calls) must stay valid until the work on the given stream completes.
 *    The library owns all device memory it allocates until cwpir_free_db or
 *    cwpir_destroy.
 *  - Calls on one context are not thread-safe; use one context per thread
 *    or serialise (the slot calls below are the exception).  Every call
 *    returns CWPIR_OK (0) or a negative code; the message of the last
 *    failure is available from cwpir_last_error.
 */
#ifndef CWPIR_H
#define CWPIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CWPIR_ABI_VERSION 4
/* Largest number of plaintexts per database row (payload_len <= this * N). */
#define CWPIR_MAX_PLAINTEXTS 256

enum {
  CWPIR_OK = 0,
  CWPIR_EINVAL = -1,    /* an argument, shape or residue is out of range */
  CWPIR_ENOMEM = -2,    /* device or host allocation failed */
  CWPIR_ENODB = -3,     /* unknown database id */
  CWPIR_ECUDA = -4,     /* a CUDA runtime call failed */
  CWPIR_ETIMEDOUT = -5, /* a bounded device wait gave up */
  CWPIR_EBUSY = -6,     /* serving: no admission slot or memory right now */
  CWPIR_ENOKEY = -7,    /* a required Galois key was not supplied */
  CWPIR_EINTERNAL = -8  /* a device-side consistency check failed */
};

typedef struct cwpir_ctx cwpir_ctx;

/* Encryption parameters (Sec. 2.1.1; Sec. 4-5 use N in {4096, 8192, 16384}). */
typedef struct {
  uint32_t N;         /* ring degree */
  uint32_t L;         /* number of ciphertext primes */
  const uint64_t *q;  /* [L] primes, see conventions */
  uint64_t t;         /* plaintext modulus */
} cwpir_params;

/* Evaluation keys.  relin: [L][2][L][N] for w = s^2.  galois: for query
 * expansion with compression factor c the substitutions use the elements
 * N/2^a + 1 for a < c (Alg. Query Expansion); n_galois keys are given with
 * their elements in galois_elts, key g at galois + idx*L*2*L*N.  n_galois
 * may be 0 when no query is compressed. */
typedef struct {
  const uint64_t *relin;
  uint32_t n_galois;
  const uint32_t *galois_elts;
  const uint64_t *galois;
} cwpir_keys;

/* Work counters of an answer (for throughput accounting). */
typedef struct {
  uint64_t rows;            /* database rows processed */
  uint64_t mults;           /* homomorphic multiplications executed */
  uint64_t substitutions;   /* substitutions executed (expansion) */
  uint64_t ntt_polys;       /* length-N NTTs/INTTs executed (per limb) */
  uint64_t kernel_launches; /* kernels launched */
  uint64_t db_bytes_read;   /* NTT-form database bytes streamed */
} cwpir_stats;

/* ---- library information and host helpers ---- */
int cwpir_abi_version(void);
const char *cwpir_strerror(int code);
/* Message of the last failing call on ctx (or of the last failing setup in
 * this thread when ctx is NULL).  Valid until the next call on ctx. */
const char *cwpir_last_error(const cwpir_ctx *ctx);
/* The L largest primes q < 2^54 with q = 1 (mod 2N), descending (all above
 * 2^53 for N <= 16384 and L <= 8). */
int cwpir_default_primes(uint32_t N, uint32_t L, uint64_t *q_out);
/* Perfect mapping (Alg. Perfect Mapping, Sec. 3.2): x in [C(m,k)] -> the
 * x-th codeword of CW(m,k); writes its k one-positions in ascending order.
 * EINVAL if x >= C(m,k), k = 0, k > m or m > 65535. */
int cwpir_map_perfect(uint64_t x, uint32_t m, uint32_t k, uint16_t *pos_out);
/* Lossy mapping (Alg. Lossy Mapping, App. A) for domains too large for a
 * perfect mapping: draws H_1(x), H_2(x), ... in [m] and sets each new
 * position until k are set; writes the k positions in ascending order.
 * H_i(x) = (i-th output of a SplitMix64 generator seeded with x) mod m
 * (Steele, Lea, Flood 2014: mix64(x + i * 0x9E3779B97F4A7C15)); not keyed,
 * not cryptographic.  Two different x share a codeword with probability
 * 1 / C(m,k) (Theorem lossy-coll-prob); rows whose codewords coincide are
 * both selected by a query for either, so callers resolve collisions
 * before cwpir_load_db.  EINVAL if k = 0, k > m or m > 65535. */
int cwpir_map_lossy(uint64_t x, uint32_t m, uint32_t k, uint16_t *pos_out);
/* Positions 2i + y[i] (i < ell) of the plain folklore operator's factors
 * for the public ell-bit operand y.  EINVAL if ell is not in [1, 16] or
 * y >= 2^ell. */
int cwpir_map_folklore(uint64_t y, uint32_t ell, uint16_t *pos_out);
/* Smallest m with C(m,k) >= n (Sec. 3: "choose m such that C(m,k) >= n"). */
int cwpir_code_length(uint64_t n, uint32_t k, uint32_t *m_out);

/* ---- Setup (server, offline) ---- */
/* Validates params and keys, builds the device tables and uploads the keys
 * (converted to the internal NTT form).  *out receives a new context.
 * EINVAL on invalid params or key residues >= q_j; ENOMEM; ECUDA. */
int cwpir_setup(const cwpir_params *params, const cwpir_keys *keys,
                cwpir_ctx **out);
void cwpir_destroy(cwpir_ctx *ctx);

/* Database load (Setup, Sec. 3.3.1): n rows of payload_len plaintext
 * coefficients each < t (row-major [n][payload_len]), and each row's
 * codeword in CW(m,k) as k ascending one-positions < m ([n][k]).  A row is
 * s = ceil(payload_len / N) plaintexts (s = 1 for payload_len <= N;
 * payload_len <= CWPIR_MAX_PLAINTEXTS * N): plaintext p holds payload
 * coefficients p*N .. p*N + N - 1, the last one zero-padded; every answer
 * against the database returns s ciphertexts, the inner products of the one
 * selection vector with each plaintext column (Sec. 3.3.3).  For index PIR
 * the codeword of row i is the perfect mapping of i; for keyword PIR
 * (Sec. 3.3.6) the mapping of the row's keyword.  The rows are lifted to
 * centered integers and kept in HBM in NTT form: rows of one plaintext with
 * k >= 2 modulo three (four for a large t) internal 30-bit primes (12 or 16
 * bytes a coefficient; the answer multiplies them exactly as integers),
 * otherwise modulo the ciphertext primes (8 L bytes a coefficient and
 * plaintext).
 * 1 <= k <= 16, k <= m <= 16384, 1 <= n <= 2^24.  *db_id receives a handle.
 * EINVAL (including a coefficient >= t or a bad codeword), ENOMEM, ECUDA. */
int cwpir_load_db(cwpir_ctx *ctx, uint64_t n, uint32_t payload_len, uint32_t k,
                  uint32_t m, const uint32_t *items, const uint16_t *codewords,
                  int32_t *db_id);
int cwpir_free_db(cwpir_ctx *ctx, int32_t db_id);
/* Folklore PIR (Sec. 4: the same architecture with the plain folklore
 * equality operator, Eq. folklore-plain-eq, and the logarithmic binary
 * encoding of indices): n <= 2^ell rows indexed 0 .. n-1, payloads as for
 * cwpir_load_db.  Queries against the database are the ell ciphertexts of
 * the index bits x[0..ell-1] (c = 0); the server forms the leaves
 * (1 - x[0], x[0], 1 - x[1], x[1], ...) with 1 - x = (Delta - c0, -c1) and
 * selects row y by the codeword of positions 2i + y[i] (cwpir_map_folklore),
 * a product of ell factors of depth ceil(log2 ell).  1 <= ell <= 16.
 * EINVAL, ENOMEM, ECUDA. */
int cwpir_load_db_folklore(cwpir_ctx *ctx, uint64_t n, uint32_t payload_len,
                           uint32_t ell, const uint32_t *items, int32_t *db_id);

/* ---- Process (server, online) ---- */
/* Answer one query against a database (Sec. 3.3.3): expansion when c > 0
 * (Alg. Query Expansion), the selection vector by the plain constant-weight
 * equality operator (Alg. Selection Vector Calculation, Eq. plain-cw-eq,
 * balanced pairwise product tree over the ascending positions), and the
 * inner product sum_i sel_i * DB_i (Eq. baseline-pir).
 * query: [h][2][L][N] with h = m when c = 0, else h = ceil(m / 2^c) (Alg.
 * Query); c <= log2 N and needs the Galois keys for N/2^a + 1, a < c.
 * response: [s][2][L][N] (s = cwpir_db_plaintexts), written.  Host buffers;
 * blocks until done.
 * EINVAL, ENODB, ENOKEY, ECUDA, EINTERNAL. */
int cwpir_answer(cwpir_ctx *ctx, int32_t db_id, uint32_t c,
                 const uint64_t *query, uint64_t *response);
/* Same with device buffers, enqueued on `stream` (a cudaStream_t, NULL for
 * the legacy default stream), on slot 0.  Returns once the work is enqueued;
 * the device checks of that work are read with cwpir_device_status. */
int cwpir_answer_device(cwpir_ctx *ctx, int32_t db_id, uint32_t c,
                        const uint64_t *d_query, uint64_t *d_response,
                        void *stream);

/* Answer nq queries against one database together (configuration 4 of
 * the benchmark: batched answering).  Every query is answered exactly as
 * by cwpir_answer (identical response bits); the queries share each kernel
 * launch: expansion rounds, first-level products and tree levels of all nq
 * queries run in the same grids.  queries: [nq][h][2][L][N] (h as for
 * cwpir_answer, same c for all), responses: [nq][s][2][L][N].  With
 * CWPIR_OPT_USE_GRAPH the launch sequence for (database, nq, c) is captured
 * once into a CUDA graph on the first call and replayed afterwards.
 * EINVAL also when nq times the tree's widest level exceeds the
 * multiplications per launch (CWPIR_OPT_MAX_JOBS), or nq * s exceeds it. */
int cwpir_answer_batch(cwpir_ctx *ctx, int32_t db_id, uint32_t c, uint32_t nq,
                       const uint64_t *queries, uint64_t *responses);
int cwpir_answer_batch_device(cwpir_ctx *ctx, int32_t db_id, uint32_t c,
                              uint32_t nq, const uint64_t *d_queries,
                              uint64_t *d_responses, void *stream);
/* Batched answering across databases (configuration 4 of the benchmark):
 * the queries of several resident databases, possibly of different
 * contexts (ring degrees, primes, code weights) on one device, in one
 * launch sequence.  Each item is (context, database, c, nq queries, answered
 * nq_call at a time, nq_call dividing nq; 0 = all nq at once) and gets its
 * own branch: a stream and a slot of its context (cwpir_slot_create, held
 * until cwpir_multi_destroy) with its own plan over all rows.  A call forks
 * the branches from `stream`, runs each item's sub-batches in order on its
 * branch, so that the small databases' launches fill the device while the
 * large ones run, and joins them back into `stream`; with use_graph the
 * whole forked sequence is captured once into one CUDA graph and replayed
 * afterwards (recaptured when a context's scratch was re-sized).  Every
 * response is bit-identical to cwpir_answer of the same query.  Contexts
 * and databases must outlive the object; no other call may use these
 * contexts while a cwpir_multi call runs, except the slot calls. */
typedef struct {
  cwpir_ctx *ctx;
  int32_t db_id;
  uint32_t c;        /* compression factor of the item's queries */
  uint32_t nq;       /* queries of the item per call */
  uint32_t nq_call;  /* queries per batched answer in the branch (0 = nq) */
} cwpir_multi_item;
typedef struct cwpir_multi cwpir_multi;
/* EINVAL (contexts on different devices, nq not a multiple of nq_call, a
 * bad c), ENODB, ENOKEY, ENOMEM, ECUDA. */
int cwpir_multi_create(const cwpir_multi_item *items, uint32_t count,
                       cwpir_multi **out);
/* d_queries[i]: item i's [nq][h][2][L][N] device queries, d_responses[i]:
 * its [nq][s][2][L][N] responses; enqueued on `stream` (a cudaStream_t,
 * NULL: legacy default stream), returns once enqueued.  ENODB if a database
 * was freed. */
int cwpir_multi_answer_device(cwpir_multi *mb, const uint64_t *const *d_queries,
                              uint64_t *const *d_responses, int use_graph,
                              void *stream);
/* Waits for `stream` and reads every branch's device check flag
 * (cwpir_device_status): CWPIR_EINTERNAL if any check failed. */
int cwpir_multi_status(cwpir_multi *mb, void *stream);
/* Work counters of the last enqueued (or captured) sequence, all items. */
int cwpir_multi_stats(const cwpir_multi *mb, cwpir_stats *out);
const char *cwpir_multi_last_error(const cwpir_multi *mb);
void cwpir_multi_destroy(cwpir_multi *mb);

/* Exchange step of a database sharded by rows over several GPUs (one
 * context per GPU, each holding a disjoint set of the rows with their own
 * codewords).  The response is linear in the rows: r = sum over rows i of
 * sel_i * DB_i mod Q (Eq. baseline-pir, Sec. 2.3; the Inner Product of
 * Sec. 3.3.3), so each shard answers over its rows and the response is the
 * sum of the partial responses modulo each q_j, bit-identical to answering
 * over all rows on one GPU.  d_parts: [count][s][2][L][N] partial responses
 * in coefficient form (residues below q_j, as returned by
 * cwpir_answer_device), d_out: [s][2][L][N]; both device memory on ctx's
 * GPU, owned by the caller, and d_out must not overlap d_parts.  stream: a
 * cudaStream_t (NULL: legacy default stream); returns once enqueued.
 * EINVAL for a null pointer, count = 0, or s = 0 or s > CWPIR_MAX_PLAINTEXTS.
 * Moving the partials between GPUs (an all-gather) is the caller's. */
int cwpir_sum_responses_device(cwpir_ctx *ctx, uint32_t count, uint32_t s,
                               const uint64_t *d_parts, uint64_t *d_out,
                               void *stream);

/* The same exchange as one all-reduce: d_sums [s][2][L][N] holds the
 * element-wise u64 sums (wrapping modulo 2^64 is the caller's to avoid: at
 * most 1023 partial responses of residues below 2^54) of the partial
 * responses of the shards; d_out [s][2][L][N] = d_sums mod q_j, the
 * response.  d_out may equal d_sums.  Device memory on ctx's GPU; returns
 * once enqueued on `stream`.  EINVAL for a null pointer or s out of range. */
int cwpir_reduce_responses_device(cwpir_ctx *ctx, uint32_t s, const uint64_t *d_sums,
                                  uint64_t *d_out, void *stream);

/* Autotuner: times answers of the nq device queries (as for
 * cwpir_answer_batch_device) for each candidate number of multiplications
 * per launch in `candidates` (count entries, 0 = automatic), keeps the
 * fastest on ctx (CWPIR_OPT_MAX_JOBS) and writes it and its time per call
 * in milliseconds.  d_responses is scratch of [nq][s][2][L][N]. */
int cwpir_autotune(cwpir_ctx *ctx, int32_t db_id, uint32_t c, uint32_t nq,
                   const uint64_t *d_queries, uint64_t *d_responses,
                   const int64_t *candidates, uint32_t count, int64_t *best,
                   double *best_ms);
/* The autotuner over a grid: every (multiplications per launch, row-group
 * waves) pair of jobs[n_jobs] x waves[n_waves] (n_waves = 0: the default
 * waves only); keeps the fastest pair on ctx (CWPIR_OPT_MAX_JOBS,
 * CWPIR_OPT_ROW_GROUP_WAVES) and writes it (best_waves may be NULL) with
 * its time per call.  Reads slot 0's device check flag at the end. */
int cwpir_autotune_grid(cwpir_ctx *ctx, int32_t db_id, uint32_t c, uint32_t nq,
                        const uint64_t *d_queries, uint64_t *d_responses,
                        const int64_t *jobs, uint32_t n_jobs, const int64_t *waves,
                        uint32_t n_waves, int64_t *best_jobs, int64_t *best_waves,
                        double *best_ms);

/* Device memory (bytes, an upper estimate) that the first
 * cwpir_answer_batch(_device) call for (db_id, nq, c) would allocate for
 * its plan and, if not yet allocated, the context's scratch; 0 when the
 * plan is cached.  Used for admission by free device memory. */
int cwpir_plan_bytes(cwpir_ctx *ctx, int32_t db_id, uint32_t nq, uint32_t c,
                     uint64_t *bytes);
/* Frees the cached plans (and graphs) of one database, or of all databases
 * of ctx when db_id < 0; waits for the device first. */
int cwpir_release_plans(cwpir_ctx *ctx, int32_t db_id);

/* ---- the steps of Process, one at a time (host buffers) ---- */
/* Homomorphic multiplication M of two ciphertexts with relinearisation. */
int cwpir_mul(cwpir_ctx *ctx, const uint64_t *a, const uint64_t *b,
              uint64_t *out);
/* Substitution Sub_g (Sec. 2.1.1): automorphism x -> x^g plus key switch
 * with the Galois key of g.  ENOKEY if no key for g was supplied. */
int cwpir_substitute(cwpir_ctx *ctx, uint32_t g, const uint64_t *ct,
                     uint64_t *out);
/* Query expansion (Alg. Query Expansion): h = ceil(m / 2^c) ciphertexts ->
 * the first m expanded ciphertexts, out: [m][2][L][N].  1 <= c. */
int cwpir_expand(cwpir_ctx *ctx, uint32_t c, uint32_t m, const uint64_t *query,
                 uint64_t *out);
/* Selection-vector entries sel_i (Alg. Selection Vector Calculation) for
 * `count` rows of a database: out: [count][2][L][N]. */
int cwpir_selection(cwpir_ctx *ctx, int32_t db_id, uint32_t c,
                    const uint64_t *query, uint64_t count,
                    const uint64_t *rows, uint64_t *out);
/* Arithmetic constant-weight equality operator (Alg. Arithmetic
 * Constant-weight Equality Operator, Sec. 3.1) on two encrypted operands,
 * slot-wise when the plaintexts are batch-encoded: x, y: [m][2][L][N]
 * (ciphertext i holds bit i of the codewords), out: [2][L][N] =
 * (1/k!) prod_{i<k} (sum_j x_j y_j - i), which decrypts to 1 where the
 * codewords agree and 0 elsewhere; m + k - 1 multiplications, depth
 * 1 + ceil(log2 k).  1 <= k <= 16, k <= m <= 8192.  Host buffers (pinned
 * ones copy fastest).  The residues are checked on the device (EINVAL once
 * the call has run).  The call keeps its device buffers and product plans
 * for the next call with the same (m, k), until cwpir_release_plans(ctx,
 * -1) or an option change that drops the answer plans.
 * EINVAL, ENOMEM, ECUDA, EINTERNAL. */
int cwpir_arith_cw_eq(cwpir_ctx *ctx, uint32_t m, uint32_t k, const uint64_t *x,
                      const uint64_t *y, uint64_t *out);
/* Plain multiplication PM of a ciphertext by row `row` of a database: by
 * each of the row's s plaintexts, out: [s][2][L][N].  EINTERNAL if a device
 * consistency check fails. */
int cwpir_plain_mul(cwpir_ctx *ctx, int32_t db_id, uint64_t row,
                    const uint64_t *ct, uint64_t *out);

/* ---- options ---- */
enum {
  /* 1 (default): compute each distinct first-level product of the tree once
   * per query and share it between rows; 0: every row's tree in full.  The
   * response bits are identical either way. */
  CWPIR_OPT_SHARE_LEVEL1 = 1,
  /* rows per device batch (0 = automatic) */
  CWPIR_OPT_BATCH_ROWS = 2,
  /* 0 (default): enqueue every kernel of an answer; 1: capture the launch
   * sequence of each (database, queries per call, c, slot) once into a CUDA
   * graph and replay it (the batched and served paths switch it on) */
  CWPIR_OPT_USE_GRAPH = 3,
  /* 1: bracket every kernel launch with CUDA events on its stream and add
   * the durations per kernel class (read with cwpir_kernel_times); 0
   * (default): no events */
  CWPIR_OPT_KERNEL_TIMING = 4,
  /* multiplications per kernel launch (0 = automatic, at most 2048); sizes
   * the context's scratch: setting it waits for the device, frees the
   * scratch and the answer plans, which the next call rebuilds */
  CWPIR_OPT_MAX_JOBS = 5,
  /* 1 (default): databases loaded afterwards with one plaintext per row and
   * k >= 2 are held in the row basis of internal primes (cwpir_load_db); 0:
   * modulo the ciphertext primes.  The response bits are identical either
   * way; already loaded databases keep their form. */
  CWPIR_OPT_ROW_BASIS = 6,
  /* cap, in bytes, on the device memory the context's buffers may hold
   * (databases, scratch, plans; 0 = no cap, the default): an allocation
   * that would pass it fails with CWPIR_ENOMEM before cudaMalloc is
   * called, and the context stays usable.  Lowering it frees nothing. */
  CWPIR_OPT_MEM_LIMIT = 7,
  /* row sums of the last tree level: split into row groups until about
   * this many waves of the device's resident threads cover it (0 = the
   * default, 2); drops the cached plans.  Response bits are unchanged. */
  CWPIR_OPT_ROW_GROUP_WAVES = 8,
  /* 0 (default): the scale-down after each multiplication rounds t d / Q
   * with a fixed-point sum and hands the rare coefficients it cannot decide
   * (about one in 2^21) to an exact path; 1: every coefficient takes the
   * exact path (slower: a check of that path).  Drops the cached plans.
   * Response bits are unchanged. */
  CWPIR_OPT_SCALE_EXACT = 9
};
/* Both return EINVAL for an unknown option or a value out of range. */
int cwpir_set_option(cwpir_ctx *ctx, int option, int64_t value);
int cwpir_get_option(cwpir_ctx *ctx, int option, int64_t *value);
/* Device bytes the context's buffers hold now (what CWPIR_OPT_MEM_LIMIT
 * caps). */
int cwpir_mem_used(const cwpir_ctx *ctx, uint64_t *bytes);

/* ---- slots: concurrent answers on one context ----
 * A slot is one set of the multiplication kernels' scratch buffers (up to
 * 8 GiB, sized by CWPIR_OPT_MAX_JOBS) with its own device consistency
 * flag; answers on different slots may run at the same time on different
 * streams.  Slot 0 exists from cwpir_setup on and serves every call that
 * takes no slot.  The calls in this group may be made from several threads
 * on one context (they serialise their host-side work on a per-context
 * lock; the device work of different slots overlaps); one slot must not be
 * used by two streams at once. */
/* Adds a slot; *slot receives its index.  Its buffers are allocated by its
 * first answer.  ENOMEM, ECUDA. */
int cwpir_slot_create(cwpir_ctx *ctx, uint32_t *slot);
/* Waits for the device, frees the slot's buffers and its cached plans; the
 * index may be handed out again by cwpir_slot_create.  EINVAL for slot 0
 * or a slot not in use. */
int cwpir_slot_release(cwpir_ctx *ctx, uint32_t slot);
/* cwpir_answer_batch_device with the scratch of `slot`; the plans (and
 * graphs) it builds are cached per slot. */
int cwpir_answer_batch_slot(cwpir_ctx *ctx, uint32_t slot, int32_t db_id, uint32_t c,
                            uint32_t nq, const uint64_t *d_queries, uint64_t *d_responses,
                            void *stream);
/* cwpir_plan_bytes for a slot: includes the slot's scratch if it has none
 * yet. */
int cwpir_plan_bytes_slot(cwpir_ctx *ctx, uint32_t slot, int32_t db_id, uint32_t nq,
                          uint32_t c, uint64_t *bytes);
/* Status of the device work of a slot: waits for `stream` (a cudaStream_t;
 * NULL: the legacy default stream), then reads and clears the slot's
 * consistency flag.  CWPIR_EINTERNAL if one of the device checks of the
 * scale-down or of the row-basis rounding failed since the flag was last
 * read (the responses computed meanwhile must not be used), else CWPIR_OK.
 * The *_device and *_slot answer calls return once their work is enqueued
 * and cannot report it themselves: call this after them.  The host-buffer
 * calls read and clear slot 0's flag themselves. */
int cwpir_device_status(cwpir_ctx *ctx, uint32_t slot, void *stream);
/* Test hook for the path above: sets the slot's consistency flag as a
 * failed device check would (a host-to-device copy of one word; no kernel
 * runs, nothing faults).  The next status read reports CWPIR_EINTERNAL. */
int cwpir_inject_status(cwpir_ctx *ctx, uint32_t slot);

/* Homomorphic multiplication M (as cwpir_mul) on device buffers that
 * allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 * The paper has no counterpart; this call serves callers that cannot
 * allocate device memory where they multiply (a fixed pre-partitioned
 * memory pool, a section where an allocation would stall or is forbidden).
 * d_a, d_b: [2][L][N] ciphertexts, d_out: [2][L][N], device memory owned by
 * the caller; every residue of limb j must be below q_j, as for the other
 * device-buffer calls (not checked here: the inputs are never copied to the
 * host; an unreduced residue gives a wrong product, not an error).
 * stream: a cudaStream_t (NULL: legacy default stream).  The call blocks
 * until the result is complete.
 * Intermediates live in one file-scope device array of 2^20 u64 words
 * (8 MiB) plus a 64-word header, held by every GPU that loads the library
 * until the process exits.  One multiplication needs (L^2 + 14L + 7K/2) * N
 * words, K the 30-bit extension primes of the tensor (K = 5, 8, 12, 15, 19,
 * 23, 26, 30 for L = 1 ... 8): N = 4096 allows L <= 7, N = 8192 allows
 * L <= 4, N = 16384 allows L <= 2; larger sizes are rejected with EINVAL.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the rest of the process; make
 * that first call before any stream capture.  The address belongs to the
 * device's primary context: after cudaDeviceReset on that device the call
 * must not be used again in the process.
 * All calls share the array and it keeps
 * the previous call's contents (the error flag is cleared each call): calls
 * that overlap on the GPU, from any context or stream, race.  ctx must be a
 * set-up context (it supplies the tables and the relinearisation key). */
int cwpir_mul_noalloc(cwpir_ctx *ctx, const uint64_t *d_a, const uint64_t *d_b,
                      uint64_t *d_out, void *stream);

/* Shape of a loaded database: ring degree, number of primes, code length. */
int cwpir_db_shape(const cwpir_ctx *ctx, int32_t db_id, uint32_t *N, uint32_t *L,
                   uint32_t *m);
/* Query ciphertexts h of one query against a database with compression c:
 * m (c = 0), ceil(m / 2^c), or ell for a folklore database (c = 0 only). */
int cwpir_query_cts(cwpir_ctx *ctx, int32_t db_id, uint32_t c, uint32_t *h);
/* Plaintexts per row s of a loaded database (responses are [s][2][L][N]). */
int cwpir_db_plaintexts(const cwpir_ctx *ctx, int32_t db_id, uint32_t *s);
/* CUDA device of the context. */
int cwpir_ctx_device(const cwpir_ctx *ctx, int *device);

/* ---- online serving (configuration 5 of the benchmark) ---- */
/* A server answers queries for registered targets (a context, one of its
 * databases, and the compression factor c of that target's queries).  Each
 * target gets lanes_per_target worker lanes: a host thread with its own
 * stream and its own slot on the target's context (cwpir_slot_create, so
 * up to 8 GiB of scratch per lane, held until the server is destroyed).
 * Whenever a lane is free it takes the waiting requests of its target, up
 * to the largest power of two <= max_batch whose answer plan fits in free
 * device memory minus hbm_reserve_bytes (the target's cached plans are
 * released when nothing fits), and answers them with one
 * cwpir_answer_batch_slot call replayed from a CUDA graph (continuous
 * batching).  Lanes of all targets run concurrently, so a request that
 * arrives while others are on the GPU starts at once on an idle lane of
 * its target and its kernels overlap with theirs; when every lane of its
 * target is busy it joins the next batch of the first lane to finish.
 * After each batch the lane reads its slot's device check flag
 * (cwpir_device_status): a failed check fails that batch's requests with
 * CWPIR_EINTERNAL.  Each response is bit-identical to cwpir_answer for the
 * same query.  While a server runs, its contexts may be used by other
 * threads only through the slot calls.  Requests beyond max_pending
 * waiting or running are refused with EBUSY. */
typedef struct cwpir_server cwpir_server;
typedef struct {
  cwpir_ctx *ctx;
  int32_t db_id;
  uint32_t c;
} cwpir_target;
typedef struct {
  uint32_t max_batch;         /* most requests one lane answers at once, >= 1 */
  uint32_t lanes_per_target;  /* 1 .. 16 */
  uint32_t max_pending;       /* requests waiting or running, >= 1 */
  uint64_t hbm_reserve_bytes; /* free device memory admission leaves untouched */
} cwpir_server_config;
typedef struct {
  uint64_t submitted, completed, batches, max_batch_seen, rejected_busy;
  uint64_t failed;         /* requests completed with an error status */
  uint64_t max_concurrent; /* most batches running at the same time */
  double busy_s;           /* summed wall time of the lanes' batches */
} cwpir_server_stats;
/* EINVAL for a bad target or configuration; ENOMEM; the slot errors. */
int cwpir_server_create(const cwpir_target *targets, uint32_t n_targets,
                        const cwpir_server_config *cfg, cwpir_server **out);
/* Queues one query ([h][2][L][N] host memory, copied) for a target;
 * *ticket identifies it.  Non-blocking; EBUSY when max_pending is reached. */
int cwpir_submit(cwpir_server *srv, uint32_t target, const uint64_t *query,
                 uint64_t *ticket);
/* Non-blocking: *status = 0 while waiting or running; when done, 1 (the
 * response [s][2][L][N] is written, latency_s = completion - submission) or
 * a negative error code; a finished ticket is forgotten after it is read. */
int cwpir_poll(cwpir_server *srv, uint64_t ticket, uint64_t *response,
               int32_t *status, double *latency_s);
/* Blocking variant of cwpir_poll; ETIMEDOUT after timeout_s seconds. */
int cwpir_wait(cwpir_server *srv, uint64_t ticket, uint64_t *response,
               int32_t *status, double *latency_s, double timeout_s);
int cwpir_server_get_stats(cwpir_server *srv, cwpir_server_stats *out);
/* Finishes the waiting requests, stops the lanes and frees the server. */
void cwpir_server_destroy(cwpir_server *srv);

/* ---- measurement ---- */
/* Integer-pipe throughput of a device, measured (no counterpart in the
 * paper: the denominator of the answer kernels' roofline, whose work is
 * modular multiplication on the integer pipes).  Each rate is operations
 * per second over all SMs, from a probe kernel of independent dependency
 * chains on every SM (2048 threads per SM) timed with CUDA events; the
 * multiply probes pair each multiply with one XOR, which runs on another
 * pipe.  Takes well under a second; uses the current clocks. */
typedef struct {
  double imad32_per_s;   /* 32-bit multiply-add, low word (IMAD) */
  double mulhi32_per_s;  /* high word of a 32 x 32-bit product */
  double mullo64_per_s;  /* low 64 bits of a 64 x 64-bit product */
  double mulhi64_per_s;  /* high 64 bits of a 64 x 64-bit product */
  double iadd32_per_s;   /* three-input 32-bit add (IADD3) */
  int sms;               /* streaming multiprocessors */
  double max_sm_mhz;     /* the device's maximum SM clock */
} cwpir_int_peaks;
/* EINVAL for a bad device or null out; ENOMEM; ECUDA. */
int cwpir_measure_int_peaks(int device, cwpir_int_peaks *out);

/* Work counters of the last answer on ctx (cwpir_stats, above). */
int cwpir_last_stats(const cwpir_ctx *ctx, cwpir_stats *out);

/* Kernel classes of the answer path, for cwpir_kernel_times. */
enum {
  CWPIR_K_TENSOR = 0,  /* tensor product + inverse NTT ("tensor") */
  CWPIR_K_SCALE = 1,   /* exact scale-down round(t d / Q) ("scale") */
  CWPIR_K_RELIN = 2,   /* key switching fused with plain multiplication
                          ("relin_pm"; on a row-basis database: the row sums
                          and the once-per-group conversions) */
  CWPIR_K_LIFT = 3,    /* centered base conversion Q -> P ("lift") */
  CWPIR_K_NTT = 4,     /* stand-alone NTTs ("ntt") */
  CWPIR_K_ACC = 5,     /* accumulation of partial products ("accumulate") */
  CWPIR_K_EXPAND = 6,  /* automorphisms, substitution key switches, combine
                          ("expand") */
  CWPIR_K_ROWS = 7,    /* the row transforms of the last tree level on a
                          row-basis database ("row_ntt") */
  CWPIR_K_CLASSES = 8
};
/* With CWPIR_OPT_KERNEL_TIMING on: waits for the recorded work, then writes
 * per class the summed milliseconds (ms) and launch counts (launches),
 * arrays of CWPIR_K_CLASSES entries, for all launches since the previous
 * call, and resets the sums. */
int cwpir_kernel_times(cwpir_ctx *ctx, double *ms, uint64_t *launches);
const char *cwpir_kernel_class_name(int cls);

#ifdef __cplusplus
}
#endif
#endif
