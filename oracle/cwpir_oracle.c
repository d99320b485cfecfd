/*
 * cwpir_oracle.c -- plain CPU oracle for the constant-weight PIR answer path.
 *
 * TEST INFRASTRUCTURE ONLY (see cwpir_oracle.h).  Nothing here is shared with
 * the product library.  Speed is not a goal: every step is written the plain
 * way so that it can be checked against the paper by eye.
 *
 * What it computes, with the paper's sections:
 *   FV/BFV ring operations (Sec. 2.1.1): Add, Plain Multiplication PM,
 *     Multiplication M (tensor, exact scale by t/Q, relinearisation) and
 *     Substitution Sub_g (automorphism plus key switch).
 *   Plain constant-weight equality operator (Sec. 3.1, Eq. plain-cw-eq):
 *     product of the query ciphertexts at the one-positions of a codeword.
 *   Perfect mapping and its inverse (Alg. Perfect Mapping, App. A).
 *   Query construction (Alg. Query), query expansion (Alg. Query Expansion),
 *     selection vector (Alg. Selection Vector Calculation) and the inner
 *     product with the database (Sec. 3.3.3), keyword variant (Sec. 3.3.6).
 * Readings where the paper is silent (FV textbook choices) are stated at the
 * function that makes them.
 */
#include "cwpir_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

#define MAXL 8    /* ciphertext primes */
#define MAXK 24   /* auxiliary primes for exact products */
#define BW 20     /* big-integer width in 64-bit words (1280 bits) */

static void die(const char *msg) {
  fprintf(stderr, "cwpir_oracle: fatal: %s\n", msg);
  abort();
}

/* ------------------------------------------------------------------ */
/* Word-size modular arithmetic (p < 2^63).                            */
/* ------------------------------------------------------------------ */
static inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) {
  return (uint64_t)(((u128)a * b) % p);
}
static inline uint64_t addmod(uint64_t a, uint64_t b, uint64_t p) {
  uint64_t s = a + b;
  return s >= p ? s - p : s;
}
static inline uint64_t submod(uint64_t a, uint64_t b, uint64_t p) {
  return a >= b ? a - b : a + p - b;
}
static uint64_t powmod(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1 % p;
  a %= p;
  while (e) {
    if (e & 1) r = mulmod(r, a, p);
    a = mulmod(a, a, p);
    e >>= 1;
  }
  return r;
}
static uint64_t invmod(uint64_t a, uint64_t p) { return powmod(a, p - 2, p); }

int orc_is_prime(uint64_t n) {
  static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return 0;
  for (int i = 0; i < 12; ++i) {
    if (n == bases[i]) return 1;
    if (n % bases[i] == 0) return 0;
  }
  uint64_t d = n - 1;
  int r = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++r;
  }
  for (int i = 0; i < 12; ++i) {
    uint64_t x = powmod(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    int composite = 1;
    for (int j = 1; j < r; ++j) {
      x = mulmod(x, x, n);
      if (x == n - 1) {
        composite = 0;
        break;
      }
    }
    if (composite) return 0;
  }
  return 1;
}

int orc_primes(uint32_t N, uint32_t count, uint32_t bits, uint64_t *out) {
  if (N < 2 || (N & (N - 1)) || bits < 8 || bits > 62) return -1;
  uint64_t step = 2 * (uint64_t)N;
  if (step >= (1ull << bits)) return -1;
  /* 2^bits is a multiple of 2N, so 2^bits - 2N + 1 is the largest value
   * below 2^bits that is 1 mod 2N. */
  uint64_t p = (1ull << bits) - step + 1;
  uint32_t got = 0;
  while (got < count) {
    if (p <= step) return -2;
    if (orc_is_prime(p)) out[got++] = p;
    p -= step;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Unsigned and signed big integers (fixed width, little-endian).      */
/* ------------------------------------------------------------------ */
typedef struct {
  uint64_t w[BW];
} bu;
typedef struct {
  int neg;
  bu m;
} bs;

static void bu_zero(bu *a) { memset(a, 0, sizeof *a); }
static void bu_set(bu *a, uint64_t v) {
  bu_zero(a);
  a->w[0] = v;
}
static int bu_is_zero(const bu *a) {
  for (int i = 0; i < BW; ++i)
    if (a->w[i]) return 0;
  return 1;
}
static int bu_cmp(const bu *a, const bu *b) {
  for (int i = BW - 1; i >= 0; --i)
    if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
  return 0;
}
static void bu_add(bu *r, const bu *a, const bu *b) {
  u128 c = 0;
  for (int i = 0; i < BW; ++i) {
    c += (u128)a->w[i] + b->w[i];
    r->w[i] = (uint64_t)c;
    c >>= 64;
  }
  if (c) die("big integer overflow in add");
}
/* r = a - b, requires a >= b */
static void bu_sub(bu *r, const bu *a, const bu *b) {
  uint64_t borrow = 0;
  for (int i = 0; i < BW; ++i) {
    u128 d = (u128)a->w[i] - b->w[i] - borrow;
    r->w[i] = (uint64_t)d;
    borrow = (uint64_t)(d >> 64) ? 1 : 0;
  }
  if (borrow) die("big integer underflow in sub");
}
/* r += a * m */
static void bu_addmul(bu *r, const bu *a, uint64_t m) {
  u128 c = 0;
  for (int i = 0; i < BW; ++i) {
    c += (u128)a->w[i] * m + r->w[i];
    r->w[i] = (uint64_t)c;
    c >>= 64;
  }
  if (c) die("big integer overflow in addmul");
}
static void bu_mul_u64(bu *r, const bu *a, uint64_t m) {
  bu t;
  bu_zero(&t);
  bu_addmul(&t, a, m);
  *r = t;
}
/* q = floor(a / d), returns a mod d */
static uint64_t bu_divmod(bu *q, const bu *a, uint64_t d) {
  u128 rem = 0;
  for (int i = BW - 1; i >= 0; --i) {
    u128 cur = (rem << 64) | a->w[i];
    q->w[i] = (uint64_t)(cur / d);
    rem = cur % d;
  }
  return (uint64_t)rem;
}
static uint64_t bu_mod(const bu *a, uint64_t d) {
  u128 rem = 0;
  for (int i = BW - 1; i >= 0; --i) rem = ((rem << 64) | a->w[i]) % d;
  return (uint64_t)rem;
}
/* r = a * b (full product, must fit) */
static void bu_mul(bu *r, const bu *a, const bu *b) {
  bu acc, sh;
  bu_zero(&acc);
  for (int i = 0; i < BW; ++i) {
    if (!b->w[i]) continue;
    bu_zero(&sh);
    for (int j = 0; j + i < BW; ++j) sh.w[j + i] = a->w[j];
    for (int j = BW - i; j < BW; ++j)
      if (a->w[j]) die("big integer overflow in mul");
    bu_addmul(&acc, &sh, b->w[i]);
  }
  *r = acc;
}
static void bu_shr1(bu *r, const bu *a) {
  for (int i = 0; i < BW; ++i) {
    uint64_t hi = (i + 1 < BW) ? a->w[i + 1] : 0;
    r->w[i] = (a->w[i] >> 1) | (hi << 63);
  }
}
static int bu_bitlen(const bu *a) {
  for (int i = BW - 1; i >= 0; --i)
    if (a->w[i]) return 64 * i + (64 - __builtin_clzll(a->w[i]));
  return 0;
}
static double bu_log2(const bu *a) {
  int b = bu_bitlen(a);
  if (b == 0) return -INFINITY;
  if (b <= 64) return log2((double)a->w[0]);
  /* top 128 bits as a double times 2^shift */
  int shift = b - 64;
  int wi = shift / 64, bi = shift % 64;
  uint64_t top = a->w[wi] >> bi;
  if (bi && wi + 1 < BW) top |= a->w[wi + 1] << (64 - bi);
  return log2((double)top) + shift;
}

static uint64_t bs_mod(const bs *a, uint64_t p) {
  uint64_t r = bu_mod(&a->m, p);
  return (a->neg && r) ? p - r : r;
}

/* ------------------------------------------------------------------ */
/* Negacyclic NTT modulo one prime (the oracle's own).                 */
/* ------------------------------------------------------------------ */
typedef struct {
  uint64_t p;
  uint32_t N;
  uint64_t *psi;  /* psi^i, i < N; psi a primitive 2N-th root of unity */
  uint64_t *ipsi; /* psi^-i * N^-1 */
  uint64_t *w;    /* omega^j, j < N/2, omega = psi^2 */
  uint64_t *iw;   /* omega^-j */
} ntab;

static int ntab_init(ntab *T, uint32_t N, uint64_t p) {
  memset(T, 0, sizeof *T);
  if ((p - 1) % (2 * (uint64_t)N)) return -1;
  T->p = p;
  T->N = N;
  uint64_t psi = 0;
  for (uint64_t g = 2; g < 1000; ++g) {
    uint64_t cand = powmod(g, (p - 1) / (2 * (uint64_t)N), p);
    if (powmod(cand, N, p) == p - 1) {
      psi = cand;
      break;
    }
  }
  if (!psi) return -2;
  T->psi = malloc(N * sizeof(uint64_t));
  T->ipsi = malloc(N * sizeof(uint64_t));
  T->w = malloc((N / 2 + 1) * sizeof(uint64_t));
  T->iw = malloc((N / 2 + 1) * sizeof(uint64_t));
  uint64_t ipsi = invmod(psi, p), ninv = invmod(N, p);
  uint64_t x = 1, y = ninv;
  for (uint32_t i = 0; i < N; ++i) {
    T->psi[i] = x;
    T->ipsi[i] = y;
    x = mulmod(x, psi, p);
    y = mulmod(y, ipsi, p);
  }
  uint64_t om = mulmod(psi, psi, p), iom = invmod(om, p);
  x = 1;
  y = 1;
  for (uint32_t j = 0; j <= N / 2; ++j) {
    T->w[j] = x;
    T->iw[j] = y;
    x = mulmod(x, om, p);
    y = mulmod(y, iom, p);
  }
  return 0;
}
static void ntab_free(ntab *T) {
  free(T->psi);
  free(T->ipsi);
  free(T->w);
  free(T->iw);
  memset(T, 0, sizeof *T);
}

/* Cyclic NTT of length N, natural order in and out (iterative radix 2). */
static void cyclic_ntt(uint64_t *a, uint32_t N, const uint64_t *wt, uint64_t p) {
  for (uint32_t i = 1, j = 0; i < N; ++i) {
    uint32_t bit = N >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      uint64_t t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
  for (uint32_t len = 2; len <= N; len <<= 1) {
    uint32_t half = len / 2, step = N / len;
    for (uint32_t i = 0; i < N; i += len)
      for (uint32_t j = 0; j < half; ++j) {
        uint64_t u = a[i + j];
        uint64_t v = mulmod(a[i + j + half], wt[j * step], p);
        a[i + j] = addmod(u, v, p);
        a[i + j + half] = submod(u, v, p);
      }
  }
}
/* Negacyclic transform: twist by psi^i then cyclic NTT with omega. */
static void nega_fwd(const ntab *T, uint64_t *a) {
  for (uint32_t i = 0; i < T->N; ++i) a[i] = mulmod(a[i], T->psi[i], T->p);
  cyclic_ntt(a, T->N, T->w, T->p);
}
static void nega_inv(const ntab *T, uint64_t *a) {
  cyclic_ntt(a, T->N, T->iw, T->p);
  for (uint32_t i = 0; i < T->N; ++i) a[i] = mulmod(a[i], T->ipsi[i], T->p);
}
/* out = a * b in Z_p[x]/(x^N + 1); out may alias a or b. */
static void nega_mul(const ntab *T, const uint64_t *a, const uint64_t *b,
                     uint64_t *out) {
  uint32_t N = T->N;
  uint64_t *x = malloc(N * sizeof(uint64_t)), *y = malloc(N * sizeof(uint64_t));
  memcpy(x, a, N * sizeof(uint64_t));
  memcpy(y, b, N * sizeof(uint64_t));
  nega_fwd(T, x);
  nega_fwd(T, y);
  for (uint32_t i = 0; i < N; ++i) x[i] = mulmod(x[i], y[i], T->p);
  nega_inv(T, x);
  memcpy(out, x, N * sizeof(uint64_t));
  free(x);
  free(y);
}

int orc_negacyclic_mul_mod(uint32_t N, uint64_t p, const uint64_t *a,
                           const uint64_t *b, uint64_t *out) {
  if (N < 2 || (N & (N - 1)) || p >= (1ull << 62)) return -1;
  ntab T;
  if (ntab_init(&T, N, p)) return -2;
  uint64_t *ar = malloc(N * sizeof(uint64_t)), *br = malloc(N * sizeof(uint64_t));
  for (uint32_t i = 0; i < N; ++i) {
    ar[i] = a[i] % p;
    br[i] = b[i] % p;
  }
  nega_mul(&T, ar, br, out);
  free(ar);
  free(br);
  ntab_free(&T);
  return 0;
}

/* ------------------------------------------------------------------ */
/* CRT bases: reconstruction of x in [0, M) from residues.             */
/* ------------------------------------------------------------------ */
typedef struct {
  uint32_t K;
  uint64_t p[MAXK];
  bu M, Mhalf;      /* product, floor(product / 2) */
  bu hat[MAXK];     /* M / p_k */
  uint64_t hatinv[MAXK]; /* (M / p_k)^-1 mod p_k */
} crt;

static void crt_init(crt *B, const uint64_t *p, uint32_t K) {
  B->K = K;
  bu_set(&B->M, 1);
  for (uint32_t k = 0; k < K; ++k) {
    B->p[k] = p[k];
    bu_mul_u64(&B->M, &B->M, p[k]);
  }
  bu_shr1(&B->Mhalf, &B->M);
  for (uint32_t k = 0; k < K; ++k) {
    bu_set(&B->hat[k], 1);
    for (uint32_t l = 0; l < K; ++l)
      if (l != k) bu_mul_u64(&B->hat[k], &B->hat[k], p[l]);
    B->hatinv[k] = invmod(bu_mod(&B->hat[k], p[k]), p[k]);
  }
}
/* x = sum_k [r_k * hatinv_k]_{p_k} * hat_k, reduced into [0, M). */
static void crt_reconstruct(const crt *B, const uint64_t *r, size_t stride,
                            bu *x) {
  bu_zero(x);
  for (uint32_t k = 0; k < B->K; ++k) {
    uint64_t y = mulmod(r[k * stride] % B->p[k], B->hatinv[k], B->p[k]);
    bu_addmul(x, &B->hat[k], y);
  }
  while (bu_cmp(x, &B->M) >= 0) bu_sub(x, x, &B->M);
}
/* Centered representative in (-M/2, M/2]. */
static void crt_centered(const crt *B, const uint64_t *r, size_t stride,
                         bs *x) {
  crt_reconstruct(B, r, stride, &x->m);
  x->neg = 0;
  if (bu_cmp(&x->m, &B->Mhalf) > 0) {
    bu_sub(&x->m, &B->M, &x->m);
    x->neg = 1;
  }
  if (bu_is_zero(&x->m)) x->neg = 0;
}

/* ------------------------------------------------------------------ */
/* Context                                                             */
/* ------------------------------------------------------------------ */
struct orc_ctx {
  uint32_t N, L;
  uint64_t t;
  uint64_t q[MAXL];
  ntab qt[MAXL];
  crt Qb;          /* ciphertext modulus Q = prod q_j */
  bu Qhalf;        /* floor(Q/2) */
  bu Delta;        /* floor(Q/t) */
  uint64_t delta_mod[MAXL];
  uint64_t g_mod[MAXL][MAXL]; /* g_i mod q_j, g_i = (Q/q_i)[(Q/q_i)^-1]_{q_i} */
  crt Mb;          /* auxiliary primes for exact integer products */
  ntab mt[MAXK];
};

uint32_t orc_aux_count(const orc_ctx *ctx) { return ctx->Mb.K; }

orc_ctx *orc_create(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t) {
  if (N < 4 || N > 65536 || (N & (N - 1)) || L < 1 || L > MAXL) return NULL;
  if (t < 2 || t >= (1ull << 32)) return NULL;
  for (uint32_t j = 0; j < L; ++j) {
    if (q[j] >= (1ull << 62) || !orc_is_prime(q[j])) return NULL;
    if ((q[j] - 1) % (2 * (uint64_t)N)) return NULL;
    if (q[j] == t) return NULL;
    for (uint32_t l = 0; l < j; ++l)
      if (q[l] == q[j]) return NULL;
  }
  orc_ctx *c = calloc(1, sizeof *c);
  c->N = N;
  c->L = L;
  c->t = t;
  for (uint32_t j = 0; j < L; ++j) {
    c->q[j] = q[j];
    if (ntab_init(&c->qt[j], N, q[j])) die("ntt table for q");
  }
  crt_init(&c->Qb, q, L);
  bu_shr1(&c->Qhalf, &c->Qb.M);
  bu_divmod(&c->Delta, &c->Qb.M, t);
  for (uint32_t j = 0; j < L; ++j) c->delta_mod[j] = bu_mod(&c->Delta, q[j]);
  for (uint32_t i = 0; i < L; ++i) {
    bu g;
    bu_mul_u64(&g, &c->Qb.hat[i], c->Qb.hatinv[i]);
    for (uint32_t j = 0; j < L; ++j) c->g_mod[i][j] = bu_mod(&g, q[j]);
  }
  /* Auxiliary primes (61-62 bits, = 1 mod 2N) until their product exceeds
   * 2 * N * Q^2: the exact products have |d| <= 2 * N * (Q/2)^2. */
  bu need, Q2;
  bu_mul(&Q2, &c->Qb.M, &c->Qb.M);
  bu_mul_u64(&need, &Q2, 2 * (uint64_t)N);
  uint64_t aux[MAXK];
  uint32_t K = 0;
  bu prod;
  bu_set(&prod, 1);
  uint64_t p = (1ull << 62) - 2 * (uint64_t)N + 1;
  while (bu_cmp(&prod, &need) <= 0) {
    if (K == MAXK) die("too many auxiliary primes");
    while (!orc_is_prime(p)) p -= 2 * (uint64_t)N;
    aux[K++] = p;
    bu_mul_u64(&prod, &prod, p);
    p -= 2 * (uint64_t)N;
  }
  crt_init(&c->Mb, aux, K);
  for (uint32_t k = 0; k < K; ++k)
    if (ntab_init(&c->mt[k], N, aux[k])) die("ntt table for aux prime");
  return c;
}

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  for (uint32_t j = 0; j < c->L; ++j) ntab_free(&c->qt[j]);
  for (uint32_t k = 0; k < c->Mb.K; ++k) ntab_free(&c->mt[k]);
  free(c);
}

#define LN(c) ((size_t)(c)->L * (c)->N)

/* ------------------------------------------------------------------ */
/* Exact tensor and scale-down (BFV multiplication, FV textbook).      */
/* ------------------------------------------------------------------ */

/* Centered lift of an R_Q polynomial: coefficient i -> integer in
 * (-Q/2, Q/2] with the given residues. */
static void lift_poly(const orc_ctx *c, const uint64_t *poly, bs *out) {
  for (uint32_t i = 0; i < c->N; ++i) crt_centered(&c->Qb, poly + i, c->N, &out[i]);
}

/* Exact integer negacyclic products of centered lifts.  n_out products:
 * out[l] = sum over pairs (A[l][u], B[l][u]) for u < terms[l].  Each
 * product is formed modulo every auxiliary prime through the NTT and the
 * integer is rebuilt by CRT (the auxiliary product exceeds twice the
 * largest possible magnitude). */
static void exact_products(const orc_ctx *c, int n_in, const bs *const *in,
                           int n_out, const int (*pairs)[2][2],
                           const int *terms, bs **out) {
  uint32_t N = c->N, K = c->Mb.K;
  uint64_t *res = malloc((size_t)n_out * K * N * sizeof(uint64_t));
  uint64_t *tr = malloc((size_t)n_in * N * sizeof(uint64_t));
  uint64_t *acc = malloc((size_t)N * sizeof(uint64_t));
  for (uint32_t k = 0; k < K; ++k) {
    const ntab *T = &c->mt[k];
    for (int v = 0; v < n_in; ++v) {
      for (uint32_t i = 0; i < N; ++i) tr[(size_t)v * N + i] = bs_mod(&in[v][i], T->p);
      nega_fwd(T, tr + (size_t)v * N);
    }
    for (int l = 0; l < n_out; ++l) {
      memset(acc, 0, N * sizeof(uint64_t));
      for (int u = 0; u < terms[l]; ++u) {
        const uint64_t *x = tr + (size_t)pairs[l][u][0] * N;
        const uint64_t *y = tr + (size_t)pairs[l][u][1] * N;
        for (uint32_t i = 0; i < N; ++i)
          acc[i] = addmod(acc[i], mulmod(x[i], y[i], T->p), T->p);
      }
      nega_inv(T, acc);
      memcpy(res + ((size_t)l * K + k) * N, acc, N * sizeof(uint64_t));
    }
  }
  for (int l = 0; l < n_out; ++l)
    for (uint32_t i = 0; i < N; ++i)
      crt_centered(&c->Mb, res + (size_t)l * K * N + i, N, &out[l][i]);
  free(res);
  free(tr);
  free(acc);
}

/* floor(X / Q) for a signed X, by successive floor divisions by the primes
 * of Q (floor(floor(X/a)/b) = floor(X/(ab)) for X >= 0). */
static void floordiv_Q(const orc_ctx *c, const bs *X, bs *out) {
  bu a = X->m;
  if (X->neg) {
    /* floor(-A/Q) = -floor((A + Q - 1)/Q) */
    bu one;
    bu_set(&one, 1);
    bu_add(&a, &a, &c->Qb.M);
    bu_sub(&a, &a, &one);
  }
  for (uint32_t j = 0; j < c->L; ++j) bu_divmod(&a, &a, c->q[j]);
  out->m = a;
  out->neg = X->neg && !bu_is_zero(&a);
}

/* e = round(t * d / Q) = floor((t*d + floor(Q/2)) / Q), reduced mod q_j.
 * Q is odd and coprime to t, so t*d/Q is never exactly half an integer and
 * the rounding direction of ties never matters. */
static void scale_round(const orc_ctx *c, const bs *d, uint64_t *res, size_t stride) {
  bs X;
  bu_mul_u64(&X.m, &d->m, c->t);
  X.neg = d->neg;
  /* X += floor(Q/2) */
  if (!X.neg) {
    bu_add(&X.m, &X.m, &c->Qhalf);
  } else if (bu_cmp(&X.m, &c->Qhalf) > 0) {
    bu_sub(&X.m, &X.m, &c->Qhalf);
  } else {
    bu_sub(&X.m, &c->Qhalf, &X.m);
    X.neg = 0;
  }
  if (bu_is_zero(&X.m)) X.neg = 0;
  bs e;
  floordiv_Q(c, &X, &e);
  for (uint32_t j = 0; j < c->L; ++j) res[j * stride] = bs_mod(&e, c->q[j]);
}

int orc_exact_product(const orc_ctx *c, const uint64_t *a, const uint64_t *b,
                      uint32_t words, int32_t *sign, uint64_t *mag) {
  if (words > BW) return -1;
  uint32_t N = c->N;
  bs *A = malloc(N * sizeof(bs)), *B = malloc(N * sizeof(bs)), *D = malloc(N * sizeof(bs));
  lift_poly(c, a, A);
  lift_poly(c, b, B);
  const bs *in[2] = {A, B};
  static const int pairs[1][2][2] = {{{0, 1}, {0, 0}}};
  static const int terms[1] = {1};
  bs *outs[1] = {D};
  exact_products(c, 2, in, 1, pairs, terms, outs);
  int rc = 0;
  for (uint32_t i = 0; i < N; ++i) {
    sign[i] = D[i].neg;
    for (uint32_t w = words; w < BW; ++w)
      if (D[i].m.w[w]) rc = -2;
    memcpy(mag + (size_t)i * words, D[i].m.w, words * sizeof(uint64_t));
  }
  free(A);
  free(B);
  free(D);
  return rc;
}

int orc_scale_round(const orc_ctx *c, int32_t sign, const uint64_t *mag,
                    uint32_t words, uint64_t *out) {
  if (words > BW) return -1;
  bs d;
  bu_zero(&d.m);
  memcpy(d.m.w, mag, words * sizeof(uint64_t));
  d.neg = sign && !bu_is_zero(&d.m);
  scale_round(c, &d, out, 1);
  return 0;
}

/* Tensor: with a = (a0, a1), b = (b0, b1) lifted to centered integers,
 * d0 = a0*b0, d1 = a0*b1 + a1*b0, d2 = a1*b1 exactly, then each
 * coefficient is scaled by t/Q and rounded (FV multiplication). */
int orc_tensor(const orc_ctx *c, const uint64_t *a, const uint64_t *b,
               uint64_t *out3) {
  uint32_t N = c->N;
  size_t ln = LN(c);
  bs *buf = malloc((size_t)7 * N * sizeof(bs));
  bs *A0 = buf, *A1 = buf + N, *B0 = buf + 2 * N, *B1 = buf + 3 * N;
  bs *D[3] = {buf + 4 * N, buf + 5 * N, buf + 6 * N};
  lift_poly(c, a, A0);
  lift_poly(c, a + ln, A1);
  lift_poly(c, b, B0);
  lift_poly(c, b + ln, B1);
  const bs *in[4] = {A0, A1, B0, B1};
  static const int pairs[3][2][2] = {
      {{0, 2}, {0, 0}}, {{0, 3}, {1, 2}}, {{1, 3}, {0, 0}}};
  static const int terms[3] = {1, 2, 1};
  exact_products(c, 4, in, 3, pairs, terms, D);
  for (int l = 0; l < 3; ++l)
    for (uint32_t i = 0; i < N; ++i) scale_round(c, &D[l][i], out3 + l * ln + i, N);
  free(buf);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Key switching (RNS-digit decomposition, no special modulus).        */
/* ------------------------------------------------------------------ */
/* z in R_Q.  Digit i is D_i = [z]_{q_i} taken as an integer in [0, q_i);
 * since sum_i D_i * g_i = z (mod Q), a key with b_i = -a_i*s + e_i + g_i*w
 * gives (sum D_i b_i) + (sum D_i a_i) * s = z*w + sum D_i e_i (mod Q). */
int orc_keyswitch(const orc_ctx *c, const uint64_t *z, const uint64_t *key,
                  uint64_t *out) {
  uint32_t N = c->N, L = c->L;
  size_t ln = LN(c);
  /* Output limb j: sum_i (D_i mod q_j) * key_ij in Z_{q_j}[x]/(x^N+1); the
   * products are summed in the NTT domain and transformed back once. */
#pragma omp parallel for schedule(static)
  for (uint32_t j = 0; j < L; ++j) {
    const ntab *T = &c->qt[j];
    uint64_t *d = malloc(N * sizeof(uint64_t)), *kp = malloc(N * sizeof(uint64_t));
    uint64_t *acc[2] = {calloc(N, sizeof(uint64_t)), calloc(N, sizeof(uint64_t))};
    for (uint32_t i = 0; i < L; ++i) {
      for (uint32_t x = 0; x < N; ++x) d[x] = z[(size_t)i * N + x] % c->q[j];
      nega_fwd(T, d);
      for (int comp = 0; comp < 2; ++comp) {
        memcpy(kp, key + ((size_t)i * 2 + comp) * ln + (size_t)j * N, N * sizeof(uint64_t));
        nega_fwd(T, kp);
        for (uint32_t x = 0; x < N; ++x)
          acc[comp][x] = addmod(acc[comp][x], mulmod(d[x], kp[x], T->p), T->p);
      }
    }
    for (int comp = 0; comp < 2; ++comp) {
      nega_inv(T, acc[comp]);
      memcpy(out + comp * ln + (size_t)j * N, acc[comp], N * sizeof(uint64_t));
      free(acc[comp]);
    }
    free(d);
    free(kp);
  }
  return 0;
}

static void poly_add(const orc_ctx *c, const uint64_t *a, const uint64_t *b,
                     uint64_t *out) {
  for (uint32_t j = 0; j < c->L; ++j)
    for (uint32_t i = 0; i < c->N; ++i) {
      size_t x = (size_t)j * c->N + i;
      out[x] = addmod(a[x], b[x], c->q[j]);
    }
}
static void poly_sub(const orc_ctx *c, const uint64_t *a, const uint64_t *b,
                     uint64_t *out) {
  for (uint32_t j = 0; j < c->L; ++j)
    for (uint32_t i = 0; i < c->N; ++i) {
      size_t x = (size_t)j * c->N + i;
      out[x] = submod(a[x], b[x], c->q[j]);
    }
}

/* M: tensor, scale-down, then relinearise the s^2 component. */
int orc_bfv_mul(const orc_ctx *c, const uint64_t *a, const uint64_t *b,
                const uint64_t *rlk, uint64_t *out) {
  size_t ln = LN(c);
  uint64_t *t3 = malloc(3 * ln * sizeof(uint64_t)), *ks = malloc(2 * ln * sizeof(uint64_t));
  orc_tensor(c, a, b, t3);
  orc_keyswitch(c, t3 + 2 * ln, rlk, ks);
  poly_add(c, t3, ks, out);
  poly_add(c, t3 + ln, ks + ln, out + ln);
  free(t3);
  free(ks);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Automorphism, monomials, substitution, expansion                    */
/* ------------------------------------------------------------------ */
int orc_automorphism(const orc_ctx *c, uint32_t g, const uint64_t *in,
                     uint64_t *out) {
  uint32_t N = c->N;
  uint64_t twoN = 2 * (uint64_t)N;
  if (!(g & 1) || g >= twoN) return -1;
  for (uint32_t j = 0; j < c->L; ++j)
    for (uint32_t i = 0; i < N; ++i) {
      /* x^i -> x^(i*g mod 2N), and x^(N + r) = -x^r */
      uint64_t e = ((uint64_t)i * g) % twoN;
      uint64_t v = in[(size_t)j * N + i];
      if (e >= N) {
        e -= N;
        v = v ? c->q[j] - v : 0;
      }
      out[(size_t)j * N + e] = v;
    }
  return 0;
}

int orc_monomial(const orc_ctx *c, int64_t e, const uint64_t *in, uint64_t *out) {
  int64_t twoN = 2 * (int64_t)c->N;
  if (e <= -twoN || e >= twoN) return -1;
  uint64_t r = (uint64_t)((e % twoN + twoN) % twoN);
  uint32_t N = c->N;
  for (uint32_t j = 0; j < c->L; ++j)
    for (uint32_t i = 0; i < N; ++i) {
      uint64_t d = i + r, v = in[(size_t)j * N + i];
      if (d >= 2 * (uint64_t)N) {
        d -= 2 * (uint64_t)N;
      } else if (d >= N) {
        d -= N;
        v = v ? c->q[j] - v : 0;
      }
      out[(size_t)j * N + d] = v;
    }
  return 0;
}

/* Sub_g(c0, c1) = (tau_g(c0), 0) + KeySwitch(tau_g(c1)) with the key for
 * s(x^g): decrypts to tau_g(c0 + c1 s) = Delta*mu(x^g) + noise. */
int orc_substitute(const orc_ctx *c, uint32_t g, const uint64_t *ct,
                   const uint64_t *gkey, uint64_t *out) {
  size_t ln = LN(c);
  uint64_t *t0 = malloc(ln * sizeof(uint64_t)), *t1 = malloc(ln * sizeof(uint64_t));
  uint64_t *ks = malloc(2 * ln * sizeof(uint64_t));
  if (orc_automorphism(c, g, ct, t0) || orc_automorphism(c, g, ct + ln, t1)) {
    free(t0);
    free(t1);
    free(ks);
    return -1;
  }
  orc_keyswitch(c, t1, gkey, ks);
  poly_add(c, t0, ks, out);
  memcpy(out + ln, ks + ln, ln * sizeof(uint64_t));
  free(t0);
  free(t1);
  free(ks);
  return 0;
}

static void ct_monomial(const orc_ctx *c, int64_t e, const uint64_t *in, uint64_t *out) {
  size_t ln = LN(c);
  orc_monomial(c, e, in, out);
  orc_monomial(c, e, in + ln, out + ln);
}
static void ct_add(const orc_ctx *c, const uint64_t *a, const uint64_t *b, uint64_t *out) {
  size_t ln = LN(c);
  poly_add(c, a, b, out);
  poly_add(c, a + ln, b + ln, out + ln);
}
static void ct_sub(const orc_ctx *c, const uint64_t *a, const uint64_t *b, uint64_t *out) {
  size_t ln = LN(c);
  poly_sub(c, a, b, out);
  poly_sub(c, a + ln, b + ln, out + ln);
}

/* Alg. Query Expansion: for each input ciphertext, c rounds; in round a the
 * b-th entry (b < 2^a) is split with one substitution by N/2^a + 1 and two
 * monomial multiplications by x^(-2^a).  The outputs of all input cts are
 * concatenated and the first m kept. */
int orc_expand(const orc_ctx *c, uint32_t h, const uint64_t *query, uint32_t cf,
               uint32_t m, const uint64_t *gkeys, uint64_t *out) {
  uint32_t N = c->N;
  size_t ln = LN(c), ctw = 2 * ln;
  if ((1u << cf) > N || m > (uint64_t)h << cf) return -1;
  uint32_t B = 1u << cf;
  uint64_t *cts = malloc((size_t)B * ctw * sizeof(uint64_t));
  uint32_t written = 0;
  for (uint32_t j = 0; j < h && written < m; ++j) {
    memcpy(cts, query + (size_t)j * ctw, ctw * sizeof(uint64_t));
    for (uint32_t a = 0; a < cf; ++a) {
      uint32_t two_a = 1u << a;
      uint32_t g = N / two_a + 1;
      const uint64_t *gk = gkeys + (size_t)a * c->L * ctw;
      /* the iterations over b touch disjoint entries: run them in parallel */
#pragma omp parallel for schedule(dynamic, 1)
      for (uint32_t b = 0; b < two_a; ++b) {
        uint64_t *c0 = malloc(ctw * sizeof(uint64_t)), *c1 = malloc(ctw * sizeof(uint64_t));
        uint64_t *cb = cts + (size_t)b * ctw, *cb2 = cts + (size_t)(b + two_a) * ctw;
        orc_substitute(c, g, cb, gk, c0);          /* c0 <- Sub(cts[b])        */
        ct_monomial(c, -(int64_t)two_a, c0, c1);  /* c1 <- x^-2^a * c0        */
        ct_monomial(c, -(int64_t)two_a, cb, cb2); /* cts[b+2^a] <- x^-2^a cts[b] */
        ct_add(c, cb, c0, cb);                    /* cts[b] += c0             */
        ct_sub(c, cb2, c1, cb2);                  /* cts[b+2^a] -= c1         */
        free(c0);
        free(c1);
      }
    }
    for (uint32_t b = 0; b < B && written < m; ++b, ++written)
      memcpy(out + (size_t)written * ctw, cts + (size_t)b * ctw, ctw * sizeof(uint64_t));
  }
  free(cts);
  return 0;
}

/* Alg. SealPIR Oblivious Expansion, loop only: cts[b] = c0 + Sub(c0) and
 * cts[b+2^a] = c1 + Sub(c1) with c1 = x^(-2^a) c0. */
int orc_expand_sealpir(const orc_ctx *c, const uint64_t *ct, uint32_t cf,
                       const uint64_t *gkeys, uint64_t *out) {
  uint32_t N = c->N;
  size_t ln = LN(c), ctw = 2 * ln;
  if ((1u << cf) > N) return -1;
  uint64_t *c0 = malloc(ctw * sizeof(uint64_t)), *c1 = malloc(ctw * sizeof(uint64_t));
  uint64_t *sb = malloc(ctw * sizeof(uint64_t));
  memcpy(out, ct, ctw * sizeof(uint64_t));
  for (uint32_t a = 0; a < cf; ++a) {
    uint32_t two_a = 1u << a, g = N / two_a + 1;
    const uint64_t *gk = gkeys + (size_t)a * c->L * ctw;
    for (uint32_t b = 0; b < two_a; ++b) {
      memcpy(c0, out + (size_t)b * ctw, ctw * sizeof(uint64_t));
      ct_monomial(c, -(int64_t)two_a, c0, c1);
      orc_substitute(c, g, c0, gk, sb);
      ct_add(c, c0, sb, out + (size_t)b * ctw);
      orc_substitute(c, g, c1, gk, sb);
      ct_add(c, c1, sb, out + (size_t)(b + two_a) * ctw);
    }
  }
  free(c0);
  free(c1);
  free(sb);
  return 0;
}

int orc_scalar_mul(const orc_ctx *c, const uint64_t *ct, uint64_t scalar,
                   uint64_t *out) {
  size_t ln = LN(c);
  for (uint32_t p = 0; p < 2; ++p)
    for (uint32_t j = 0; j < c->L; ++j)
      for (uint32_t i = 0; i < c->N; ++i) {
        size_t x = p * ln + (size_t)j * c->N + i;
        out[x] = mulmod(ct[x], scalar % c->q[j], c->q[j]);
      }
  return 0;
}

/* Homomorphic 1 - mu: the constant plaintext 1 minus the ciphertext,
 * (Delta * 1 - c0, -c1) in R_Q; decrypts to 1 - mu (mod t) with the noise
 * negated.  The factor (1 - x[i]) of Eq. folklore-plain-eq. */
int orc_one_minus(const orc_ctx *c, const uint64_t *ct, uint64_t *out) {
  size_t ln = LN(c);
  for (uint32_t j = 0; j < c->L; ++j) {
    uint64_t q = c->q[j];
    for (uint32_t i = 0; i < c->N; ++i) {
      size_t x = (size_t)j * c->N + i;
      uint64_t c0 = ct[x], c1 = ct[ln + x];
      uint64_t d = i == 0 ? c->delta_mod[j] : 0; /* Delta times the constant 1 */
      out[x] = d >= c0 ? d - c0 : d + q - c0;
      out[ln + x] = c1 ? q - c1 : 0;
    }
  }
  return 0;
}

/* Leaves of the plain folklore operator (Eq. folklore-plain-eq) for an
 * ell-bit public operand y: the factor of bit i is (1 - x[i]) when y[i] = 0
 * and x[i] when y[i] = 1.  With the 2*ell leaves ordered
 * (1 - x[0], x[0], 1 - x[1], x[1], ...), the factors of y sit at positions
 * 2i + y[i], ascending, so the product is a selection over a weight-ell
 * codeword of length 2*ell. */
int orc_folklore_codeword(uint64_t y, uint32_t ell, uint16_t *pos) {
  if (ell == 0 || ell > 64 || (ell < 64 && (y >> ell))) return -1;
  for (uint32_t i = 0; i < ell; ++i) pos[i] = (uint16_t)(2 * i + ((y >> i) & 1));
  return 0;
}

/* ------------------------------------------------------------------ */
/* Plain multiplication, selection vector, answer                      */
/* ------------------------------------------------------------------ */
/* The item plaintext mu (coefficients in [0, t), zero beyond payload_len)
 * is lifted to its centered integer (v > t/2 -> v - t) and multiplied into
 * both ciphertext polynomials in R_Q. */
int orc_plain_mul(const orc_ctx *c, const uint64_t *ct, const uint32_t *mu,
                  uint32_t payload_len, uint64_t *out) {
  uint32_t N = c->N;
  size_t ln = LN(c);
  if (payload_len > N) return -1;
  uint64_t *m = malloc(N * sizeof(uint64_t));
  for (uint32_t j = 0; j < c->L; ++j) {
    uint64_t qj = c->q[j];
    for (uint32_t i = 0; i < N; ++i) {
      uint64_t v = i < payload_len ? mu[i] % c->t : 0;
      m[i] = (v > c->t / 2) ? qj - (c->t - v) : v;
    }
    for (int p = 0; p < 2; ++p)
      nega_mul(&c->qt[j], ct + p * ln + (size_t)j * N, m, out + p * ln + (size_t)j * N);
  }
  free(m);
  return 0;
}

/* Plain constant-weight equality operator as a product tree: the ciphertexts
 * at the ascending positions form the first level; each level multiplies
 * neighbours (2r, 2r+1) and carries an odd last element up unchanged. */
int orc_selection(const orc_ctx *c, const uint64_t *ctxts,
                  const uint16_t *positions, uint32_t k, const uint64_t *rlk,
                  uint64_t *out) {
  size_t ctw = 2 * LN(c);
  if (k == 0) return -1;
  uint64_t *level = malloc((size_t)k * ctw * sizeof(uint64_t));
  uint64_t *next = malloc((size_t)k * ctw * sizeof(uint64_t));
  for (uint32_t u = 0; u < k; ++u)
    memcpy(level + u * ctw, ctxts + (size_t)positions[u] * ctw, ctw * sizeof(uint64_t));
  uint32_t len = k;
  while (len > 1) {
    uint32_t nl = 0;
    for (uint32_t r = 0; 2 * r + 1 < len; ++r, ++nl)
      orc_bfv_mul(c, level + 2 * r * ctw, level + (2 * r + 1) * ctw, rlk, next + nl * ctw);
    if (len & 1) {
      memcpy(next + nl * ctw, level + (len - 1) * ctw, ctw * sizeof(uint64_t));
      ++nl;
    }
    uint64_t *tmp = level;
    level = next;
    next = tmp;
    len = nl;
  }
  memcpy(out, level, ctw * sizeof(uint64_t));
  free(level);
  free(next);
  return 0;
}

/* Alg. Arithmetic Constant-weight Equality Operator on encrypted operands
 * x, y ([m] ciphertexts each, bit i of every SIMD slot's codeword):
 *   k' = sum_i x[i] * y[i]             (m multiplications M, then adds)
 *   e  = (1/k!) prod_{i<k} (k' - i)     (k' - i: the constant plaintext i
 *                                        subtracted; the product by the
 *                                        balanced tree; 1/k! mod t as a
 *                                        scalar)
 * Depth 1 + ceil(log2 k). */
int orc_arith_cw_eq(const orc_ctx *c, uint32_t m, uint32_t k, const uint64_t *x,
                    const uint64_t *y, const uint64_t *rlk, uint64_t *out) {
  size_t ctw = 2 * LN(c);
  if (k == 0 || k > m) return -1;
  uint64_t *kp = calloc(ctw, sizeof(uint64_t)), *prod = malloc(ctw * sizeof(uint64_t));
  for (uint32_t i = 0; i < m; ++i) {
    orc_bfv_mul(c, x + (size_t)i * ctw, y + (size_t)i * ctw, rlk, prod);
    ct_add(c, kp, prod, kp);
  }
  uint64_t *fac = malloc((size_t)k * ctw * sizeof(uint64_t));
  uint16_t *pos = malloc(k * sizeof(uint16_t));
  for (uint32_t i = 0; i < k; ++i) {
    uint64_t *f = fac + (size_t)i * ctw;
    memcpy(f, kp, ctw * sizeof(uint64_t));
    for (uint32_t j = 0; j < c->L; ++j) /* c0 - Delta * i at x^0 */
      f[(size_t)j * c->N] = submod(f[(size_t)j * c->N], mulmod(c->delta_mod[j], i, c->q[j]),
                                   c->q[j]);
    pos[i] = (uint16_t)i;
  }
  orc_selection(c, fac, pos, k, rlk, prod);
  uint64_t kf = 1; /* k! mod t */
  for (uint32_t i = 2; i <= k; ++i) kf = mulmod(kf, i, c->t);
  orc_scalar_mul(c, prod, invmod(kf, c->t), out);
  free(kp);
  free(prod);
  free(fac);
  free(pos);
  return 0;
}

/* SIMD batch encoding over Z_t (t prime, t = 1 mod 2N): slot i of a
 * plaintext mu is mu evaluated at psi^(2i+1), psi = 3^((t-1)/2N) a
 * primitive 2N-th root of unity (3 generates Z_t^* for t = 65537).  The
 * slots of a product mod (x^N + 1, t) are the slot-wise products.
 * Evaluated directly, O(N^2). */
static uint64_t batch_psi(const orc_ctx *c) {
  return powmod(3, (c->t - 1) / (2 * c->N), c->t);
}

int orc_batch_decode(const orc_ctx *c, const uint32_t *mu, uint32_t *slots) {
  uint64_t t = c->t, psi = batch_psi(c);
  if ((t - 1) % (2 * c->N)) return -1;
  for (uint32_t i = 0; i < c->N; ++i) {
    uint64_t w = powmod(psi, 2 * i + 1, t), pw = 1, v = 0;
    for (uint32_t j = 0; j < c->N; ++j) {
      v = (v + mulmod(mu[j] % t, pw, t)) % t;
      pw = mulmod(pw, w, t);
    }
    slots[i] = (uint32_t)v;
  }
  return 0;
}

int orc_batch_encode(const orc_ctx *c, const uint32_t *slots, uint32_t *mu) {
  uint64_t t = c->t, psi = batch_psi(c);
  if ((t - 1) % (2 * c->N)) return -1;
  /* mu_j = N^-1 sum_i slot_i w_i^-j with w_i = psi^(2i+1); cur[i] runs
   * through slot_i w_i^-j as j grows */
  uint64_t ninv = invmod(c->N % t, t);
  uint64_t *cur = malloc(c->N * sizeof(uint64_t)), *winv = malloc(c->N * sizeof(uint64_t));
  for (uint32_t i = 0; i < c->N; ++i) {
    cur[i] = slots[i] % t;
    winv[i] = invmod(powmod(psi, 2 * i + 1, t), t);
  }
  for (uint32_t j = 0; j < c->N; ++j) {
    uint64_t v = 0;
    for (uint32_t i = 0; i < c->N; ++i) {
      v += cur[i];
      cur[i] = mulmod(cur[i], winv[i], t);
    }
    mu[j] = (uint32_t)mulmod(v % t, ninv, t);
  }
  free(cur);
  free(winv);
  return 0;
}

int orc_answer(const orc_ctx *c, uint64_t n, uint32_t payload_len,
               const uint32_t *items, const uint16_t *codewords, uint32_t k,
               uint32_t m, uint32_t cf, const uint64_t *query,
               const uint64_t *rlk, const uint64_t *gkeys, int nthreads,
               uint64_t *resp) {
  size_t ctw = 2 * LN(c);
  /* Sec. 3.3.1: a row holds s >= 1 plaintexts; plaintext p carries payload
   * coefficients p*N .. p*N + N - 1 (the last one zero-padded). */
  const uint32_t s = payload_len == 0 ? 1 : (payload_len + c->N - 1) / c->N;
  if (k == 0 || k > m || s > ORC_MAX_PLAINTEXTS) return -1;
  for (uint64_t i = 0; i < n; ++i)
    for (uint32_t u = 0; u < k; ++u) {
      uint16_t p = codewords[i * k + u];
      if (p >= m || (u && p <= codewords[i * k + u - 1])) return -2;
    }
  /* Query expansion (only when the query is compressed). */
  const uint64_t *ctxts = query;
  uint64_t *expanded = NULL;
  if (cf > 0) {
    if (!gkeys) return -3;
    uint32_t h = (m + (1u << cf) - 1) >> cf;
    expanded = malloc((size_t)m * ctw * sizeof(uint64_t));
    orc_expand(c, h, query, cf, m, gkeys, expanded);
    ctxts = expanded;
  }
  memset(resp, 0, (size_t)s * ctw * sizeof(uint64_t));
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    uint64_t *local = calloc((size_t)s * ctw, sizeof(uint64_t));
    uint64_t *sel = malloc(ctw * sizeof(uint64_t)), *pm = malloc(ctw * sizeof(uint64_t));
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
      /* one selection entry per row, then s inner products (Sec. 3.3.3) */
      orc_selection(c, ctxts, codewords + (size_t)i * k, k, rlk, sel);
      for (uint32_t p = 0; p < s; ++p) {
        uint32_t lo = p * c->N, len = payload_len - lo < c->N ? payload_len - lo : c->N;
        orc_plain_mul(c, sel, items + (size_t)i * payload_len + lo, len, pm);
        ct_add(c, local + (size_t)p * ctw, pm, local + (size_t)p * ctw);
      }
    }
#pragma omp critical
    for (uint32_t p = 0; p < s; ++p)
      ct_add(c, resp + (size_t)p * ctw, local + (size_t)p * ctw, resp + (size_t)p * ctw);
    free(local);
    free(sel);
    free(pm);
  }
  free(expanded);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Client side: keys, encryption, query construction, decryption       */
/* ------------------------------------------------------------------ */
static void small_to_mod(const orc_ctx *c, uint32_t j, const int64_t *v, uint64_t *out) {
  uint64_t q = c->q[j];
  for (uint32_t i = 0; i < c->N; ++i) {
    int64_t x = v[i] % (int64_t)q;
    out[i] = x < 0 ? (uint64_t)(x + (int64_t)q) : (uint64_t)x;
  }
}

/* Switching key for w (given as a signed small polynomial):
 * b_i = -a_i*s + e_i + g_i*w (mod Q), component a_i. */
static void keygen_switch(const orc_ctx *c, const int8_t *s, const int64_t *w,
                          const uint64_t *a, const int32_t *e, uint64_t *key) {
  uint32_t N = c->N, L = c->L;
  size_t ln = LN(c);
  int64_t *tmp = malloc(N * sizeof(int64_t));
  uint64_t *sm = malloc(N * sizeof(uint64_t)), *wm = malloc(N * sizeof(uint64_t));
  uint64_t *as = malloc(N * sizeof(uint64_t)), *em = malloc(N * sizeof(uint64_t));
  for (uint32_t i = 0; i < L; ++i)
    for (uint32_t j = 0; j < L; ++j) {
      uint64_t q = c->q[j];
      for (uint32_t x = 0; x < N; ++x) tmp[x] = s[x];
      small_to_mod(c, j, tmp, sm);
      small_to_mod(c, j, w, wm);
      for (uint32_t x = 0; x < N; ++x) tmp[x] = e[(size_t)i * N + x];
      small_to_mod(c, j, tmp, em);
      const uint64_t *aij = a + (size_t)i * ln + (size_t)j * N;
      nega_mul(&c->qt[j], aij, sm, as);
      uint64_t *b = key + ((size_t)i * 2 + 0) * ln + (size_t)j * N;
      uint64_t *ak = key + ((size_t)i * 2 + 1) * ln + (size_t)j * N;
      for (uint32_t x = 0; x < N; ++x) {
        uint64_t v = submod(em[x], as[x], q);
        v = addmod(v, mulmod(c->g_mod[i][j], wm[x], q), q);
        b[x] = v;
        ak[x] = aij[x] % q;
      }
    }
  free(tmp);
  free(sm);
  free(wm);
  free(as);
  free(em);
}

int orc_keygen_relin(const orc_ctx *c, const int8_t *s, const uint64_t *a,
                     const int32_t *e, uint64_t *key) {
  uint32_t N = c->N;
  /* s^2 in Z[x]/(x^N+1), schoolbook over the small integers */
  int64_t *w = calloc(N, sizeof(int64_t));
  for (uint32_t i = 0; i < N; ++i) {
    if (!s[i]) continue;
    for (uint32_t j = 0; j < N; ++j) {
      int64_t v = (int64_t)s[i] * s[j];
      uint32_t d = i + j;
      if (d >= N) w[d - N] -= v;
      else w[d] += v;
    }
  }
  keygen_switch(c, s, w, a, e, key);
  free(w);
  return 0;
}

int orc_keygen_galois(const orc_ctx *c, uint32_t g, const int8_t *s,
                      const uint64_t *a, const int32_t *e, uint64_t *key) {
  uint32_t N = c->N;
  uint64_t twoN = 2 * (uint64_t)N;
  if (!(g & 1) || g >= twoN) return -1;
  int64_t *w = calloc(N, sizeof(int64_t));
  for (uint32_t i = 0; i < N; ++i) {
    uint64_t d = ((uint64_t)i * g) % twoN;
    if (d >= N) w[d - N] = -s[i];
    else w[d] = s[i];
  }
  keygen_switch(c, s, w, a, e, key);
  free(w);
  return 0;
}

int orc_encrypt(const orc_ctx *c, const uint32_t *mu, const int8_t *s,
                const uint64_t *a, const int32_t *e, uint64_t *ct) {
  uint32_t N = c->N;
  size_t ln = LN(c);
  int64_t *tmp = malloc(N * sizeof(int64_t));
  uint64_t *sm = malloc(N * sizeof(uint64_t)), *as = malloc(N * sizeof(uint64_t));
  for (uint32_t j = 0; j < c->L; ++j) {
    uint64_t q = c->q[j];
    for (uint32_t x = 0; x < N; ++x) tmp[x] = s[x];
    small_to_mod(c, j, tmp, sm);
    const uint64_t *aj = a + (size_t)j * N;
    nega_mul(&c->qt[j], aj, sm, as);
    for (uint32_t x = 0; x < N; ++x) {
      int64_t ev = e[x] % (int64_t)q;
      uint64_t em = ev < 0 ? (uint64_t)(ev + (int64_t)q) : (uint64_t)ev;
      uint64_t v = mulmod(c->delta_mod[j], mu[x] % c->t, q);
      v = submod(v, as[x], q);
      v = addmod(v, em, q);
      ct[(size_t)j * N + x] = v;
      ct[ln + (size_t)j * N + x] = aj[x] % q;
    }
  }
  free(tmp);
  free(sm);
  free(as);
  return 0;
}

/* Alg. Query: E_q's bits packed 2^c per plaintext, each multiplied by
 * 2^-c mod t, then encrypted under the secret key. */
int orc_make_query(const orc_ctx *c, const uint16_t *positions, uint32_t k,
                   uint32_t m, uint32_t cf, const int8_t *s, const uint64_t *a,
                   const int32_t *e, uint64_t *query) {
  uint32_t N = c->N;
  size_t ln = LN(c);
  if ((1u << cf) > N) return -1;
  uint32_t B = 1u << cf, h = (m + B - 1) / B;
  uint8_t *bits = calloc(m, 1);
  for (uint32_t u = 0; u < k; ++u) {
    if (positions[u] >= m) {
      free(bits);
      return -2;
    }
    bits[positions[u]] = 1;
  }
  uint64_t inv = invmod(powmod(2, cf, c->t), c->t); /* t prime */
  uint32_t *mu = malloc(N * sizeof(uint32_t));
  for (uint32_t i = 0; i < h; ++i) {
    memset(mu, 0, N * sizeof(uint32_t));
    for (uint32_t j = 0; j < B; ++j) {
      uint32_t idx = i * B + j;
      if (idx < m && bits[idx]) mu[j] = (uint32_t)inv;
    }
    orc_encrypt(c, mu, s, a + (size_t)i * ln, e + (size_t)i * N, query + (size_t)i * 2 * ln);
  }
  free(mu);
  free(bits);
  return 0;
}

/* Decryption: x = [c0 + c1 s (+ c2 s^2)]_Q, mu = round(t x / Q) mod t.
 * The invariant noise is w = t x - Q round(t x / Q); the budget is
 * log2(Q) - 1 - log2(max |w|) bits (decryption is correct while it is > 0). */
int orc_decrypt(const orc_ctx *c, const uint64_t *ct, uint32_t size,
                const int8_t *s, uint32_t *mu, double *budget) {
  uint32_t N = c->N;
  size_t ln = LN(c);
  if (size < 2 || size > 3) return -1;
  uint64_t *x = malloc(ln * sizeof(uint64_t)), *sm = malloc(N * sizeof(uint64_t));
  uint64_t *s2 = malloc(N * sizeof(uint64_t)), *tmp = malloc(N * sizeof(uint64_t));
  int64_t *si = malloc(N * sizeof(int64_t));
  for (uint32_t i = 0; i < N; ++i) si[i] = s[i];
  for (uint32_t j = 0; j < c->L; ++j) {
    uint64_t q = c->q[j];
    small_to_mod(c, j, si, sm);
    nega_mul(&c->qt[j], ct + ln + (size_t)j * N, sm, tmp);
    for (uint32_t i = 0; i < N; ++i)
      x[(size_t)j * N + i] = addmod(ct[(size_t)j * N + i], tmp[i], q);
    if (size == 3) {
      nega_mul(&c->qt[j], sm, sm, s2);
      nega_mul(&c->qt[j], ct + 2 * ln + (size_t)j * N, s2, tmp);
      for (uint32_t i = 0; i < N; ++i)
        x[(size_t)j * N + i] = addmod(x[(size_t)j * N + i], tmp[i], q);
    }
  }
  bu maxw;
  bu_zero(&maxw);
  for (uint32_t i = 0; i < N; ++i) {
    bu v, tx, r, prod;
    crt_reconstruct(&c->Qb, x + i, N, &v);
    bu_mul_u64(&tx, &v, c->t);
    bu_add(&r, &tx, &c->Qhalf);
    for (uint32_t j = 0; j < c->L; ++j) bu_divmod(&r, &r, c->q[j]);
    /* r = round(t x / Q) >= 0; |w| = |t x - Q r| */
    mu[i] = (uint32_t)bu_mod(&r, c->t);
    bu_mul(&prod, &r, &c->Qb.M);
    bu w;
    if (bu_cmp(&tx, &prod) >= 0) bu_sub(&w, &tx, &prod);
    else bu_sub(&w, &prod, &tx);
    if (bu_cmp(&w, &maxw) > 0) maxw = w;
  }
  if (budget) {
    double lq = bu_log2(&c->Qb.M);
    *budget = bu_is_zero(&maxw) ? lq : lq - 1.0 - bu_log2(&maxw);
  }
  free(x);
  free(sm);
  free(s2);
  free(tmp);
  free(si);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Constant-weight codes (Sec. 3.2, App. A)                            */
/* ------------------------------------------------------------------ */
static const u128 SAT = ((u128)1) << 127;

static u128 binom128(uint64_t n, uint64_t r) {
  if (r > n) return 0;
  if (r > n - r) r = n - r;
  u128 v = 1;
  for (uint64_t i = 1; i <= r; ++i) {
    /* v * (n - r + i) / i is exact: v*(n-r+i) = C(n-r+i, i) * i */
    uint64_t f = n - r + i;
    if (v > SAT / f) return SAT;
    v = v * f / i;
  }
  return v;
}

void orc_binom(uint64_t n, uint64_t r, uint64_t *lo, uint64_t *hi) {
  u128 v = binom128(n, r);
  *lo = (uint64_t)v;
  *hi = (uint64_t)(v >> 64);
}

/* Alg. Perfect Mapping: scan m' = m-1 down to 0; whenever the remainder r is
 * at least C(m', h) set bit m', subtract, and lower h; stop at h = 0. */
int orc_map_perfect(uint64_t x, uint32_t m, uint32_t k, uint16_t *pos) {
  if (k == 0 || k > m || m > 65535) return -1;
  if ((u128)x >= binom128(m, k)) return -2;
  u128 r = x;
  uint32_t h = k;
  for (int64_t mp = (int64_t)m - 1; mp >= 0 && h > 0; --mp) {
    u128 b = binom128((uint64_t)mp, h);
    if (r >= b) {
      pos[h - 1] = (uint16_t)mp; /* filled from the top: ascending order */
      r -= b;
      h -= 1;
    }
  }
  return h == 0 ? 0 : -3;
}

/* Alg. Lossy Mapping (App. A).  The hash family: H_i(x) is the i-th output
 * of a SplitMix64 generator seeded with x, reduced mod m.  SplitMix64 keeps
 * a 64-bit state that advances by the odd constant 0x9E3779B97F4A7C15 and
 * returns the state passed through a xor-shift-multiply mixer. */
static uint64_t orc_splitmix_next(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int orc_map_lossy(uint64_t x, uint32_t m, uint32_t k, uint16_t *pos) {
  if (k == 0 || k > m || m > 65535) return -1;
  unsigned char *y = calloc(m, 1); /* the codeword y = 0^m */
  uint64_t state = x;
  uint32_t cnt = 0;
  for (uint64_t draws = 0; cnt < k && draws < 64ull * m + 1024; ++draws) {
    uint32_t mp = (uint32_t)(orc_splitmix_next(&state) % m); /* m' = H_i(x) */
    if (y[mp] == 0) {
      y[mp] = 1;
      cnt += 1;
    }
  }
  uint32_t h = 0;
  for (uint32_t i = 0; i < m && cnt == k; ++i)
    if (y[i]) pos[h++] = (uint16_t)i;
  free(y);
  return cnt == k ? 0 : -2;
}

/* Alg. Inverse Perfect Mapping: x = sum over ascending one-positions m' of
 * C(m', h) with h = 1, 2, ... */
int orc_map_inverse(const uint16_t *pos, uint32_t k, uint64_t *x) {
  u128 v = 0;
  for (uint32_t h = 1; h <= k; ++h) {
    if (h > 1 && pos[h - 1] <= pos[h - 2]) return -1;
    v += binom128(pos[h - 1], h);
  }
  if (v >> 64) return -2;
  *x = (uint64_t)v;
  return 0;
}

uint64_t orc_code_length(uint32_t bits, uint32_t k, uint64_t limit) {
  if (bits > 64 || k == 0) return 0;
  u128 need = ((u128)1) << bits;
  for (uint64_t m = k; m <= limit; ++m)
    if (binom128(m, k) >= need) return m;
  return 0;
}
