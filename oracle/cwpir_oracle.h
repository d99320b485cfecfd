/*
 * cwpir_oracle.h -- plain, slow CPU oracle for the constant-weight PIR server
 * answer path (Mahdavi & Kerschbaum, "Constant-weight PIR", arXiv 2202.07569).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product library
 * (paper_2202_07569_gb300) never includes, links or calls it, and this file
 * shares no code with it.
 *
 * Arithmetic is exact: every value is an integer residue or a big integer.
 * Each function follows the definition it cites, step by step; the only
 * library-style primitive is a negacyclic NTT (written here) used to form
 * exact ring products.
 *
 * Layouts (all little-endian u64 residues, coefficient form):
 *   poly         [L][N]            limb j holds residues mod q_j
 *   ciphertext   [2][L][N]         (c0, c1): decrypts as c0 + c1*s
 *   size-3 ct    [3][L][N]         decrypts as c0 + c1*s + c2*s^2
 *   switch key   [L][2][L][N]      digit i, component (0 = b_i, 1 = a_i), limb j
 *   galois keys  [c][L][2][L][N]   key for element N/2^a + 1 at index a
 * Secret s: int8 [N] in {-1,0,1}; errors: int32 [N]; plaintexts: u32 [N] < t.
 *
 * Return codes: 0 ok, negative on invalid arguments.
 */
#ifndef CWPIR_ORACLE_H
#define CWPIR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_ctx orc_ctx;

/* Deterministic Miller-Rabin for 64-bit integers. */
int orc_is_prime(uint64_t p);
/* The `count` largest primes p < 2^bits with p = 1 (mod 2N), descending. */
int orc_primes(uint32_t N, uint32_t count, uint32_t bits, uint64_t *out);

orc_ctx *orc_create(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t);
void orc_destroy(orc_ctx *ctx);
/* Number of auxiliary primes used to form exact integer products. */
uint32_t orc_aux_count(const orc_ctx *ctx);

/* Negacyclic product mod p of two [N] vectors through the oracle's NTT. */
int orc_negacyclic_mul_mod(uint32_t N, uint64_t p, const uint64_t *a,
                           const uint64_t *b, uint64_t *out);

/* Exact integer negacyclic product of the centered lifts of two R_Q
 * polynomials a, b ([L][N] residues).  Coefficient i is returned as
 * sign[i] (0 or 1 = negative) and magnitude mag[i*words .. +words). */
int orc_exact_product(const orc_ctx *ctx, const uint64_t *a, const uint64_t *b,
                      uint32_t words, int32_t *sign, uint64_t *mag);
/* round(t*d/Q) mod q_j for one signed big integer d (magnitude in `words`
 * little-endian u64 words); writes L residues. */
int orc_scale_round(const orc_ctx *ctx, int32_t sign, const uint64_t *mag,
                    uint32_t words, uint64_t *out);

/* BFV tensor with exact scale-down (no relinearisation): [3][L][N]. */
int orc_tensor(const orc_ctx *ctx, const uint64_t *a, const uint64_t *b,
               uint64_t *out3);
/* Key switch of z ([L][N]) with an RNS-digit key: ([2][L][N]). */
int orc_keyswitch(const orc_ctx *ctx, const uint64_t *z, const uint64_t *key,
                  uint64_t *out);
/* Homomorphic multiplication M: tensor, scale-down, relinearisation. */
int orc_bfv_mul(const orc_ctx *ctx, const uint64_t *a, const uint64_t *b,
                const uint64_t *rlk, uint64_t *out);
/* Automorphism x -> x^g on every limb of one [L][N] polynomial (g odd). */
int orc_automorphism(const orc_ctx *ctx, uint32_t g, const uint64_t *in,
                     uint64_t *out);
/* Multiply one [L][N] polynomial by the monomial x^e, e in (-2N, 2N). */
int orc_monomial(const orc_ctx *ctx, int64_t e, const uint64_t *in,
                 uint64_t *out);
/* Substitution Sub_g: automorphism plus key switch with the Galois key. */
int orc_substitute(const orc_ctx *ctx, uint32_t g, const uint64_t *ct,
                   const uint64_t *gkey, uint64_t *out);
/* Query expansion (modified algorithm): h cts -> the first m expanded cts. */
int orc_expand(const orc_ctx *ctx, uint32_t h, const uint64_t *query,
               uint32_t c, uint32_t m, const uint64_t *gkeys, uint64_t *out);
/* SealPIR expansion loop (two substitutions per inner step) on one ct,
 * without the final 2^-c scaling: writes 2^c cts. */
int orc_expand_sealpir(const orc_ctx *ctx, const uint64_t *ct, uint32_t c,
                       const uint64_t *gkeys, uint64_t *out);
/* Multiply a ciphertext by an integer scalar in [0, t). */
int orc_scalar_mul(const orc_ctx *ctx, const uint64_t *ct, uint64_t scalar,
                   uint64_t *out);
/* (Delta - c0, -c1): the constant plaintext 1 minus ct (decrypts to 1 - mu). */
int orc_one_minus(const orc_ctx *ctx, const uint64_t *ct, uint64_t *out);
/* Positions 2i + y[i], i < ell, of the plain folklore operator's factors
 * among the leaves (1 - x[0], x[0], 1 - x[1], x[1], ...). */
int orc_folklore_codeword(uint64_t y, uint32_t ell, uint16_t *pos);
/* Plain multiplication by an item plaintext (payload_len coefficients < t,
 * zero-padded, centered lift). */
int orc_plain_mul(const orc_ctx *ctx, const uint64_t *ct, const uint32_t *mu,
                  uint32_t payload_len, uint64_t *out);
/* Selection-vector entry for one item: product of ctxts at `positions`
 * (k ascending) by the balanced pairwise tree. */
int orc_selection(const orc_ctx *ctx, const uint64_t *ctxts,
                  const uint16_t *positions, uint32_t k, const uint64_t *rlk,
                  uint64_t *out);
/* Alg. Arithmetic Constant-weight Equality Operator on encrypted
 * operands x, y ([m][2][L][N] each): (1/k!) prod_{i<k} (sum_j x_j y_j - i). */
int orc_arith_cw_eq(const orc_ctx *ctx, uint32_t m, uint32_t k, const uint64_t *x,
                    const uint64_t *y, const uint64_t *rlk, uint64_t *out);
/* SIMD batch encoding: slot i = mu(psi^(2i+1)) mod t, psi = 3^((t-1)/2N). */
int orc_batch_encode(const orc_ctx *ctx, const uint32_t *slots, uint32_t *mu);
int orc_batch_decode(const orc_ctx *ctx, const uint32_t *mu, uint32_t *slots);
/* Full server answer: expansion (c > 0), selection vector, inner product.
 * query: [h][2][L][N] with h = m when c = 0, else ceil(m / 2^c).
 * items: [n][payload_len]; a row is s = ceil(payload_len / N) plaintexts
 * (Sec. 3.3.1), plaintext p holding coefficients p*N .. p*N + N - 1, and the
 * answer is s inner products with the same selection vector (Sec. 3.3.3):
 * resp [s][2][L][N].  codewords: [n][k] ascending positions < m.
 * gkeys may be NULL when c = 0.  nthreads <= 0 uses the OpenMP default. */
#define ORC_MAX_PLAINTEXTS 256
int orc_answer(const orc_ctx *ctx, uint64_t n, uint32_t payload_len,
               const uint32_t *items, const uint16_t *codewords, uint32_t k,
               uint32_t m, uint32_t c, const uint64_t *query,
               const uint64_t *rlk, const uint64_t *gkeys, int nthreads,
               uint64_t *resp);

/* ---- client side (key generation, query, extract) ---- */
/* Switching key for the secret w*s-image: digit i component b_i =
 * -a_i*s + e_i + g_i*w, a_i uniform ([L][L][N]), e_i ([L][N]).
 * orc_keygen_relin uses w = s^2; orc_keygen_galois uses w = s(x^g). */
int orc_keygen_relin(const orc_ctx *ctx, const int8_t *s, const uint64_t *a,
                     const int32_t *e, uint64_t *key);
int orc_keygen_galois(const orc_ctx *ctx, uint32_t g, const int8_t *s,
                      const uint64_t *a, const int32_t *e, uint64_t *key);
/* Secret-key encryption of mu ([N] < t): ([Delta*mu - a*s + e]_Q, a). */
int orc_encrypt(const orc_ctx *ctx, const uint32_t *mu, const int8_t *s,
                const uint64_t *a, const int32_t *e, uint64_t *ct);
/* Query construction: the k positions of E_q, packed 2^c bits per
 * plaintext with the 2^-c pre-scale; a: [h][L][N], e: [h][N]. */
int orc_make_query(const orc_ctx *ctx, const uint16_t *positions, uint32_t k,
                   uint32_t m, uint32_t c, const int8_t *s, const uint64_t *a,
                   const int32_t *e, uint64_t *query);
/* Decryption of a size-2 (size=2) or size-3 (size=3) ciphertext.  Writes mu
 * ([N] < t) and, if budget != NULL, the invariant noise budget in bits. */
int orc_decrypt(const orc_ctx *ctx, const uint64_t *ct, uint32_t size,
                const int8_t *s, uint32_t *mu, double *budget);

/* ---- constant-weight codes ---- */
/* Binomial coefficient, saturating at 2^127. */
void orc_binom(uint64_t n, uint64_t r, uint64_t *lo, uint64_t *hi);
/* Perfect mapping x -> CW(m,k); writes the k one-positions ascending. */
int orc_map_perfect(uint64_t x, uint32_t m, uint32_t k, uint16_t *pos);
/* Alg. Lossy Mapping (App. A) with H_i(x) = i-th SplitMix64 output of
 * seed x, mod m; ascending positions. */
int orc_map_lossy(uint64_t x, uint32_t m, uint32_t k, uint16_t *pos);
/* Inverse perfect mapping of k ascending positions. */
int orc_map_inverse(const uint16_t *pos, uint32_t k, uint64_t *x);
/* Smallest m with C(m,k) >= 2^bits (bits <= 64), or 0 if m > limit. */
uint64_t orc_code_length(uint32_t bits, uint32_t k, uint64_t limit);

#ifdef __cplusplus
}
#endif
#endif
