// kernels.cuh -- device data structures and kernel entry points of the
// constant-weight PIR answer path (arXiv 2202.07569, Sec. 3.3.3).
#pragma once
#include <cuda_runtime.h>

#include "arith.cuh"

namespace cw {

// 32-bit NTT data of a 30-bit extension prime, in device memory.
struct ExtNtt {
  ExtPrime e;
  const u32 *psi2;   // [N][2]: psi^bitrev(i) and floor(psi^bitrev(i) 2^32 / p)
  const u32 *ipsi2;  // [N][2]: the same for psi^-1
};

// Row-sum waves: the row sums of the last tree level are split into row
// groups until about this many waves of resident threads cover the device.
constexpr u32 kDefaultRowWaves = 2;

// All per-context constants the kernels read, in device memory.  sms,
// sm_threads (read from the device at setup) and row_waves size launch
// grids on the host.
struct DevTables {
  u32 N, logN, L, K;
  u32 sms, sm_threads, row_waves;
  u64 t;
  u64 delta[kMaxL];       // Delta = floor(Q / t) mod q_j
  NttPrime prime[kMaxL];  // ciphertext primes q_0..q_{L-1}
  ExtNtt ext[kMaxK];      // extension primes p_0..p_{K-1} (30-bit)
  LiftTab lift;           // centered Q -> P conversion (leaves, nodes)
  ScaleTab scale;         // exact round(t d / Q) from residues modulo Q and P
  ScaleTabP scalep;       // round(t d / Q) from residues modulo P alone
  RowTab rows;            // row basis: first nr extension primes -> Q
  RowTab ksr;             // key-switch basis: first five extension primes -> Q
};

// Primes of the key-switch basis (the first kKsrPrimes extension primes).
constexpr u32 kKsrPrimes = 5;

// QP layout of one polynomial (NTT domain or, for the tensor buffer,
// coefficients): L limbs of N u64 residues mod q_j, then K limbs of N u32
// residues mod the 30-bit p_k; L N + K N / 2 u64 words in all.
CW_HD u64 qp_poly_words(u32 L, u32 K, u32 N) { return (u64)L * N + (u64)K * N / 2; }
// The tensor buffer: per job three polynomials (N d0, N d1, N d2) of K
// limbs of N u32 residues modulo the extension primes, K N / 2 u64 words
// each.
CW_HD u64 tensor_poly_words(u32 K, u32 N) { return (u64)K * N / 2; }
CW_HD u32 *ext_limb(u64 *poly, u32 L, u32 N, u32 k) {
  return reinterpret_cast<u32 *>(poly + (u64)L * N) + (u64)k * N;
}
CW_HD const u32 *ext_limb(const u64 *poly, u32 L, u32 N, u32 k) {
  return reinterpret_cast<const u32 *>(poly + (u64)L * N) + (u64)k * N;
}

// One homomorphic multiplication of two ciphertexts held in "QP-NTT" form:
// two polynomials in QP layout, NTT domain.
struct MulJob {
  const u64 *a;
  const u64 *b;
  u64 *dst;   // internal node: QP-NTT destination; root: output slot (SEL)
  u64 row;    // root: database row
};

// Substitution job: source ciphertext [2][L][N] coefficient form.
struct SubJob {
  const u64 *src;
  u64 *dst;   // [2][L][N] coefficient form result
};

enum RootMode : int {
  ROOT_PM = 0,    // sel * DB[row] -> partial products
  ROOT_SEL = 1,   // sel in coefficient form -> dst ([2][L][N])
  INTERNAL = 2    // sel -> the extension limbs of a QP-NTT ciphertext at dst
};


// ---- launchers (kernels.cu); all enqueue on `st` and return the launch
// error.  Buffers are described in kernels.cu next to each kernel. ----
// rows of plen payload coefficients, sp = ceil(plen / N) plaintexts each,
// into db [rows][sp][L][N] (NTT form).
cudaError_t launch_db_load(const DevTables *T, const DevTables &h, const u32 *items,
                           u64 rows, u32 plen, u32 sp, u64 *db, cudaStream_t st);
cudaError_t launch_ntt(const DevTables *T, const DevTables &h, u64 *base, u32 units,
                       u64 unit_stride, u32 limb_begin, u32 limb_end, bool inverse,
                       const u64 *src, u64 src_unit_stride, cudaStream_t st);
cudaError_t launch_lift(const DevTables *T, const DevTables &h, const u64 *src,
                        u64 src_stride, u64 *dst, u64 dst_stride, u32 units,
                        bool copy_q, cudaStream_t st);
cudaError_t launch_lift_jobs(const DevTables *T, const DevTables &h, const u64 *C,
                             const MulJob *jobs, u32 njobs, cudaStream_t st);
cudaError_t launch_ntt_jobs_p(const DevTables *T, const DevTables &h, const MulJob *jobs,
                              u32 njobs, cudaStream_t st);
cudaError_t launch_tensor(const DevTables *T, const DevTables &h, const MulJob *jobs,
                               u32 njobs, u64 *Tbuf, cudaStream_t st);
cudaError_t launch_scale(const DevTables *T, const DevTables &h, const u64 *Tbuf, u32 njobs,
                         u64 *E, int *err, cudaStream_t st);
// Relinearisation of the scaled tensor E with its consumer.  DN: scratch
// [njobs][L+2][L][N].  mode ROOT_PM: the jobs form `segs` equal segments
// (one per query), database rows hold sp plaintexts ([rows][sp][L][N]);
// out = partials [segs * G][sp][2][L][N] with
// G = relin_pm_groups(h, segs, njobs / segs, sp, cap) <= cap / (segs sp)
// (sums of sel * DB over row groups); with sp > 1, S is scratch
// [njobs][2][L][N] for the NTT-form selection entries.  INTERNAL: NTT-form
// Q limbs to jobs[].dst and coefficient form to out ([njobs][2][L][N]);
// ROOT_SEL: coefficient form to jobs[].dst, out is scratch [njobs][2][L][N].
cudaError_t launch_relin(const DevTables *T, const DevTables &h, const u64 *E, u32 njobs,
                         u32 segs, const MulJob *jobs, int mode, const u64 *rlk,
                         const u64 *rlk_s, const u64 *db, u32 sp, u32 cap, u64 *DN, u64 *S,
                         u64 *out, cudaStream_t st);
u32 relin_pm_groups(const DevTables &h, u32 segs, u32 seg_len, u32 sp, u32 cap);

// ---- row basis (RowTab): databases of one plaintext per row held as
// [rows][nr][N] u32, NTT form modulo the first nr extension primes ----
u32 relin_rows_groups(const DevTables &h, u32 segs, u32 seg_len, u32 gcap);
cudaError_t launch_db_load_rows(const DevTables *T, const DevTables &h, const u32 *items,
                                u64 rows, u32 plen, u32 *dbr, cudaStream_t st);
// The row transforms of the scaled tensor E ([njobs][3][L][N]): the limbs
// of e0, e1 and the digits of e2 (the limbs of e2) reduced modulo each row
// prime and transformed, D = [njobs][3L][nr][N] u32 (NTT form).
cudaError_t launch_rows_transforms(const DevTables *T, const DevTables &h, const u64 *E,
                                   u32 njobs, u32 *D, cudaStream_t st);
// Relinearisation of the scaled tensor with the plain multiplication by the
// rows of a row-basis database, summed over row groups, from its row
// transforms D (launch_rows_transforms of the same jobs): the transforms
// are multiplied with the rows exactly in the row basis, summed, brought
// back to the ciphertext primes and multiplied by the key once per group.
// The jobs form `segs` segments (one per query); out = partials
// [segs * G][2][L][N], NTT form, G = relin_rows_groups(h, segs, njobs /
// segs, gcap) <= gcap.  Scratch: S [gcap][3L][nr][N] u32; DNQ
// [gcap][L+2][L][N].  E is not read.
cudaError_t launch_relin_rows(const DevTables *T, const DevTables &h, const u64 *E, u32 njobs,
                              u32 segs, const MulJob *jobs, const u64 *rlk, const u64 *rlk_s,
                              const u32 *dbr, u32 gcap, u32 *D, u32 *S, u64 *DNQ, int *err,
                              u64 *out, cudaStream_t st);
// Plain multiplication of ct ([2][L][N] coefficient form) by row `row` of a
// row-basis database: out [2][L][N] coefficient form.  D: [2L][nr][N] u32,
// S: [2L][nr][N] u32; job: one device MulJob whose row is read.
cudaError_t launch_plain_mul_rows(const DevTables *T, const DevTables &h, const u64 *ct,
                                  const MulJob *job, const u32 *dbr, u32 *D, u32 *S, int *err,
                                  u64 *out, cudaStream_t st);
// Key switching of the internal tree nodes through the key-switch basis
// (RowTab ksr): the digits of e2 (its limbs, integers below q_i) and the
// switching key (integers below q_j) multiply exactly as integer
// polynomials modulo five 30-bit primes, |sum_i D_i * key_ij| < L N q^2 <
// 2^125 < R/2, and the sums come back to each q_j by an exact CRT.  The
// result C[job][2][L][N] = (e0 + sum_i D_i b_i, e1 + sum_i D_i a_i) mod q_j
// is in coefficient form.  ks: the key in the basis ([L][2][L][5][N] u32,
// NTT form); D: scratch [njobs][L][5][N] u32; O: scratch
// [njobs][2L][5][N] u32.
cudaError_t launch_relin_ksr(const DevTables *T, const DevTables &h, const u64 *E, u32 njobs,
                             const u32 *ks, u32 *D, u32 *O, int *err, u64 *C, cudaStream_t st);
// The switching key [L][2][L][N] (coefficient form, residues below q_j)
// into the key-switch basis: ks [L][2][L][5][N] u32, NTT form.
cudaError_t launch_ksr_key(const DevTables *T, const DevTables &h, const u64 *key, u32 *ks,
                           cudaStream_t st);
// k = 1: P[job][sp][2][L][N] = leaf * DB[row][p].
cudaError_t launch_pm_leaf(const DevTables *T, const DevTables &h, const MulJob *jobs,
                           u32 njobs, u32 sp, const u64 *db, u64 *P, cudaStream_t st);
// acc[s] += sum of P[s * per_seg .. (s+1) * per_seg) for s < segs; each
// entry is [sp][2][L][N].
cudaError_t launch_accumulate(const DevTables &h, const DevTables *T, const u64 *P, u32 segs,
                              u32 per_seg, u32 sp, u64 *acc, cudaStream_t st);
cudaError_t launch_automorph(const DevTables *T, const DevTables &h, const SubJob *jobs,
                             u32 njobs, u32 g, u64 *tau, cudaStream_t st);
// Sub_g key switch: tau [njobs][2][L][N] (automorphism images) ->
// sjobs[].dst = (tau0 + u0, u1) in coefficient form.  DN: scratch
// [njobs][L+1][L][N]; O: scratch [njobs][2][L][N].
cudaError_t launch_sub_keyswitch(const DevTables *T, const DevTables &h, const u64 *tau,
                                 u32 njobs, const SubJob *jobs, const u64 *key,
                                 const u64 *key_s, u64 *DN, u64 *O, cudaStream_t st);
cudaError_t launch_expand_combine(const DevTables *T, const DevTables &h, const u64 *cur,
                                  const u64 *S, u64 *next, u32 h_in, u32 cfac, u32 a,
                                  cudaStream_t st);
cudaError_t launch_pm_ntt(const DevTables *T, const DevTables &h, const u64 *ct_ntt,
                          const u64 *db_row, u64 *out, cudaStream_t st);
// Folklore leaves (Eq. folklore-plain-eq): query [nq][ell] bit ciphertexts
// x[i] -> out [nq][2 ell] = (1 - x[0], x[0], 1 - x[1], x[1], ...) with
// 1 - x = (Delta - c0, -c1), coefficient form.
cudaError_t launch_folklore_leaves(const DevTables *T, const DevTables &h, const u64 *query,
                                   u32 count, u64 *out, cudaStream_t st);
// Element-wise ciphertext steps of the arithmetic operator (coefficient
// form [2][L][N]): out = sum of `count` ciphertexts in[x * in_stride]
// (residues below q_j; also the sum of a sharded database's partial
// responses); out[f] = in minus the constant plaintext f (Delta f off c0 at
// x^0), f < count; out = s * in.
cudaError_t launch_ct_sum(const DevTables *T, const DevTables &h, const u64 *in, u32 count,
                          u64 in_stride, u64 *out, cudaStream_t st);
// out[x] = in[x] mod q_j for `count` ciphertexts [2][L][N] of u64 values
// (sums of residues below 2^64).
cudaError_t launch_ct_reduce(const DevTables *T, const DevTables &h, const u64 *in, u32 count,
                             u64 *out, cudaStream_t st);
cudaError_t launch_minus_consts(const DevTables *T, const DevTables &h, const u64 *in,
                                u32 count, u64 *out, cudaStream_t st);
// *flag |= 1 if a residue of ct [count][2][L][N] is not below its q_j (the
// flag is not cleared here).
cudaError_t launch_check_residues(const DevTables *T, const DevTables &h, const u64 *ct,
                                  u64 count, int *flag, cudaStream_t st);
cudaError_t launch_ct_scalar(const DevTables *T, const DevTables &h, const u64 *in, u64 s,
                             u64 *out, cudaStream_t st);
cudaError_t launch_key_prep(const DevTables *T, const DevTables &h, u64 *key, u64 *key_s,
                            u32 nkeys, cudaStream_t st);

}  // namespace cw
