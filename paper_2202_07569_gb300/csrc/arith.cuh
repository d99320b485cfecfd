// arith.cuh -- word-size modular arithmetic and per-coefficient RNS steps of
// the BFV multiplication (FV scheme, arXiv 2202.07569 Sec. 2.1.1), written
// for the 32-bit integer pipes of sm_103a.  Every function is exact.
//
// Ciphertext residues are u64 values below primes q < 2^54; the extension
// basis of the tensor product uses 30-bit primes held in 32-bit words.  The
// functions are __host__ __device__ so that the same arithmetic can be
// exercised on the CPU by the test suite.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define CW_HD __host__ __device__ __forceinline__
#define CW_HDM __host__ __device__ __forceinline__
#else
#define CW_HD static inline
#define CW_HDM inline
#endif

namespace cw {

typedef uint64_t u64;
typedef uint32_t u32;

constexpr int kMaxL = 8;       // ciphertext primes
constexpr int kMaxK = 30;      // extension primes (30-bit)

// Extension primes used with L ciphertext primes: the smallest count of
// 30-bit primes (each above 2^29.98) whose product P is at least 2 N Q^2
// for 54-bit q_j and N <= 2^14.  The tensor of two centered lifts
// (|d| <= N Q^2 / 2) then lies within P/4 of zero, so the extension basis
// alone holds it exactly; P >= 2^17 t N Q (t < 2^20) follows as well, the
// bound of the exact scale-down scale_coeff.
CW_HD constexpr int ext_count(int L) {
  return L <= 1 ? 5 : L == 2 ? 8 : L == 3 ? 12 : L == 4 ? 15 : L == 5 ? 19 : L == 6 ? 23
       : L == 7 ? 26 : 30;
}

CW_HD u64 mulhi(u64 a, u64 b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (u64)(((unsigned __int128)a * b) >> 64);
#endif
}
CW_HD u32 mulhi32(u32 a, u32 b) {
#if defined(__CUDA_ARCH__)
  return __umulhi(a, b);
#else
  return (u32)(((u64)a * b) >> 32);
#endif
}

// v - m if v >= m, else v (m <= 2^31): the unsigned minimum of v and
// v - m, since v - m wraps above v exactly when v < m (one IADD and one
// IMNMX instead of a compare, a subtraction and a select).
CW_HD u32 csub32(u32 v, u32 m) {
#if defined(__CUDA_ARCH__)
  return umin(v, v - m);
#else
  return v >= m ? v - m : v;
#endif
}

CW_HD u64 addq(u64 a, u64 b, u64 q) {
  u64 s = a + b;
  return s >= q ? s - q : s;
}
CW_HD u64 subq(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// Shoup multiplication by a constant w < q with ws = floor(w * 2^64 / q):
// for any a < 2^64, a*w - mulhi(a, ws)*q lies in [0, 2q).  Result < q.
CW_HD u64 shoup(u64 a, u64 w, u64 ws, u64 q) {
  u64 r = a * w - mulhi(a, ws) * q;
  return r >= q ? r - q : r;
}

// Barrett multiplication of two variables a, b < 2q (product < 2^110) for a
// prime 2^53 < q < 2^54 with mu = floor(2^116 / q) < 2^63.
// With x = a*b, x1 = floor(x / 2^52), qh = floor(x1 * mu / 2^64):
//   qh <= x/q  and  qh > x/q - x/2^116 - 2^52/q - 1 > x/q - 2,
// so r = x - qh*q is in [0, 2q) and one subtraction finishes it.
CW_HD u64 barrett(u64 a, u64 b, u64 q, u64 mu) {
  u64 lo = a * b, hi = mulhi(a, b);
  u64 x1 = (hi << 12) | (lo >> 52);
  u64 qh = mulhi(x1, mu);
  u64 r = lo - qh * q;
  return r >= q ? r - q : r;
}

// Reduction of X = hi 2^64 + lo < 2^112 modulo a prime 2^53 < q < 2^54
// with mu = floor(2^116 / q): x1 = floor(X / 2^52) < 2^60 and
// qh = floor(x1 mu / 2^64) > X/q - X/2^116 - 2^52/q - 1 > X/q - 1.57, so
// X - qh q lies in [0, 2q).
CW_HD u64 barrett_reduce(u64 hi, u64 lo, u64 q, u64 mu) {
  u64 x1 = (hi << 12) | (lo >> 52);
  u64 qh = mulhi(x1, mu);
  u64 r = lo - qh * q;
  return r >= q ? r - q : r;
}

// 128-bit accumulator of exact products of residues (< 2^108 each); at most
// 16 terms keep the sum below 2^112.
struct Acc128 {
  u64 hi = 0, lo = 0;
  CW_HDM void mac(u64 a, u64 b) {
    u64 p = a * b;
    u64 h = mulhi(a, b);
    lo += p;
    hi += h + (lo < p ? 1 : 0);
  }
  CW_HDM void add(u64 a) {
    lo += a;
    hi += lo < a ? 1 : 0;
  }
};

// Full 64-bit product of two 32-bit words: one wide multiply-add on the
// integer pipe, where a product of u64 operands would take three.  The
// callers narrow to u32 only values they know to be below 2^32.
CW_HD u64 wmul(u32 a, u32 b) { return (u64)a * b; }

// 27-bit halves of a constant b < 2^54: b = out[1] 2^27 + out[0].
constexpr u32 kMask27 = (1u << 27) - 1;
// the halves of a residue below 2^54
CW_HD u32 lo27(u64 y) { return (u32)y & kMask27; }
CW_HD u32 hi27(u64 y) { return (u32)(y >> 27); }
CW_HD void split27(u64 b, u32 *out) {
  out[0] = (u32)b & kMask27;
  out[1] = (u32)(b >> 27);
}

// ---------------------------------------------------------------------
// NTT butterflies (negacyclic, psi = primitive 2N-th root of unity).
// Twiddles are stored as (value, Shoup companion) pairs.
// Forward: Cooley-Tukey with the powers of psi in bit-reversed order,
// natural-order input, bit-reversed output.  Inverse: Gentleman-Sande with
// the powers of psi^-1, bit-reversed input, natural output, then * N^-1.
// Stage s of the forward transform has m = 2^s groups of half-length
// len = N / 2^(s+1); butterfly b (< N/2) is in group b / len.
// ---------------------------------------------------------------------
CW_HD void fwd_bfly(u64 *a, u32 b, u32 logh, u32 m, const u64 *psi2, u64 q) {
  u32 len = 1u << logh, g = b >> logh, pos = b & (len - 1);
  u32 j = (g << (logh + 1)) + pos;
  u64 U = a[j];
  u64 V = shoup(a[j + len], psi2[2 * (m + g)], psi2[2 * (m + g) + 1], q);
  a[j] = addq(U, V, q);
  a[j + len] = subq(U, V, q);
}
CW_HD void inv_bfly(u64 *a, u32 b, u32 logh, u32 m, const u64 *ipsi2, u64 q) {
  u32 len = 1u << logh, g = b >> logh, pos = b & (len - 1);
  u32 j = (g << (logh + 1)) + pos;
  u64 U = a[j], V = a[j + len];
  a[j] = addq(U, V, q);
  a[j + len] = shoup(subq(U, V, q), ipsi2[2 * (m + g)], ipsi2[2 * (m + g) + 1], q);
}

// Per-prime NTT data of a ciphertext prime, in device memory.
struct NttPrime {
  u64 q, mu;          // prime, Barrett constant floor(2^116/q)
  u64 ninv, ninv_s;   // N^-1 mod q and Shoup companion
  const u64 *psi2;    // [N][2]: psi^bitrev(i) and its Shoup companion
  const u64 *ipsi2;   // [N][2]: psi^-bitrev(i) and its Shoup companion
};

// ---------------------------------------------------------------------
// 30-bit extension primes 2^29 < p < 2^30 in 32-bit words.
// ---------------------------------------------------------------------
struct ExtPrime {
  u32 p;
  u32 mu60;   // floor(2^60 / p), in (2^30, 2^31)
  u64 mu64;   // floor(2^64 / p)
  u32 c32;    // 2^32 mod p
  u32 mu61;   // floor(2^61 / p), in (2^31, 2^32)
};

// v mod p for any v < 2^64: qh = floor(v mu64 / 2^64) lies in
// (v/p - v/2^64 - 1, v/p], so v - qh p is in [0, 2p).
CW_HD u32 reduce_ext(u64 v, const ExtPrime &E) {
  return csub32((u32)(v - mulhi(v, E.mu64) * E.p), E.p);
}

// v mod p for v < 2^62, on 32-bit words (the row transforms' loads; in the
// scale-down's register-heavy sums reduce_ext measured faster): the high
// word folds back,
// x = (v >> 32) (2^32 mod p) + (v mod 2^32) < 2^60 + 2^32, then with
// x1 = floor(x / 2^29) < 2^32, qh = floor(x1 mu61 / 2^32) satisfies
// x/p - x/2^61 - 2^29/p < qh <= x/p, i.e. x/p - 1.51 < qh, so
// r = x - qh p is in [0, 3p) (the low word suffices) and two subtractions
// finish it.
// The same reduction left lazy in [0, 3p) (below 2^32): the input of a
// forward 32-bit transform, which accepts values below 4p.
CW_HD u32 reduce_ext62_lazy(u64 v, const ExtPrime &E) {
  const u64 x = (u64)(u32)(v >> 32) * E.c32 + (u32)v;
  return (u32)x - mulhi32((u32)(x >> 29), E.mu61) * E.p;
}
CW_HD u32 reduce_ext62(u64 v, const ExtPrime &E) {
  const u64 x = (u64)(u32)(v >> 32) * E.c32 + (u32)v;
  const u32 qh = mulhi32((u32)(x >> 29), E.mu61);
  return csub32(csub32((u32)x - qh * E.p, 2 * E.p), E.p);
}

// a b mod p in [0, 2p) for a, b < p (Barrett on 32-bit words): with
// x = a b < 2^60 and x1 = floor(x / 2^28) < 2^32, qh = floor(x1 mu60 / 2^32)
// satisfies x/p - 1.5 < qh <= x/p, so r = x - qh p is in [0, 3p) (below
// 2^32: the low word suffices) and one subtraction of 2p brings it below 2p.
CW_HD u32 mulmod_ext_lazy(u32 a, u32 b, const ExtPrime &E) {
  const u64 x = (u64)a * b;
  const u32 qh = mulhi32((u32)(x >> 28), E.mu60);
  return csub32((u32)x - qh * E.p, 2 * E.p);
}

// ---------------------------------------------------------------------
// Exact centered conversion out of the ciphertext basis Q = q_0 ... q_{L-1}.
//
// x is given by its residues x_j.  With y_j = [x_j (Q/q_j)^-1]_{q_j},
// sum_j y_j (Q/q_j) = x + v Q with v = floor(sum_j y_j / q_j), and the
// centered representative of x is x_c = sum_j y_j (Q/q_j) - rho Q with
// rho = round(sum_j y_j / q_j) (Q is odd, so the sum is never a half
// integer).
//
// rho is read from a 64.64 fixed-point sum of phi_j <= y_j 2^64 / q_j,
// each low by less than 2 units, so the sum is low by less than 2L units:
// rho = hi(2^63 + sum phi) unless the low word is within 2L of 2^64; in
// that case x is within 2L Q/2^64 of Q/2 and the exact comparison of x
// with (Q-1)/2 in mixed radix (Garner) decides.
// ---------------------------------------------------------------------
struct QConv {
  u64 q[kMaxL];
  u64 mu[kMaxL];                      // floor(2^116 / q_j)
  u64 theta[kMaxL], theta_s[kMaxL];   // (Q/q_j)^-1 mod q_j
  u64 w_hi[kMaxL], w_lo[kMaxL];       // floor(2^128 / q_j)
  u64 mrinv[kMaxL][kMaxL], mrinv_s[kMaxL][kMaxL];  // q_i^-1 mod q_j, i < j
  u64 half_mr[kMaxL];                 // mixed-radix digits of (Q-1)/2
};

// 1 if x > (Q-1)/2, by exact mixed-radix comparison (x_j < q_j).
template <int L>
CW_HD u64 mr_greater_half(const u64 *x, const QConv &C) {
  u64 a[L];
  for (int j = 0; j < L; ++j) {
    u64 qj = C.q[j], v = x[j];
    for (int i = 0; i < j; ++i) {
      u64 ai = a[i] >= qj ? a[i] - qj : a[i];
      v = shoup(subq(v, ai, qj), C.mrinv[i][j], C.mrinv_s[i][j], qj);
    }
    a[j] = v;
  }
  for (int j = L - 1; j >= 0; --j)
    if (a[j] != C.half_mr[j]) return a[j] > C.half_mr[j] ? 1 : 0;
  return 0;  // equal: x = (Q-1)/2 is not greater
}

// hi(2^63 + sum_j phi_j) with phi_j = y_j w_j / 2^64 and w_j = floor(2^128 /
// s_j) (y_j < s_j), and whether the low word is in the ambiguous zone.
template <int NS>
CW_HD u64 round_sum(const u64 *y, const u64 *w_hi, const u64 *w_lo, bool *ambiguous) {
  u64 lo = 0x8000000000000000ull, hi = 0;
  for (int j = 0; j < NS; ++j) {
    u64 phi = y[j] * w_hi[j] + mulhi(y[j], w_lo[j]);
    lo += phi;
    hi += (lo < phi) ? 1 : 0;
  }
  *ambiguous = lo > ~0ull - 2ull * NS;
  return hi;
}

// Centered conversion Q -> extension primes of one coefficient:
// out_k = [sum_j y_j (Q/q_j) - rho Q]_{p_k}.  Each y_j < 2^54 is split into
// 27-bit halves, y_j = yh 2^27 + yl, so every product of a half with a
// 30-bit constant is below 2^57 and the 2L products plus rho (-Q mod p_k)
// sum below 2^62 in one 64-bit word, reduced once.
struct LiftTab {
  QConv Q;
  ExtPrime ext[kMaxK];
  u32 h[kMaxL][kMaxK], h27[kMaxL][kMaxK];  // (Q/q_j) mod p_k, 2^27 (Q/q_j) mod p_k
  u32 negq[kMaxK];                         // (-Q) mod p_k
};

template <int L, int K>
CW_HD void lift_ext(const u64 *x, u32 *out, const LiftTab &C) {
  u64 y[L];
  for (int j = 0; j < L; ++j) y[j] = shoup(x[j], C.Q.theta[j], C.Q.theta_s[j], C.Q.q[j]);
  bool amb;
  u64 rho = round_sum<L>(y, C.Q.w_hi, C.Q.w_lo, &amb);
  if (amb) rho += mr_greater_half<L>(x, C.Q);
  // rho <= L: one 32-bit word; the halves of y_j are below 2^27
  for (int k = 0; k < K; ++k) {
    u64 s = wmul((u32)rho, C.negq[k]);
    for (int j = 0; j < L; ++j) s += wmul(lo27(y[j]), C.h[j][k]) + wmul(hi27(y[j]), C.h27[j][k]);
    out[k] = reduce_ext(s, C.ext[k]);
  }
}

// ---------------------------------------------------------------------
// Exact scale-down e = round(t d / Q) mod q_j of one tensor coefficient d,
// known modulo Q (residues dq) and modulo P = prod p_k (residues dp), with
// |d| < N Q^2 / 2 and P > 2^17 t N Q.
//   eps = [t d]_Q centered: y_j = [d_j * t (Q/q_j)^-1]_{q_j}, rho as above,
//   r = (t d - eps)/Q = round(t d / Q) exactly; modulo p_k:
//   r_k = [t Q^-1]_{p_k} d_k - sum_j y_j [q_j^-1]_{p_k} + rho, and its
//   conversion digit yb_k = [r_k (P/p_k)^-1]_{p_k} is formed directly.
//   |r| <= t N Q / 2 + 1 < P/2, so the centered conversion of r from the
//   p-basis to the q-basis is exact (and never near the ambiguous zone).
// ---------------------------------------------------------------------
// The residues handed to scale_coeff are those of f*d for a fixed factor f
// (f = N: the inverse transforms that produce d skip their N^-1); every
// constant that multiplies d carries f^-1.
struct ScaleTab {
  QConv Q;
  u64 t_theta[kMaxL], t_theta_s[kMaxL]; // t f^-1 (Q/q_j)^-1 mod q_j
  u64 t_mod[kMaxL], t_mod_s[kMaxL];     // t f^-1 mod q_j (ambiguous path)
  ExtPrime ext[kMaxK];
  // yb_k = [A_k (f d)_k + sum_j (B_jk yl_j + B27_jk yh_j) + C_k rho]_{p_k}
  u32 A[kMaxK];                          // t f^-1 Q^-1 (P/p_k)^-1 mod p_k
  u32 B[kMaxL][kMaxK], B27[kMaxL][kMaxK]; // -q_j^-1 (P/p_k)^-1 mod p_k, times 2^27
  u32 Cr[kMaxK];                         // (P/p_k)^-1 mod p_k
  u32 pw58[kMaxK];                       // floor(2^58 / p_k)
  // e_j = [sum_k yb_k (P/p_k) + rho2 (-P)]_{q_j}, constants as 27-bit halves
  u32 hat2[kMaxK][kMaxL][2], negp2[kMaxL][2];
};

// dq: residues of f*d below 2^55 (lazy [0, 2q) values are fine); dp:
// residues below 2^31 (lazy [0, 2p)).
//
// The conversion of r back to Q needs rho2 = round(sum_k yb_k / p_k).  As
// sum_k yb_k / p_k = rho2 + r/P with |r|/P < 2^-18 (P > 2^17 t N Q), the sum
// lies within 2^-18 of the integer rho2, and a 6.58 fixed-point sum of
// yb_k floor(2^58 / p_k), each term low by less than yb_k < 2^30 units of
// 2^-58, i.e. the sum low by less than 30 * 2^-28, rounds to it exactly.
// Returns false if that sum is ever 2^-17 or more away from an integer
// (which the bound rules out); callers record it as an internal error.
template <int L>
CW_HD bool scale_coeff(const u64 *dq, const u64 *dp, u64 *out, const ScaleTab &S) {
  constexpr int K = ext_count(L);
  u64 y[L];
#pragma unroll 1
  for (int j = 0; j < L; ++j)
    y[j] = shoup(dq[j], S.t_theta[j], S.t_theta_s[j], S.Q.q[j]);
  bool amb;
  u64 rho = round_sum<L>(y, S.Q.w_hi, S.Q.w_lo, &amb);
  if (amb) {
    u64 eps[L];
#pragma unroll 1
    for (int j = 0; j < L; ++j)
      eps[j] = shoup(dq[j], S.t_mod[j], S.t_mod_s[j], S.Q.q[j]);
    rho += mr_greater_half<L>(eps, S.Q);
  }
  // dp_k A_k < 2^61, 2L products of 27-bit halves with 30-bit constants
  // below 2^57 each (2^61 for L = 8), rho C_k < 2^34: the sum fits 2^62
  // every factor is below 2^32: dp_k < 2^31, rho <= L, the halves of y_j,
  // so each product is one wide 32 x 32-bit multiply
  u32 yb[K];
#pragma unroll 1
  for (int k = 0; k < K; ++k) {
    u64 s = wmul((u32)dp[k], S.A[k]) + wmul((u32)rho, S.Cr[k]);
#pragma unroll 1
    for (int j = 0; j < L; ++j) s += wmul(lo27(y[j]), S.B[j][k]) + wmul(hi27(y[j]), S.B27[j][k]);
    yb[k] = reduce_ext(s, S.ext[k]);
  }
  u64 fix = 0;
#pragma unroll 1
  for (int k = 0; k < K; ++k) fix += wmul(yb[k], S.pw58[k]);  // each < 2^58: sum < 2^63 (K <= 30)
  const u64 rho2 = (fix + (1ull << 57)) >> 58;
  const u64 frac = (fix + (1ull << 57)) & ((1ull << 58) - 1);  // offset + 1/2, in 2^-58
  const bool far = frac < (1ull << 57) - (1ull << 41) || frac > (1ull << 57) + (1ull << 41);
  // K + 1 <= 31 products of values below 2^30 with 27-bit halves: the words
  // ll and x stay below 31 * 2^57 < 2^62; the sum ll + x 2^27 < 2^90
#pragma unroll 1
  for (int j = 0; j < L; ++j) {  // rho2 <= K
    u64 ll = wmul((u32)rho2, S.negp2[j][0]), x = wmul((u32)rho2, S.negp2[j][1]);
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      ll += wmul(yb[k], S.hat2[k][j][0]);
      x += wmul(yb[k], S.hat2[k][j][1]);
    }
    const u64 lo = ll + (x << 27);
    const u64 hi = (x >> 37) + (lo < ll ? 1 : 0);
    out[j] = barrett_reduce(hi, lo, S.Q.q[j], S.Q.mu[j]);
  }
  return !far;
}

// ---------------------------------------------------------------------
// Exact scale-down e = round(t d / Q) mod q_j from the extension basis
// alone.  The tensor of two centered lifts, |d| <= N Q^2 / 2, is held
// exactly by its residues modulo the K extension primes (P >= 2 N Q^2):
//   x_k = [d (P/p_k)^-1]_{p_k},   d = sum_k x_k (P/p_k) - v P,
//   v = round(sum_k x_k / p_k)    (the sum lies within |d|/P <= 1/4 of v).
// Split t (P/p_k) / Q = I_k + f_k and t P / Q = I_P + f_P into integer
// and fractional parts; then t d / Q = sum_k x_k I_k - v I_P + G with
// G = sum_k x_k f_k - v f_P, so that exactly
//   round(t d / Q) = sum_k x_k I_k - v I_P + round(G).
// G comes from a 58-bit fixed-point sum of x_k floor(f_k 2^58) - v
// floor(f_P 2^58), which errs by less than sum_k x_k + v < 2^35 units of
// 2^-58 (below 2^-23); the rounding is taken from it unless its fraction
// lies within 2^-22 of 1/2, which happens for about one coefficient in 2^21.
// Those go to scale_exact, which forms N d mod q_j from the same digits and
// runs scale_coeff.  Q is odd and t d / Q never a half integer, so the
// rounding is unique.
//
// The residues handed over are those of N d (the inverse transforms skip
// N^-1): c_k carries N^-1.
// ---------------------------------------------------------------------
struct ScaleTabP {
  ExtPrime ext[kMaxK];
  u32 c[kMaxK], cs[kMaxK];    // N^-1 (P/p_k)^-1 mod p_k, floor(c_k 2^32 / p_k)
  u32 pw58[kMaxK];            // floor(2^58 / p_k)
  u32 fh[kMaxK], fl[kMaxK];   // floor(f_k 2^58) = fh_k 2^29 + fl_k
  u64 fP;                     // floor(f_P 2^58)
  u32 I2[kMaxK][kMaxL][2];    // I_k mod q_j, 27-bit halves
  u32 nIP2[kMaxL][2];         // -I_P mod q_j, 27-bit halves
  u64 q[kMaxL], mu[kMaxL];    // q_j, floor(2^116 / q_j)
  u64 nq[kMaxL], nq_s[kMaxL]; // N mod q_j and its Shoup companion (exact path)
  u32 exact_all;              // 1: every coefficient takes the exact path
};

// Sum of x_k times 27-bit halves h[k][j] of residues modulo q_j, plus
// `extra` and v times the halves g: with extra below 2^62 - (K + 1) 2^57
// (at least 2^57 for K <= 30) the words stay below 2^62 and their
// combination below 2^90; reduced modulo q_j.
template <int K>
CW_HD u64 sum_to_q(const u32 *x, const u32 (*h)[kMaxL][2], int j, u64 v, const u32 *g,
                   u64 extra, u64 q, u64 mu) {
  u64 ll = extra + wmul((u32)v, g[0]), hh = wmul((u32)v, g[1]);  // v <= K
#pragma unroll
  for (int k = 0; k < K; ++k) {
    ll += wmul(x[k], h[k][j][0]);
    hh += wmul(x[k], h[k][j][1]);
  }
  const u64 lo = ll + (hh << 27);
  const u64 hi = (hh >> 37) + (lo < ll ? 1 : 0);
  return barrett_reduce(hi, lo, q, mu);
}

// The digits x_k of d from dp_k = N d mod p_k below 2^31 (lazy [0, 2p)),
// and v; false if the sum for v is not within 1/4 + 2^-20 of an integer
// (which the bound on |d| rules out).  A and B: the two halves of the
// fixed-point sum for G.
template <int K>
CW_HD bool scale_digits(const u32 *dp, u32 *x, u64 *v, u64 *A, u64 *B, const ScaleTabP &S) {
  u64 fix = 0, a = 0, b = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const u32 d = dp[k], p = S.ext[k].p;
    x[k] = csub32(d * S.c[k] - mulhi32(d, S.cs[k]) * p, p);  // Shoup: [0, 2p) -> [0, p)
    fix += wmul(x[k], S.pw58[k]);  // each < 2^58
    a += wmul(x[k], S.fh[k]);      // each < 2^59: K <= 30 terms fit 64 bits
    b += wmul(x[k], S.fl[k]);
  }
  *A = a;
  *B = b;
  const u64 vs = fix + (1ull << 57), vfrac = vs & ((1ull << 58) - 1);
  *v = vs >> 58;
  // fix / 2^58 is in (v + d/P - 2^-23, v + d/P] with |d/P| <= 1/4
  return vfrac >= (1ull << 56) - (1ull << 38) && vfrac <= 3 * (1ull << 56);
}

// The fast path: writes e and returns 0, or returns 1 when the rounding is
// left to the exact path (e not written), or 2 when scale_digits fails.
template <int L>
CW_HD int scale_fast(const u32 *dp, u64 *e, const ScaleTabP &S) {
  constexpr int K = ext_count(L);
  u32 x[K];
  u64 v, A, B;
  if (!scale_digits<K>(dp, x, &v, &A, &B, S)) return 2;
  // T = A 2^29 + B + 2^57 + 64 2^58 - v fP >= 0 (128-bit): the rounding
  // of G offset by 64
  u64 lo = A << 29, hi = (A >> 35) + 1;
  lo += B;
  hi += lo < B ? 1 : 0;
  lo += 1ull << 57;
  hi += lo < (1ull << 57) ? 1 : 0;
  const u64 vf = v * S.fP;  // v <= K, fP < 2^58
  hi -= lo < vf ? 1 : 0;
  lo -= vf;
  const u64 phi = lo & ((1ull << 58) - 1);
  if (S.exact_all || phi < (1ull << 36) || phi > (1ull << 58) - (1ull << 36)) return 1;
  const u64 r64 = (hi << 6) | (lo >> 58);  // round(G) + 64 < 2^36 + 64
#pragma unroll
  for (int j = 0; j < L; ++j)  // + (q_j - 64) takes the offset back out
    e[j] = sum_to_q<K>(x, S.I2, j, v, S.nIP2[j], r64 + S.q[j] - 64, S.q[j], S.mu[j]);
  return 0;
}

// The exact path: N d mod q_j = N (sum_k x_k (P/p_k) - v P) mod q_j from
// scale_coeff's own constants (P/p_k and -P modulo q_j), then scale_coeff
// on the residues of N d modulo Q and P.
template <int L>
CW_HD bool scale_exact(const u32 *dp, u64 *e, const ScaleTabP &SP, const ScaleTab &S) {
  constexpr int K = ext_count(L);
  u32 x[K];
  u64 v, A, B, dq[L], dp64[K];
  if (!scale_digits<K>(dp, x, &v, &A, &B, SP)) return false;
#pragma unroll 1
  for (int j = 0; j < L; ++j) {  // sum_to_q, kept rolled up on this rare path
    u64 ll = wmul((u32)v, S.negp2[j][0]), hh = wmul((u32)v, S.negp2[j][1]);
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      ll += wmul(x[k], S.hat2[k][j][0]);
      hh += wmul(x[k], S.hat2[k][j][1]);
    }
    const u64 lo = ll + (hh << 27);
    const u64 hi = (hh >> 37) + (lo < ll ? 1 : 0);
    dq[j] = shoup(barrett_reduce(hi, lo, SP.q[j], SP.mu[j]), SP.nq[j], SP.nq_s[j], SP.q[j]);
  }
#pragma unroll 1
  for (int k = 0; k < K; ++k) dp64[k] = dp[k];
  return scale_coeff<L>(dq, dp64, e, S);
}

// ---------------------------------------------------------------------
// Exact products with database rows in a "row basis" of nr = 3 or 4 primes.
//
// The plaintext rows are small integers (|v| <= (t-1)/2 after the centered
// lift), and the inputs of the last tree level's key switch (the limbs of
// e0, e1 and the digits of e2) are residues below the largest ciphertext
// prime.  A sum over a group of rows of their negacyclic products with the
// rows is an integer x with |x| <= rows N q_max (t-1)/2; the library keeps
// the rows per group low enough that |x| < (1 - 2^-23) R/2 (R the product
// of the first nr extension primes), so the residues modulo the r_k hold x
// exactly.  row_digits recovers x from N x mod r_k (the inverse transforms
// leave the factor N): y_k = [(N x)_k (R/r_k)^-1 N^-1]_{r_k},
// x = sum_k y_k (R/r_k) - rho R with rho = round(sum_k y_k / r_k); the sum
// is at least 2^-24 away from a half integer, and a 6.58 fixed-point sum of
// y_k floor(2^58 / r_k), low by less than nr 2^-28, rounds to rho exactly.
// ---------------------------------------------------------------------
constexpr int kRowPrimes = 5;  // at most (the key-switch basis uses five)

struct RowTab {
  u32 nr;                             // primes in use: 3 or 4 (rows), 5 (key switch)
  u32 rmax;                           // rows per group the basis holds exactly
  ExtPrime r[kRowPrimes];
  u32 theta[kRowPrimes];              // (R/r_k)^-1 N^-1 mod r_k
  u32 rw58[kRowPrimes];               // floor(2^58 / r_k)
  u32 hat2[kRowPrimes][kMaxL][2];     // (R/r_k) mod q_j, 27-bit halves
  u32 negr2[kMaxL][2];                // (-R) mod q_j, 27-bit halves
  u64 q[kMaxL], q_mu[kMaxL];          // ciphertext primes, floor(2^116 / q_j)
};

// xr: N x mod r_k (k < nr), below 2^31 (lazy [0, 2r)); y: the digits y_k;
// returns rho, and true in *far if the fixed-point sum comes within 2^-25 of
// a half integer (ruled out by the bound on |x|).
CW_HD u64 row_digits(const u32 *xr, u32 *y, const RowTab &T, bool *far) {
  u64 fix = 0;
  for (int k = 0; k < kRowPrimes; ++k) {
    if ((u32)k >= T.nr) break;
    const u32 v = xr[k] >= T.r[k].p ? xr[k] - T.r[k].p : xr[k];
    const u32 m = mulmod_ext_lazy(v, T.theta[k], T.r[k]);
    y[k] = m >= T.r[k].p ? m - T.r[k].p : m;
    fix += (u64)y[k] * T.rw58[k];
  }
  const u64 frac = (fix + (1ull << 57)) & ((1ull << 58) - 1);
  *far = frac < (1ull << 33) || frac > (1ull << 58) - (1ull << 33);
  return (fix + (1ull << 57)) >> 58;
}

// x mod q_j from the digits: sum_k y_k (R/r_k) - rho R (at most six
// products of values below 2^30 with 27-bit halves, sum below 2^88).
CW_HD u64 row_to_q(const u32 *y, u64 rho, int j, const RowTab &T) {
  u64 ll = wmul((u32)rho, T.negr2[j][0]), x = wmul((u32)rho, T.negr2[j][1]);  // rho <= nr
  for (int k = 0; k < kRowPrimes; ++k) {
    if ((u32)k >= T.nr) break;
    ll += (u64)y[k] * T.hat2[k][j][0];
    x += (u64)y[k] * T.hat2[k][j][1];
  }
  const u64 lo = ll + (x << 27);
  const u64 hi = (x >> 37) + (lo < ll ? 1 : 0);
  return barrett_reduce(hi, lo, T.q[j], T.q_mu[j]);
}

}  // namespace cw
