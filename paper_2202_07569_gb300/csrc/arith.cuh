// arith.cuh -- word-size modular arithmetic and per-coefficient RNS steps of
// the BFV multiplication (FV scheme, arXiv 2202.07569 Sec. 2.1.1), written
// for the 32-bit integer pipes of sm_103a.  Every function is exact.
//
// Residues are u64 values below primes q < 2^54.  The functions are
// __host__ __device__ so that the same arithmetic can be exercised on the
// CPU by the test suite.
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
constexpr int kMaxK = 9;       // extension primes (L + 1)
constexpr int kMaxP = kMaxL + kMaxK;

CW_HD u64 mulhi(u64 a, u64 b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (u64)(((unsigned __int128)a * b) >> 64);
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

// Exact sum of a few products a * b with a < 2^55 and constants b < 2^54
// given as 27-bit halves (b = b1 2^27 + b0): with a = a1 2^27 + a0 each
// product is four 32 x 32 + 64 multiply-adds into the words
// ll = sum a0 b0, x = sum (a0 b1 + a1 b0), hh = sum a1 b1 (partials below
// 2^55, so up to 8 terms cannot overflow 64 bits), and the sum is
// ll + x 2^27 + hh 2^54.
constexpr u32 kMask27 = (1u << 27) - 1;
CW_HD void split27(u64 b, u32 *out) {
  out[0] = (u32)b & kMask27;
  out[1] = (u32)(b >> 27);
}
struct Acc3 {
  u64 ll = 0, x = 0, hh = 0;
  CW_HDM void mac(u64 a, const u32 *b) {
    const u32 a0 = (u32)a & kMask27, a1 = (u32)(a >> 27);
    ll += (u64)a0 * b[0];
    x += (u64)a0 * b[1];
    x += (u64)a1 * b[0];
    hh += (u64)a1 * b[1];
  }
  CW_HDM void add(u64 v) { ll += v; }
  // the sum as hi 2^64 + lo (the caller bounds it below 2^112)
  CW_HDM void get(u64 &hi, u64 &lo) const {
    const u64 l1 = ll + (x << 27);
    const u64 l2 = l1 + (hh << 54);
    hi = (x >> 37) + (hh >> 10) + (l1 < ll ? 1 : 0) + (l2 < l1 ? 1 : 0);
    lo = l2;
  }
};

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

// Per-prime NTT data in device memory.
struct NttPrime {
  u64 q, mu;          // prime, Barrett constant floor(2^116/q)
  u64 ninv, ninv_s;   // N^-1 mod q and Shoup companion
  const u64 *psi2;    // [N][2]: psi^bitrev(i) and its Shoup companion
  const u64 *ipsi2;   // [N][2]: psi^-bitrev(i) and its Shoup companion
};

// ---------------------------------------------------------------------
// Exact centered base conversion between RNS bases.
//
// x is given by residues x_j modulo the source primes s_j (product S).
// With y_j = [x_j * (S/s_j)^-1]_{s_j}, sum_j y_j (S/s_j) = x + v S where
// v = floor(sum_j y_j / s_j), and the centered representative of x is
// x_c = sum_j y_j (S/s_j) - rho S with rho = round(sum_j y_j / s_j)
// (S is odd, so sum_j y_j/s_j is never a half integer).
//
// rho is read from a 64.64 fixed-point sum of phi_j <= y_j 2^64 / s_j,
// each low by less than 2 units, so the sum is low by less than 2*ns units:
// rho = hi(2^63 + sum phi) unless the low word is within 2*ns of 2^64; in
// that case x is within 2*ns*S/2^64 of S/2 and the exact comparison of x
// with (S-1)/2 in mixed radix (Garner) decides.
// ---------------------------------------------------------------------
struct BaseConv {
  u32 ns, nd;
  u64 s[kMaxK];                 // source primes
  u64 theta[kMaxK], theta_s[kMaxK]; // (S/s_j)^-1 mod s_j
  u64 w_hi[kMaxK], w_lo[kMaxK];     // floor(2^128 / s_j)
  u64 d[kMaxK];                 // target primes
  u64 hat[kMaxK][kMaxK], hat_s[kMaxK][kMaxK]; // (S/s_j) mod d_k
  u64 smod[kMaxK], smod_s[kMaxK];   // S mod d_k
  u64 negsmod[kMaxK];           // (-S) mod d_k
  u64 d_mu[kMaxK];              // floor(2^116 / d_k)
  u64 mrinv[kMaxK][kMaxK], mrinv_s[kMaxK][kMaxK]; // s_i^-1 mod s_j, i < j
  u64 half_mr[kMaxK];           // mixed-radix digits of (S-1)/2
};

// 1 if x > (S-1)/2, by exact mixed-radix comparison.
template <int NS>
CW_HD u64 mr_greater_half(const u64 *x, const BaseConv &C) {
  u64 a[NS];
  for (int j = 0; j < NS; ++j) {
    u64 sj = C.s[j], v = x[j];
    for (int i = 0; i < j; ++i) {
      u64 ai = a[i] >= sj ? a[i] - sj : a[i];
      v = shoup(subq(v, ai, sj), C.mrinv[i][j], C.mrinv_s[i][j], sj);
    }
    a[j] = v;
  }
  for (int j = NS - 1; j >= 0; --j)
    if (a[j] != C.half_mr[j]) return a[j] > C.half_mr[j] ? 1 : 0;
  return 0;  // equal: x = (S-1)/2 is not greater
}

// hi(2^63 + sum_j phi_j) and whether the low word is in the ambiguous zone.
template <int NS>
CW_HD u64 round_sum(const u64 *y, const BaseConv &C, bool *ambiguous) {
  u64 lo = 0x8000000000000000ull, hi = 0;
  for (int j = 0; j < NS; ++j) {
    u64 phi = y[j] * C.w_hi[j] + mulhi(y[j], C.w_lo[j]);
    lo += phi;
    hi += (lo < phi) ? 1 : 0;
  }
  *ambiguous = lo > ~0ull - 2ull * NS;
  return hi;
}

// Centered conversion of one coefficient: x (NS source residues) -> out
// (ND target residues of x_c): out_k = [sum_j y_j (S/s_j) - rho S]_{d_k},
// accumulated exactly in 128 bits and reduced once.
template <int NS, int ND>
CW_HD void lift_centered(const u64 *x, u64 *out, const BaseConv &C) {
  u64 y[NS];
  for (int j = 0; j < NS; ++j) y[j] = shoup(x[j], C.theta[j], C.theta_s[j], C.s[j]);
  bool amb;
  u64 rho = round_sum<NS>(y, C, &amb);
  if (amb) rho += mr_greater_half<NS>(x, C);
  for (int k = 0; k < ND; ++k) {
    Acc128 a;
    for (int j = 0; j < NS; ++j) a.mac(y[j], C.hat[j][k]);
    a.mac(rho, C.negsmod[k]);
    out[k] = barrett_reduce(a.hi, a.lo, C.d[k], C.d_mu[k]);
  }
}

// ---------------------------------------------------------------------
// Exact scale-down e = round(t d / Q) mod q_j of one tensor coefficient d,
// known modulo Q (residues dq) and modulo P = prod p_k (residues dp), with
// |d| < 2N(Q/2)^2 and P > t N Q + 1.
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
  u64 t_theta[kMaxL], t_theta_s[kMaxL]; // t f^-1 (Q/q_j)^-1 mod q_j
  u64 t_mod[kMaxL], t_mod_s[kMaxL];     // t f^-1 mod q_j (ambiguous path)
  // yb_k = [r_k (P/p_k)^-1]_{p_k} = [A_k (f d)_k + sum_j B_jk y_j + C_k rho]_{p_k}
  u64 A[kMaxK];          // t f^-1 Q^-1 (P/p_k)^-1 mod p_k
  u64 B[kMaxL][kMaxK];   // -q_j^-1 (P/p_k)^-1 mod p_k
  u64 Cr[kMaxK];         // (P/p_k)^-1 mod p_k
  BaseConv q2b;  // Q -> P conversion data (fraction and Garner parts used)
  BaseConv b2q;  // P -> Q conversion
  // the constants of the two multiply-accumulate stages as 27-bit halves
  u32 A2[kMaxK][2], B2[kMaxL][kMaxK][2], Cr2[kMaxK][2];
  u32 hat2[kMaxK][kMaxL][2], negs2[kMaxL][2];  // b2q.hat[k][j], b2q.negsmod[j]
};

// dq, dp: residues of f*d below 2^55 (lazy [0, 2q) values are fine).
// Returns false if the P-basis rounding ever lands in the ambiguous zone,
// which the bound on |r| rules out; callers record it as an internal error.
template <int L>
CW_HD bool scale_coeff(const u64 *dq, const u64 *dp, u64 *out, const ScaleTab &S) {
  constexpr int K = L + 1;
  u64 y[L];
  for (int j = 0; j < L; ++j)
    y[j] = shoup(dq[j], S.t_theta[j], S.t_theta_s[j], S.q2b.s[j]);
  bool amb;
  u64 rho = round_sum<L>(y, S.q2b, &amb);
  if (amb) {
    u64 eps[L];
    for (int j = 0; j < L; ++j)
      eps[j] = shoup(dq[j], S.t_mod[j], S.t_mod_s[j], S.q2b.s[j]);
    rho += mr_greater_half<L>(eps, S.q2b);
  }
  // L + 2 and K + 1 products below 2^55 * 2^54 each: sums below 2^112
  u64 yb[K];
  for (int k = 0; k < K; ++k) {
    Acc3 a;
    a.mac(dp[k], S.A2[k]);
    for (int j = 0; j < L; ++j) a.mac(y[j], S.B2[j][k]);
    a.mac(rho, S.Cr2[k]);
    u64 hi, lo;
    a.get(hi, lo);
    yb[k] = barrett_reduce(hi, lo, S.b2q.s[k], S.q2b.d_mu[k]);
  }
  bool amb2;
  u64 rho2 = round_sum<K>(yb, S.b2q, &amb2);
  for (int j = 0; j < L; ++j) {
    Acc3 a;
    for (int k = 0; k < K; ++k) a.mac(yb[k], S.hat2[k][j]);
    a.mac(rho2, S.negs2[j]);
    u64 hi, lo;
    a.get(hi, lo);
    out[j] = barrett_reduce(hi, lo, S.b2q.d[j], S.b2q.d_mu[j]);
  }
  return !amb2;
}

}  // namespace cw
