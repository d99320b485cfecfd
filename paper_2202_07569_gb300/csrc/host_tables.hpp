// host_tables.hpp -- host-side number theory and the constant tables the
// kernels read: NTT twiddles (bit-reversed powers of a primitive 2N-th root
// of unity), exact base-conversion data and the scale-down constants.
// Header-only C++, no CUDA runtime dependency.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "arith.cuh"

namespace cw {
namespace host {

typedef unsigned __int128 u128;

inline u64 hmul(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }
inline u64 hpow(u64 a, u64 e, u64 m) {
  u64 r = 1 % m;
  a %= m;
  for (; e; e >>= 1) {
    if (e & 1) r = hmul(r, a, m);
    a = hmul(a, a, m);
  }
  return r;
}
inline u64 hinv(u64 a, u64 p) { return hpow(a, p - 2, p); }  // p prime
inline u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

inline bool miller_rabin(u64 n) {
  if (n < 2) return false;
  static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (u64 p : small) {
    if (n == p) return true;
    if (n % p == 0) return false;
  }
  u64 d = n - 1;
  int r = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++r;
  }
  for (u64 a : small) {
    u64 x = hpow(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < r && comp; ++i) {
      x = hmul(x, x, n);
      if (x == n - 1) comp = false;
    }
    if (comp) return false;
  }
  return true;
}

// primes p = 1 mod 2N with 2^53 < p < 2^54, descending, skipping `avoid`.
inline std::vector<u64> ntt_primes(u32 N, u32 count, const std::vector<u64> &avoid) {
  std::vector<u64> out;
  const u64 step = 2ull * N;
  for (u64 p = (1ull << 54) - step + 1; out.size() < count && p > (1ull << 53); p -= step)
    if (miller_rabin(p) && std::find(avoid.begin(), avoid.end(), p) == avoid.end())
      out.push_back(p);
  return out;
}

// extension primes: p = 1 mod 2N with 2^29 < p < 2^30, descending.
inline std::vector<u64> ext_primes(u32 N, u32 count) {
  std::vector<u64> out;
  const u64 step = 2ull * N;
  for (u64 p = (1ull << 30) - step + 1; out.size() < count && p > (1ull << 29); p -= step)
    if (miller_rabin(p)) out.push_back(p);
  return out;
}

inline u64 primitive_2n_root(u64 p, u32 N) {
  for (u64 g = 2; g < 100000; ++g) {
    u64 r = hpow(g, (p - 1) / (2ull * N), p);
    if (hpow(r, N, p) == p - 1) return r;
  }
  return 0;
}

inline u32 bitrev(u32 x, u32 bits) {
  u32 r = 0;
  for (u32 i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}

// Centered conversion data of the ciphertext basis (see QConv in arith.cuh).
inline void fill_qconv(cw::QConv &C, const std::vector<u64> &q) {
  memset(&C, 0, sizeof C);
  const u32 L = (u32)q.size();
  for (u32 j = 0; j < L; ++j) {
    const u64 qj = q[j];
    C.q[j] = qj;
    C.mu[j] = (u64)(((u128)1 << 116) / qj);
    u64 hat = 1;
    for (u32 l = 0; l < L; ++l)
      if (l != j) hat = hmul(hat, q[l] % qj, qj);
    C.theta[j] = hinv(hat, qj);
    C.theta_s[j] = shoup_of(C.theta[j], qj);
    const u128 W = (~(u128)0) / qj;  // floor(2^128 / q_j): q_j is not a power of 2
    C.w_hi[j] = (u64)(W >> 64);
    C.w_lo[j] = (u64)W;
  }
  // Garner data: q_i^-1 mod q_j (i < j) and the mixed-radix digits of
  // (Q-1)/2, whose residue mod q_j is (q_j - 1)/2.
  for (u32 j = 0; j < L; ++j)
    for (u32 i = 0; i < j; ++i) {
      C.mrinv[i][j] = hinv(q[i] % q[j], q[j]);
      C.mrinv_s[i][j] = shoup_of(C.mrinv[i][j], q[j]);
    }
  u64 a[cw::kMaxL];
  for (u32 j = 0; j < L; ++j) {
    const u64 qj = q[j];
    u64 v = (qj - 1) / 2;
    for (u32 i = 0; i < j; ++i) v = hmul((v + qj - a[i] % qj) % qj, C.mrinv[i][j], qj);
    a[j] = v;
    C.half_mr[j] = v;
  }
}

inline cw::ExtPrime ext_prime(u64 p) {
  cw::ExtPrime E;
  E.p = (u32)p;
  E.mu60 = (u32)((1ull << 60) / p);
  E.mu64 = (u64)(((u128)1 << 64) / p);
  E.c32 = (u32)((1ull << 32) % p);
  E.mu61 = (u32)((1ull << 61) / p);
  return E;
}

// (product of src) / src[j] mod m
inline u64 hat_mod(const std::vector<u64> &src, u32 j, u64 m) {
  u64 h = 1;
  for (u32 l = 0; l < src.size(); ++l)
    if (l != j) h = hmul(h, src[l] % m, m);
  return h;
}
inline u64 prod_mod(const std::vector<u64> &src, u64 m) {
  u64 h = 1;
  for (u64 v : src) h = hmul(h, v % m, m);
  return h;
}

// Centered Q -> P conversion constants (see LiftTab in arith.cuh).
inline void fill_lift(cw::LiftTab &T, const std::vector<u64> &q, const std::vector<u64> &p) {
  memset(&T, 0, sizeof T);
  fill_qconv(T.Q, q);
  for (u32 k = 0; k < p.size(); ++k) {
    const u64 pk = p[k];
    T.ext[k] = ext_prime(pk);
    for (u32 j = 0; j < q.size(); ++j) {
      const u64 h = hat_mod(q, j, pk);
      T.h[j][k] = (u32)h;
      T.h27[j][k] = (u32)hmul(h, 1ull << 27, pk);
    }
    const u64 Qm = prod_mod(q, pk);
    T.negq[k] = (u32)(Qm ? pk - Qm : 0);
  }
}

// Forward pairs (psi^bitrev(i), Shoup) at tw[0..2N), inverse pairs
// (psi^-bitrev(i), Shoup) at tw[2N..4N).  Returns false if q has no
// primitive 2N-th root of unity.
inline bool make_twiddles(u64 q, u32 N, u32 logN, u64 *tw) {
  u64 psi = primitive_2n_root(q, N);
  if (!psi) return false;
  u64 ipsi = hinv(psi, q);
  for (u32 i = 0; i < N; ++i) {
    u32 e = bitrev(i, logN);
    u64 f = hpow(psi, e, q), b = hpow(ipsi, e, q);
    tw[2 * i] = f;
    tw[2 * i + 1] = shoup_of(f, q);
    tw[2 * N + 2 * i] = b;
    tw[2 * N + 2 * i + 1] = shoup_of(b, q);
  }
  return true;
}

// 32-bit twiddles of an extension prime: forward pairs (psi^bitrev(i),
// floor(psi^bitrev(i) 2^32 / p)) at tw[0..2N), inverse pairs at tw[2N..4N).
inline bool make_twiddles32(u64 p, u32 N, u32 logN, u32 *tw) {
  const u64 psi = primitive_2n_root(p, N);
  if (!psi) return false;
  const u64 ipsi = hinv(psi, p);
  for (u32 i = 0; i < N; ++i) {
    const u32 e = bitrev(i, logN);
    const u64 f = hpow(psi, e, p), b = hpow(ipsi, e, p);
    tw[2 * i] = (u32)f;
    tw[2 * i + 1] = (u32)((f << 32) / p);
    tw[2 * N + 2 * i] = (u32)b;
    tw[2 * N + 2 * i + 1] = (u32)((b << 32) / p);
  }
  return true;
}

// Scale-down constants for round(t d / Q) (see ScaleTab in arith.cuh),
// for residues given as f*d: the constants that multiply d carry f^-1 (the
// tensor kernel leaves the factor N of its inverse transforms in place).
inline void fill_scale(cw::ScaleTab &S, const std::vector<u64> &q, const std::vector<u64> &p,
                       u64 t, u64 f) {
  memset(&S, 0, sizeof S);
  const u32 L = (u32)q.size(), K = (u32)p.size();
  fill_qconv(S.Q, q);
  for (u32 j = 0; j < L; ++j) {
    const u64 qj = q[j];
    S.t_mod[j] = hmul(t % qj, hinv(f % qj, qj), qj);
    S.t_mod_s[j] = shoup_of(S.t_mod[j], qj);
    S.t_theta[j] = hmul(S.t_mod[j], S.Q.theta[j], qj);
    S.t_theta_s[j] = shoup_of(S.t_theta[j], qj);
  }
  for (u32 k = 0; k < K; ++k) {
    const u64 pk = p[k];
    S.ext[k] = ext_prime(pk);
    const u64 th = hinv(hat_mod(p, k, pk), pk);  // (P/p_k)^-1 mod p_k
    const u64 Qm = prod_mod(q, pk);
    S.A[k] = (u32)hmul(hmul(hmul(t % pk, hinv(Qm, pk), pk), th, pk), hinv(f % pk, pk), pk);
    S.Cr[k] = (u32)th;
    for (u32 j = 0; j < L; ++j) {
      const u64 v = hmul(hinv(q[j] % pk, pk), th, pk);
      const u64 b = v ? pk - v : 0;
      S.B[j][k] = (u32)b;
      S.B27[j][k] = (u32)hmul(b, 1ull << 27, pk);
    }
    S.pw58[k] = (u32)((1ull << 58) / pk);
  }
  for (u32 j = 0; j < L; ++j) {
    const u64 qj = q[j];
    for (u32 k = 0; k < K; ++k) split27(hat_mod(p, k, qj), S.hat2[k][j]);
    const u64 Pm = prod_mod(p, qj);
    split27(Pm ? qj - Pm : 0, S.negp2[j]);
  }
}

// Unsigned multi-precision integers (32-bit words, least significant
// first), for the few setup constants that need exact products and
// quotients of the moduli.
struct Big {
  std::vector<u32> w;
  static Big of(u64 v) {
    Big b;
    b.w = {(u32)v, (u32)(v >> 32)};
    b.trim();
    return b;
  }
  void trim() {
    while (!w.empty() && w.back() == 0) w.pop_back();
  }
  u32 bits() const {
    if (w.empty()) return 0;
    u32 n = 32 * (u32)(w.size() - 1), top = w.back();
    while (top) ++n, top >>= 1;
    return n;
  }
  bool bit(u32 i) const { return i / 32 < w.size() && ((w[i / 32] >> (i % 32)) & 1u); }
  void mul(u64 m) {  // *= m
    u128 carry = 0;
    for (u32 &x : w) {
      const u128 v = (u128)x * m + carry;
      x = (u32)v;
      carry = v >> 32;
    }
    while (carry) w.push_back((u32)carry), carry >>= 32;
    trim();
  }
  void shl1_or(u32 b) {  // = 2 * this + b
    u32 carry = b;
    for (u32 &x : w) {
      const u32 top = x >> 31;
      x = (x << 1) | carry;
      carry = top;
    }
    if (carry) w.push_back(carry);
  }
  bool geq(const Big &o) const {
    if (w.size() != o.w.size()) return w.size() > o.w.size();
    for (size_t i = w.size(); i-- > 0;)
      if (w[i] != o.w[i]) return w[i] > o.w[i];
    return true;
  }
  void sub(const Big &o) {  // this >= o
    u64 borrow = 0;
    for (size_t i = 0; i < w.size(); ++i) {
      const u64 d = (u64)w[i] - (i < o.w.size() ? o.w[i] : 0) - borrow;
      w[i] = (u32)d;
      borrow = (d >> 63) & 1;
    }
    trim();
  }
  u64 mod(u64 m) const {
    u128 r = 0;
    for (size_t i = w.size(); i-- > 0;) r = ((r << 32) | w[i]) % m;
    return (u64)r;
  }
  u64 low64() const {
    return (w.size() > 0 ? w[0] : 0) | (w.size() > 1 ? (u64)w[1] << 32 : 0);
  }
};

// a = quo b + rem, 0 <= rem < b (b > 0), by binary long division.
inline void big_divmod(const Big &a, const Big &b, Big &quo, Big &rem) {
  quo.w.assign(a.w.size(), 0);
  rem.w.clear();
  for (u32 i = a.bits(); i-- > 0;) {
    rem.shl1_or(a.bit(i) ? 1u : 0u);
    if (rem.geq(b)) {
      rem.sub(b);
      quo.w[i / 32] |= 1u << (i % 32);
    }
  }
  quo.trim();
}

inline Big big_prod(const std::vector<u64> &v, int skip = -1) {
  Big b = Big::of(1);
  for (size_t i = 0; i < v.size(); ++i)
    if ((int)i != skip) b.mul(v[i]);
  return b;
}

// floor(num / den) mod each q_j into 27-bit halves, and floor(frac(num /
// den) 2^58).
inline u64 split_quotient(const Big &num, const Big &den, const std::vector<u64> &q,
                          u32 (*halves)[2]) {
  Big quo, rem;
  big_divmod(num, den, quo, rem);
  for (size_t j = 0; j < q.size(); ++j) split27(quo.mod(q[j]), halves[j]);
  for (int b = 0; b < 58; ++b) rem.mul(2);
  Big f, r2;
  big_divmod(rem, den, f, r2);
  return f.low64();
}

// Constants of the scale-down from the extension basis (ScaleTabP in
// arith.cuh); N is the factor the residues carry.
inline void fill_scale_p(cw::ScaleTabP &S, const std::vector<u64> &q, const std::vector<u64> &p,
                         u64 t, u64 N) {
  memset(&S, 0, sizeof S);
  const u32 L = (u32)q.size(), K = (u32)p.size();
  const Big Q = big_prod(q);
  for (u32 k = 0; k < K; ++k) {
    const u64 pk = p[k];
    S.ext[k] = ext_prime(pk);
    const u64 c = hmul(hinv(hat_mod(p, k, pk), pk), hinv(N % pk, pk), pk);
    S.c[k] = (u32)c;
    S.cs[k] = (u32)((c << 32) / pk);
    S.pw58[k] = (u32)((1ull << 58) / pk);
    Big num = big_prod(p, (int)k);
    num.mul(t);
    u32 halves[cw::kMaxL][2];
    const u64 f = split_quotient(num, Q, q, halves);
    S.fh[k] = (u32)(f >> 29);
    S.fl[k] = (u32)(f & ((1u << 29) - 1));
    for (u32 j = 0; j < L; ++j) {
      S.I2[k][j][0] = halves[j][0];
      S.I2[k][j][1] = halves[j][1];
    }
  }
  Big num = big_prod(p);
  num.mul(t);
  u32 halves[cw::kMaxL][2];
  S.fP = split_quotient(num, Q, q, halves);
  for (u32 j = 0; j < L; ++j) {
    const u64 qj = q[j];
    const u64 ip = ((u64)halves[j][1] << 27) | halves[j][0];
    split27(ip ? qj - ip : 0, S.nIP2[j]);
    S.q[j] = qj;
    S.mu[j] = (u64)(((u128)1 << 116) / qj);
    S.nq[j] = N % qj;
    S.nq_s[j] = shoup_of(S.nq[j], qj);
  }
}

// Largest number of rows per group for which the row basis of the first nr
// extension primes holds the group sums exactly: rows N q_max (t-1)/2 <=
// (1 - 2^-23) R/2 (see RowTab in arith.cuh).
inline u64 row_group_limit(const std::vector<u64> &q, const std::vector<u64> &p, u32 nr,
                           u64 N, u64 t) {
  long double lr = 0;
  for (u32 k = 0; k < nr; ++k) lr += log2l((long double)p[k]);
  const u64 qmax = *std::max_element(q.begin(), q.end());
  const long double lim =
      lr - 1 + log2l(1.0L - 1.0L / (1 << 23)) - log2l((long double)N) -
      log2l((long double)qmax) - log2l((long double)((t - 1) / 2));
  if (lim >= 40) return 1ull << 40;
  return lim < 0 ? 0 : (u64)floorl(exp2l(lim));
}

// Row-basis constants (see RowTab in arith.cuh): r = the first nr
// extension primes, N the transform length.
inline void fill_rows(cw::RowTab &T, const std::vector<u64> &q, const std::vector<u64> &p,
                      u64 N, u32 nr) {
  memset(&T, 0, sizeof T);
  T.nr = nr;
  std::vector<u64> r(p.begin(), p.begin() + nr);
  for (u32 k = 0; k < nr; ++k) {
    const u64 rk = r[k];
    T.r[k] = ext_prime(rk);
    T.theta[k] = (u32)hmul(hinv(hat_mod(r, k, rk), rk), hinv(N % rk, rk), rk);
    T.rw58[k] = (u32)((1ull << 58) / rk);
    for (u32 j = 0; j < q.size(); ++j) split27(hat_mod(r, k, q[j]), T.hat2[k][j]);
  }
  for (u32 j = 0; j < q.size(); ++j) {
    const u64 Rm = prod_mod(r, q[j]);
    split27(Rm ? q[j] - Rm : 0, T.negr2[j]);
    T.q[j] = q[j];
    T.q_mu[j] = (u64)(((u128)1 << 116) / q[j]);
  }
}

}  // namespace host
}  // namespace cw
