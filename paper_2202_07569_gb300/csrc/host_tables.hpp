// host_tables.hpp -- host-side number theory and the constant tables the
// kernels read: NTT twiddles (bit-reversed powers of a primitive 2N-th root
// of unity), exact base-conversion data and the scale-down constants.
// Header-only C++, no CUDA runtime dependency.
#pragma once
#include <algorithm>
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

// Exact centered base conversion data (see BaseConv in arith.cuh).
inline void fill_conv(cw::BaseConv &C, const std::vector<u64> &src, const std::vector<u64> &dst) {
  memset(&C, 0, sizeof C);
  C.ns = (u32)src.size();
  C.nd = (u32)dst.size();
  for (u32 j = 0; j < C.ns; ++j) {
    u64 s = src[j];
    C.s[j] = s;
    u64 hat = 1;
    for (u32 l = 0; l < C.ns; ++l)
      if (l != j) hat = hmul(hat, src[l] % s, s);
    C.theta[j] = hinv(hat, s);
    C.theta_s[j] = shoup_of(C.theta[j], s);
    u128 W = (~(u128)0) / s;  // floor((2^128 - 1)/s) = floor(2^128/s): s is not a power of 2
    C.w_hi[j] = (u64)(W >> 64);
    C.w_lo[j] = (u64)W;
  }
  for (u32 k = 0; k < C.nd; ++k) {
    u64 d = dst[k];
    C.d[k] = d;
    u64 smod = 1;
    for (u32 j = 0; j < C.ns; ++j) smod = hmul(smod, src[j] % d, d);
    C.smod[k] = smod;
    C.smod_s[k] = shoup_of(smod, d);
    C.negsmod[k] = smod ? d - smod : 0;
    C.d_mu[k] = (u64)(((u128)1 << 116) / d);
    for (u32 j = 0; j < C.ns; ++j) {
      u64 hat = 1;
      for (u32 l = 0; l < C.ns; ++l)
        if (l != j) hat = hmul(hat, src[l] % d, d);
      C.hat[j][k] = hat;
      C.hat_s[j][k] = shoup_of(hat, d);
    }
  }
  // Garner data: s_i^-1 mod s_j (i < j) and the mixed-radix digits of
  // (S-1)/2, whose residue mod s_j is (s_j - 1)/2.
  for (u32 j = 0; j < C.ns; ++j)
    for (u32 i = 0; i < j; ++i) {
      C.mrinv[i][j] = hinv(src[i] % src[j], src[j]);
      C.mrinv_s[i][j] = shoup_of(C.mrinv[i][j], src[j]);
    }
  u64 a[cw::kMaxK];
  for (u32 j = 0; j < C.ns; ++j) {
    u64 sj = src[j], v = (sj - 1) / 2;
    for (u32 i = 0; i < j; ++i) v = hmul((v + sj - a[i] % sj) % sj, C.mrinv[i][j], sj);
    a[j] = v;
    C.half_mr[j] = v;
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

// Scale-down constants for round(t d / Q) (see ScaleTab in arith.cuh),
// for residues given as f*d: the constants that multiply d carry f^-1 (the
// tensor kernel leaves the factor N of its inverse transforms in place).
inline void fill_scale(cw::ScaleTab &S, const std::vector<u64> &q, const std::vector<u64> &p,
                       u64 t, u64 f) {
  const u32 L = (u32)q.size(), K = (u32)p.size();
  fill_conv(S.q2b, q, p);
  fill_conv(S.b2q, p, q);
  for (u32 j = 0; j < L; ++j) {
    u64 qj = q[j];
    S.t_mod[j] = hmul(t % qj, hinv(f % qj, qj), qj);
    S.t_mod_s[j] = shoup_of(S.t_mod[j], qj);
    S.t_theta[j] = hmul(S.t_mod[j], S.q2b.theta[j], qj);
    S.t_theta_s[j] = shoup_of(S.t_theta[j], qj);
  }
  for (u32 k = 0; k < K; ++k) {
    u64 pk = p[k];
    u64 Qm = 1;
    for (u32 j = 0; j < L; ++j) Qm = hmul(Qm, q[j] % pk, pk);
    const u64 th = S.b2q.theta[k];  // (P/p_k)^-1 mod p_k
    S.A[k] = hmul(hmul(hmul(t % pk, hinv(Qm, pk), pk), th, pk), hinv(f % pk, pk), pk);
    S.Cr[k] = th;
    for (u32 j = 0; j < L; ++j) {
      u64 v = hmul(hinv(q[j] % pk, pk), th, pk);
      S.B[j][k] = v ? pk - v : 0;
    }
  }
  for (u32 k = 0; k < K; ++k) {
    split27(S.A[k], S.A2[k]);
    split27(S.Cr[k], S.Cr2[k]);
    for (u32 j = 0; j < L; ++j) {
      split27(S.B[j][k], S.B2[j][k]);
      split27(S.b2q.hat[k][j], S.hat2[k][j]);
    }
  }
  for (u32 j = 0; j < L; ++j) split27(S.b2q.negsmod[j], S.negs2[j]);
}

}  // namespace host
}  // namespace cw
