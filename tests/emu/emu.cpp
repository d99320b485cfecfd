// emu.cpp -- TEST-ONLY host emulation of the kernels' arithmetic.
//
// Runs the per-coefficient and per-butterfly functions of csrc/arith.cuh
// with the tables of csrc/host_tables.hpp, in the order the kernels apply
// them (stage by stage for the NTTs), so that the arithmetic of the CUDA
// path can be compared with the oracle on a machine without a GPU.  It is
// not part of the library and nothing in the product calls it.
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../paper_2202_07569_gb300/csrc/host_tables.hpp"
#include "../../paper_2202_07569_gb300/csrc/ntt_pass.cuh"

using namespace cw;
using namespace cw::host;

namespace {

struct Emu {
  u32 N, logN, L, K;
  u64 t;
  std::vector<u64> q, p, all;
  std::vector<std::vector<u64>> tw;   // per prime: 4N (value, 64-bit Shoup) pairs
  std::vector<std::vector<u32>> tw32;  // per extension prime: 4N (value, 32-bit Shoup)
  std::vector<u64> ninv, ninv_s, mu;
  std::vector<ExtPrime> ext;
  LiftTab LT;
  ScaleTab S;
  ScaleTabP SP;

  Emu(u32 N_, u32 L_, const u64 *q_, u64 t_) : N(N_), L(L_), t(t_) {
    logN = 0;
    while ((1u << logN) < N) ++logN;
    q.assign(q_, q_ + L);
    K = (u32)ext_count((int)L);
    p = ext_primes(N, K);
    all = q;
    all.insert(all.end(), p.begin(), p.end());
    for (u64 pr : all) {
      std::vector<u64> w(4 * N);
      make_twiddles(pr, N, logN, w.data());
      tw.push_back(w);
      ninv.push_back(hinv(N % pr, pr));
      ninv_s.push_back(shoup_of(ninv.back(), pr));
      mu.push_back((u64)(((u128)1 << 116) / pr));
    }
    for (u64 pr : p) {
      std::vector<u32> w(4 * N);
      make_twiddles32(pr, N, logN, w.data());
      tw32.push_back(w);
      ext.push_back(ext_prime(pr));
    }
    fill_lift(LT, q, p);
    fill_scale(S, q, p, t, N);
    fill_scale_p(SP, q, p, t, N);
  }
  void fwd(u64 *a, u32 l) {
    const u64 *w = tw[l].data();
    for (u32 st = 0; st < logN; ++st)
      for (u32 b = 0; b < N / 2; ++b) fwd_bfly(a, b, logN - 1 - st, 1u << st, w, all[l]);
  }
  void inv(u64 *a, u32 l) {
    const u64 *w = tw[l].data();
    for (u32 st = 0; st < logN; ++st)
      for (u32 b = 0; b < N / 2; ++b) inv_bfly(a, b, st, N >> (st + 1), w + 2 * N, all[l]);
    for (u32 c = 0; c < N; ++c) a[c] = shoup(a[c], ninv[l], ninv_s[l], all[l]);
  }
  // coefficient ct [2][L][N] -> QP-NTT [2][L+K][N]
  void to_qp(const u64 *ct, u64 *out) {
    const u32 LK = L + K;
    u64 x[kMaxL], y[kMaxK];
    for (u32 poly = 0; poly < 2; ++poly) {
      for (u32 c = 0; c < N; ++c) {
        for (u32 j = 0; j < L; ++j) x[j] = ct[(poly * L + j) * N + c];
        lift(x, y);
        for (u32 j = 0; j < L; ++j) out[(poly * LK + j) * N + c] = x[j];
        for (u32 k = 0; k < K; ++k) out[(poly * LK + L + k) * N + c] = y[k];
      }
      for (u32 l = 0; l < LK; ++l) fwd(out + (poly * LK + l) * N, l);
    }
  }
  void lift(const u64 *x, u64 *y) {
    u32 y32[kMaxK];
    switch (L) {
      case 1: lift_ext<1, ext_count(1)>(x, y32, LT); break;
      case 2: lift_ext<2, ext_count(2)>(x, y32, LT); break;
      case 3: lift_ext<3, ext_count(3)>(x, y32, LT); break;
      case 4: lift_ext<4, ext_count(4)>(x, y32, LT); break;
      case 5: lift_ext<5, ext_count(5)>(x, y32, LT); break;
      case 6: lift_ext<6, ext_count(6)>(x, y32, LT); break;
      case 7: lift_ext<7, ext_count(7)>(x, y32, LT); break;
      default: lift_ext<8, ext_count(8)>(x, y32, LT); break;
    }
    for (u32 k = 0; k < K; ++k) y[k] = y32[k];
  }
  bool scale(const u64 *dq, const u64 *dp, u64 *e) {
    switch (L) {
      case 1: return scale_coeff<1>(dq, dp, e, S);
      case 2: return scale_coeff<2>(dq, dp, e, S);
      case 3: return scale_coeff<3>(dq, dp, e, S);
      case 4: return scale_coeff<4>(dq, dp, e, S);
      case 5: return scale_coeff<5>(dq, dp, e, S);
      case 6: return scale_coeff<6>(dq, dp, e, S);
      case 7: return scale_coeff<7>(dq, dp, e, S);
      default: return scale_coeff<8>(dq, dp, e, S);
    }
  }
  // The kernels' scale-down from the extension residues dp (N d mod p_k,
  // lazy): 0 = fast path, 1 = exact path (always with force_exact), -1 =
  // a failed check.
  int scale_p(const u32 *dp, u64 *e, bool force_exact) {
    int r = 1;
    switch (L) {
#define CW_EMU_SCALE(LL)                                                          \
  case LL:                                                                        \
    if (!force_exact) r = scale_fast<LL>(dp, e, SP);                              \
    if (r == 1) return scale_exact<LL>(dp, e, SP, S) ? 1 : -1;                    \
    return r == 0 ? 0 : -1;
      CW_EMU_SCALE(1) CW_EMU_SCALE(2) CW_EMU_SCALE(3) CW_EMU_SCALE(4)
      CW_EMU_SCALE(5) CW_EMU_SCALE(6) CW_EMU_SCALE(7) CW_EMU_SCALE(8)
#undef CW_EMU_SCALE
    }
    return -1;
  }
  // key [L][2][L][N] coefficient -> NTT + Shoup companions
  void prep_key(const u64 *key, std::vector<u64> &k, std::vector<u64> &ks) {
    k.assign(key, key + 2ull * L * L * N);
    ks.assign(k.size(), 0);
    for (u32 unit = 0; unit < 2 * L; ++unit)
      for (u32 j = 0; j < L; ++j) {
        u64 *a = k.data() + ((u64)unit * L + j) * N;
        fwd(a, j);
        for (u32 c = 0; c < N; ++c) ks[((u64)unit * L + j) * N + c] = shoup_of(a[c], q[j]);
      }
  }
  // key switch of z ([L][N] coefficient digits) plus optional addends,
  // result in coefficient form [2][L][N]
  void keyswitch(const u64 *z, const u64 *add0, const u64 *add1, const std::vector<u64> &k,
                 const std::vector<u64> &ks, u64 *out) {
    std::vector<u64> s(N), a0(N), a1(N);
    for (u32 j = 0; j < L; ++j) {
      u64 qj = q[j];
      std::fill(a0.begin(), a0.end(), 0);
      std::fill(a1.begin(), a1.end(), 0);
      for (u32 i = 0; i < L; ++i) {
        for (u32 c = 0; c < N; ++c) {
          u64 d = z[(u64)i * N + c];
          s[c] = d >= qj ? d - qj : d;
        }
        fwd(s.data(), j);
        const u64 *kb = k.data() + ((u64)(i * 2) * L + j) * N, *ka = kb + (u64)L * N;
        const u64 *kbs = ks.data() + ((u64)(i * 2) * L + j) * N, *kas = kbs + (u64)L * N;
        for (u32 c = 0; c < N; ++c) {
          a0[c] = addq(a0[c], shoup(s[c], kb[c], kbs[c], qj), qj);
          a1[c] = addq(a1[c], shoup(s[c], ka[c], kas[c], qj), qj);
        }
      }
      for (int comp = 0; comp < 2; ++comp) {
        const u64 *ad = comp ? add1 : add0;
        if (!ad) continue;
        memcpy(s.data(), ad + (u64)j * N, N * 8);
        fwd(s.data(), j);
        std::vector<u64> &acc = comp ? a1 : a0;
        for (u32 c = 0; c < N; ++c) acc[c] = addq(acc[c], s[c], qj);
      }
      inv(a0.data(), j);
      inv(a1.data(), j);
      memcpy(out + (u64)j * N, a0.data(), N * 8);
      memcpy(out + ((u64)L + j) * N, a1.data(), N * 8);
    }
  }
};

}  // namespace

extern "C" {

// One homomorphic multiplication in the kernels' order: the tensor on the
// extension limbs alone, the scale-down from them (every coefficient through
// the exact path when force_exact), the key switch.  Returns 0, or 1 if a
// scale-down check tripped.
int emu_bfv_mul(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t, const uint64_t *rlk,
                const uint64_t *a, const uint64_t *b, uint64_t *out, int force_exact) {
  Emu E(N, L, q, t);
  const u32 LK = L + E.K;
  std::vector<u64> A(2ull * LK * N), B(2ull * LK * N);
  E.to_qp(a, A.data());
  E.to_qp(b, B.data());
  std::vector<u32> Tb(3ull * E.K * N);
  std::vector<u64> o(N), Eb(3ull * L * N);
  for (u32 which = 0; which < 3; ++which)
    for (u32 k = 0; k < E.K; ++k) {
      const u32 l = L + k;
      const u64 pr = E.all[l];
      const u64 *a0 = A.data() + (u64)l * N, *a1 = a0 + (u64)LK * N;
      const u64 *b0 = B.data() + (u64)l * N, *b1 = b0 + (u64)LK * N;
      // the kernels' 32-bit products, lazy [0, 2p)
      const ExtPrime &X = E.ext[k];
      const u32 p2 = 2 * X.p;
      for (u32 c = 0; c < N; ++c) {
        u32 v;
        if (which == 0) v = mulmod_ext_lazy((u32)a0[c], (u32)b0[c], X);
        else if (which == 2) v = mulmod_ext_lazy((u32)a1[c], (u32)b1[c], X);
        else {
          v = reduce_ext62_lazy(wmul((u32)a0[c], (u32)b1[c]) + wmul((u32)a1[c], (u32)b0[c]), X);
          v = v >= p2 ? v - p2 : v;
        }
        o[c] = v >= X.p ? v - X.p : v;
      }
      E.inv(o.data(), l);  // canonical d; the scale-down takes N d as the kernels hand it over
      for (u32 c = 0; c < N; ++c)
        Tb[((u64)which * E.K + k) * N + c] = (u32)(hmul(o[c], N % pr, pr) + ((c & 1) ? pr : 0));
    }
  int bad = 0;
  u32 dp[kMaxK];
  u64 e[kMaxL];
  for (u32 which = 0; which < 3; ++which)
    for (u32 c = 0; c < N; ++c) {
      for (u32 k = 0; k < E.K; ++k) dp[k] = Tb[((u64)which * E.K + k) * N + c];
      if (E.scale_p(dp, e, force_exact != 0) < 0) bad = 1;
      for (u32 j = 0; j < L; ++j) Eb[((u64)which * L + j) * N + c] = e[j];
    }
  std::vector<u64> k, ks;
  E.prep_key(rlk, k, ks);
  E.keyswitch(Eb.data() + 2ull * L * N, Eb.data(), Eb.data() + (u64)L * N, k, ks, out);
  return bad;
}

// The scale-down from the extension residues for n coefficients: dp [n][K]
// (N d mod p_k, below 2^31), out [n][L]; path[i] = 0 (fast), 1 (exact),
// -1 (a failed check).
void emu_scale_p(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t, uint64_t n,
                 const uint32_t *dp, uint64_t *out, int force_exact, int32_t *path) {
  Emu E(N, L, q, t);
  for (u64 i = 0; i < n; ++i)
    path[i] = E.scale_p(dp + i * E.K, out + i * L, force_exact != 0);
}

// Centered Q -> P conversion of one coefficient vector ([L] residues).
void emu_lift(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t, const uint64_t *x,
              uint64_t *y) {
  Emu E(N, L, q, t);
  E.lift(x, y);
}

// The number of extension primes and the primes the library chooses for
// these parameters (p holds ext_count(L) entries).
uint32_t emu_ext_count(uint32_t L) { return (uint32_t)ext_count((int)L); }
void emu_ext_primes(uint32_t N, uint32_t L, const uint64_t *q, uint64_t *p) {
  (void)q;
  std::vector<u64> v = ext_primes(N, (u32)ext_count((int)L));
  for (u32 i = 0; i < v.size(); ++i) p[i] = v[i];
}

// Sub_g: automorphism then key switch with the Galois key (coefficient form).
void emu_substitute(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t, uint32_t g,
                    const uint64_t *gkey, const uint64_t *ct, uint64_t *out) {
  Emu E(N, L, q, t);
  std::vector<u64> tau(2ull * L * N);
  for (u32 pl = 0; pl < 2 * L; ++pl) {
    u64 qj = q[pl % L];
    for (u32 i = 0; i < N; ++i) {
      u64 v = ct[(u64)pl * N + i];
      u32 e = (u32)(((u64)i * g) & (2ull * N - 1));
      if (e >= N) {
        e -= N;
        v = v ? qj - v : 0;
      }
      tau[(u64)pl * N + e] = v;
    }
  }
  std::vector<u64> k, ks;
  E.prep_key(gkey, k, ks);
  E.keyswitch(tau.data() + (u64)L * N, tau.data(), nullptr, k, ks, out);
}

}  // extern "C"

extern "C" {
// Rows per group that the row basis of nr primes holds exactly.
uint64_t emu_row_limit(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t, uint32_t nr) {
  Emu E(N, L, q, t);
  return row_group_limit(E.q, E.p, nr, N, t);
}

// reduce_ext62 on `count` values below 2^62 for the 30-bit prime p.
void emu_reduce62(uint64_t p, const uint64_t *v, uint64_t count, uint32_t *out) {
  const ExtPrime E = ext_prime(p);
  for (uint64_t i = 0; i < count; ++i) out[i] = reduce_ext62(v[i], E);
}

// x mod q_j (j < L) from N x mod the nr row primes (lazy below 2r);
// returns 1 if the fixed-point check tripped.
int emu_row_crt(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t, uint32_t nr,
                const uint32_t *xr, uint64_t *out) {
  Emu E(N, L, q, t);
  RowTab T;
  fill_rows(T, E.q, E.p, N, nr);
  u32 y[kRowPrimes];
  bool far;
  const u64 rho = row_digits(xr, y, T, &far);
  for (u32 j = 0; j < L; ++j) out[j] = row_to_q(y, rho, (int)j, T);
  return far ? 1 : 0;
}

// round(t d / Q) mod q_j for one coefficient given by its residues mod the
// q_j (dq) and the extension primes (dp); returns 0 if the check tripped.
int emu_scale(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t, const uint64_t *dq,
              const uint64_t *dp, uint64_t *out) {
  Emu E(N, L, q, t);
  return E.scale(dq, dp, out) ? 1 : 0;
}
}

namespace {
// The register-blocked schedule of the kernels, thread by thread: every
// pass reads the thread's 2^RB slots, runs its butterflies, writes them back.
template <int LOGN, int RB>
void pass_ntt(u64 *a, const u64 *tw, u64 q, bool inverse, u64 ninv, u64 ninv_s) {
  constexpr u32 R = 1u << RB;
  const u32 N = 1u << LOGN, T = N / R;
  std::vector<u64> s(smem_words<RB>(N));
  for (u32 i = 0; i < N; ++i) s[sidx<RB>(i)] = a[i];
  for (int p = 0; p < Passes<LOGN, RB>::count; ++p) {
    u32 lo, c, w;
    if (inverse) Passes<LOGN, RB>::inv(p, lo, c, w);
    else Passes<LOGN, RB>::fwd(p, lo, c, w);
    for (u32 t = 0; t < T; ++t) {
      u64 x[R];
      for (u32 r = 0; r < R; ++r) x[r] = s[sidx<RB>(pass_idx<RB>(t, r, w))];
      if (inverse) inv_pass<LOGN, RB>(x, t, lo, c, w, tw + 2 * N, q);
      else fwd_pass<LOGN, RB>(x, t, lo, c, w, tw, q);
      if (p == Passes<LOGN, RB>::count - 1)
        for (u32 r = 0; r < R; ++r)
          x[r] = inverse ? shoup(x[r], ninv, ninv_s, q) : reduce4(x[r], q);
      for (u32 r = 0; r < R; ++r) s[sidx<RB>(pass_idx<RB>(t, r, w))] = x[r];
    }
  }
  for (u32 i = 0; i < N; ++i) a[i] = s[sidx<RB>(i)];
}

// The 32-bit schedule of the extension primes (forward from [0, 4p) to
// canonical; inverse from [0, 2p) to N times the coefficient in [0, 2p)).
template <int LOGN, int RB>
void pass_ntt32(u32 *a, const u32 *tw, u32 p, bool inverse) {
  constexpr u32 R = 1u << RB;
  const u32 N = 1u << LOGN, T = N / R;
  std::vector<u32> s(smem_words<RB>(N));
  for (u32 i = 0; i < N; ++i) s[sidx<RB>(i)] = a[i];
  for (int pp = 0; pp < Passes<LOGN, RB>::count; ++pp) {
    u32 lo, c, w;
    if (inverse) Passes<LOGN, RB>::inv(pp, lo, c, w);
    else Passes<LOGN, RB>::fwd(pp, lo, c, w);
    for (u32 t = 0; t < T; ++t) {
      u32 x[R];
      for (u32 r = 0; r < R; ++r) x[r] = s[sidx<RB>(pass_idx<RB>(t, r, w))];
      if (inverse) inv_pass32<LOGN, RB>(x, t, lo, c, w, tw + 2 * N, p);
      else fwd_pass32<LOGN, RB>(x, t, lo, c, w, tw, p);
      if (pp == Passes<LOGN, RB>::count - 1 && !inverse)
        for (u32 r = 0; r < R; ++r) x[r] = reduce4_32(x[r], p);
      for (u32 r = 0; r < R; ++r) s[sidx<RB>(pass_idx<RB>(t, r, w))] = x[r];
    }
  }
  for (u32 i = 0; i < N; ++i) a[i] = s[sidx<RB>(i)];
}

// Three 32-bit inverse transforms of one prime in lock-step (inv_pass32m),
// thread by thread as the extension tensor runs them: registers per
// thread, exchanges through one shared array per transform with the
// tensor's slot mapping (xslot) between the windows of consecutive passes;
// a slot collision or an out-of-range slot would corrupt the result.
template <int LOGN, int RB>
void pass_ntt32_x3(u32 *a, const u32 *tw, u32 p) {
  constexpr u32 R = 1u << RB;
  const u32 N = 1u << LOGN, T = N / R, SW = smem_words<RB>(N);
  std::vector<u32> reg(3ull * T * R), s(3ull * SW, 0xFFFFFFFFu);
  u32 lo, c, w, wprev = 0;
  Passes<LOGN, RB>::inv(0, lo, c, w);
  for (u32 t = 0; t < T; ++t)
    for (int i = 0; i < 3; ++i)
      for (u32 r = 0; r < R; ++r) reg[(t * 3 + i) * R + r] = a[i * N + pass_idx<RB>(t, r, w)];
  for (int pp = 0; pp < Passes<LOGN, RB>::count; ++pp) {
    Passes<LOGN, RB>::inv(pp, lo, c, w);
    if (pp > 0) {
      for (u32 t = 0; t < T; ++t)
        for (int i = 0; i < 3; ++i)
          for (u32 r = 0; r < R; ++r) {
            const u32 slot = xslot<RB>(pass_idx<RB>(t, r, wprev), wprev, w);
            if (slot >= SW) return;  // leaves a unchanged: the caller's comparison fails
            s[i * SW + slot] = reg[(t * 3 + i) * R + r];
          }
      for (u32 t = 0; t < T; ++t)
        for (int i = 0; i < 3; ++i)
          for (u32 r = 0; r < R; ++r)
            reg[(t * 3 + i) * R + r] = s[i * SW + xslot<RB>(pass_idx<RB>(t, r, w), wprev, w)];
    }
    for (u32 t = 0; t < T; ++t) inv_pass32m<LOGN, RB, 3>(&reg[t * 3 * R], t, lo, c, w, tw + 2 * N, p);
    wprev = w;
  }
  for (u32 t = 0; t < T; ++t)
    for (int i = 0; i < 3; ++i)
      for (u32 r = 0; r < R; ++r) a[i * N + pass_idx<RB>(t, r, wprev)] = reg[(t * 3 + i) * R + r];
}

template <int RB>
void pass_ntt32_n(u32 logN, u32 *a, const u32 *tw, u32 p, bool inverse) {
  switch (logN) {
    case 10: pass_ntt32<10, RB>(a, tw, p, inverse); break;
    case 11: pass_ntt32<11, RB>(a, tw, p, inverse); break;
    case 12: pass_ntt32<12, RB>(a, tw, p, inverse); break;
    case 13: pass_ntt32<13, RB>(a, tw, p, inverse); break;
    default: pass_ntt32<14, RB>(a, tw, p, inverse); break;
  }
}

template <int RB>
void pass_ntt_n(u32 logN, u64 *a, const u64 *tw, u64 q, bool inverse, u64 ninv, u64 ninv_s) {
  switch (logN) {
    case 10: pass_ntt<10, RB>(a, tw, q, inverse, ninv, ninv_s); break;
    case 11: pass_ntt<11, RB>(a, tw, q, inverse, ninv, ninv_s); break;
    case 12: pass_ntt<12, RB>(a, tw, q, inverse, ninv, ninv_s); break;
    case 13: pass_ntt<13, RB>(a, tw, q, inverse, ninv, ninv_s); break;
    default: pass_ntt<14, RB>(a, tw, q, inverse, ninv, ninv_s); break;
  }
}
}  // namespace

extern "C" {
// Runs the pass schedule (windows of rb = 4 or 5 bits) and the stage-by-
// stage transform on the same data for every prime of the parameter set;
// returns the number of mismatches.
uint64_t emu_ntt_compare(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t,
                         const uint64_t *data, uint32_t rb) {
  Emu E(N, L, q, t);
  uint64_t bad = 0;
  auto run = rb == 4 ? pass_ntt_n<4> : pass_ntt_n<5>;
  auto run32 = rb == 4 ? pass_ntt32_n<4> : pass_ntt32_n<5>;
  for (u32 l = 0; l < E.all.size(); ++l) {
    u64 pr = E.all[l];
    if (l >= L) {  // extension prime: the 32-bit schedule
      std::vector<u64> a(N);
      std::vector<u32> b(N);
      for (u32 i = 0; i < N; ++i) {
        a[i] = data[i] % pr;
        b[i] = (u32)(a[i] + (data[i] >> 62) * pr);  // lazy input below 4p
      }
      E.fwd(a.data(), l);
      run32(E.logN, b.data(), E.tw32[l - L].data(), (u32)pr, false);
      for (u32 i = 0; i < N; ++i) bad += a[i] != b[i];
      for (u32 i = 0; i < N; ++i) b[i] += (u32)(((data[i] >> 59) & 1) * pr);  // below 2p
      E.inv(a.data(), l);
      run32(E.logN, b.data(), E.tw32[l - L].data(), (u32)pr, true);
      // the 32-bit inverse leaves N times the coefficient in [0, 2p)
      for (u32 i = 0; i < N; ++i)
        bad += b[i] >= 2 * pr || b[i] % pr != hmul(a[i], N % pr, pr) ||
               a[i] != data[i] % pr;
      continue;
    }
    std::vector<u64> a(N), b(N);
    // the schedule accepts lazy inputs: below 4q forward, below 2q inverse
    for (u32 i = 0; i < N; ++i) {
      a[i] = data[i] % pr;
      b[i] = a[i] + (data[i] >> 62) * pr;
    }
    E.fwd(a.data(), l);
    run(E.logN, b.data(), E.tw[l].data(), pr, false, 0, 0);
    for (u32 i = 0; i < N; ++i) bad += a[i] != b[i];
    for (u32 i = 0; i < N; ++i) b[i] += ((data[i] >> 59) & 1) * pr;
    E.inv(a.data(), l);
    run(E.logN, b.data(), E.tw[l].data(), pr, true, E.ninv[l], E.ninv_s[l]);
    for (u32 i = 0; i < N; ++i) bad += a[i] != b[i] || b[i] != data[i] % pr;
  }
  return bad;
}
}

extern "C" {
// The tensor kernel's inverse transforms (N = 2^logN, logN 13 or 14, 16
// coefficients a thread): the three-transform 32-bit schedule with the
// kernel's exchanges on every extension prime must leave each of three
// inputs (below 2p) as the single schedule does.  Returns the number of
// mismatches.
uint64_t emu_tensor_intt_compare(uint32_t logN, uint32_t L, const uint64_t *q, uint64_t t,
                                 const uint64_t *data) {
  const u32 N = 1u << logN;
  Emu E(N, L, q, t);
  uint64_t bad = 0;
  for (u32 k = 0; k < E.K; ++k) {
    const u64 pr = E.p[k];
    std::vector<u32> x3(3 * N), x1(N);
    for (u32 i = 0; i < 3 * N; ++i) x3[i] = (u32)(data[(7 * i + 3) % 8192] % (2 * pr));  // below 2p
    std::vector<u32> y(x3);
    if (logN == 13) pass_ntt32_x3<13, 4>(y.data(), E.tw32[k].data(), (u32)pr);
    else pass_ntt32_x3<14, 4>(y.data(), E.tw32[k].data(), (u32)pr);
    for (int j = 0; j < 3; ++j) {
      for (u32 i = 0; i < N; ++i) x1[i] = x3[j * N + i];
      if (logN == 13) pass_ntt32<13, 4>(x1.data(), E.tw32[k].data(), (u32)pr, true);
      else pass_ntt32<14, 4>(x1.data(), E.tw32[k].data(), (u32)pr, true);
      for (u32 i = 0; i < N; ++i) bad += y[j * N + i] != x1[i];
    }
  }
  return bad;
}
}

extern "C" {
// The row-basis path of the last tree level for one polynomial limb: out =
// sum_r z_r * lift(db_r) mod q_j (negacyclic, j < L) through the row
// primes, in the order of the row kernels: each limb z_r (below 2^62)
// reduced modulo r_k and transformed, each row centered-lifted and
// transformed, the pointwise products summed modulo r_k, the sum inverse-
// transformed (N x in [0, 2r)), and the exact CRT to the q_j.  z:
// [rows][N] u64, db: [rows][N] u32 below t, out: [L][N].  Returns the
// number of coefficients whose fixed-point check tripped.
uint64_t emu_row_sum(uint32_t N, uint32_t L, const uint64_t *q, uint64_t t, uint32_t nr,
                     uint64_t rows, const uint64_t *z, const uint32_t *db, uint64_t *out) {
  Emu E(N, L, q, t);
  RowTab T;
  fill_rows(T, E.q, E.p, N, nr);
  std::vector<u32> x((u64)nr * N), a(N), b(N);
  for (u32 k = 0; k < nr; ++k) {
    const ExtPrime &P = T.r[k];
    const u32 p = P.p;
    std::vector<u64> acc(N, 0);
    for (u64 r = 0; r < rows; ++r) {
      for (u32 c = 0; c < N; ++c) {
        a[c] = reduce_ext62(z[r * N + c], P);
        const u32 v = db[r * N + c];
        b[c] = v > (u32)t / 2 ? p - (u32)(t - v) : v;
      }
      pass_ntt32_n<4>(E.logN, a.data(), E.tw32[k].data(), p, false);
      pass_ntt32_n<4>(E.logN, b.data(), E.tw32[k].data(), p, false);
      for (u32 c = 0; c < N; ++c) acc[c] = reduce_ext(acc[c] + (u64)a[c] * b[c], P);
    }
    for (u32 c = 0; c < N; ++c) a[c] = (u32)acc[c];
    pass_ntt32_n<4>(E.logN, a.data(), E.tw32[k].data(), p, true);
    for (u32 c = 0; c < N; ++c) x[(u64)c * nr + k] = a[c];
  }
  uint64_t tripped = 0;
  for (u32 c = 0; c < N; ++c) {
    u32 xr[kRowPrimes] = {0, 0, 0, 0}, y[kRowPrimes];
    for (u32 k = 0; k < nr; ++k) xr[k] = x[(u64)c * nr + k];
    bool far;
    const u64 rho = row_digits(xr, y, T, &far);
    tripped += far;
    for (u32 j = 0; j < L; ++j) out[(u64)j * N + c] = row_to_q(y, rho, (int)j, T);
  }
  return tripped;
}
}
