// ntt_pass.cuh -- register-blocked negacyclic NTT passes (host/device).
//
// The transform is the one of fwd_bfly/inv_bfly in arith.cuh (same
// butterflies, same twiddles, same output order); only the schedule
// differs.  Index bit b of the transform is "butterfly bit" b: the forward
// transform processes b = n-1 down to 0 (pairs idx, idx + 2^b, group
// g = idx >> (b+1), twiddle psi[N/2^(b+1) + g]); the inverse processes
// b = 0 up to n-1.  A pass takes up to four consecutive butterfly bits:
// each of the N/16 threads holds 16 coefficients whose indices differ in a
// 4-bit window [w, w+4) that contains the pass's bits, so all butterflies
// of the pass are on registers.  Between passes the coefficients go
// through shared memory, stored with one pad word after every 16 so that
// the strided layouts of the passes are free of bank conflicts.
#pragma once
#include "arith.cuh"

namespace cw {

// shared-memory slot of coefficient i (one pad word per 16)
CW_HD u32 sidx(u32 i) { return i + (i >> 4); }
// words of shared memory for an N-point transform
CW_HD u32 smem_words(u32 N) { return N + N / 16; }

// coefficient index held in register r by thread t in a pass whose 4-bit
// window starts at bit w
CW_HD u32 pass_idx(u32 t, u32 r, u32 w) {
  return (t & ((1u << w) - 1)) | (r << w) | ((t >> w) << (w + 4));
}

// Forward butterflies for bits lo+c-1 .. lo of one thread's 16 values.
template <int LOGN>
CW_HD void fwd_pass(u64 *x, u32 t, u32 lo, u32 c, u32 w, const u64 *psi, const u64 *psi_s,
                    u64 q) {
#pragma unroll
  for (int bi = 3; bi >= 0; --bi) {
    if ((u32)bi >= c) continue;
    const u32 b = lo + bi, rb = b - w, m = 1u << (LOGN - 1 - b);
#pragma unroll
    for (u32 r = 0; r < 16; ++r) {
      if (r & (1u << rb)) continue;
      const u32 g = pass_idx(t, r, w) >> (b + 1);
      const u64 W = psi[m + g], Ws = psi_s[m + g];
      const u64 U = x[r], V = shoup(x[r | (1u << rb)], W, Ws, q);
      x[r] = addq(U, V, q);
      x[r | (1u << rb)] = subq(U, V, q);
    }
  }
}

// Inverse (Gentleman-Sande) butterflies for bits lo .. lo+c-1.
template <int LOGN>
CW_HD void inv_pass(u64 *x, u32 t, u32 lo, u32 c, u32 w, const u64 *ipsi, const u64 *ipsi_s,
                    u64 q) {
#pragma unroll
  for (int bi = 0; bi < 4; ++bi) {
    if ((u32)bi >= c) continue;
    const u32 b = lo + bi, rb = b - w, m = 1u << (LOGN - 1 - b);
#pragma unroll
    for (u32 r = 0; r < 16; ++r) {
      if (r & (1u << rb)) continue;
      const u32 g = pass_idx(t, r, w) >> (b + 1);
      const u64 U = x[r], V = x[r | (1u << rb)];
      x[r] = addq(U, V, q);
      x[r | (1u << rb)] = shoup(subq(U, V, q), ipsi[m + g], ipsi_s[m + g], q);
    }
  }
}

// Pass schedule: forward passes take bits from the top in chunks of four,
// inverse passes from the bottom; a pass of c < 4 bits uses the window
// clamped into [0, n).
template <int LOGN>
struct Passes {
  static constexpr int count = (LOGN + 3) / 4;
  CW_HD static void fwd(int p, u32 &lo, u32 &c, u32 &w) {
    int hi = LOGN - 4 * p;
    c = hi >= 4 ? 4 : hi;
    lo = hi - c;
    w = lo < LOGN - 4 ? lo : LOGN - 4;
  }
  CW_HD static void inv(int p, u32 &lo, u32 &c, u32 &w) {
    lo = 4 * p;
    c = LOGN - (int)lo >= 4 ? 4 : LOGN - lo;
    w = lo < LOGN - 4 ? lo : LOGN - 4;
  }
};

}  // namespace cw
