// ntt_pass.cuh -- register-blocked negacyclic NTT passes (host/device).
//
// The transform is the one of fwd_bfly/inv_bfly in arith.cuh (same
// butterflies, same twiddles, same output order); only the schedule
// differs.  Index bit b of the transform is "butterfly bit" b: the forward
// transform processes b = n-1 down to 0 (pairs idx, idx + 2^b, group
// g = idx >> (b+1), twiddle psi[N/2^(b+1) + g]); the inverse processes
// b = 0 up to n-1.  A pass takes up to RB consecutive butterfly bits: each
// of the N/2^RB threads holds R = 2^RB coefficients whose indices differ in
// an RB-bit window [w, w+RB) that contains the pass's bits, so all
// butterflies of the pass are on registers.  Between passes the
// coefficients go through shared memory, stored with one pad word after
// every R so that the strided layouts of the passes are free of bank
// conflicts.
#pragma once
#include "arith.cuh"

namespace cw {

// shared-memory slot of coefficient i (one pad word per 2^RB)
template <int RB>
CW_HD u32 sidx(u32 i) { return i + (i >> RB); }
// Shared-memory slot of coefficient i in an exchange of 32-bit words
// between the layouts of windows wa and wb: one pad word per 16 (a warp's
// indices are strided when a window is below 5) or, when both windows are
// at least 5 (a warp then touches 32 consecutive indices, which one pad
// per 16 puts two to a bank), one per 32.  Used by the extension tensor
// (tensor 82.3 -> 81.4 ms per metric answer); in the single-transform
// kernels its addressing cost registers (the row transforms 63.3 -> 67.1 ms).
template <int RB>
CW_HD u32 xslot(u32 i, u32 wa, u32 wb) {
  return (wa >= 5 && wb >= 5) ? i + (i >> 5) : sidx<RB>(i);
}

// words of shared memory for an N-point transform
template <int RB>
CW_HD u32 smem_words(u32 N) { return N + (N >> RB); }

// coefficient index held in register r by thread t in a pass whose RB-bit
// window starts at bit w
template <int RB>
CW_HD u32 pass_idx(u32 t, u32 r, u32 w) {
  return (t & ((1u << w) - 1)) | (r << w) | ((t >> w) << (w + RB));
}
// One (twiddle, Shoup companion) pair: a 16-byte read-only load on the
// device.
CW_HD void ld_pair(const u64 *p, u64 &a, u64 &b) {
#if defined(__CUDA_ARCH__)
  const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(p));
  a = v.x;
  b = v.y;
#else
  a = p[0];
  b = p[1];
#endif
}

// Shoup product without the final correction: a*w mod q in [0, 2q) for any
// a < 2^64.
CW_HD u64 shoup_lazy(u64 a, u64 w, u64 ws, u64 q) { return a * w - mulhi(a, ws) * q; }

// Forward butterflies (Harvey's lazy Cooley-Tukey) for bits lo+c-1 .. lo of
// one thread's 2^RB values: values stay in [0, 4q) (q < 2^54 keeps 4q far
// below 2^64); U is brought into [0, 2q), V = W x in [0, 2q), outputs
// U + V and U - V + 2q.
template <int LOGN, int RB>
CW_HD void fwd_pass(u64 *x, u32 t, u32 lo, u32 c, u32 w, const u64 *psi2, u64 q) {
  const u64 q2 = 2 * q;
  constexpr u32 R = 1u << RB;
#pragma unroll
  for (int bi = RB - 1; bi >= 0; --bi) {
    if ((u32)bi >= c) continue;
    const u32 b = lo + bi, rb = b - w, m = 1u << (LOGN - 1 - b);
    // registers r and r | 2^rb pair up; the twiddle depends only on the
    // bits of r above rb, so each distinct twiddle is loaded once
#pragma unroll
    for (u32 hv = 0; hv < (R >> (rb + 1)); ++hv) {
      const u32 r0 = hv << (rb + 1);
      const u32 g = pass_idx<RB>(t, r0, w) >> (b + 1);
      u64 W, Ws;
      ld_pair(psi2 + 2 * (m + g), W, Ws);
#pragma unroll
      for (u32 lv = 0; lv < (1u << rb); ++lv) {
        const u32 r = r0 | lv;
        u64 U = x[r];
        U = U >= q2 ? U - q2 : U;
        const u64 V = shoup_lazy(x[r | (1u << rb)], W, Ws, q);
        x[r] = U + V;
        x[r | (1u << rb)] = U - V + q2;
      }
    }
  }
}

// Inverse butterflies (lazy Gentleman-Sande) for bits lo .. lo+c-1: inputs
// and outputs in [0, 2q); U + V is brought back into [0, 2q), the difference
// U - V + 2q < 4q goes through a lazy Shoup product.
template <int LOGN, int RB>
CW_HD void inv_pass(u64 *x, u32 t, u32 lo, u32 c, u32 w, const u64 *ipsi2, u64 q) {
  const u64 q2 = 2 * q;
  constexpr u32 R = 1u << RB;
#pragma unroll
  for (int bi = 0; bi < RB; ++bi) {
    if ((u32)bi >= c) continue;
    const u32 b = lo + bi, rb = b - w, m = 1u << (LOGN - 1 - b);
#pragma unroll
    for (u32 hv = 0; hv < (R >> (rb + 1)); ++hv) {
      const u32 r0 = hv << (rb + 1);
      const u32 g = pass_idx<RB>(t, r0, w) >> (b + 1);
      u64 W, Ws;
      ld_pair(ipsi2 + 2 * (m + g), W, Ws);
#pragma unroll
      for (u32 lv = 0; lv < (1u << rb); ++lv) {
        const u32 r = r0 | lv;
        const u64 U = x[r], V = x[r | (1u << rb)];
        const u64 S = U + V;
        x[r] = S >= q2 ? S - q2 : S;
        x[r | (1u << rb)] = shoup_lazy(U - V + q2, W, Ws, q);
      }
    }
  }
}

// [0, 4q) -> [0, q)
CW_HD u64 reduce4(u64 v, u64 q) {
  const u64 q2 = 2 * q;
  v = v >= q2 ? v - q2 : v;
  return v >= q ? v - q : v;
}

// ---- the same passes on 32-bit words, for the 30-bit extension primes
// (p < 2^30 keeps 4p below 2^32); twiddles are (w, floor(w 2^32 / p)) pairs.
CW_HD void ld_pair32(const u32 *p, u32 &a, u32 &b) {
#if defined(__CUDA_ARCH__)
  const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
  a = v.x;
  b = v.y;
#else
  a = p[0];
  b = p[1];
#endif
}

// Two consecutive (twiddle, Shoup) pairs from an even pair index: one
// 16-byte load on the device.
CW_HD void ld_pair32x2(const u32 *p, u32 &a0, u32 &b0, u32 &a1, u32 &b1) {
#if defined(__CUDA_ARCH__)
  const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
  a0 = v.x;
  b0 = v.y;
  a1 = v.z;
  b1 = v.w;
#else
  a0 = p[0];
  b0 = p[1];
  a1 = p[2];
  b1 = p[3];
#endif
}

// a*w mod p in [0, 2p) for any a < 2^32
CW_HD u32 shoup32_lazy(u32 a, u32 w, u32 ws, u32 p) { return a * w - mulhi32(a, ws) * p; }

template <int LOGN, int RB>
CW_HD void fwd_pass32(u32 *x, u32 t, u32 lo, u32 c, u32 w, const u32 *psi2, u32 p) {
  const u32 p2 = 2 * p;
  constexpr u32 R = 1u << RB;
#pragma unroll
  for (int bi = RB - 1; bi >= 0; --bi) {
    if ((u32)bi >= c) continue;
    const u32 b = lo + bi, rb = b - w, m = 1u << (LOGN - 1 - b);
    // the level's twiddles of this thread: R >> (rb + 1) consecutive pairs
    // from m + ((t >> w) << (RB - 1 - rb)) (hv fills the low bits of
    // pass_idx >> (b + 1)); with two or more of them b <= LOGN - 2, so m
    // and the start are even and two pairs come in one 16-byte load
    const u32 nh = R >> (rb + 1), g0 = m + ((t >> w) << (RB - 1 - rb));
#pragma unroll
    for (u32 hv = 0; hv < nh; hv += 2) {
      u32 W[2], Ws[2];
      if (nh == 1) ld_pair32(psi2 + 2 * g0, W[0], Ws[0]);
      else ld_pair32x2(psi2 + 2 * (g0 + hv), W[0], Ws[0], W[1], Ws[1]);
#pragma unroll
      for (u32 h = 0; h < 2 && hv + h < nh; ++h) {
        const u32 r0 = (hv + h) << (rb + 1);
#pragma unroll
        for (u32 lv = 0; lv < (1u << rb); ++lv) {
          const u32 r = r0 | lv;
          const u32 U = csub32(x[r], p2);
          const u32 V = shoup32_lazy(x[r | (1u << rb)], W[h], Ws[h], p);
          x[r] = U + V;
          x[r | (1u << rb)] = U - V + p2;
        }
      }
    }
  }
}

// Inverse butterflies on M transforms of the same prime at once (one
// twiddle load serves the M butterflies): x[i * R + r] is register r of
// transform i.
template <int LOGN, int RB, int M>
CW_HD void inv_pass32m(u32 *x, u32 t, u32 lo, u32 c, u32 w, const u32 *ipsi2, u32 p) {
  const u32 p2 = 2 * p;
  constexpr u32 R = 1u << RB;
#pragma unroll
  for (int bi = 0; bi < RB; ++bi) {
    if ((u32)bi >= c) continue;
    const u32 b = lo + bi, rb = b - w, m = 1u << (LOGN - 1 - b);
    const u32 nh = R >> (rb + 1), g0 = m + ((t >> w) << (RB - 1 - rb));
#pragma unroll
    for (u32 hv = 0; hv < nh; hv += 2) {
      u32 W[2], Ws[2];
      if (nh == 1) ld_pair32(ipsi2 + 2 * g0, W[0], Ws[0]);
      else ld_pair32x2(ipsi2 + 2 * (g0 + hv), W[0], Ws[0], W[1], Ws[1]);
#pragma unroll
      for (u32 h = 0; h < 2 && hv + h < nh; ++h) {
        const u32 r0 = (hv + h) << (rb + 1);
#pragma unroll
        for (u32 lv = 0; lv < (1u << rb); ++lv) {
#pragma unroll
          for (int i = 0; i < M; ++i) {
            const u32 r = i * R + (r0 | lv);
            const u32 U = x[r], V = x[r + (1u << rb)];
            x[r] = csub32(U + V, p2);
            x[r + (1u << rb)] = shoup32_lazy(U - V + p2, W[h], Ws[h], p);
          }
        }
      }
    }
  }
}

template <int LOGN, int RB>
CW_HD void inv_pass32(u32 *x, u32 t, u32 lo, u32 c, u32 w, const u32 *ipsi2, u32 p) {
  inv_pass32m<LOGN, RB, 1>(x, t, lo, c, w, ipsi2, p);
}

CW_HD u32 reduce4_32(u32 v, u32 p) { return csub32(csub32(v, 2 * p), p); }

// Pass schedule: forward passes take bits from the top in chunks of RB,
// inverse passes from the bottom; a pass of c < RB bits uses the window
// clamped into [0, n).
template <int LOGN, int RB>
struct Passes {
  static constexpr int count = (LOGN + RB - 1) / RB;
  CW_HDM static void fwd(int p, u32 &lo, u32 &c, u32 &w) {
    int hi = LOGN - RB * p;
    c = hi >= RB ? RB : hi;
    lo = hi - c;
    w = lo < LOGN - RB ? lo : LOGN - RB;
  }
  CW_HDM static void inv(int p, u32 &lo, u32 &c, u32 &w) {
    lo = RB * p;
    c = LOGN - (int)lo >= RB ? RB : LOGN - lo;
    w = lo < LOGN - RB ? lo : LOGN - RB;
  }
};

// Shape of the device transforms of length 2^LOGN: 2^RB coefficients per
// thread, N / 2^RB threads per block, at least min_blocks resident blocks
// per SM (64 registers per thread up to N = 8192).  Sixteen coefficients
// per thread: with 32 (256-thread blocks, 128 registers) a bare transform
// is 10% faster, but the tensor kernel, which loads four operands per
// coefficient before its transform, is 14% slower.
template <int LOGN>
struct NttShape {
  static constexpr int RB = 4;
  static constexpr int R = 1 << RB;
  static constexpr int threads = (1 << LOGN) / R;
  static constexpr int min_blocks = LOGN <= 13 ? 2 : 1;
};

// Shape of the 32-bit transforms (30-bit extension and row primes): 2^RB
// coefficients per thread, N / 2^RB threads per block and up to 2048
// resident threads per SM (at most four blocks), so that the operand loads
// of some blocks overlap the transforms of others.  NTT-domain arrays of
// these primes are produced and consumed by 32-bit kernels only, so their
// storage order may differ from the 54-bit one.
template <int LOGN>
struct NttShape32 {
  static constexpr int RB = 4;
  static constexpr int R = 1 << RB;
  static constexpr int threads = (1 << LOGN) / R;
  static constexpr int min_blocks = 2048 / threads > 4 ? 4 : 2048 / threads;
};

}  // namespace cw
