// kernels.cu -- sm_103a kernels of the constant-weight PIR answer path.
//
// Layout conventions (u64 residues mod q_j, u32 residues mod the 30-bit
// extension primes p_k, limb-major):
//   coefficient ciphertext   [2][L][N]
//   QP-NTT ciphertext        [2] polynomials in QP layout (kernels.cuh): L limbs
//                            of u64, then K limbs of u32; NTT form
//   database                 [rows][L][N] NTT form (centered plaintext lift)
//   tensor buffer  Tbuf      [jobs][3][K][N] u32: N d0, N d1, N d2 modulo the
//                            extension primes (lazy residues)
//   scaled buffer  E         [jobs][3][L][N]   round(t d / Q) mod q_j
//   partials       P         [jobs][2][L][N]   NTT-form sel * DB rows
//
// NTT kernels run one length-N transform per CTA of N/R threads; each
// thread holds R = 2^RB coefficients in registers (ntt_pass.cuh, NttShape).
// A forward transform takes coefficient t + r N/R in register r of thread t
// and leaves NTT-domain value R t + r there; the inverse goes the other way.
// NTT-domain arrays are stored permuted (ntt_pos) so that both ends of a
// transform move through global memory coalesced.
#include "kernels.cuh"
#include "ntt_pass.cuh"

namespace cw {

namespace {

template <int LOGN>
__device__ __forceinline__ u32 strided_idx(u32 t, u32 r) {
  return t | (r << (LOGN - NttShape<LOGN>::RB));
}
// Storage position of NTT-domain coefficient R t + r (the value thread t
// holds in register r after a forward transform): t + r N/R, so that
// stores after a forward transform and loads before an inverse transform
// are coalesced.  Every NTT-domain array (database, keys, QP-NTT
// ciphertexts, digit transforms, accumulators) uses this order; element-wise
// kernels are indifferent to it and the ABI never exposes it.
template <int LOGN>
__device__ __forceinline__ u32 ntt_pos(u32 t, u32 r) {
  return t | (r << (LOGN - NttShape<LOGN>::RB));
}

// The same two orders for the arrays of the 32-bit primes (NttShape32).
template <int LOGN>
__device__ __forceinline__ u32 strided_idx32(u32 t, u32 r) {
  return t | (r << (LOGN - NttShape32<LOGN>::RB));
}
template <int LOGN>
__device__ __forceinline__ u32 ntt_pos32(u32 t, u32 r) {
  return t | (r << (LOGN - NttShape32<LOGN>::RB));
}

// registers of one transform per thread
template <int LOGN>
using NttRegs = u64[NttShape<LOGN>::R];

// Forward transform: x[r] = coefficient t + r N/R (< 4q) -> x[r] = NTT
// value R t + r, canonical.  Uses s (smem_words(N) words) and all
// threads of the block; s may be reused after return.
template <int LOGN>
__device__ __forceinline__ void ntt_fwd(NttRegs<LOGN> &x, u64 *s, const NttPrime &P) {
  constexpr int RB = NttShape<LOGN>::RB, R = NttShape<LOGN>::R;
  constexpr int NP = Passes<LOGN, RB>::count;
  const u32 t = threadIdx.x;
  u32 wprev = 0;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    u32 lo, c, w;
    Passes<LOGN, RB>::fwd(p, lo, c, w);
    if (p > 0) {
#pragma unroll
      for (u32 r = 0; r < R; ++r) s[sidx<RB>(pass_idx<RB>(t, r, wprev))] = x[r];
      __syncthreads();
#pragma unroll
      for (u32 r = 0; r < R; ++r) x[r] = s[sidx<RB>(pass_idx<RB>(t, r, w))];
      __syncthreads();
    }
    fwd_pass<LOGN, RB>(x, t, lo, c, w, P.psi2, P.q);
    wprev = w;
  }
#pragma unroll
  for (u32 r = 0; r < R; ++r) x[r] = reduce4(x[r], P.q);
}

// Inverse transform: x[r] = NTT value R t + r (< 2q) -> x[r] = coefficient
// t + r N/R.  With SCALE the factor N^-1 is applied and the output is
// canonical; without it the output is N times the coefficient, in [0, 2q).
template <int LOGN, bool SCALE = true>
__device__ __forceinline__ void ntt_inv(NttRegs<LOGN> &x, u64 *s, const NttPrime &P) {
  constexpr int RB = NttShape<LOGN>::RB, R = NttShape<LOGN>::R;
  constexpr int NP = Passes<LOGN, RB>::count;
  const u32 t = threadIdx.x;
  u32 wprev = 0;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    u32 lo, c, w;
    Passes<LOGN, RB>::inv(p, lo, c, w);
    if (p > 0) {
#pragma unroll
      for (u32 r = 0; r < R; ++r) s[sidx<RB>(pass_idx<RB>(t, r, wprev))] = x[r];
      __syncthreads();
#pragma unroll
      for (u32 r = 0; r < R; ++r) x[r] = s[sidx<RB>(pass_idx<RB>(t, r, w))];
      __syncthreads();
    }
    inv_pass<LOGN, RB>(x, t, lo, c, w, P.ipsi2, P.q);
    wprev = w;
  }
  if (SCALE) {
#pragma unroll
    for (u32 r = 0; r < R; ++r) x[r] = shoup(x[r], P.ninv, P.ninv_s, P.q);
  }
}

// The same transforms on 32-bit words for a 30-bit extension prime: the
// forward one from [0, 4p) to canonical values, the inverse one from
// [0, 2p) to N times the coefficient in [0, 2p) (no N^-1: the scale-down
// absorbs it).
template <int LOGN>
using NttRegs32 = u32[NttShape32<LOGN>::R];

template <int LOGN>
__device__ __forceinline__ void ntt_fwd32(NttRegs32<LOGN> &x, u32 *s, const ExtNtt &P) {
  constexpr int RB = NttShape32<LOGN>::RB, R = NttShape32<LOGN>::R;
  constexpr int NP = Passes<LOGN, RB>::count;
  const u32 t = threadIdx.x;
  u32 wprev = 0;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    u32 lo, c, w;
    Passes<LOGN, RB>::fwd(p, lo, c, w);
    if (p > 0) {
#pragma unroll
      for (u32 r = 0; r < R; ++r) s[sidx<RB>(pass_idx<RB>(t, r, wprev))] = x[r];
      __syncthreads();
#pragma unroll
      for (u32 r = 0; r < R; ++r) x[r] = s[sidx<RB>(pass_idx<RB>(t, r, w))];
      __syncthreads();
    }
    fwd_pass32<LOGN, RB>(x, t, lo, c, w, P.psi2, P.e.p);
    wprev = w;
  }
#pragma unroll
  for (u32 r = 0; r < R; ++r) x[r] = reduce4_32(x[r], P.e.p);
}

template <int LOGN>
__device__ __forceinline__ void ntt_inv32(NttRegs32<LOGN> &x, u32 *s, const ExtNtt &P) {
  constexpr int RB = NttShape32<LOGN>::RB, R = NttShape32<LOGN>::R;
  constexpr int NP = Passes<LOGN, RB>::count;
  const u32 t = threadIdx.x;
  u32 wprev = 0;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    u32 lo, c, w;
    Passes<LOGN, RB>::inv(p, lo, c, w);
    if (p > 0) {
#pragma unroll
      for (u32 r = 0; r < R; ++r) s[sidx<RB>(pass_idx<RB>(t, r, wprev))] = x[r];
      __syncthreads();
#pragma unroll
      for (u32 r = 0; r < R; ++r) x[r] = s[sidx<RB>(pass_idx<RB>(t, r, w))];
      __syncthreads();
    }
    inv_pass32<LOGN, RB>(x, t, lo, c, w, P.ipsi2, P.e.p);
    wprev = w;
  }
}

template <int LOGN>
constexpr size_t ntt_smem_bytes() {
  return (size_t)((1u << LOGN) + ((1u << LOGN) >> NttShape<LOGN>::RB)) * sizeof(u64);
}

template <typename F>
cudaError_t allow_smem(F *kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ---------------------------------------------------------------------
// Database load: row r, plaintext p (payload coefficients p N .. p N + N-1,
// zero-padded), limb j: centered lift (v > t/2 -> v - t), forward NTT into
// db[r][p][j].  grid (sp L, rows).
// ---------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN>::threads, NttShape<LOGN>::min_blocks)
    k_db_load(const DevTables *T, const u32 *items, u32 plen, u32 sp, u64 *db) {
  extern __shared__ u64 s[];
  constexpr u32 N = 1u << LOGN;
  const u32 L = T->L, p = blockIdx.x / L, j = blockIdx.x % L, t = threadIdx.x;
  const u64 row = blockIdx.y;
  const NttPrime P = T->prime[j];
  const u64 tt = T->t;
  NttRegs<LOGN> x;
  constexpr u32 R = NttShape<LOGN>::R;
#pragma unroll
  for (u32 r = 0; r < R; ++r) {
    const u32 c = p * N + strided_idx<LOGN>(t, r);
    const u64 v = c < plen ? (u64)items[row * plen + c] : 0;
    x[r] = v > tt / 2 ? P.q - (tt - v) : v;
  }
  ntt_fwd<LOGN>(x, s, P);
  u64 *out = db + ((row * sp + p) * L + j) * N;
#pragma unroll
  for (u32 r = 0; r < R; ++r) out[ntt_pos<LOGN>(t, r)] = x[r];
}

// ---------------------------------------------------------------------
// Batched NTT: unit u, limb l (prime l < L): base + u*unit_stride + l*N,
// read from src (same limb offset, src_unit_stride) when src != nullptr.
// grid (limb_end - limb_begin, units).  k_ntt32: the forward transform of
// extension limb k (limbs L + k of units in QP layout), grid (k_end -
// k_begin, units).
// ---------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(NttShape32<LOGN>::threads, NttShape32<LOGN>::min_blocks)
    k_ntt32(const DevTables *T, u64 *base, u64 unit_stride, u32 k_begin, const u64 *src,
            u64 src_unit_stride) {
  extern __shared__ u32 s32[];
  constexpr u32 N = 1u << LOGN, R = NttShape32<LOGN>::R;
  const u32 L = T->L, k = k_begin + blockIdx.x, t = threadIdx.x;
  const u64 u = blockIdx.y;
  const u64 *unit_in = src ? src + u * src_unit_stride : base + u * unit_stride;
  const ExtNtt E = T->ext[k];
  const u32 *in = ext_limb(unit_in, L, N, k);
  u32 *out = ext_limb(base + u * unit_stride, L, N, k);
  NttRegs32<LOGN> y;
#pragma unroll
  for (u32 r = 0; r < R; ++r) y[r] = in[strided_idx32<LOGN>(t, r)];
  ntt_fwd32<LOGN>(y, s32, E);  // contains barriers: all loads precede all stores
#pragma unroll
  for (u32 r = 0; r < R; ++r) out[ntt_pos32<LOGN>(t, r)] = y[r];
}

template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN>::threads, NttShape<LOGN>::min_blocks)
    k_ntt(const DevTables *T, u64 *base, u64 unit_stride, u32 limb_begin, int inverse,
          const u64 *src, u64 src_unit_stride) {
  extern __shared__ u64 s[];
  constexpr u32 N = 1u << LOGN;
  const u32 l = limb_begin + blockIdx.x, t = threadIdx.x;
  const u64 u = blockIdx.y;
  constexpr u32 R = NttShape<LOGN>::R;
  const u64 *unit_in = src ? src + u * src_unit_stride : base + u * unit_stride;
  u64 *unit_out = base + u * unit_stride;
  const NttPrime P = T->prime[l];
  const u64 *in = unit_in + (u64)l * N;
  u64 *out = unit_out + (u64)l * N;
  NttRegs<LOGN> x;
  if (inverse) {
#pragma unroll
    for (u32 r = 0; r < R; ++r) x[r] = in[ntt_pos<LOGN>(t, r)];
    ntt_inv<LOGN>(x, s, P);
#pragma unroll
    for (u32 r = 0; r < R; ++r) out[strided_idx<LOGN>(t, r)] = x[r];
  } else {
#pragma unroll
    for (u32 r = 0; r < R; ++r) x[r] = in[strided_idx<LOGN>(t, r)];
    ntt_fwd<LOGN>(x, s, P);
#pragma unroll
    for (u32 r = 0; r < R; ++r) out[ntt_pos<LOGN>(t, r)] = x[r];
  }
}

// Forward NTT of the P limbs of every job's destination (both polys),
// in place.  grid (K, 2 * njobs).
template <int LOGN>
__global__ void __launch_bounds__(NttShape32<LOGN>::threads, NttShape32<LOGN>::min_blocks)
    k_ntt_jobs_p(const DevTables *T, const MulJob *jobs) {
  extern __shared__ u32 s32[];
  constexpr u32 N = 1u << LOGN;
  const u32 L = T->L, t = threadIdx.x;
  const u32 job = blockIdx.y >> 1, poly = blockIdx.y & 1;
  const ExtNtt E = T->ext[blockIdx.x];
  u32 *p = ext_limb(jobs[job].dst + poly * qp_poly_words(L, T->K, N), L, N, blockIdx.x);
  NttRegs32<LOGN> x;
  constexpr u32 R = NttShape32<LOGN>::R;
#pragma unroll
  for (u32 r = 0; r < R; ++r) x[r] = p[strided_idx32<LOGN>(t, r)];
  // contains barriers: all loads precede all stores
  ntt_fwd32<LOGN>(x, s32, E);
#pragma unroll
  for (u32 r = 0; r < R; ++r) p[ntt_pos32<LOGN>(t, r)] = x[r];
}

// ---------------------------------------------------------------------
// Centered Q -> P conversion of coefficient-form polynomials.
// unit u: src + u*src_stride ([L][N]) -> dst + u*dst_stride (a polynomial
// in QP layout: P limbs written; Q limbs copied when copy_q).
// grid (N/256, units).
// ---------------------------------------------------------------------
// The conversion tables are passed by value (__grid_constant__): they sit
// in the constant bank and the integer multiplies read them as operands.
template <int L>
__global__ void k_lift(const DevTables *T, const u64 *src, u64 src_stride, u64 *dst,
                       u64 dst_stride, int copy_q, const __grid_constant__ LiftTab C) {
  constexpr int K = ext_count(L);
  const u32 N = T->N;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u64 u = blockIdx.y;
  const u64 *in = src + u * src_stride;
  u64 *out = dst + u * dst_stride;
  u64 x[L];
  u32 y[K];
#pragma unroll
  for (int j = 0; j < L; ++j) x[j] = in[(u64)j * N + c];
  lift_ext<L, K>(x, y, C);
  if (copy_q) {
#pragma unroll
    for (int j = 0; j < L; ++j) out[(u64)j * N + c] = x[j];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) ext_limb(out, L, N, k)[c] = y[k];
}

// Internal tree nodes: C ([jobs][2][L][N] coefficient form) -> the P limbs
// of jobs[j].dst.  grid (N/256, 2 * njobs).
template <int L>
__global__ void k_lift_jobs(const DevTables *T, const u64 *C, const MulJob *jobs,
                            const __grid_constant__ LiftTab Cv) {
  constexpr int K = ext_count(L);
  const u32 N = T->N;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u32 job = blockIdx.y >> 1, poly = blockIdx.y & 1;
  const u64 *in = C + ((u64)job * 2 + poly) * L * N;
  u64 *out = jobs[job].dst + poly * qp_poly_words(L, K, N);
  u64 x[L];
  u32 y[K];
#pragma unroll
  for (int j = 0; j < L; ++j) x[j] = in[(u64)j * N + c];
  lift_ext<L, K>(x, y, Cv);
#pragma unroll
  for (int k = 0; k < K; ++k) ext_limb(out, L, N, k)[c] = y[k];
}

// ---------------------------------------------------------------------
// Tensor of two QP-NTT ciphertexts followed by the inverse NTT:
// d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1, on the K extension limbs
// alone (their product P >= 2 N Q^2 holds the tensor of two centered lifts
// exactly, and the scale-down reads nothing else).  One block per job and
// prime computes all three outputs, so that the four operand loads of a
// coefficient serve its three products and one twiddle load serves three
// butterflies.  grid (njobs, K); the prime varies slowest so that the
// blocks resident on one SM share its twiddles in L1.
// ---------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(NttShape32<LOGN>::threads, LOGN <= 13 ? 2 : 1)
    k_tensor_ext(const DevTables *T, const MulJob *jobs, u64 *Tbuf) {
  extern __shared__ u32 s32[];
  constexpr u32 N = 1u << LOGN, R = NttShape32<LOGN>::R, RB = NttShape32<LOGN>::RB;
  constexpr int NP = Passes<LOGN, RB>::count;
  constexpr u32 SW = (1u << LOGN) + ((1u << LOGN) >> RB);  // one transform's shared words
  const u32 L = T->L, k = blockIdx.y, t = threadIdx.x;
  const u64 job = blockIdx.x;
  const MulJob J = jobs[job];
  const u64 ps = qp_poly_words(L, T->K, N), ts = 2 * tensor_poly_words(T->K, N);
  const ExtNtt E = T->ext[k];
  const u32 p2 = 2 * E.e.p;
  const u32 *a0 = ext_limb(J.a, L, N, k), *a1 = ext_limb(J.a + ps, L, N, k);
  const u32 *b0 = ext_limb(J.b, L, N, k), *b1 = ext_limb(J.b + ps, L, N, k);
  u32 y[3 * R];  // the three outputs' registers
#pragma unroll
  for (u32 r = 0; r < R; ++r) {  // products in [0, 2p)
    const u32 c = ntt_pos32<LOGN>(t, r);
    const u32 x0 = a0[c], x1 = a1[c], z0 = b0[c], z1 = b1[c];
    y[r] = mulmod_ext_lazy(x0, z0, E.e);
    // d1: both products summed exactly (below 2^61), one reduction
    y[R + r] = csub32(reduce_ext62_lazy(wmul(x0, z1) + wmul(x1, z0), E.e), p2);
    y[2 * R + r] = mulmod_ext_lazy(x1, z1, E.e);
  }
  // the three inverse transforms in lock-step: N d in [0, 2p)
  u32 wprev = 0;
#pragma unroll
  for (int pp = 0; pp < NP; ++pp) {
    u32 lo, c, w;
    Passes<LOGN, RB>::inv(pp, lo, c, w);
    if (pp > 0) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (u32 r = 0; r < R; ++r) s32[i * SW + xslot<RB>(pass_idx<RB>(t, r, wprev), wprev, w)] = y[i * R + r];
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (u32 r = 0; r < R; ++r) y[i * R + r] = s32[i * SW + xslot<RB>(pass_idx<RB>(t, r, w), wprev, w)];
      __syncthreads();
    }
    inv_pass32m<LOGN, RB, 3>(y, t, lo, c, w, E.ipsi2, E.e.p);
    wprev = w;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    u32 *out = reinterpret_cast<u32 *>(Tbuf) + (job * 3 + i) * ts + (u64)k * N;
#pragma unroll
    for (u32 r = 0; r < R; ++r) out[strided_idx32<LOGN>(t, r)] = y[i * R + r];
  }
}

// ---------------------------------------------------------------------
// Exact scale-down of every tensor coefficient from its K extension
// residues (scale_fast); the few coefficients whose fixed-point rounding is
// too close to call go through scale_exact, kept out of line so that its
// registers do not weigh on the common path.  grid (N/256, 3*njobs).
// ---------------------------------------------------------------------
// the exact path for coefficient c of the polynomial at `in`, out of line:
// it reloads its residues, so that nothing of the caller's stays live
template <int L>
__device__ __noinline__ bool scale_exact_at(const DevTables *T, const u32 *in, u64 *out, u32 c) {
  constexpr int K = ext_count(L);
  const u32 N = T->N;
  u32 dp[K];
  u64 e[L];
  for (int k = 0; k < K; ++k) dp[k] = in[(u64)k * N + c];
  const bool ok = scale_exact<L>(dp, e, T->scalep, T->scale);
  for (int j = 0; j < L; ++j) out[(u64)j * N + c] = e[j];
  return ok;
}

// Six resident blocks per SM at L <= 4 (at most 42 registers): 47.8 against
// 48.6 ms per metric answer with the five that 44 registers allow; four
// (64 registers) above.
template <int L>
__global__ void __launch_bounds__(256, L <= 4 ? 6 : 4) k_scale(const DevTables *T, const u64 *Tbuf, u64 *E, int *err,
                        const __grid_constant__ ScaleTabP S) {
  constexpr int K = ext_count(L);
  const u32 N = T->N;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u64 jw = blockIdx.y;
  const u32 *in = reinterpret_cast<const u32 *>(Tbuf) + jw * K * N;
  u64 *out = E + jw * L * N;
  u32 dp[K];
  u64 e[L];
#pragma unroll
  for (int k = 0; k < K; ++k) dp[k] = in[(u64)k * N + c];
  const int r = scale_fast<L>(dp, e, S);
  if (r == 0) {
#pragma unroll
    for (int j = 0; j < L; ++j) out[(u64)j * N + c] = e[j];
  } else if (r == 2 || !scale_exact_at<L>(T, in, out, c)) {
    atomicOr(err, 1);
  }
}

// ---------------------------------------------------------------------
// Key switching with RNS digits in two kernels.
//
// (A) k_ks_ntt: for job `job`, output limb j and unit d: d < L is digit
//     [z_d]_{q_j} (z_d in [0, q_d) < 2 q_j, one subtraction reduces it),
//     d = L is add0 (limb j), d = L+1 is add1; forward NTT mod q_j into
//     DN[job][d][j][N].  grid (L + n_add, L, njobs).
// (B) element-wise over the NTT domain:
//     acc0 = DN[L] + sum_i DN[i] * b_ij, acc1 = DN[L+1] + sum_i DN[i] * a_ij,
//     followed by the consumer (plain multiplication summed over rows, or
//     the NTT-form result).
// ---------------------------------------------------------------------
struct KsArgs {
  const u64 *z;
  u64 z_stride;
  const u64 *add0;
  u64 add0_stride;
  const u64 *add1;
  u64 add1_stride;
  u32 n_add;
};

template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN>::threads, NttShape<LOGN>::min_blocks) k_ks_ntt(const DevTables *T, KsArgs A,
                                                             u64 *DN) {
  extern __shared__ u64 s[];
  constexpr u32 N = 1u << LOGN;
  const u32 L = T->L, t = threadIdx.x, d = blockIdx.x, j = blockIdx.z;
  const u64 job = blockIdx.y;
  const NttPrime P = T->prime[j];
  const u64 q = P.q;
  NttRegs<LOGN> x;
  constexpr u32 R = NttShape<LOGN>::R;
  if (d < L) {
    const u64 *zi = A.z + job * A.z_stride + (u64)d * N;
#pragma unroll
    for (u32 r = 0; r < R; ++r) {
      const u64 v = zi[strided_idx<LOGN>(t, r)];
      x[r] = v >= q ? v - q : v;
    }
  } else {
    const u64 *ad = (d == L ? A.add0 + job * A.add0_stride : A.add1 + job * A.add1_stride) +
                    (u64)j * N;
#pragma unroll
    for (u32 r = 0; r < R; ++r) x[r] = ad[strided_idx<LOGN>(t, r)];
  }
  ntt_fwd<LOGN>(x, s, P);
  u64 *o = DN + ((job * (L + A.n_add) + d) * L + j) * N;
#pragma unroll
  for (u32 r = 0; r < R; ++r) o[ntt_pos<LOGN>(t, r)] = x[r];
}

// acc0/acc1 of one coefficient c of limb j for one job (see (B) above).
template <int L>
__device__ __forceinline__ void ks_mac(const u64 *DN, u64 job, u32 n_add, u32 j, u32 c, u32 N,
                                       const u64 *kb, const u64 *kbs, const u64 *ka,
                                       const u64 *kas, u64 q, u64 &a0, u64 &a1) {
  const u64 unit = (u64)L * N;
  const u64 *base = DN + job * (L + n_add) * unit + (u64)j * N + c;
  a0 = n_add >= 1 ? base[L * unit] : 0;
  a1 = n_add >= 2 ? base[(L + 1) * unit] : 0;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const u64 v = base[i * unit];
    a0 = addq(a0, shoup(v, kb[i], kbs[i], q), q);
    a1 = addq(a1, shoup(v, ka[i], kas[i], q), q);
  }
}

// Exact sum of products a * m of residues below q: 128-bit accumulation,
// folded back below q every 15 terms (15 q^2 + q < 2^112).
struct LazySum {
  Acc128 acc;
  __device__ __forceinline__ void mac(u64 a, u64 m) { acc.mac(a, m); }
  __device__ __forceinline__ void fold(u64 q, u64 mu) {
    acc.lo = barrett_reduce(acc.hi, acc.lo, q, mu);
    acc.hi = 0;
  }
  __device__ __forceinline__ u64 value(u64 q, u64 mu) const {
    return barrett_reduce(acc.hi, acc.lo, q, mu);
  }
};

// (B) for the answer's last level, rows of one plaintext.  The launch's
// jobs form `segs` segments of seg_len consecutive jobs (one segment per
// query); block z = s*G + g handles jobs g, g+G, ... of segment s.  The key
// switch is linear in the digits, so its key products move out of the row
// sum: modulo q_j, exactly,
//   sum_rows sel * DB = (sum_rows e0 DB + sum_d b_d sum_rows D_d DB,
//                        sum_rows e1 DB + sum_d a_d sum_rows D_d DB),
// so each thread keeps L + 2 row sums (digits d < L, then e0, e1) and
// multiplies the digit sums by the key once at the end.  Output
// P[s*G + g][2][L][N].  grid (N/256, L, segs*G).
template <int L>
__global__ void k_ks_mac_pm(const DevTables *T, const u64 *DN, u32 n_add, u32 seg_len, u32 G,
                            const MulJob *jobs, const u64 *key, const u64 *key_s,
                            const u64 *db, u64 *P) {
  const u32 N = T->N, c = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  const u32 sg = blockIdx.z, seg = sg / G, g = sg % G;
  const NttPrime Pr = T->prime[j];
  const u64 q = Pr.q;
  const u64 LN = (u64)L * N;
  LazySum acc[L + 2];
  u32 terms = 0;
  // the next row's index is loaded one iteration ahead so that the row's
  // database load issues together with the digit loads
  u64 job = (u64)seg * seg_len + g;
  u64 row = g < seg_len ? jobs[job].row : 0;
  for (u32 x = g; x < seg_len; x += G, job += G) {
    const u64 m = db[row * LN + (u64)j * N + c];
    if (x + G < seg_len) row = jobs[job + G].row;
    const u64 *dn = DN + job * (L + n_add) * LN + (u64)j * N + c;
#pragma unroll
    for (int d = 0; d < L + 2; ++d) acc[d].mac(dn[d * LN], m);
    if (++terms == 15) {
#pragma unroll
      for (int d = 0; d < L + 2; ++d) acc[d].fold(q, Pr.mu);
      terms = 1;  // the folded residue counts as one term
    }
  }
  u64 o0 = acc[L].value(q, Pr.mu), o1 = acc[L + 1].value(q, Pr.mu);
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const u64 v = acc[i].value(q, Pr.mu);
    const u64 ob = ((u64)(i * 2 + 0) * L + j) * N + c, oa = ((u64)(i * 2 + 1) * L + j) * N + c;
    o0 = addq(o0, shoup(v, key[ob], key_s[ob], q), q);
    o1 = addq(o1, shoup(v, key[oa], key_s[oa], q), q);
  }
  u64 *o = P + (u64)sg * 2 * LN + (u64)j * N + c;
  o[0] = o0;
  o[LN] = o1;
}

// Rows of sp > 1 plaintexts: the selection entries of the launch's jobs are
// first formed in NTT form (k_ks_mac_out into S[job][2][L][N]); block
// z = (s*G + g) * pcn + pc then sums S[job] * DB[row][p] over jobs g, g+G,
// ... of segment s for the plaintexts p of chunk pc (at most PPT) into
// P[s*G + g][p][2][L][N].  Two rows are loaded ahead of their products.
// grid (N/256, L, segs*G*pcn).
template <int PPT>
__global__ void k_pm_rows(const DevTables *T, const u64 *S, u32 seg_len, u32 G, u32 sp,
                          u32 pcn, const MulJob *jobs, const u64 *db, u64 *P) {
  const u32 N = T->N, L = T->L, c = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  const u32 pc = blockIdx.z % pcn, sg = blockIdx.z / pcn, seg = sg / G, g = sg % G;
  const u32 per = (sp + pcn - 1) / pcn, p0 = pc * per;
  const u32 np = sp - p0 < per ? sp - p0 : per;
  const NttPrime Pr = T->prime[j];
  const u64 q = Pr.q;
  const u64 LN = (u64)L * N, off = (u64)j * N + c;
  LazySum s0[PPT], s1[PPT];
  u32 terms = 0;
  u64 job = (u64)seg * seg_len + g;
  for (u32 x = g; x < seg_len; x += 2 * G, job += 2 * G) {
    const bool two = x + G < seg_len;
    const u64 r0 = jobs[job].row, r1 = two ? jobs[job + G].row : r0;
    const u64 *e0 = S + job * 2 * LN + off, *e1 = S + (two ? job + G : job) * 2 * LN + off;
    const u64 a00 = e0[0], a01 = e0[LN], a10 = e1[0], a11 = e1[LN];
    const u64 *d0 = db + (r0 * sp + p0) * LN + off, *d1 = db + (r1 * sp + p0) * LN + off;
    u64 m0[PPT], m1[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      m0[k] = (u32)k < np ? d0[k * LN] : 0;
      m1[k] = (u32)k < np && two ? d1[k * LN] : 0;
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      s0[k].mac(a00, m0[k]);
      s1[k].mac(a01, m0[k]);
      s0[k].mac(a10, m1[k]);
      s1[k].mac(a11, m1[k]);
    }
    terms += 2;
    if (terms >= 14) {
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        s0[k].fold(q, Pr.mu);
        s1[k].fold(q, Pr.mu);
      }
      terms = 1;
    }
  }
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if ((u32)k < np) {
      u64 *o = P + ((u64)sg * sp + p0 + k) * 2 * LN + off;
      o[0] = s0[k].value(q, Pr.mu);
      o[LN] = s1[k].value(q, Pr.mu);
    }
  }
}

// ---------------------------------------------------------------------
// Row basis (RowTab in arith.cuh): the database rows and the last tree
// level's key-switch inputs multiply exactly as integers modulo the first
// four extension primes r_k, on 32-bit words.
// ---------------------------------------------------------------------
// Database load: row `row`, prime k: centered lift of the payload (at most
// N coefficients, zero-padded), forward NTT into dbr[row][k][N].
// grid (4, rows).
template <int LOGN>
__global__ void __launch_bounds__(NttShape32<LOGN>::threads, NttShape32<LOGN>::min_blocks)
    k_db_load_rows(const DevTables *T, const u32 *items, u32 plen, u32 *dbr) {
  extern __shared__ u32 s32[];
  constexpr u32 N = 1u << LOGN, R = NttShape32<LOGN>::R;
  const u32 k = blockIdx.x, t = threadIdx.x, nr = T->rows.nr;
  const u64 row = blockIdx.y;
  const ExtNtt E = T->ext[k];
  const u32 tt = (u32)T->t, p = E.e.p;
  NttRegs32<LOGN> x;
#pragma unroll
  for (u32 r = 0; r < R; ++r) {
    const u32 c = strided_idx32<LOGN>(t, r);
    const u32 v = c < plen ? items[row * plen + c] : 0;
    x[r] = v > tt / 2 ? p - (tt - v) : v;
  }
  ntt_fwd32<LOGN>(x, s32, E);
  u32 *out = dbr + (row * nr + k) * N;
#pragma unroll
  for (u32 r = 0; r < R; ++r) out[ntt_pos32<LOGN>(t, r)] = x[r];
}

// Limb l of unit u of E (unit stride ustride u64 words, limbs of N
// residues below 2^54) reduced modulo the extension prime k < np and
// transformed: D[u][l][k][N] u32.  grid (np, nl, units).
template <int LOGN>
__global__ void __launch_bounds__(NttShape32<LOGN>::threads, NttShape32<LOGN>::min_blocks)
    k_rows_ntt(const DevTables *T, const u64 *Ein, u64 ustride, u32 nl, u32 np, u32 *D) {
  extern __shared__ u32 s32[];
  constexpr u32 N = 1u << LOGN, R = NttShape32<LOGN>::R;
  const u32 k = blockIdx.x, l = blockIdx.y, t = threadIdx.x;
  const u64 u = blockIdx.z;
  const ExtNtt E = T->ext[k];
  const u64 *in = Ein + u * ustride + (u64)l * N;
  NttRegs32<LOGN> x;
#pragma unroll
  for (u32 r = 0; r < R; ++r) x[r] = reduce_ext62_lazy(in[strided_idx32<LOGN>(t, r)], E.e);
  ntt_fwd32<LOGN>(x, s32, E);
  u32 *out = D + ((u * nl + l) * np + k) * N;
#pragma unroll
  for (u32 r = 0; r < R; ++r) out[ntt_pos32<LOGN>(t, r)] = x[r];
}

// Row sums: block z = s*G + g sums D[job][l][k] * dbr[row][k] over the jobs
// g, g+G, ... of segment seg0 + s, modulo r_k, into S[s*G + g][nl][nr][N];
// a thread takes one coefficient of one prime and NLT of the nl limbs
// (blockIdx.y = k * (nl / NLT) + part, limbs part * NLT ...).  RPI rows per
// iteration: all their loads are in flight before the products (the loop
// waits on memory: twelve rows and four limbs a thread took the metric's
// row sums from 27 to 15 ms a query against two rows and all twelve limbs).
// Products of residues below 2^30 are below 2^60, so fifteen terms fit 64
// bits.  grid (N/256, nr * nl / NLT, nseg * G).
constexpr int kMacRows = 12;  // rows per iteration
constexpr int kMacLimbs = 4;  // most limbs per thread

template <int NLT, int RPI>
__global__ void k_rows_mac(const DevTables *T, const u32 *D, u32 nl, u32 seg0, u32 seg_len,
                           u32 G, const MulJob *jobs, const u32 *dbr, u32 *S) {
  const u32 N = T->N, c = blockIdx.x * blockDim.x + threadIdx.x, parts = nl / NLT;
  const u32 k = blockIdx.y / parts, l0 = (blockIdx.y % parts) * NLT;
  const u32 sg = blockIdx.z, seg = seg0 + sg / G, g = sg % G;
  const ExtPrime E = T->ext[k].e;
  const u64 kN = (u64)T->rows.nr * N;
  u64 acc[NLT];
#pragma unroll
  for (int l = 0; l < NLT; ++l) acc[l] = 0;
  static_assert(RPI >= 1 && RPI <= 14, "RPI products and a folded residue must fit 64 bits");
  u32 terms = 0;
  const u64 kc = (u64)k * N + c + l0 * kN, jstride = (u64)nl * kN;
  u64 job = (u64)seg * seg_len + g;
  u32 x = g;
  for (; x + (RPI - 1) * G < seg_len; x += RPI * G, job += RPI * G) {
    u32 m[RPI], a[RPI][NLT];
#pragma unroll
    for (int i = 0; i < RPI; ++i) m[i] = dbr[jobs[job + i * G].row * kN + (u64)k * N + c];
#pragma unroll
    for (int i = 0; i < RPI; ++i)
#pragma unroll
      for (int l = 0; l < NLT; ++l) a[i][l] = D[(job + i * G) * jstride + kc + l * kN];
#pragma unroll
    for (int l = 0; l < NLT; ++l) {
      u64 s = 0;
#pragma unroll
      for (int i = 0; i < RPI; ++i) s += wmul(a[i][l], m[i]);
      acc[l] += s;
    }
    terms += RPI;
    if (terms + RPI > 15) {  // at most 15 terms below 2^60 each: below 2^64
#pragma unroll
      for (int l = 0; l < NLT; ++l) acc[l] = reduce_ext(acc[l], E);
      terms = 1;  // the folded residue counts as one term
    }
  }
  for (; x < seg_len; x += G, job += G) {  // the last rows (fewer than RPI)
    const u32 m0 = dbr[jobs[job].row * kN + (u64)k * N + c];
    const u32 *d0 = D + job * jstride + kc;
#pragma unroll
    for (int l = 0; l < NLT; ++l) acc[l] += wmul(d0[l * kN], m0);
  }
  u32 *o = S + (u64)sg * nl * kN + kc;
#pragma unroll
  for (int l = 0; l < NLT; ++l) o[l * kN] = reduce_ext(acc[l], E);
}

// Inverse transform (without N^-1) of S[u][l][k] (k < np) in place:
// coefficient order, values N x mod p_k below 2p_k.  grid (np, nl, units).
template <int LOGN>
__global__ void __launch_bounds__(NttShape32<LOGN>::threads, NttShape32<LOGN>::min_blocks)
    k_rows_intt(const DevTables *T, u32 *S, u32 nl, u32 np) {
  extern __shared__ u32 s32[];
  constexpr u32 N = 1u << LOGN, R = NttShape32<LOGN>::R;
  const u32 k = blockIdx.x, l = blockIdx.y, t = threadIdx.x;
  const u64 u = blockIdx.z;
  const ExtNtt E = T->ext[k];
  u32 *p = S + ((u * nl + l) * np + k) * N;
  NttRegs32<LOGN> x;
#pragma unroll
  for (u32 r = 0; r < R; ++r) x[r] = p[ntt_pos32<LOGN>(t, r)];
  ntt_inv32<LOGN>(x, s32, E);  // contains barriers: all loads precede all stores
#pragma unroll
  for (u32 r = 0; r < R; ++r) p[strided_idx32<LOGN>(t, r)] = x[r];
}

// Row sums back to the ciphertext primes (row_digits, row_to_q): limb
// l < 2L (e0 and e1, or the two polynomials of a plain product) goes to
// Eo[u][l] modulo q_{l mod L}; limb l >= 2L (digit i = l - 2L of e2) to
// Do[u][i][j] for every j < L.  Eo, Do: [.][N] u64 rows with unit strides.
// grid (N/256, nl, units).
template <int L>
__global__ void k_rows_crt(const DevTables *T, const u32 *S, u32 nl, u64 *Eo, u64 eo_stride,
                           u64 *Do, u64 do_stride, int *err, const __grid_constant__ RowTab RT) {
  const u32 N = T->N, c = blockIdx.x * blockDim.x + threadIdx.x, l = blockIdx.y;
  const u64 u = blockIdx.z;
  const u32 *src = S + (u * nl + l) * RT.nr * N + c;
  u32 xr[kRowPrimes], y[kRowPrimes];
#pragma unroll
  for (int k = 0; k < kRowPrimes; ++k) xr[k] = (u32)k < RT.nr ? src[(u64)k * N] : 0;
  bool far;
  const u64 rho = row_digits(xr, y, RT, &far);
  if (far) atomicOr(err, 2);
  if (l < 2 * L) {
    Eo[u * eo_stride + (u64)l * N + c] = row_to_q(y, rho, (int)(l % L), RT);
  } else {
    u64 *o = Do + u * do_stride + (u64)(l - 2 * L) * L * N + c;
#pragma unroll
    for (int j = 0; j < L; ++j) o[(u64)j * N] = row_to_q(y, rho, j, RT);
  }
}

// Key switch in the key-switch basis (launch_relin_ksr), the pointwise
// step: O[job][c L + j][k] = sum_i D[job][i][k] * ks[i][c][j][k] modulo
// p_k, k < 5, for c < 2 and j < L.  The L products of residues below 2^30
// sum below L 2^60 <= 2^63 and are reduced once.  grid (N/256, 5, njobs).
template <int L>
__global__ void k_ksr_mac(const DevTables *T, const u32 *D, const u32 *ks, u32 *O) {
  constexpr u32 NP = kKsrPrimes;
  const u32 N = T->N, c = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
  const u64 job = blockIdx.z;
  const ExtPrime E = T->ext[k].e;
  const u64 kc = (u64)k * N + c;
  u32 d[L];
#pragma unroll
  for (int i = 0; i < L; ++i) d[i] = D[(job * L + i) * NP * N + kc];
#pragma unroll
  for (int o = 0; o < 2 * L; ++o) {
    u64 acc = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) acc += wmul(d[i], ks[((u64)i * 2 * L + o) * NP * N + kc]);
    O[(job * 2 * L + o) * NP * N + kc] = reduce_ext(acc, E);
  }
}

// Key switch in the key-switch basis, the way back: the five residues of
// N x (x = sum_i D_i key_i, an integer below 2^125 in magnitude) give x
// modulo q_j exactly (row_digits, row_to_q with the basis tables), and
// C[job][c][j] = (x + e_c,j) mod q_j.  grid (N/256, 2L, njobs).
template <int L>
__global__ void k_ksr_crt(const DevTables *T, const u32 *O, const u64 *E, int *err, u64 *C,
                          const __grid_constant__ RowTab KT) {
  constexpr u32 NP = kKsrPrimes;
  const u32 N = T->N, c = blockIdx.x * blockDim.x + threadIdx.x, o = blockIdx.y;
  const u32 j = o % L, comp = o / L;
  const u64 job = blockIdx.z;
  const u32 *src = O + (job * 2 * L + o) * NP * N + c;
  u32 xr[kRowPrimes], y[kRowPrimes];
#pragma unroll
  for (int k = 0; k < kRowPrimes; ++k) xr[k] = (u32)k < NP ? src[(u64)k * N] : 0;
  bool far;
  const u64 rho = row_digits(xr, y, KT, &far);
  if (far) atomicOr(err, 4);
  const u64 x = row_to_q(y, rho, (int)j, KT);
  const u64 e = E[(job * 3 + comp) * L * N + (u64)j * N + c];
  C[(job * 2 + comp) * L * N + (u64)j * N + c] = addq(x, e, KT.q[j]);
}

// (B) producing the NTT-form result: INTERNAL mode writes it to the Q
// limbs of jobs[job].dst (QP layout), other modes to O[job][2][L][N].
// grid (N/256, L, njobs).
template <int L>
__global__ void k_ks_mac_out(const DevTables *T, const u64 *DN, u32 n_add, const MulJob *jobs,
                             int internal, const u64 *key, const u64 *key_s, u64 *O) {
  const u32 N = T->N, c = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  const u64 job = blockIdx.z;
  const u64 q = T->prime[j].q;
  u64 kb[L], kbs[L], ka[L], kas[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const u64 ob = ((u64)(i * 2 + 0) * L + j) * N + c, oa = ((u64)(i * 2 + 1) * L + j) * N + c;
    kb[i] = key[ob];
    kbs[i] = key_s[ob];
    ka[i] = key[oa];
    kas[i] = key_s[oa];
  }
  u64 a0, a1;
  ks_mac<L>(DN, job, n_add, j, c, N, kb, kbs, ka, kas, q, a0, a1);
  if (internal) {
    u64 *d = jobs[job].dst;
    d[(u64)j * N + c] = a0;
    d[qp_poly_words(L, T->K, N) + (u64)j * N + c] = a1;
  } else {
    O[(job * 2 + 0) * L * N + (u64)j * N + c] = a0;
    O[(job * 2 + 1) * L * N + (u64)j * N + c] = a1;
  }
}

// Inverse NTT of NTT-form results into coefficient form.  Source: the Q
// limbs of jobs[job].dst (src_from_jobs, QP layout) or O[job][2][L][N];
// destination: C[job][2][L][N] (dst_to_jobs = 0), jobs[job].dst (1) or
// sjobs[job].dst (2), both [2][L][N].  grid (L, 2 * njobs).
template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN>::threads, NttShape<LOGN>::min_blocks)
    k_intt_jobs(const DevTables *T, const MulJob *jobs, const SubJob *sjobs, int src_from_jobs,
                const u64 *O, int dst_to_jobs, u64 *C) {
  extern __shared__ u64 s[];
  constexpr u32 N = 1u << LOGN;
  const u32 L = T->L, t = threadIdx.x, j = blockIdx.x;
  const u32 job = blockIdx.y >> 1, poly = blockIdx.y & 1;
  const NttPrime P = T->prime[j];
  const u64 *in = src_from_jobs ? jobs[job].dst + poly * qp_poly_words(L, T->K, N) + (u64)j * N
                                : O + (((u64)job * 2 + poly) * L + j) * N;
  u64 *out;
  if (dst_to_jobs == 1) out = jobs[job].dst + ((u64)poly * L + j) * N;
  else if (dst_to_jobs == 2) out = sjobs[job].dst + ((u64)poly * L + j) * N;
  else out = C + (((u64)job * 2 + poly) * L + j) * N;
  NttRegs<LOGN> x;
  constexpr u32 R = NttShape<LOGN>::R;
#pragma unroll
  for (u32 r = 0; r < R; ++r) x[r] = in[ntt_pos<LOGN>(t, r)];
  ntt_inv<LOGN>(x, s, P);
#pragma unroll
  for (u32 r = 0; r < R; ++r) out[strided_idx<LOGN>(t, r)] = x[r];
}

// k = 1: the selection entry is the leaf itself (Q limbs in NTT form);
// P[job][p][2][L][N] = leaf * DB[row][p].  grid (N/256, sp L, njobs).
__global__ void k_pm_leaf(const DevTables *T, const MulJob *jobs, u32 sp, const u64 *db,
                          u64 *P) {
  const u32 N = T->N, L = T->L, K = T->K, p = blockIdx.y / L, j = blockIdx.y % L;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u64 job = blockIdx.z;
  const NttPrime Pr = T->prime[j];
  const MulJob J = jobs[job];
  const u64 LN = (u64)L * N;
  const u64 m = db[((u64)J.row * sp + p) * LN + (u64)j * N + c];
  const u64 ps = qp_poly_words(L, K, N);
  u64 *o = P + (job * sp + p) * 2 * LN + (u64)j * N + c;
  o[0] = barrett(J.a[(u64)j * N + c], m, Pr.q, Pr.mu);
  o[LN] = barrett(J.a[ps + (u64)j * N + c], m, Pr.q, Pr.mu);
}

// acc[s][sp][2][L][N] += sum over x < per_seg of P[s*per_seg + x][sp][2][L][N]
// (mod q_j) for every segment s.  grid (N/256, 2 L sp, segs).
__global__ void k_accumulate(const DevTables *T, const u64 *P, u32 per_seg, u32 sp, u64 *acc) {
  const u32 N = T->N, L = T->L;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u32 pl = blockIdx.y, j = pl % L, seg = blockIdx.z;
  const u64 q = T->prime[j].q;
  const u64 stride = 2ull * sp * L * N, off = (u64)pl * N + c;
  const u64 *ps = P + (u64)seg * per_seg * stride;
  u64 *as = acc + (u64)seg * stride;
  u64 a = as[off];
  for (u32 x = 0; x < per_seg; ++x) a = addq(a, ps[x * stride + off], q);
  as[off] = a;
}

// tau[job] = (tau_g(c0), tau_g(c1)) of sjobs[job].src, x^i -> x^(i g mod 2N)
// with x^N = -1.  grid (N/256, 2L, njobs).
__global__ void k_automorph(const DevTables *T, const SubJob *jobs, u32 g, u64 *tau) {
  const u32 N = T->N, L = T->L;
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  const u32 pl = blockIdx.y, j = pl % L;
  const u64 job = blockIdx.z;
  const u64 q = T->prime[j].q;
  u64 v = jobs[job].src[(u64)pl * N + i];
  u32 e = (u32)(((u64)i * g) & (2ull * N - 1));
  if (e >= N) {
    e -= N;
    v = v ? q - v : 0;
  }
  tau[(job * 2 * L + pl) * N + e] = v;
}

// Folklore leaves: for query bit ciphertext src = s*ell + i, leaves 2 src
// (the constant plaintext 1 minus x: Delta - c0 at x^0, -c0 elsewhere, and
// -c1) and 2 src + 1 (x itself).  grid (N/256, 2L, nq * ell).
__global__ void k_folklore_leaves(const DevTables *T, const u64 *query, u64 *out) {
  const u32 N = T->N, L = T->L;
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x, pl = blockIdx.y, j = pl % L;
  const u64 src = blockIdx.z;
  const u64 q = T->prime[j].q, ctw = 2ull * L * N, off = (u64)pl * N + i;
  const u64 v = query[src * ctw + off];
  u64 w;
  if (pl < L) {
    const u64 d = i == 0 ? T->delta[j] : 0;
    w = d >= v ? d - v : d + q - v;
  } else {
    w = v ? q - v : 0;
  }
  out[2 * src * ctw + off] = w;
  out[(2 * src + 1) * ctw + off] = v;
}

// Arithmetic operator steps, coefficient form; grid (N/256, 2L[, count]).
__global__ void k_ct_sum(const DevTables *T, const u64 *in, u32 count, u64 in_stride,
                         u64 *out) {
  const u32 N = T->N, L = T->L, i = blockIdx.x * blockDim.x + threadIdx.x, pl = blockIdx.y;
  const u64 q = T->prime[pl % L].q, off = (u64)pl * N + i;
  u64 a = 0;
  for (u32 x = 0; x < count; ++x) a = addq(a, in[x * in_stride + off], q);
  out[off] = a;
}

// Element-wise sums v < 2^64 of residues (one all-reduce of partial
// responses) -> v mod q_j (Barrett on v below 2^112).  grid (N/256, 2L, s).
__global__ void k_ct_reduce(const DevTables *T, const u64 *in, u64 *out) {
  const u32 N = T->N, L = T->L, i = blockIdx.x * blockDim.x + threadIdx.x, pl = blockIdx.y;
  const NttPrime P = T->prime[pl % L];
  const u64 off = ((u64)blockIdx.z * 2 * L + pl) * N + i;
  out[off] = barrett_reduce(0, in[off], P.q, P.mu);
}

__global__ void k_minus_consts(const DevTables *T, const u64 *in, u64 *out) {
  const u32 N = T->N, L = T->L, i = blockIdx.x * blockDim.x + threadIdx.x, pl = blockIdx.y;
  const u32 f = blockIdx.z, j = pl % L;
  const u64 q = T->prime[j].q, off = (u64)pl * N + i;
  u64 v = in[off];
  if (pl < L && i == 0) {
    const u64 d = (u64)(((unsigned __int128)T->delta[j] * f) % q);
    v = subq(v, d, q);
  }
  out[(u64)f * 2 * L * N + off] = v;
}

__global__ void k_ct_scalar(const DevTables *T, const u64 *in, u64 s, u64 *out) {
  const u32 N = T->N, L = T->L, i = blockIdx.x * blockDim.x + threadIdx.x, pl = blockIdx.y;
  const NttPrime P = T->prime[pl % L];
  const u64 off = (u64)pl * N + i;
  out[off] = barrett(in[off], s % P.q, P.q, P.mu);
}

// One round a of Alg. Query Expansion for all (input j, entry b < 2^a):
// next[b] = cur[b] + S_b, next[b + 2^a] = x^(-2^a) (cur[b] - S_b), where
// S_b = Sub(cur[b]); entries are indexed j * 2^c + b.
// grid (N/256, 2L, h_in * 2^a).
__global__ void k_expand_combine(const DevTables *T, const u64 *cur, const u64 *S, u64 *next,
                                 u32 cfac, u32 a) {
  const u32 N = T->N, L = T->L;
  const u32 o = blockIdx.x * blockDim.x + threadIdx.x;
  const u32 pl = blockIdx.y, jl = pl % L;
  const u32 job = blockIdx.z, ja = job >> a, b = job & ((1u << a) - 1);
  const u64 q = T->prime[jl].q;
  const u64 ctw = 2ull * L * N;
  const u64 src = ((u64)ja << cfac) + b, hi = src + (1u << a);
  const u64 *cb = cur + src * ctw + (u64)pl * N;
  const u64 *sb = S + (u64)job * ctw + (u64)pl * N;
  next[src * ctw + (u64)pl * N + o] = addq(cb[o], sb[o], q);
  const u32 e = 1u << a;
  u64 v;
  if (o + e < N) v = subq(cb[o + e], sb[o + e], q);
  else {
    u64 w = subq(cb[o + e - N], sb[o + e - N], q);
    v = w ? q - w : 0;
  }
  next[hi * ctw + (u64)pl * N + o] = v;
}

// out = ct * db_row in the NTT domain ([2][L][N] and [L][N]).
// grid (N/256, 2L).
__global__ void k_pm_ntt(const DevTables *T, const u64 *ct, const u64 *dbr, u64 *out) {
  const u32 N = T->N, L = T->L;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u32 pl = blockIdx.y, j = pl % L;
  const NttPrime P = T->prime[j];
  out[(u64)pl * N + c] = barrett(ct[(u64)pl * N + c], dbr[(u64)j * N + c], P.q, P.mu);
}

// Switching keys [nkeys][L][2][L][N]: forward NTT of every limb (prime =
// limb index) and the Shoup companion floor(w 2^64 / q) by long division.
// grid (L, nkeys*2*L).
template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN>::threads, NttShape<LOGN>::min_blocks)
    k_key_prep(const DevTables *T, u64 *key, u64 *key_s) {
  extern __shared__ u64 s[];
  constexpr u32 N = 1u << LOGN;
  const u32 j = blockIdx.x, t = threadIdx.x;
  const u64 unit = blockIdx.y;
  const NttPrime P = T->prime[j];
  u64 *p = key + (unit * T->L + j) * N;
  u64 *ps = key_s + (unit * T->L + j) * N;
  NttRegs<LOGN> x;
  constexpr u32 R = NttShape<LOGN>::R;
#pragma unroll
  for (u32 r = 0; r < R; ++r) x[r] = p[strided_idx<LOGN>(t, r)];
  ntt_fwd<LOGN>(x, s, P);
#pragma unroll
  for (u32 r = 0; r < R; ++r) {
    u64 w = x[r], rem = w, quo = 0;
    for (int b = 0; b < 64; ++b) {
      rem <<= 1;
      const u64 bit = rem >= P.q ? 1 : 0;
      if (bit) rem -= P.q;
      quo = (quo << 1) | bit;
    }
    p[ntt_pos<LOGN>(t, r)] = w;
    ps[ntt_pos<LOGN>(t, r)] = quo;
  }
}

// blockDim of the transform kernels: N / R threads.
template <int LOGN>
inline dim3 ntt_block() { return dim3(NttShape<LOGN>::threads); }
template <int LOGN>
inline dim3 ntt_block32() { return dim3(NttShape32<LOGN>::threads); }
// shared memory of one 32-bit transform (one pad word per 2^RB)
template <int LOGN>
constexpr size_t smem32_bytes() {
  return (size_t)((1u << LOGN) + ((1u << LOGN) >> NttShape32<LOGN>::RB)) * sizeof(u32);
}

#define CW_DISPATCH_LOGN(LOGN_, ...)                       \
  switch (LOGN_) {                                         \
    case 10: { constexpr int LG = 10; __VA_ARGS__; } break; \
    case 11: { constexpr int LG = 11; __VA_ARGS__; } break; \
    case 12: { constexpr int LG = 12; __VA_ARGS__; } break; \
    case 13: { constexpr int LG = 13; __VA_ARGS__; } break; \
    case 14: { constexpr int LG = 14; __VA_ARGS__; } break; \
    default: return cudaErrorInvalidValue;                 \
  }

}  // namespace

// ---------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------
#define CW_DISPATCH_L(L_, KERNEL, GRID, BLOCK, SMEM, STREAM, ...)      \
  switch (L_) {                                                       \
    case 1: KERNEL<1><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break; \
    case 2: KERNEL<2><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break; \
    case 3: KERNEL<3><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break; \
    case 4: KERNEL<4><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break; \
    case 5: KERNEL<5><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break; \
    case 6: KERNEL<6><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break; \
    case 7: KERNEL<7><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break; \
    case 8: KERNEL<8><<<GRID, BLOCK, SMEM, STREAM>>>(__VA_ARGS__); break; \
    default: return cudaErrorInvalidValue;                            \
  }

cudaError_t launch_db_load(const DevTables *T, const DevTables &h, const u32 *items, u64 rows,
                           u32 plen, u32 sp, u64 *db, cudaStream_t st) {
  const u64 chunk = 32768;
  for (u64 r0 = 0; r0 < rows; r0 += chunk) {
    u64 nr = rows - r0 < chunk ? rows - r0 : chunk;
    CW_DISPATCH_LOGN(h.logN, {
      cudaError_t e = allow_smem(k_db_load<LG>, ntt_smem_bytes<LG>());
      if (e != cudaSuccess) return e;
      k_db_load<LG><<<dim3(sp * h.L, (u32)nr), ntt_block<LG>(), ntt_smem_bytes<LG>(), st>>>(
          T, items + r0 * plen, plen, sp, db + r0 * sp * h.L * h.N);
    });
  }
  return cudaGetLastError();
}

cudaError_t launch_ntt(const DevTables *T, const DevTables &h, u64 *base, u32 units,
                       u64 unit_stride, u32 limb_begin, u32 limb_end, bool inverse,
                       const u64 *src, u64 src_unit_stride, cudaStream_t st) {
  if (!units || limb_end <= limb_begin) return cudaSuccess;
  if (inverse && limb_end > h.L) return cudaErrorInvalidValue;  // extension limbs: forward only
  const u32 chunk = 32768;
  const u32 qb = limb_begin, qe = limb_end < h.L ? limb_end : h.L;   // ciphertext limbs
  const u32 kb = (limb_begin > h.L ? limb_begin : h.L) - h.L;         // extension limbs
  const u32 ke = limb_end > h.L ? limb_end - h.L : 0;
  for (u32 u0 = 0; u0 < units; u0 += chunk) {
    u32 nu = units - u0 < chunk ? units - u0 : chunk;
    u64 *b0 = base + (u64)u0 * unit_stride;
    const u64 *s0 = src ? src + (u64)u0 * src_unit_stride : nullptr;
    CW_DISPATCH_LOGN(h.logN, {
      if (qe > qb) {
        cudaError_t e = allow_smem(k_ntt<LG>, ntt_smem_bytes<LG>());
        if (e != cudaSuccess) return e;
        k_ntt<LG><<<dim3(qe - qb, nu), ntt_block<LG>(), ntt_smem_bytes<LG>(), st>>>(
            T, b0, unit_stride, qb, inverse ? 1 : 0, s0, src_unit_stride);
      }
      if (ke > kb) {
        cudaError_t e = allow_smem(k_ntt32<LG>, smem32_bytes<LG>());
        if (e != cudaSuccess) return e;
        k_ntt32<LG><<<dim3(ke - kb, nu), ntt_block32<LG>(), smem32_bytes<LG>(), st>>>(
            T, b0, unit_stride, kb, s0, src_unit_stride);
      }
    });
  }
  return cudaGetLastError();
}

cudaError_t launch_lift(const DevTables *T, const DevTables &h, const u64 *src,
                        u64 src_stride, u64 *dst, u64 dst_stride, u32 units, bool copy_q,
                        cudaStream_t st) {
  const u32 chunk = 32768;
  for (u32 u0 = 0; u0 < units; u0 += chunk) {
    u32 nu = units - u0 < chunk ? units - u0 : chunk;
    dim3 grid(h.N / 256, nu);
    CW_DISPATCH_L(h.L, k_lift, grid, 256, 0, st, T, src + (u64)u0 * src_stride, src_stride,
                  dst + (u64)u0 * dst_stride, dst_stride, copy_q ? 1 : 0, h.lift);
  }
  return cudaGetLastError();
}

cudaError_t launch_lift_jobs(const DevTables *T, const DevTables &h, const u64 *C,
                             const MulJob *jobs, u32 njobs, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  dim3 grid(h.N / 256, 2 * njobs);
  CW_DISPATCH_L(h.L, k_lift_jobs, grid, 256, 0, st, T, C, jobs, h.lift);
  return cudaGetLastError();
}

cudaError_t launch_ntt_jobs_p(const DevTables *T, const DevTables &h, const MulJob *jobs,
                              u32 njobs, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  CW_DISPATCH_LOGN(h.logN, {
    cudaError_t e = allow_smem(k_ntt_jobs_p<LG>, smem32_bytes<LG>());
    if (e != cudaSuccess) return e;
    k_ntt_jobs_p<LG><<<dim3(h.K, 2 * njobs), ntt_block32<LG>(), smem32_bytes<LG>(), st>>>(T, jobs);
  });
  return cudaGetLastError();
}

cudaError_t launch_tensor(const DevTables *T, const DevTables &h, const MulJob *jobs,
                               u32 njobs, u64 *Tbuf, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  CW_DISPATCH_LOGN(h.logN, {
    cudaError_t e = allow_smem(k_tensor_ext<LG>, 3 * smem32_bytes<LG>());
    if (e != cudaSuccess) return e;
    k_tensor_ext<LG><<<dim3(njobs, h.K), ntt_block32<LG>(), 3 * smem32_bytes<LG>(), st>>>(
        T, jobs, Tbuf);
  });
  return cudaGetLastError();
}

cudaError_t launch_scale(const DevTables *T, const DevTables &h, const u64 *Tbuf, u32 njobs,
                         u64 *E, int *err, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  dim3 grid(h.N / 256, 3 * njobs);
  CW_DISPATCH_L(h.L, k_scale, grid, 256, 0, st, T, Tbuf, E, err, h.scalep);
  return cudaGetLastError();
}

static cudaError_t launch_ks_ntt(const DevTables *T, const DevTables &h, const KsArgs &A,
                                 u32 njobs, u64 *DN, cudaStream_t st) {
  CW_DISPATCH_LOGN(h.logN, {
    cudaError_t e = allow_smem(k_ks_ntt<LG>, ntt_smem_bytes<LG>());
    if (e != cudaSuccess) return e;
    k_ks_ntt<LG><<<dim3(h.L + A.n_add, njobs, h.L), ntt_block<LG>(), ntt_smem_bytes<LG>(), st>>>(T, A, DN);
  });
  return cudaGetLastError();
}

static cudaError_t launch_intt_jobs(const DevTables *T, const DevTables &h, const MulJob *jobs,
                                    const SubJob *sjobs, u32 njobs, int src_from_jobs,
                                    const u64 *O, int dst_to_jobs, u64 *C, cudaStream_t st) {
  CW_DISPATCH_LOGN(h.logN, {
    cudaError_t e = allow_smem(k_intt_jobs<LG>, ntt_smem_bytes<LG>());
    if (e != cudaSuccess) return e;
    k_intt_jobs<LG><<<dim3(h.L, 2 * njobs), ntt_block<LG>(), ntt_smem_bytes<LG>(), st>>>(
        T, jobs, sjobs, src_from_jobs, O, dst_to_jobs, C);
  });
  return cudaGetLastError();
}

// plaintexts per k_pm_rows thread (PPT) and the chunks covering sp
constexpr u32 kPmPPT = 2;  // fewer per thread keeps more warps resident
u32 pm_chunks(u32 sp) { return sp <= 1 ? 1 : (sp + kPmPPT - 1) / kPmPPT; }

u32 pm_groups(const DevTables &h, u32 segs, u32 seg_len, u32 sp, u32 cap) {
  // row groups per segment: about row_waves waves of the device's resident
  // threads over the segs * L * N * (plaintext chunks) threads, at most
  // seg_len, and at most cap partial slots of [sp][2][L][N] in all
  u64 lanes = (u64)segs * h.L * h.N * pm_chunks(sp);
  u64 g = ((u64)h.row_waves * h.sms * h.sm_threads + lanes - 1) / lanes;
  g = g < seg_len ? g : seg_len;
  const u64 gcap = cap / ((u64)segs * sp);
  g = g < gcap ? g : gcap;
  return (u32)(g < 1 ? 1 : g);
}

cudaError_t launch_relin(const DevTables *T, const DevTables &h, const u64 *E, u32 njobs,
                         u32 segs, const MulJob *jobs, int mode, const u64 *rlk, const u64 *rlk_s,
                         const u64 *db, u32 sp, u32 cap, u64 *DN, u64 *S, u64 *out,
                         cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  const u64 LN = (u64)h.L * h.N;
  KsArgs A;
  A.z = E + 2 * LN;
  A.z_stride = 3 * LN;
  A.add0 = E;
  A.add0_stride = 3 * LN;
  A.add1 = E + LN;
  A.add1_stride = 3 * LN;
  A.n_add = 2;
  cudaError_t e = launch_ks_ntt(T, h, A, njobs, DN, st);
  if (e != cudaSuccess) return e;
  if (mode == ROOT_PM) {
    const u32 seg_len = njobs / segs, G = pm_groups(h, segs, seg_len, sp, cap);
    if (sp == 1) {
      dim3 grid(h.N / 256, h.L, segs * G);
      CW_DISPATCH_L(h.L, k_ks_mac_pm, grid, 256, 0, st, T, DN, 2u, seg_len, G, jobs, rlk, rlk_s,
                    db, out);
      return cudaGetLastError();
    }
    // selection entries in NTT form into S, then the rows' plaintexts
    dim3 grid_s(h.N / 256, h.L, njobs);
    CW_DISPATCH_L(h.L, k_ks_mac_out, grid_s, 256, 0, st, T, DN, 2u, jobs, 0, rlk, rlk_s, S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const u32 pcn = pm_chunks(sp);
    k_pm_rows<kPmPPT><<<dim3(h.N / 256, h.L, segs * G * pcn), 256, 0, st>>>(
        T, S, seg_len, G, sp, pcn, jobs, db, out);
    return cudaGetLastError();
  }
  dim3 grid(h.N / 256, h.L, njobs);
  const int internal = mode == INTERNAL ? 1 : 0;
  CW_DISPATCH_L(h.L, k_ks_mac_out, grid, 256, 0, st, T, DN, 2u, jobs, internal, rlk, rlk_s, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (internal) return launch_intt_jobs(T, h, jobs, nullptr, njobs, 1, nullptr, 0, out, st);
  return launch_intt_jobs(T, h, jobs, nullptr, njobs, 0, out, 1, nullptr, st);
}

u32 relin_pm_groups(const DevTables &h, u32 segs, u32 seg_len, u32 sp, u32 cap) {
  return pm_groups(h, segs, seg_len, sp, cap);
}

// ---- row basis ----
// Row groups per segment: as for the ciphertext basis (at most gcap / segs),
// and at least enough that no group sums more rows than the basis holds.
u32 relin_rows_groups(const DevTables &h, u32 segs, u32 seg_len, u32 gcap) {
  const u32 g = pm_groups(h, segs, seg_len, 1, gcap);
  const u32 need = (seg_len + h.rows.rmax - 1) / h.rows.rmax;
  return g > need ? g : need;
}


// Row sums for nl limbs: NLT = the largest divisor of nl that is at most
// kMacLimbs, nr * nl / NLT blocks in y.
static cudaError_t rows_mac(const DevTables &h, const DevTables *T, const u32 *D, u32 nl,
                            u32 seg0, u32 seg_len, u32 G, const MulJob *jobs, const u32 *dbr,
                            u32 *S, u32 units, cudaStream_t st) {
  u32 nlt = kMacLimbs < (int)nl ? kMacLimbs : nl;
  while (nl % nlt) --nlt;
  const dim3 grid(h.N / 256, h.rows.nr * (nl / nlt), units);
  switch (nlt) {
#define CW_MAC_CASE(V) \
    case V: k_rows_mac<V, kMacRows><<<grid, 256, 0, st>>>(T, D, nl, seg0, seg_len, G, jobs, dbr, S); break;
    CW_MAC_CASE(1) CW_MAC_CASE(2) CW_MAC_CASE(3) CW_MAC_CASE(4) CW_MAC_CASE(5) CW_MAC_CASE(6)
    CW_MAC_CASE(7) CW_MAC_CASE(8) CW_MAC_CASE(9) CW_MAC_CASE(10) CW_MAC_CASE(11) CW_MAC_CASE(12)
#undef CW_MAC_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_db_load_rows(const DevTables *T, const DevTables &h, const u32 *items,
                                u64 rows, u32 plen, u32 *dbr, cudaStream_t st) {
  const u64 chunk = 32768;
  for (u64 r0 = 0; r0 < rows; r0 += chunk) {
    const u64 nr = rows - r0 < chunk ? rows - r0 : chunk;
    CW_DISPATCH_LOGN(h.logN, {
      cudaError_t e = allow_smem(k_db_load_rows<LG>, smem32_bytes<LG>());
      if (e != cudaSuccess) return e;
      k_db_load_rows<LG><<<dim3(h.rows.nr, (u32)nr), ntt_block32<LG>(), smem32_bytes<LG>(), st>>>(
          T, items + r0 * plen, plen, dbr + r0 * h.rows.nr * h.N);
    });
  }
  return cudaGetLastError();
}

// units of nl limbs (unit stride ustride) -> D[u][l][k < np] (k_rows_ntt)
static cudaError_t rns_ntt(const DevTables *T, const DevTables &h, const u64 *E, u64 ustride,
                           u32 nl, u32 np, u32 units, u32 *D, cudaStream_t st) {
  CW_DISPATCH_LOGN(h.logN, {
    cudaError_t e = allow_smem(k_rows_ntt<LG>, smem32_bytes<LG>());
    if (e != cudaSuccess) return e;
    k_rows_ntt<LG><<<dim3(np, nl, units), ntt_block32<LG>(), smem32_bytes<LG>(), st>>>(
        T, E, ustride, nl, np, D);
  });
  return cudaGetLastError();
}

static cudaError_t rns_intt(const DevTables *T, const DevTables &h, u32 *S, u32 nl, u32 np,
                            u32 units, cudaStream_t st) {
  CW_DISPATCH_LOGN(h.logN, {
    cudaError_t e = allow_smem(k_rows_intt<LG>, smem32_bytes<LG>());
    if (e != cudaSuccess) return e;
    k_rows_intt<LG><<<dim3(np, nl, units), ntt_block32<LG>(), smem32_bytes<LG>(), st>>>(
        T, S, nl, np);
  });
  return cudaGetLastError();
}

static cudaError_t rows_ntt(const DevTables *T, const DevTables &h, const u64 *E, u32 nl,
                            u32 units, u32 *D, cudaStream_t st) {
  return rns_ntt(T, h, E, (u64)nl * h.N, nl, h.rows.nr, units, D, st);
}

static cudaError_t rows_intt(const DevTables *T, const DevTables &h, u32 *S, u32 nl, u32 units,
                             cudaStream_t st) {
  return rns_intt(T, h, S, nl, h.rows.nr, units, st);
}

cudaError_t launch_relin_ksr(const DevTables *T, const DevTables &h, const u64 *E, u32 njobs,
                             const u32 *ks, u32 *D, u32 *O, int *err, u64 *C, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  const u32 L = h.L, N = h.N;
  const u64 LN = (u64)L * N;
  // the digits of e2 (its limbs) into the basis
  cudaError_t e = rns_ntt(T, h, E + 2 * LN, 3 * LN, L, kKsrPrimes, njobs, D, st);
  if (e != cudaSuccess) return e;
  CW_DISPATCH_L(L, k_ksr_mac, dim3(N / 256, kKsrPrimes, njobs), 256, 0, st, T, D, ks, O);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = rns_intt(T, h, O, 2 * L, kKsrPrimes, njobs, st)) != cudaSuccess) return e;
  CW_DISPATCH_L(L, k_ksr_crt, dim3(N / 256, 2 * L, njobs), 256, 0, st, T, O, E, err, C, h.ksr);
  return cudaGetLastError();
}

cudaError_t launch_ksr_key(const DevTables *T, const DevTables &h, const u64 *key, u32 *ks,
                           cudaStream_t st) {
  // every [N] limb of the key is one unit of one limb
  return rns_ntt(T, h, key, h.N, 1, kKsrPrimes, 2 * h.L * h.L, ks, st);
}


cudaError_t launch_rows_transforms(const DevTables *T, const DevTables &h, const u64 *E,
                                   u32 njobs, u32 *D, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  return rows_ntt(T, h, E, 3 * h.L, njobs, D, st);
}

cudaError_t launch_relin_rows(const DevTables *T, const DevTables &h, const u64 *E, u32 njobs,
                              u32 segs, const MulJob *jobs, const u64 *rlk, const u64 *rlk_s,
                              const u32 *dbr, u32 gcap, u32 *D, u32 *S, u64 *DNQ, int *err,
                              u64 *out, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  const u32 L = h.L, nl = 3 * L, N = h.N;
  const u64 LN = (u64)L * N, unit = (u64)(L + 2) * LN;
  cudaError_t e;
  const u32 seg_len = njobs / segs, G = relin_rows_groups(h, segs, seg_len, gcap);
  const u32 spp = G >= gcap ? 1 : gcap / G;  // segments per pass
  for (u32 s0 = 0; s0 < segs; s0 += spp) {
    const u32 nseg = segs - s0 < spp ? segs - s0 : spp, units = nseg * G;
    if ((e = rows_mac(h, T, D, nl, s0, seg_len, G, jobs, dbr, S, units, st)) != cudaSuccess)
      return e;
    if ((e = rows_intt(T, h, S, nl, units, st)) != cudaSuccess) return e;
    CW_DISPATCH_L(L, k_rows_crt, dim3(N / 256, nl, units), 256, 0, st, T, S, nl, DNQ + L * LN,
                  unit, DNQ, unit, err, h.rows);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // digit sums, e0 and e1 sums to NTT form modulo q_j, then the key
    if ((e = launch_ntt(T, h, DNQ, units * (L + 2), LN, 0, L, false, nullptr, 0, st)) !=
        cudaSuccess)
      return e;
    CW_DISPATCH_L(L, k_ks_mac_out, dim3(N / 256, L, units), 256, 0, st, T, DNQ, 2u, nullptr, 0,
                  rlk, rlk_s, out + (u64)s0 * G * 2 * LN);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_plain_mul_rows(const DevTables *T, const DevTables &h, const u64 *ct,
                                  const MulJob *job, const u32 *dbr, u32 *D, u32 *S, int *err,
                                  u64 *out, cudaStream_t st) {
  const u32 L = h.L, nl = 2 * L, N = h.N;
  cudaError_t e = rows_ntt(T, h, ct, nl, 1, D, st);
  if (e != cudaSuccess) return e;
  if ((e = rows_mac(h, T, D, nl, 0, 1, 1, job, dbr, S, 1, st)) != cudaSuccess) return e;
  if ((e = rows_intt(T, h, S, nl, 1, st)) != cudaSuccess) return e;
  CW_DISPATCH_L(L, k_rows_crt, dim3(N / 256, nl, 1), 256, 0, st, T, S, nl, out,
                (u64)2 * L * N, (u64 *)nullptr, (u64)0, err, h.rows);
  return cudaGetLastError();
}

cudaError_t launch_pm_leaf(const DevTables *T, const DevTables &h, const MulJob *jobs,
                           u32 njobs, u32 sp, const u64 *db, u64 *P, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  k_pm_leaf<<<dim3(h.N / 256, sp * h.L, njobs), 256, 0, st>>>(T, jobs, sp, db, P);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(const DevTables &h, const DevTables *T, const u64 *P, u32 segs,
                              u32 per_seg, u32 sp, u64 *acc, cudaStream_t st) {
  if (!segs || !per_seg) return cudaSuccess;
  k_accumulate<<<dim3(h.N / 256, 2 * h.L * sp, segs), 256, 0, st>>>(T, P, per_seg, sp, acc);
  return cudaGetLastError();
}

cudaError_t launch_folklore_leaves(const DevTables *T, const DevTables &h, const u64 *query,
                                   u32 count, u64 *out, cudaStream_t st) {
  if (!count) return cudaSuccess;
  k_folklore_leaves<<<dim3(h.N / 256, 2 * h.L, count), 256, 0, st>>>(T, query, out);
  return cudaGetLastError();
}

cudaError_t launch_ct_sum(const DevTables *T, const DevTables &h, const u64 *in, u32 count,
                          u64 in_stride, u64 *out, cudaStream_t st) {
  k_ct_sum<<<dim3(h.N / 256, 2 * h.L), 256, 0, st>>>(T, in, count, in_stride, out);
  return cudaGetLastError();
}

cudaError_t launch_ct_reduce(const DevTables *T, const DevTables &h, const u64 *in, u32 count,
                            u64 *out, cudaStream_t st) {
  if (!count) return cudaSuccess;
  k_ct_reduce<<<dim3(h.N / 256, 2 * h.L, count), 256, 0, st>>>(T, in, out);
  return cudaGetLastError();
}

cudaError_t launch_minus_consts(const DevTables *T, const DevTables &h, const u64 *in,
                                u32 count, u64 *out, cudaStream_t st) {
  if (!count) return cudaSuccess;
  k_minus_consts<<<dim3(h.N / 256, 2 * h.L, count), 256, 0, st>>>(T, in, out);
  return cudaGetLastError();
}

cudaError_t launch_ct_scalar(const DevTables *T, const DevTables &h, const u64 *in, u64 s,
                             u64 *out, cudaStream_t st) {
  k_ct_scalar<<<dim3(h.N / 256, 2 * h.L), 256, 0, st>>>(T, in, s, out);
  return cudaGetLastError();
}

// *flag |= 1 if any residue of ct[count][2][L][N] is not below its prime
// q_j.  grid (N/256, min(rows, 65535)) over the 2 L count limb rows.
__global__ void k_check_residues(const DevTables *T, const u64 *ct, u64 rows, int *flag) {
  const u32 N = T->N, L = T->L, c = blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  for (u64 r = blockIdx.y; r < rows; r += gridDim.y) bad |= ct[r * N + c] >= T->prime[r % L].q;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t launch_check_residues(const DevTables *T, const DevTables &h, const u64 *ct,
                                  u64 count, int *flag, cudaStream_t st) {
  const u64 rows = 2ull * h.L * count;
  if (!rows) return cudaSuccess;
  k_check_residues<<<dim3(h.N / 256, (u32)(rows < 65535 ? rows : 65535)), 256, 0, st>>>(
      T, ct, rows, flag);
  return cudaGetLastError();
}

cudaError_t launch_automorph(const DevTables *T, const DevTables &h, const SubJob *jobs,
                             u32 njobs, u32 g, u64 *tau, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  k_automorph<<<dim3(h.N / 256, 2 * h.L, njobs), 256, 0, st>>>(T, jobs, g, tau);
  return cudaGetLastError();
}

cudaError_t launch_sub_keyswitch(const DevTables *T, const DevTables &h, const u64 *tau,
                                 u32 njobs, const SubJob *jobs, const u64 *key,
                                 const u64 *key_s, u64 *DN, u64 *O, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  const u64 LN = (u64)h.L * h.N;
  KsArgs A;
  A.z = tau + LN;
  A.z_stride = 2 * LN;
  A.add0 = tau;
  A.add0_stride = 2 * LN;
  A.add1 = nullptr;
  A.add1_stride = 0;
  A.n_add = 1;
  cudaError_t e = launch_ks_ntt(T, h, A, njobs, DN, st);
  if (e != cudaSuccess) return e;
  dim3 grid(h.N / 256, h.L, njobs);
  CW_DISPATCH_L(h.L, k_ks_mac_out, grid, 256, 0, st, T, DN, 1u, nullptr, 0, key, key_s, O);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_intt_jobs(T, h, nullptr, jobs, njobs, 0, O, 2, nullptr, st);
}

cudaError_t launch_expand_combine(const DevTables *T, const DevTables &h, const u64 *cur,
                                  const u64 *S, u64 *next, u32 h_in, u32 cfac, u32 a,
                                  cudaStream_t st) {
  u32 njobs = h_in << a;
  if (!njobs) return cudaSuccess;
  k_expand_combine<<<dim3(h.N / 256, 2 * h.L, njobs), 256, 0, st>>>(T, cur, S, next, cfac, a);
  return cudaGetLastError();
}

cudaError_t launch_pm_ntt(const DevTables *T, const DevTables &h, const u64 *ct_ntt,
                          const u64 *db_row, u64 *out, cudaStream_t st) {
  k_pm_ntt<<<dim3(h.N / 256, 2 * h.L), 256, 0, st>>>(T, ct_ntt, db_row, out);
  return cudaGetLastError();
}

cudaError_t launch_key_prep(const DevTables *T, const DevTables &h, u64 *key, u64 *key_s,
                            u32 nkeys, cudaStream_t st) {
  if (!nkeys) return cudaSuccess;
  CW_DISPATCH_LOGN(h.logN, {
    cudaError_t e = allow_smem(k_key_prep<LG>, ntt_smem_bytes<LG>());
    if (e != cudaSuccess) return e;
    k_key_prep<LG><<<dim3(h.L, nkeys * 2 * h.L), ntt_block<LG>(), ntt_smem_bytes<LG>(), st>>>(T, key,
                                                                                  key_s);
  });
  return cudaGetLastError();
}

}  // namespace cw
