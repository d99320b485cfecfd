// kernels.cu -- sm_103a kernels of the constant-weight PIR answer path.
//
// Layout conventions (u64 residues, limb-major):
//   coefficient ciphertext   [2][L][N]
//   QP-NTT ciphertext        [2][L+K][N]  NTT form over q_0..q_{L-1}, p_0..p_{K-1}
//   database                 [rows][L][N] NTT form (centered plaintext lift)
//   tensor buffer  Tbuf      [jobs][3][L+K][N] coefficient form of d0, d1, d2
//   scaled buffer  E         [jobs][3][L][N]   round(t d / Q) mod q_j
//   partials       P         [jobs][2][L][N]   NTT-form sel * DB rows
// NTT kernels run one length-N transform per CTA in shared memory with
// blockDim = N / 16 threads.
#include "kernels.cuh"

namespace cw {

namespace {

__device__ __forceinline__ void smem_ntt_fwd(u64 *s, const NttPrime &P, u32 logN) {
  const u32 half = 1u << (logN - 1);
  for (u32 st = 0; st < logN; ++st) {
    const u32 m = 1u << st, logh = logN - 1 - st;
    for (u32 b = threadIdx.x; b < half; b += blockDim.x)
      fwd_bfly(s, b, logh, m, P.psi, P.psi_s, P.q);
    __syncthreads();
  }
}

__device__ __forceinline__ void smem_ntt_inv(u64 *s, const NttPrime &P, u32 logN) {
  const u32 N = 1u << logN, half = N >> 1;
  for (u32 st = 0; st < logN; ++st) {
    const u32 logh = st, m = N >> (st + 1);
    for (u32 b = threadIdx.x; b < half; b += blockDim.x)
      inv_bfly(s, b, logh, m, P.ipsi, P.ipsi_s, P.q);
    __syncthreads();
  }
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) s[c] = shoup(s[c], P.ninv, P.ninv_s, P.q);
  __syncthreads();
}

inline dim3 ntt_block(const DevTables &h) { return dim3(h.N / kCoefPerThread); }
inline size_t ntt_smem(const DevTables &h) { return (size_t)h.N * sizeof(u64); }

template <typename F>
cudaError_t allow_smem(F *kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)bytes);
}

// ---------------------------------------------------------------------
// Database load: row r, limb j: centered lift of the payload (v > t/2 ->
// v - t), zero-padded to N, forward NTT.  grid (L, rows).
// ---------------------------------------------------------------------
__global__ void k_db_load(const DevTables *T, const u32 *items, u32 plen, u64 *db) {
  extern __shared__ u64 s[];
  const u32 N = T->N, L = T->L, j = blockIdx.x;
  const u64 row = blockIdx.y;
  const NttPrime P = T->prime[j];
  const u64 t = T->t;
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) {
    u64 v = c < plen ? (u64)items[row * plen + c] : 0;
    s[c] = v > t / 2 ? P.q - (t - v) : v;
  }
  __syncthreads();
  smem_ntt_fwd(s, P, T->logN);
  u64 *out = db + (row * L + j) * N;
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) out[c] = s[c];
}

// ---------------------------------------------------------------------
// Batched NTT: unit u, limb l (prime l): base + u*unit_stride + l*N, read
// from src (same limb offset, src_unit_stride) when src != nullptr.
// grid (limb_end - limb_begin, units).
// ---------------------------------------------------------------------
__global__ void k_ntt(const DevTables *T, u64 *base, u64 unit_stride, u32 limb_begin,
                      int inverse, const u64 *src, u64 src_unit_stride) {
  extern __shared__ u64 s[];
  const u32 N = T->N, l = limb_begin + blockIdx.x;
  const u64 u = blockIdx.y;
  const NttPrime P = T->prime[l];
  const u64 *in = src ? src + u * src_unit_stride + (u64)l * N : base + u * unit_stride + (u64)l * N;
  u64 *out = base + u * unit_stride + (u64)l * N;
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) s[c] = in[c];
  __syncthreads();
  if (inverse) smem_ntt_inv(s, P, T->logN);
  else smem_ntt_fwd(s, P, T->logN);
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) out[c] = s[c];
}

// Forward NTT of the P limbs of every job's destination (both polys).
// grid (K, 2 * njobs).
__global__ void k_ntt_jobs_p(const DevTables *T, const MulJob *jobs) {
  extern __shared__ u64 s[];
  const u32 N = T->N, L = T->L, K = T->K, l = L + blockIdx.x;
  const u32 job = blockIdx.y >> 1, poly = blockIdx.y & 1;
  const NttPrime P = T->prime[l];
  u64 *p = jobs[job].dst + ((u64)poly * (L + K) + l) * N;
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) s[c] = p[c];
  __syncthreads();
  smem_ntt_fwd(s, P, T->logN);
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) p[c] = s[c];
}

// ---------------------------------------------------------------------
// Centered Q -> P conversion of coefficient-form polynomials.
// unit u: src + u*src_stride ([L][N]) -> dst + u*dst_stride ([L+K][N], P
// limbs written; Q limbs copied when copy_q).  grid (N/256, units).
// ---------------------------------------------------------------------
template <int L>
__global__ void k_lift(const DevTables *T, const u64 *src, u64 src_stride, u64 *dst,
                       u64 dst_stride, int copy_q) {
  constexpr int K = L + 1;
  const u32 N = T->N;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u64 u = blockIdx.y;
  const u64 *in = src + u * src_stride;
  u64 *out = dst + u * dst_stride;
  u64 x[L], y[K];
#pragma unroll
  for (int j = 0; j < L; ++j) x[j] = in[(u64)j * N + c];
  lift_centered<L, K>(x, y, T->q2b);
  if (copy_q) {
#pragma unroll
    for (int j = 0; j < L; ++j) out[(u64)j * N + c] = x[j];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) out[(u64)(L + k) * N + c] = y[k];
}

// Internal tree nodes: C ([jobs][2][L][N] coefficient form) -> the P limbs
// of jobs[j].dst.  grid (N/256, 2 * njobs).
template <int L>
__global__ void k_lift_jobs(const DevTables *T, const u64 *C, const MulJob *jobs) {
  constexpr int K = L + 1;
  const u32 N = T->N;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u32 job = blockIdx.y >> 1, poly = blockIdx.y & 1;
  const u64 *in = C + ((u64)job * 2 + poly) * L * N;
  u64 *out = jobs[job].dst + (u64)poly * (L + K) * N;
  u64 x[L], y[K];
#pragma unroll
  for (int j = 0; j < L; ++j) x[j] = in[(u64)j * N + c];
  lift_centered<L, K>(x, y, T->q2b);
#pragma unroll
  for (int k = 0; k < K; ++k) out[(u64)(L + k) * N + c] = y[k];
}

// ---------------------------------------------------------------------
// Tensor of two QP-NTT ciphertexts, one output polynomial and limb per
// CTA, followed by the inverse NTT: d0 = a0 b0, d1 = a0 b1 + a1 b0,
// d2 = a1 b1.  grid (L+K, njobs, 3).
// ---------------------------------------------------------------------
__global__ void k_tensor_intt(const DevTables *T, const MulJob *jobs, u64 *Tbuf) {
  extern __shared__ u64 s[];
  const u32 N = T->N, LK = T->L + T->K, l = blockIdx.x, which = blockIdx.z;
  const u64 job = blockIdx.y;
  const NttPrime P = T->prime[l];
  const MulJob J = jobs[job];
  const u64 ps = (u64)LK * N;
  const u64 *a0 = J.a + (u64)l * N, *a1 = a0 + ps;
  const u64 *b0 = J.b + (u64)l * N, *b1 = b0 + ps;
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) {
    u64 v;
    if (which == 0) v = barrett(a0[c], b0[c], P.q, P.mu);
    else if (which == 2) v = barrett(a1[c], b1[c], P.q, P.mu);
    else v = addq(barrett(a0[c], b1[c], P.q, P.mu), barrett(a1[c], b0[c], P.q, P.mu), P.q);
    s[c] = v;
  }
  __syncthreads();
  smem_ntt_inv(s, P, T->logN);
  u64 *out = Tbuf + ((job * 3 + which) * LK + l) * N;
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) out[c] = s[c];
}

// ---------------------------------------------------------------------
// Exact scale-down of every tensor coefficient.  grid (N/256, 3*njobs).
// ---------------------------------------------------------------------
template <int L>
__global__ void k_scale(const DevTables *T, const u64 *Tbuf, u64 *E, int *err) {
  constexpr int K = L + 1;
  const u32 N = T->N;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u64 jw = blockIdx.y;
  const u64 *in = Tbuf + jw * (L + K) * N;
  u64 dq[L], dp[K], e[L];
#pragma unroll
  for (int j = 0; j < L; ++j) dq[j] = in[(u64)j * N + c];
#pragma unroll
  for (int k = 0; k < K; ++k) dp[k] = in[(u64)(L + k) * N + c];
  if (!scale_coeff<L>(dq, dp, e, T->scale)) atomicOr(err, 1);
  u64 *out = E + jw * L * N;
#pragma unroll
  for (int j = 0; j < L; ++j) out[(u64)j * N + c] = e[j];
}

// ---------------------------------------------------------------------
// Key switching with RNS digits, fused with its consumers.  For job `job`
// and output limb j: acc0 = NTT(add0_j) + sum_i NTT([z_i]_{q_j}) * b_ij,
// acc1 = NTT(add1_j) + sum_i NTT([z_i]_{q_j}) * a_ij (digits z_i in
// [0, q_i) < 2 q_j, so one subtraction reduces them).  grid (L, njobs).
// ---------------------------------------------------------------------
struct KsArgs {
  const u64 *z;
  u64 z_stride;
  const u64 *add0;
  u64 add0_stride;
  const u64 *add1;
  u64 add1_stride;
  const u64 *key;
  const u64 *key_s;
  int mode;  // RootMode, or 3 = substitution output
  const MulJob *jobs;
  const SubJob *sjobs;
  const u64 *db;
  u64 *out;
};

template <int BD>
__global__ void __launch_bounds__(BD) k_keyswitch(const DevTables *T, KsArgs A) {
  extern __shared__ u64 s[];
  const u32 N = T->N, L = T->L, logN = T->logN, bd = blockDim.x, tid = threadIdx.x;
  const u32 j = blockIdx.x;
  const u64 job = blockIdx.y;
  const NttPrime P = T->prime[j];
  const u64 q = P.q;
  u64 acc0[kCoefPerThread], acc1[kCoefPerThread];
#pragma unroll
  for (int r = 0; r < kCoefPerThread; ++r) acc0[r] = acc1[r] = 0;

  const u64 *z = A.z + job * A.z_stride;
  for (u32 i = 0; i < L; ++i) {
    const u64 *zi = z + (u64)i * N;
#pragma unroll
    for (int r = 0; r < kCoefPerThread; ++r) {
      u32 c = tid + r * bd;
      u64 d = zi[c];
      s[c] = d >= q ? d - q : d;
    }
    __syncthreads();
    smem_ntt_fwd(s, P, logN);
    const u64 *kb = A.key + ((u64)(i * 2 + 0) * L + j) * N;
    const u64 *ka = A.key + ((u64)(i * 2 + 1) * L + j) * N;
    const u64 *kbs = A.key_s + ((u64)(i * 2 + 0) * L + j) * N;
    const u64 *kas = A.key_s + ((u64)(i * 2 + 1) * L + j) * N;
#pragma unroll
    for (int r = 0; r < kCoefPerThread; ++r) {
      u32 c = tid + r * bd;
      u64 v = s[c];
      acc0[r] = addq(acc0[r], shoup(v, kb[c], kbs[c], q), q);
      acc1[r] = addq(acc1[r], shoup(v, ka[c], kas[c], q), q);
    }
    __syncthreads();
  }
  for (int comp = 0; comp < 2; ++comp) {
    const u64 *add = comp ? A.add1 : A.add0;
    if (!add) continue;
    const u64 *ad = add + job * (comp ? A.add1_stride : A.add0_stride) + (u64)j * N;
#pragma unroll
    for (int r = 0; r < kCoefPerThread; ++r) s[tid + r * bd] = ad[tid + r * bd];
    __syncthreads();
    smem_ntt_fwd(s, P, logN);
#pragma unroll
    for (int r = 0; r < kCoefPerThread; ++r) {
      u32 c = tid + r * bd;
      if (comp) acc1[r] = addq(acc1[r], s[c], q);
      else acc0[r] = addq(acc0[r], s[c], q);
    }
    __syncthreads();
  }

  if (A.mode == ROOT_PM) {
    const u64 *dbr = A.db + ((u64)A.jobs[job].row * L + j) * N;
    u64 *o0 = A.out + (job * 2 + 0) * L * N + (u64)j * N;
    u64 *o1 = A.out + (job * 2 + 1) * L * N + (u64)j * N;
#pragma unroll
    for (int r = 0; r < kCoefPerThread; ++r) {
      u32 c = tid + r * bd;
      u64 m = dbr[c];
      o0[c] = barrett(acc0[r], m, q, P.mu);
      o1[c] = barrett(acc1[r], m, q, P.mu);
    }
    return;
  }
  if (A.mode == INTERNAL) {
    u64 *d = A.jobs[job].dst;
    const u64 ps = (u64)(L + T->K) * N;
#pragma unroll
    for (int r = 0; r < kCoefPerThread; ++r) {
      u32 c = tid + r * bd;
      d[(u64)j * N + c] = acc0[r];
      d[ps + (u64)j * N + c] = acc1[r];
    }
  }
  // coefficient-form output of both polys
  u64 *dst;
  if (A.mode == INTERNAL) dst = A.out + job * 2 * L * N;
  else if (A.mode == ROOT_SEL) dst = A.jobs[job].dst;
  else dst = A.sjobs[job].dst;
  for (int comp = 0; comp < 2; ++comp) {
#pragma unroll
    for (int r = 0; r < kCoefPerThread; ++r) s[tid + r * bd] = comp ? acc1[r] : acc0[r];
    __syncthreads();
    smem_ntt_inv(s, P, logN);
    u64 *o = dst + ((u64)comp * L + j) * N;
#pragma unroll
    for (int r = 0; r < kCoefPerThread; ++r) o[tid + r * bd] = s[tid + r * bd];
    __syncthreads();
  }
}

// k = 1: the selection entry is the leaf itself (Q limbs in NTT form).
// grid (N/256, L, njobs).
__global__ void k_pm_leaf(const DevTables *T, const MulJob *jobs, const u64 *db, u64 *P) {
  const u32 N = T->N, L = T->L, K = T->K, j = blockIdx.y;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u64 job = blockIdx.z;
  const NttPrime Pr = T->prime[j];
  const MulJob J = jobs[job];
  const u64 m = db[((u64)J.row * L + j) * N + c];
  const u64 ps = (u64)(L + K) * N;
  P[(job * 2 + 0) * L * N + (u64)j * N + c] = barrett(J.a[(u64)j * N + c], m, Pr.q, Pr.mu);
  P[(job * 2 + 1) * L * N + (u64)j * N + c] = barrett(J.a[ps + (u64)j * N + c], m, Pr.q, Pr.mu);
}

// acc[2][L][N] += sum over jobs of P[job][2][L][N] (mod q_j).
// grid (N/256, 2L).
__global__ void k_accumulate(const DevTables *T, const u64 *P, u32 njobs, u64 *acc) {
  const u32 N = T->N, L = T->L;
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  const u32 pl = blockIdx.y, j = pl % L;
  const u64 q = T->prime[j].q;
  const u64 off = (u64)pl * N + c, stride = 2ull * L * N;
  u64 a = acc[off];
  for (u32 x = 0; x < njobs; ++x) a = addq(a, P[x * stride + off], q);
  acc[off] = a;
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
__global__ void k_key_prep(const DevTables *T, u64 *key, u64 *key_s) {
  extern __shared__ u64 s[];
  const u32 N = T->N, j = blockIdx.x;
  const u64 unit = blockIdx.y;
  const NttPrime P = T->prime[j];
  u64 *p = key + (unit * T->L + j) * N;
  u64 *ps = key_s + (unit * T->L + j) * N;
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) s[c] = p[c];
  __syncthreads();
  smem_ntt_fwd(s, P, T->logN);
  for (u32 c = threadIdx.x; c < N; c += blockDim.x) {
    u64 w = s[c], rem = w, quo = 0;
    for (int b = 0; b < 64; ++b) {
      rem <<= 1;
      u64 bit = rem >= P.q ? 1 : 0;
      if (bit) rem -= P.q;
      quo = (quo << 1) | bit;
    }
    p[c] = w;
    ps[c] = quo;
  }
}

// blockDim = N / 16: 1024 threads at N = 16384, at most 512 below.
cudaError_t launch_ks(const DevTables *T, const DevTables &h, const KsArgs &A, u32 njobs,
                      cudaStream_t st) {
  cudaError_t e;
  if (h.N / kCoefPerThread > 512) {
    e = allow_smem(k_keyswitch<1024>, ntt_smem(h));
    if (e != cudaSuccess) return e;
    k_keyswitch<1024><<<dim3(h.L, njobs), ntt_block(h), ntt_smem(h), st>>>(T, A);
  } else {
    e = allow_smem(k_keyswitch<512>, ntt_smem(h));
    if (e != cudaSuccess) return e;
    k_keyswitch<512><<<dim3(h.L, njobs), ntt_block(h), ntt_smem(h), st>>>(T, A);
  }
  return cudaGetLastError();
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
                           u32 plen, u64 *db, cudaStream_t st) {
  cudaError_t e = allow_smem(k_db_load, ntt_smem(h));
  if (e != cudaSuccess) return e;
  const u64 chunk = 32768;
  for (u64 r0 = 0; r0 < rows; r0 += chunk) {
    u64 nr = rows - r0 < chunk ? rows - r0 : chunk;
    k_db_load<<<dim3(h.L, (u32)nr), ntt_block(h), ntt_smem(h), st>>>(
        T, items + r0 * plen, plen, db + r0 * h.L * h.N);
  }
  return cudaGetLastError();
}

cudaError_t launch_ntt(const DevTables *T, const DevTables &h, u64 *base, u32 units,
                       u64 unit_stride, u32 limb_begin, u32 limb_end, bool inverse,
                       const u64 *src, u64 src_unit_stride, cudaStream_t st) {
  if (!units || limb_end <= limb_begin) return cudaSuccess;
  cudaError_t e = allow_smem(k_ntt, ntt_smem(h));
  if (e != cudaSuccess) return e;
  const u32 chunk = 32768;
  for (u32 u0 = 0; u0 < units; u0 += chunk) {
    u32 nu = units - u0 < chunk ? units - u0 : chunk;
    k_ntt<<<dim3(limb_end - limb_begin, nu), ntt_block(h), ntt_smem(h), st>>>(
        T, base + (u64)u0 * unit_stride, unit_stride, limb_begin, inverse ? 1 : 0,
        src ? src + (u64)u0 * src_unit_stride : nullptr, src_unit_stride);
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
                  dst + (u64)u0 * dst_stride, dst_stride, copy_q ? 1 : 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_lift_jobs(const DevTables *T, const DevTables &h, const u64 *C,
                             const MulJob *jobs, u32 njobs, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  dim3 grid(h.N / 256, 2 * njobs);
  CW_DISPATCH_L(h.L, k_lift_jobs, grid, 256, 0, st, T, C, jobs);
  return cudaGetLastError();
}

cudaError_t launch_ntt_jobs_p(const DevTables *T, const DevTables &h, const MulJob *jobs,
                              u32 njobs, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  cudaError_t e = allow_smem(k_ntt_jobs_p, ntt_smem(h));
  if (e != cudaSuccess) return e;
  k_ntt_jobs_p<<<dim3(h.K, 2 * njobs), ntt_block(h), ntt_smem(h), st>>>(T, jobs);
  return cudaGetLastError();
}

cudaError_t launch_tensor_intt(const DevTables *T, const DevTables &h, const MulJob *jobs,
                               u32 njobs, u64 *Tbuf, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  cudaError_t e = allow_smem(k_tensor_intt, ntt_smem(h));
  if (e != cudaSuccess) return e;
  k_tensor_intt<<<dim3(h.L + h.K, njobs, 3), ntt_block(h), ntt_smem(h), st>>>(T, jobs, Tbuf);
  return cudaGetLastError();
}

cudaError_t launch_scale(const DevTables *T, const DevTables &h, const u64 *Tbuf, u32 njobs,
                         u64 *E, int *err, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  dim3 grid(h.N / 256, 3 * njobs);
  CW_DISPATCH_L(h.L, k_scale, grid, 256, 0, st, T, Tbuf, E, err);
  return cudaGetLastError();
}

cudaError_t launch_relin(const DevTables *T, const DevTables &h, const u64 *E, u32 njobs,
                         const MulJob *jobs, int mode, const u64 *rlk, const u64 *rlk_s,
                         const u64 *db, u64 *out, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  const u64 LN = (u64)h.L * h.N;
  KsArgs A;
  A.z = E + 2 * LN;
  A.z_stride = 3 * LN;
  A.add0 = E;
  A.add0_stride = 3 * LN;
  A.add1 = E + LN;
  A.add1_stride = 3 * LN;
  A.key = rlk;
  A.key_s = rlk_s;
  A.mode = mode;
  A.jobs = jobs;
  A.sjobs = nullptr;
  A.db = db;
  A.out = out;
  return launch_ks(T, h, A, njobs, st);
}

cudaError_t launch_pm_leaf(const DevTables *T, const DevTables &h, const MulJob *jobs,
                           u32 njobs, const u64 *db, u64 *P, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  k_pm_leaf<<<dim3(h.N / 256, h.L, njobs), 256, 0, st>>>(T, jobs, db, P);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(const DevTables &h, const DevTables *T, const u64 *P, u32 njobs,
                              u64 *acc, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  k_accumulate<<<dim3(h.N / 256, 2 * h.L), 256, 0, st>>>(T, P, njobs, acc);
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
                                 const u64 *key_s, cudaStream_t st) {
  if (!njobs) return cudaSuccess;
  const u64 LN = (u64)h.L * h.N;
  KsArgs A;
  A.z = tau + LN;
  A.z_stride = 2 * LN;
  A.add0 = tau;
  A.add0_stride = 2 * LN;
  A.add1 = nullptr;
  A.add1_stride = 0;
  A.key = key;
  A.key_s = key_s;
  A.mode = 3;
  A.jobs = nullptr;
  A.sjobs = jobs;
  A.db = nullptr;
  A.out = nullptr;
  return launch_ks(T, h, A, njobs, st);
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
  cudaError_t e = allow_smem(k_key_prep, ntt_smem(h));
  if (e != cudaSuccess) return e;
  k_key_prep<<<dim3(h.L, nkeys * 2 * h.L), ntt_block(h), ntt_smem(h), st>>>(T, key, key_s);
  return cudaGetLastError();
}

}  // namespace cw
