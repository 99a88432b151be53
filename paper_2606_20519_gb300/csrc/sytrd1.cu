// One-stage Householder tridiagonalisation for cones whose trailing matrix
// stays in shared memory or L2 (the medium sizes of the paper's
// process-matrix step), in a single persistent cooperative kernel.  Three
// routes share the structure below: double-float with the columns in shared
// memory, double-float with the columns in place in global memory (launches
// whose matrices fit in L2), and FP64 with the columns in L2 (larger ones).
//
// CTA r of a cone's group of G CTAs owns the columns i with i mod G = r for
// the whole reduction (both triangles are kept, so a column is contiguous).
// Step j (reflector H_j = I - tau_j v v^T from column j, v indexed from row
// j+1, m = n - j - 1 entries, v_0 = 1) needs p = tau_j A22 v, whose entries
// the owners of the columns produce, and column j+1 as the previous step
// left it.  Both are published into a write-once slab of step j (2m
// doubles) that holds a sentinel NaN until the value arrives: a reader polls
// the values themselves, so there is no group barrier per column -- a CTA
// starts step j as soon as the last value it needs has landed in L2.  After
// the poll every CTA, redundantly (the same arithmetic in each, so no column
// is handed over):
//     K = (tau_j / 2) p^T v,
//     column j+1 updated by step j:  a_t - p_t - v_t (p_0 - 2K),
//     reflector j+1 from it (its sum of squares here; beta, tau, 1/(x_0 - beta)
//     by one thread while the pass below runs);
// then one fused pass over its own columns i >= j+2 applies the rank-2 update
//     A(r, i) -= v_r (p_i - 2K v_i) + p_r v_i        (= v w^T + w v^T, w = p - K v)
// and forms the next step's p_i = tau_{j+1} u^T A(j+2:, i) (one read and one
// write of A), publishing p_i and, from the owner of column j+2, that
// column (one or two warps per column in the double-float routes, (column,
// chunk) work items over all warps in the FP64 route).
// d, e, tau and the reflectors (packed into 32-column blocks with their unit
// diagonal and zeros, ready for the blocked back-transformation) are written
// as they are formed.  The slabs live in the cone's D&C buffer QA (n^2
// doubles, unused until the divide and conquer); every CTA fills its share
// with the sentinel and one group barrier (release/acquire counters) orders
// the fill before the first publication.  Every wait is bounded
// (ST_TIMEOUT on expiry); the launch is cooperative, so every CTA is
// resident.
//
// larft1_kernel then forms, for every 32-reflector block, the triangular
// factor T of H_0 ... H_31 = I - V T V^T.
#include <limits.h>
#include <math.h>

#include "dfloat.cuh"
#include "internal.cuh"

namespace scs {

namespace {

constexpr int kSyThreads = 256;
constexpr int kNb = kSy1Block;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Sum over the CTA; every thread gets the same value (pairwise, in the same
// order).  red is [2][8]: reductions alternate halves, so the write of one
// cannot overtake the reads of the previous one.
__device__ double block_sum256(double v, double* red, int& parity) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* r = red + 8 * parity;
  parity ^= 1;
  if (lane == 0) r[w] = v;
  __syncthreads();
  static_assert(kSyThreads == 256, "tree below sums 8 warps");
  return ((r[0] + r[1]) + (r[2] + r[3])) + ((r[4] + r[5]) + (r[6] + r[7]));
}

// Barrier over the G CTAs of one cone with its arrivals spread over 8
// counters (CTA r adds to counter r mod 8, 128 bytes apart); threads 0..7
// each wait for one counter.  Returns false (in every thread) when a wait
// ran out.
constexpr int kBarLanes = 8, kBarStride = 32;
__device__ bool group_barrier8(int* counters, int rank, int G, int step, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(counters + kBarStride * (rank % kBarLanes)),
                 "r"(1)
                 : "memory");
  }
  int ok = 1;
  const int t = threadIdx.x;
  if (t < kBarLanes && t < G) {
    const int target = step * ((G - 1 - t) / kBarLanes + 1);  // CTAs with rank mod 8 == t, per step
    const int* cnt = counters + kBarStride * t;
    if (ld_acquire(cnt) < target) {
      const long long t0 = clock64();
      while (ld_acquire(cnt) < target) {
        if (clock64() - t0 > limit) { ok = 0; break; }
      }
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

constexpr int kPartMax = 2048; // work items per round (shared-memory partial sums)
constexpr size_t kSyResidentMax = 200 * 1024;  // dynamic shared memory of a launch, at most

// Householder reflector of x[0 .. len-1] in place (every thread of the CTA
// calls it; x in shared memory): H x = beta e_1 with H = I - tau u u^T,
// u_0 = 1 (LAPACK convention).  x becomes u; tau and beta are returned.
__device__ double make_reflector(double* x, int len, double* red, int& parity, double* sh, double* beta_out) {
  double ps = 0.0;
  for (int t = 1 + threadIdx.x; t < len; t += kSyThreads) ps = fma(x[t], x[t], ps);
  const double sigma = block_sum256(ps, red, parity);
  if (threadIdx.x == 0) {
    const double alpha = x[0];
    double beta = alpha, tau = 0.0, scal = 0.0;
    if (sigma != 0.0) {
      const double nrm = sqrt(fma(alpha, alpha, sigma));
      beta = alpha >= 0.0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    sh[0] = beta; sh[1] = tau; sh[2] = scal;
  }
  __syncthreads();
  const double scal = sh[2];
  for (int t = 1 + threadIdx.x; t < len; t += kSyThreads) x[t] *= scal;
  __syncthreads();
  if (threadIdx.x == 0) x[0] = 1.0;
  *beta_out = sh[0];
  return sh[1];
}

// Reflector j (u = scal * x, x indexed from row j+1) into its 32-column
// block of V1, with the unit diagonal and the zeros above; rows spread over
// the group.
__device__ void store_reflector(const ConeDev& c, int n, int j, const double* u, int rank, int G,
                                double scal = 1.0) {
  const int q = j / kNb, col = j % kNb;
  const int r0 = q * kNb + 1;               // first row of block q
  const int mq = n - r0;                    // rows of block q
  double* Vq = c.V1 + (int64_t)q * n * kNb;  // mq x 32, ld mq
  for (int r = rank * kSyThreads + threadIdx.x; r < mq; r += G * kSyThreads) {
    const int row = r0 + r;
    double val = 0.0;
    if (row == j + 1) val = 1.0;
    else if (row > j + 1) val = scal * u[row - j - 1];
    Vq[(int64_t)r + (int64_t)col * mq] = val;
  }
}

// One pass over this CTA's columns i >= r0 (i mod G = rank), rows r0 .. n-1,
// read from and written to L2: with UPDATE, first A(r, i) -= v_r w_i + w_r v_i
// (vu, wu indexed from row r0 - 1); then p_i = coef[0] (A(r0, i) + coef[1]
// sum_{r > r0} A(r, i) x_r) into pbuf[i], x indexed from row r0.  The next
// reflector is u = coef[1] x with u_0 = 1, so p_i = tau u^T A(r0:, i) without
// x having been rescaled; coef is read only after the pass's first barrier,
// so the reflector's scalars may still be in the making (by thread 0) while
// the pass starts.  Work items are (column, CH-row chunk) pairs spread over
// the warps.
template <bool UPDATE, int CH>
__device__ void column_pass(double* __restrict__ A, int n, int r0, const double* __restrict__ x, const double* coef,
                            const double* __restrict__ vu, const double* __restrict__ wu, double* pbuf,
                            double* psum, int pcap, int rank, int G) {
  constexpr int NR = CH / 32;
  const int L = n - r0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int first = r0 + ((rank - r0 % G) + G) % G;
  const int ncol = first < n ? (n - 1 - first) / G + 1 : 0;
  const int nch = (L + CH - 1) / CH;
  const int per = max(1, pcap / nch);
  for (int k0 = 0; k0 < ncol; k0 += per) {
    const int kc = min(ncol - k0, per);
    for (int it = warp; it < kc * nch; it += kSyThreads / 32) {
      const int k = k0 + it / nch, ch = it % nch;
      const int i = first + G * k;
      double* col = A + (int64_t)i * n + r0;
      const int t0 = ch * CH + lane;
      double a[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int t = t0 + 32 * r;
        a[r] = t < L ? __ldcg(col + t) : 0.0;
      }
      if (UPDATE) {
        const double vi = vu[i - r0 + 1], wi = wu[i - r0 + 1];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const int t = t0 + 32 * r;
          if (t < L) {
            a[r] = fma(-vu[t + 1], wi, fma(-wu[t + 1], vi, a[r]));
            __stcg(col + t, a[r]);
          }
        }
      }
      double acc = 0.0;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int t = t0 + 32 * r;
        if (t < L && t > 0) acc = fma(a[r], x[t], acc);
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) psum[it] = acc;
    }
    __syncthreads();
    const double tau = coef[0], scal = coef[1];
    for (int kk = tid; kk < kc; kk += kSyThreads) {
      double sdot = 0.0;
      for (int ch = 0; ch < nch; ++ch) sdot += psum[kk * nch + ch];
      const int i = first + G * (k0 + kk);
      __stcg(pbuf + i, tau * fma(scal, sdot, __ldcg(A + (int64_t)i * n + r0)));
    }
    __syncthreads();
  }
  // the caller reads the coefficients (written by thread 0 before the pass)
  // after it: a CTA without columns still passes one barrier
  if (ncol == 0) __syncthreads();
}

// Partial sums of the FP64 route's pass: (column, 64-row chunk) items per round.
__host__ __device__ inline int sytrd1_pcap(int n, int G) {
  const int items = ((n + G - 1) / G) * ((n + 63) / 64);  // up to 64-row items
  return items < kPartMax ? items : kPartMax;
}
// Shared memory of a CTA.  Resident route (double-float): two v buffers, p,
// the updated column (4n pairs) and the CTA's own columns; otherwise (FP64,
// columns in L2) v, p, column and the partial sums.
__host__ __device__ inline size_t sytrd1_bytes(int n, int G, bool res) {
  if (res) return ((size_t)4 * n + (size_t)((n + G - 1) / G) * n) * sizeof(double);
  return ((size_t)3 * n + sytrd1_pcap(n, G)) * sizeof(double);
}
// Double-float route with the columns in global memory: the 4n pairs only.
__host__ __device__ inline size_t sytrd1_glb_bytes(int n) { return (size_t)4 * n * sizeof(double); }

// ---------------------------------------------------------------- double-float path
// The shared-memory-resident route (every CTA's columns in shared memory)
// computes in double-float arithmetic (dfloat.cuh): every operation of a step
// is an FP32 pipe instruction.  The matrix is scaled by a power of two into
// [1, 2) for its largest entry first (exact; FP32's exponent range then holds
// every entry whose magnitude matters at FP64 accuracy), d and e are scaled
// back, the reflectors and tau are scale-free.  FP64 is left for the
// conversions at the boundaries (the matrix once, d, e, tau and the stored
// reflectors) and the first reflector's scalars.
__device__ __forceinline__ dfl* slab(dfl* base, int n, int j) {
  return base + (int64_t)2 * j * (n - 1) - (int64_t)j * (j - 1);
}

// Published double-float values: one 8-byte single-copy-atomic word each,
// hi in the low half.  The sentinel's hi half is a NaN with a payload FP32
// arithmetic never produces (NaN results carry the canonical payload).
constexpr unsigned long long kSentinelDf = 0xA5A5A5A5FFA5A5A5ull;
__device__ __forceinline__ void st_pub_df(dfl* p, dfl v) {
  const unsigned long long bits =
      ((unsigned long long)__float_as_uint(v.lo) << 32) | (unsigned long long)__float_as_uint(v.hi);
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(bits) : "memory");
}
__device__ __forceinline__ unsigned long long ld_pub_bits(const dfl* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ dfl df_from_bits(unsigned long long b) {
  return df_make(__uint_as_float((unsigned)(b & 0xffffffffull)), __uint_as_float((unsigned)(b >> 32)));
}

__device__ dfl block_sum_df(dfl v, dfl* red, int& parity) {
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  dfl* r = red + 8 * parity;
  parity ^= 1;
  if (lane == 0) r[w] = v;
  __syncthreads();
  return df_add(df_add(df_add(r[0], r[1]), df_add(r[2], r[3])), df_add(df_add(r[4], r[5]), df_add(r[6], r[7])));
}

// The reflector's scalars from alpha and sigma = sum of the other squares
// (double-float, one thread): beta, tau and 1 / (alpha - beta).
__device__ __forceinline__ void reflector_scalars_df(dfl alpha, dfl sigma, dfl* beta, dfl* tau, dfl* scal) {
  *beta = alpha;
  *tau = df_zero();
  *scal = df_zero();
  if (sigma.hi != 0.0f || sigma.lo != 0.0f) {
    const dfl nrm = df_sqrt(df_fma(alpha, alpha, sigma));
    *beta = alpha.hi >= 0.0f ? df_neg(nrm) : nrm;
    *tau = df_div(df_add(*beta, df_neg(alpha)), *beta);
    *scal = df_div(df_make(1.0f, 0.0f), df_add(alpha, df_neg(*beta)));
  }
}

// The reflector's scalars from alpha and sigma = sum of the other squares
// (FP64, one thread): beta, tau and 1 / (alpha - beta).
__device__ __forceinline__ void reflector_scalars(double alpha, double sigma, double* beta, double* tau,
                                                  double* scal) {
  *beta = alpha;
  *tau = 0.0;
  *scal = 0.0;
  if (sigma != 0.0) {
    const double nrm = sqrt(fma(alpha, alpha, sigma));
    *beta = alpha >= 0.0 ? -nrm : nrm;
    *tau = (*beta - alpha) / *beta;
    *scal = 1.0 / (alpha - *beta);
  }
}

// Reflector j (u = scal x, x indexed from row j+1) into V1, as store_reflector.
__device__ void store_reflector_df(const ConeDev& c, int n, int j, const dfl* u, int rank, int G, dfl scal,
                                   bool scaled) {
  const int q = j / kNb, col = j % kNb;
  const int r0 = q * kNb + 1;
  const int mq = n - r0;
  // double-float pairs (the back-transformation of this route reads them so)
  dfl* Vq = reinterpret_cast<dfl*>(c.V1) + (int64_t)q * n * kNb;
  for (int r = rank * kSyThreads + threadIdx.x; r < mq; r += G * kSyThreads) {
    const int row = r0 + r;
    dfl val = df_zero();
    if (row == j + 1) val = df_make(1.0f, 0.0f);
    else if (row > j + 1) val = scaled ? df_mul(scal, u[row - j - 1]) : u[row - j - 1];
    Vq[(int64_t)r + (int64_t)col * mq] = val;
  }
}

// Waits (bounded) until thread 0 of this CTA has announced the reflector's
// scalars for `tag`.
__device__ __forceinline__ void wait_coef(const int* coef_tag, int tag, int* status) {
  if (*(volatile const int*)coef_tag != tag) {
    long long spins = 0;
    while (*(volatile const int*)coef_tag != tag) {
      if (++spins > (1ll << 30)) { atomicOr(status, ST_TIMEOUT); break; }
    }
  }
  __threadfence_block();
}

// The double-float pass with one warp per column: the warp applies step
// j's rank-2 update to all of its column's rows, forms the column's whole dot
// product with the next reflector's source x, and its lane 0 publishes
// p_i = tau (A(r0, i) + scal sum_{r > r0} A(r, i) x_r) as soon as thread 0 has
// set the reflector's scalars (coef, announced by *coef_tag = tag).  No CTA
// barrier: columns go to warps 1, 2, .., 7, 0 (warp 0's thread 0 forms the
// scalars first).  The owner of column r0 publishes its rows to Cn.
// With at most NW / 2 columns, two warps share each column (interleaved
// chunks of rows): the second hands its part of the dot product to the
// first through half_part[k], announced by half_tag[k] = tag.
template <bool UPDATE, bool GLB>
__device__ void column_pass_dfw(dfl* __restrict__ cols, int n, int r0, const dfl* __restrict__ x, const dfl* coef,
                                const int* coef_tag, int tag, const dfl* __restrict__ vu,
                                const dfl* __restrict__ pu, dfl K2, dfl* Pn, dfl* Cn, int rank, int G,
                                int* status, int* half_tag, dfl* half_part) {
  // columns in L2 (GLB): more rows in flight per lane
  constexpr int U = GLB ? 8 : 4;
  constexpr int NW = kSyThreads / 32;
  const int L = n - r0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int first = r0 + ((rank - r0 % G) + G) % G;
  const int ncol = first < n ? (n - 1 - first) / G + 1 : 0;
  const int vw = (warp + NW - 1) % NW;  // warp 0 (whose thread 0 forms the scalars) last
  const bool split = 2 * ncol <= NW;
  const int half = split ? (vw & 1) : 0;
  const int tstride = (split ? 2 : 1) * 32 * U;
  for (int k = split ? vw / 2 : vw; k < ncol; k += split ? NW / 2 : NW) {
    const int i = first + G * k;
    dfl* col = cols + (int64_t)(GLB ? i : (i - rank) / G) * n + r0;
    const bool pub_col = i == r0;
    dfl nai = df_zero(), nvi = df_zero();
    if (UPDATE) {
      const dfl vi = vu[i - r0 + 1];
      nai = df_neg(df_fma(df_neg(K2), vi, pu[i - r0 + 1]));  // -(p_i - 2K v_i)
      nvi = df_neg(vi);
    }
    df_dot acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = df_dot_zero();
    for (int t0 = lane + half * 32 * U; t0 < L; t0 += tstride) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int t = t0 + 32 * u;
        if (t < L) {
          dfl a = col[t];
          if (UPDATE) {
            a = df_add2prod(a, vu[t + 1], nai, pu[t + 1], nvi);
            col[t] = a;
          }
          if (pub_col) st_pub_df(Cn + t, a);
          if (t > 0) acc[u] = df_dot_add(acc[u], a, x[t]);
        }
      }
    }
    dfl sdot = df_dot_value(acc[0]);
#pragma unroll
    for (int u = 1; u < U; ++u) sdot = df_add(sdot, df_dot_value(acc[u]));
    for (int o = 16; o > 0; o >>= 1) sdot = df_add(sdot, df_shfl_xor(sdot, o));
    if (split && half == 1) {
      if (lane == 0) {
        half_part[k] = sdot;
        __threadfence_block();
        *(volatile int*)(half_tag + k) = tag;
      }
      continue;  // the first warp of the pair publishes
    }
    if (lane == 0) {
      if (split) {
        wait_coef(half_tag + k, tag, status);
        sdot = df_add(sdot, half_part[k]);
      }
      // thread 0 of this CTA forms the scalars while the columns are updated
      wait_coef(coef_tag, tag, status);
      const dfl tau = coef[0], scal = coef[1];
      st_pub_df(Pn + (i - r0), df_mul(tau, df_fma(scal, sdot, col[0])));
    }
  }
}


__device__ bool poll_step_df(const dfl* P, const dfl* C, int m, const dfl* v, dfl* ps, dfl* bs, long long limit,
                             dfl* red) {
  dfl pt = df_zero();
  int ok = 1;
  for (int base = 0; base < m && ok; base += 4 * kSyThreads) {
    unsigned long long pr[4], ar[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = base + q * kSyThreads + threadIdx.x;
      pr[q] = t < m ? ld_pub_bits(P + t) : 0ull;
      ar[q] = t < m ? ld_pub_bits(C + t) : 0ull;
    }
    bool miss = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) miss = miss || pr[q] == kSentinelDf || ar[q] == kSentinelDf;
    if (miss) {
      const long long t0 = clock64();
      while (true) {
        miss = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int t = base + q * kSyThreads + threadIdx.x;
          if (pr[q] == kSentinelDf) { pr[q] = ld_pub_bits(P + t); miss = miss || pr[q] == kSentinelDf; }
          if (ar[q] == kSentinelDf) { ar[q] = ld_pub_bits(C + t); miss = miss || ar[q] == kSentinelDf; }
        }
        if (!miss) break;
        if (clock64() - t0 > limit) { ok = 0; break; }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = base + q * kSyThreads + threadIdx.x;
      if (t < m) {
        const dfl p = df_from_bits(pr[q]);
        ps[t] = p;
        bs[t] = df_add(df_from_bits(ar[q]), df_neg(p));
        pt = df_fma(p, v[t], pt);
      }
    }
  }
  // this warp's part of p^T v into red[warp] before the barrier
  for (int o = 16; o > 0; o >>= 1) pt = df_add(pt, df_shfl_xor(pt, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pt;
  return __syncthreads_and(ok) != 0;
}

// The double-float route (structure as sytrd1_body).  The CTA's own columns
// live in shared memory (GLB false: column i at slot (i - rank) / G), or, when
// they do not fit, in place of the FP64 matrix in global memory (GLB: column
// i where it was, as FP32 pairs of the same 8 bytes; only the owner touches
// it, so it stays in L2).  sh64: FP64 scalars of thread 0; shd: their
// double-float copies.
template <bool GLB>
__device__ void sytrd1_body_df(const ConeDev& c, int rank, int G, long long wait_limit, double* sy_smem,
                               dfl* red, double* sh64, dfl* shd, int* coef_tag, int* half_tag, dfl* half_part) {
  const int n = (int)c.n;
  double* A = c.A;
  dfl* base = reinterpret_cast<dfl*>(sy_smem);
  dfl* vc = base;           // v of the current step (two buffers, alternating)
  dfl* vn = base + n;
  dfl* ps = base + 2 * n;
  dfl* bs = base + 3 * n;
  dfl* cols = GLB ? reinterpret_cast<dfl*>(A) : base + 4 * n;
  double* colsd = GLB ? A : sy_smem + 4 * n;  // the same storage, first holding FP64
  auto slot = [&](int i) -> int64_t { return GLB ? i : (i - rank) / G; };
  dfl* pub = reinterpret_cast<dfl*>(c.QA);
  const int tid = threadIdx.x;
  int parity = 0;
  // ---- own columns as FP64, and the largest exponent among them
  int emax = 0;
  for (int i = rank; i < n; i += G) {
    const double* src = A + (int64_t)i * n;
    double* dst = colsd + slot(i) * n;
    for (int r = tid; r < n; r += kSyThreads) {
      const double v = __ldcg(src + r);
      if (!GLB) dst[r] = v;
      emax = max(emax, (int)((__double2hiint(v) >> 20) & 0x7FF));
    }
  }
  // GLB: column 0 and A(0, 0) are read before any owner rewrites its columns
  // in place (vc holds column 0's rows 1 .. n-1 as FP64 until the prologue)
  double a00 = 0.0;
  if (GLB && n >= 3) {
    double* v64 = reinterpret_cast<double*>(vc);
    for (int t = tid; t < n - 1; t += kSyThreads) v64[t] = __ldcg(A + 1 + t);
    a00 = __ldcg(A);
  }
  if (n < 3) {
    __syncthreads();
    if (rank == 0 && tid == 0) {
      c.d[0] = A[0];
      c.e[0] = n == 2 ? A[1] : 0.0;
      if (n == 2) { c.d[1] = A[3]; c.e[1] = 0.0; }
    }
    return;
  }
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if ((tid & 31) == 0 && emax > 0) atomicMax(c.prog + 1, emax);
  {
    const int64_t total = (int64_t)n * n - n - 2;
    const dfl sent = df_from_bits(kSentinelDf);
    for (int64_t e = (int64_t)rank * kSyThreads + tid; e < total; e += (int64_t)G * kSyThreads) pub[e] = sent;
  }
  if (!group_barrier8(c.prog, rank, G, 1, wait_limit)) {
    if (tid == 0) atomicOr(c.status, ST_TIMEOUT);
    return;
  }
  // scale 2^(1023 - eb) puts the largest entry into [1, 2); outputs scale back
  int eb = *((volatile int*)(c.prog + 1));
  eb = min(max(eb, 1), 2045);
  const double s_in = __longlong_as_double((long long)(2046 - eb) << 52);
  const double s_out = __longlong_as_double((long long)eb << 52);
  for (int i = rank; i < n; i += G) {
    dfl* dst = cols + slot(i) * n;
    const double* srcd = colsd + slot(i) * n;
    for (int r = tid; r < n; r += kSyThreads) dst[r] = df_from_d(srcd[r] * s_in);
  }
  // ---- prologue: reflector 0 from column 0 (every CTA), p_0 and column 1 into slab 0
  dfl ss = df_zero();
  for (int t = tid; t < n - 1; t += kSyThreads) {
    const double a = GLB ? reinterpret_cast<const double*>(vc)[t] : __ldcg(A + 1 + t);
    const dfl v = df_from_d(a * s_in);
    vc[t] = v;
    if (t >= 1) ss = df_fma(v, v, ss);
  }
  __syncthreads();
  {
    const dfl sig = block_sum_df(ss, red, parity);
    if (tid == 0) {
      double beta, tau, scal;
      reflector_scalars(df_to_d(vc[0]), df_to_d(sig), &beta, &tau, &scal);
      sh64[0] = beta; sh64[1] = tau;
      shd[0] = df_from_d(tau); shd[1] = df_from_d(scal);
    }
    __syncthreads();
    const dfl scal = shd[1];
    for (int t = 1 + tid; t < n - 1; t += kSyThreads) vc[t] = df_mul(scal, vc[t]);
    __syncthreads();
    if (tid == 0) vc[0] = df_make(1.0f, 0.0f);
    if (rank == 0 && tid == 0) {
      c.d[0] = GLB ? a00 : __ldcg(A);
      c.e[0] = sh64[0] * s_out;
      c.tau1[0] = sh64[1];
    }
    store_reflector_df(c, n, 0, vc, rank, G, df_zero(), false);
    if (tid == 0) {
      shd[1] = df_make(1.0f, 0.0f);  // coefficients (tau, 1): v_0 is scaled already
      *coef_tag = -1;
    }
    __syncthreads();
  }
  column_pass_dfw<false, GLB>(cols, n, 1, vc, shd, coef_tag, -1, nullptr, nullptr, df_zero(), slab(pub, n, 0),
                              slab(pub, n, 0) + (n - 1), rank, G, c.status, half_tag, half_part);
  dfl tau = shd[0];
  __syncthreads();
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    dfl* P = slab(pub, n, j);
    dfl* rp = red + 8 * parity;
    parity ^= 1;
    if (!poll_step_df(P, P + m, m, vc, ps, bs, wait_limit, rp)) {
      if (tid == 0) atomicOr(c.status, ST_TIMEOUT);
      return;
    }
    const dfl s = df_add(df_add(df_add(rp[0], rp[1]), df_add(rp[2], rp[3])),
                         df_add(df_add(rp[4], rp[5]), df_add(rp[6], rp[7])));
    const dfl K = df_mul(df_make(0.5f * tau.hi, 0.5f * tau.lo), s);
    const dfl K2 = df_make(2.0f * K.hi, 2.0f * K.lo);
    const dfl c0 = df_add(ps[0], df_neg(K2));
    const dfl nc0 = df_neg(c0);
    dfl sq = df_zero();
    for (int t = tid; t < m; t += kSyThreads) {
      const dfl nc = df_fma(vc[t], nc0, bs[t]);
      bs[t] = nc;
      if (t >= 2) sq = df_fma(nc, nc, sq);
    }
    if (j + 3 < n) {
      const dfl sig = block_sum_df(sq, red, parity);
      dfl beta1;
      if (tid == 0) {
        reflector_scalars_df(bs[1], sig, &beta1, shd, shd + 1);
        __threadfence_block();
        *(volatile int*)coef_tag = j;
      }
      dfl* Pn = slab(pub, n, j + 1);
      column_pass_dfw<true, GLB>(cols, n, j + 2, bs + 1, shd, coef_tag, j, vc, ps, K2, Pn, Pn + (m - 1), rank,
                                 G, c.status, half_tag, half_part);
      // every thread reads the scalars after thread 0 announced them
      wait_coef(coef_tag, j, c.status);
      const dfl tau1 = shd[0], scal1 = shd[1];
      if (rank == 0 && tid == 0) {
        c.d[j + 1] = df_to_d(bs[0]) * s_out;
        c.e[j + 1] = df_to_d(beta1) * s_out;
        c.tau1[j + 1] = df_to_d(tau1);
      }
      store_reflector_df(c, n, j + 1, bs + 1, rank, G, scal1, true);
      // v_{j+1} into the other buffer (the current one may still be read by a
      // warp's update), then the barrier before the next step reads it
      for (int t = tid; t < m - 1; t += kSyThreads) vn[t] = t == 0 ? df_make(1.0f, 0.0f) : df_mul(scal1, bs[1 + t]);
      tau = tau1;
      __syncthreads();
      dfl* tmp = vc;
      vc = vn;
      vn = tmp;
    } else {
      __syncthreads();
      if (rank == 0 && tid == 0) {
        c.d[n - 2] = df_to_d(bs[0]) * s_out;
        c.e[n - 2] = df_to_d(bs[1]) * s_out;
        c.e[n - 1] = 0.0;
      }
      if (rank == (n - 1) % G && tid == 0) {
        const dfl a = cols[slot(n - 1) * n + (n - 1)];
        const dfl w1 = df_fma(df_neg(K), vc[1], ps[1]);
        const dfl two_vw = df_mul(df_make(2.0f * vc[1].hi, 2.0f * vc[1].lo), w1);
        c.d[n - 1] = df_to_d(df_add(a, df_neg(two_vw))) * s_out;
      }
    }
  }
}

// The FP64 route with the columns in L2 (cones beyond the double-float
// routes' reach: launches whose matrices exceed L2).  Step j (reflector
// H_j = I - tau_j v v^T from column j, v indexed from row j+1, m = n - j - 1
// entries), with p = tau_j A22 v already in pbuf:
//   every CTA, after one group barrier per column: w = p - (tau_j / 2)(p^T v) v
//     and the updated column j+1 (rows j+1 ..) from its value in A, v and w,
//     so the next reflector is formed redundantly, with no hand-off;
//   then one pass over its own columns i >= j+2 applies A <- A - v w^T - w v^T
//     to rows j+2 .. and forms the next step's p_i (one read and one write of A).
// For matrices that stream from L2 and HBM this measured faster than the
// polled slabs of the double-float routes (4 x 4096: 661 ms against 700 ms).
__device__ void sytrd1_body(const ConeDev& c, int rank, int G, long long wait_limit, double* sy_smem, double* red,
                            double* sh) {
  const int n = (int)c.n;
  double* A = c.A;
  const int pcap = sytrd1_pcap(n, G);
  double* vc = sy_smem;             // v_j (rows j+1 ..)
  double* w = sy_smem + n;          // p_j, then w_j
  double* vx = sy_smem + 2 * n;     // updated column j+1 (rows j+1 ..), then v_{j+1} at vx + 1
  double* psum = sy_smem + 3 * n;   // pcap partial dot products
  // p, double-buffered by step parity: a CTA writes step j+2's values only
  // after every CTA has passed step j+1's barrier, i.e. finished reading
  // step j's values
  double* pbuf2 = c.X;              // 2 x n
  int* bar = c.prog;
  const int tid = threadIdx.x;
  int parity = 0, bstep = 0;
  if (n < 3) {
    __syncthreads();
    if (rank == 0 && tid == 0) {
      c.d[0] = A[0];
      c.e[0] = n == 2 ? A[1] : 0.0;
      if (n == 2) { c.d[1] = A[3]; c.e[1] = 0.0; }
    }
    return;
  }
  // ---- prologue: reflector 0 from column 0, p_0 for my columns
  double beta, tau;
  for (int t = tid; t < n - 1; t += kSyThreads) vc[t] = __ldcg(A + 1 + t);
  __syncthreads();
  tau = make_reflector(vc, n - 1, red, parity, sh, &beta);
  __syncthreads();
  if (rank == 0 && tid == 0) {
    c.d[0] = __ldcg(A);
    c.e[0] = beta;
    c.tau1[0] = tau;
  }
  store_reflector(c, n, 0, vc, rank, G);
  // v_0 is already scaled (u = v): coefficients (tau, 1)
  if (tid == 0) { sh[1] = tau; sh[2] = 1.0; }
  __syncthreads();
  if (n <= 256) column_pass<false, 128>(A, n, 1, vc, sh + 1, nullptr, nullptr, pbuf2, psum, pcap, rank, G);
  else column_pass<false, 256>(A, n, 1, vc, sh + 1, nullptr, nullptr, pbuf2, psum, pcap, rank, G);
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    const double* pbuf = pbuf2 + (j & 1) * n;
    if (!group_barrier8(bar, rank, G, ++bstep, wait_limit)) {
      if (tid == 0) atomicOr(c.status, ST_TIMEOUT);
      return;
    }
    // ---- w = p - K v and the updated column j+1, in every CTA: K = (tau / 2)
    // p^T v from the full p; all loads of a round first (one L2 round trip)
    double pt = 0.0;
    for (int base = 0; base < m; base += 4 * kSyThreads) {
      double pr[4], ar[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = base + q * kSyThreads + tid;
        pr[q] = t < m ? __ldcg(pbuf + j + 1 + t) : 0.0;
        ar[q] = t < m ? __ldcg(A + (int64_t)(j + 1 + t) + (int64_t)(j + 1) * n) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = base + q * kSyThreads + tid;
        if (t < m) {
          w[t] = pr[q];
          vx[t] = ar[q];
          pt = fma(pr[q], vc[t], pt);
        }
      }
    }
    const double K = 0.5 * tau * block_sum256(pt, red, parity);
    // w_t = p_t - K v_t, the updated column a_t - w_t v_0 - v_t w_0, and the
    // next reflector's sum of squares (rows j+3 ..); w[0] keeps p_0 (every
    // thread forms w_0 from it, and nothing later reads w[0])
    double ps = 0.0;
    {
      const double v0 = vc[0];
      const double w0 = fma(-K, v0, w[0]);
      for (int t = tid; t < m; t += kSyThreads) {
        const double wt = fma(-K, vc[t], w[t]);
        if (t > 0) w[t] = wt;
        const double nc = fma(-vc[t], w0, fma(-wt, v0, vx[t]));
        vx[t] = nc;
        if (t >= 2) ps = fma(nc, nc, ps);
      }
    }
    if (j + 3 < n) {
      // ---- reflector j+1 from rows j+2 .. of the updated column x = vx + 1:
      // thread 0 forms tau, beta and scal = 1/(x_0 - beta) while the other
      // warps already run the pass, which needs them only at its end
      const double sigma = block_sum256(ps, red, parity);
      if (tid == 0) {
        double b1, t1, sc;
        reflector_scalars(vx[1], sigma, &b1, &t1, &sc);
        sh[0] = b1; sh[1] = t1; sh[2] = sc;
      }
      double* pnext = pbuf2 + ((j + 1) & 1) * n;
      if (n <= 256) column_pass<true, 128>(A, n, j + 2, vx + 1, sh + 1, vc, w, pnext, psum, pcap, rank, G);
      else column_pass<true, 256>(A, n, j + 2, vx + 1, sh + 1, vc, w, pnext, psum, pcap, rank, G);
      const double beta1 = sh[0], tau1 = sh[1], scal1 = sh[2];
      if (rank == 0 && tid == 0) {
        c.d[j + 1] = vx[0];
        c.e[j + 1] = beta1;
        c.tau1[j + 1] = tau1;
      }
      store_reflector(c, n, j + 1, vx + 1, rank, G, scal1);
      // v_{j+1} = scal x becomes the current reflector (v_0 = 1)
      for (int t = tid; t < m - 1; t += kSyThreads) vc[t] = t == 0 ? 1.0 : scal1 * vx[1 + t];
      tau = tau1;
      __syncthreads();
    } else {
      __syncthreads();
      // the last 2 x 2 block (rows n-2, n-1); A(n-1, n-1) is current in A
      if (rank == 0 && tid == 0) {
        c.d[n - 2] = vx[0];
        c.e[n - 2] = vx[1];
        c.e[n - 1] = 0.0;
        const double a = __ldcg(A + (int64_t)(n - 1) + (int64_t)(n - 1) * n);
        c.d[n - 1] = a - fma(vc[1], w[1], w[1] * vc[1]);
      }
    }
  }
}

__global__ void __launch_bounds__(kSyThreads) sytrd1_kernel(const ConeDev* __restrict__ cones,
                                                            const int* __restrict__ cta_cone,
                                                            const int* __restrict__ cta_rank,
                                                            const int* __restrict__ cta_count,
                                                            long long wait_limit, int smem_bytes, int glb_ok) {
  extern __shared__ double sy_smem[];
  __shared__ double red[2 * (kSyThreads / 32)];
  __shared__ double sh[4];
  const ConeDev& c = cones[cta_cone[blockIdx.x]];
  const int rank = cta_rank[blockIdx.x], G = cta_count[blockIdx.x];
  if (*c.status != 0) return;
  // every CTA of a cone takes the same decision (same n, G, launch): columns
  // in shared memory and double-float arithmetic, or columns in L2 and FP64
  __shared__ int coef_tag;
  __shared__ int half_tag[kSyThreads / 64];
  __shared__ dfl half_part[kSyThreads / 64];
  // no pass has announced a part yet (the first CTA barrier of the body orders this)
  if (threadIdx.x < kSyThreads / 64) half_tag[threadIdx.x] = INT_MIN;
  const bool res = sytrd1_bytes((int)c.n, G, true) <= (size_t)smem_bytes;
  const bool glb = !res && glb_ok && sytrd1_glb_bytes((int)c.n) <= (size_t)smem_bytes;
  // the format of the reflector blocks V1: double-float pairs (both
  // double-float routes) or FP64
  if (rank == 0 && threadIdx.x == 0) c.kinfo[7] = (res || glb) ? 1 : 0;
  if (glb)
    sytrd1_body_df<true>(c, rank, G, wait_limit, sy_smem, reinterpret_cast<dfl*>(red), sh,
                         reinterpret_cast<dfl*>(sh + 2), &coef_tag, half_tag, half_part);
  else if (res)
    sytrd1_body_df<false>(c, rank, G, wait_limit, sy_smem, reinterpret_cast<dfl*>(red), sh,
                          reinterpret_cast<dfl*>(sh + 2), &coef_tag, half_tag, half_part);
  else
    sytrd1_body(c, rank, G, wait_limit, sy_smem, red, sh);
}

// T factor of each 32-reflector block (one CTA per block): G = V^T V, then
// T(a, j) = -tau_j sum_{q=a}^{j-1} T(a, q) G(q, j), T(j, j) = tau_j; written
// generically, run in double-float (the blocks are FP32 pairs on exit).
template <typename E>
__device__ void larft1_body(const ConeDev& c, int q, E (*Gm)[kNb + 1], E (*T)[kNb + 1], E (*part)[kNb]) {
  const int n = (int)c.n;
  const int r0 = q * kNb + 1, mq = n - r0;
  const int nr = min(kNb, n - 2 - q * kNb);  // reflectors in the block
  const E* Vq = reinterpret_cast<const E*>(c.V1) + (int64_t)q * n * kNb;
  const int tid = threadIdx.x;
  // partial Grams: thread = (row group, column cc); 8 row groups of 32 lanes
  const int cc = tid % kNb, grp = tid / kNb;
  E acc[kNb];
#pragma unroll
  for (int a = 0; a < kNb; ++a) g_zero(acc[a]);
  if (cc < nr)
    for (int r = grp; r < mq; r += kSyThreads / kNb) {
      const E vc = Vq[(int64_t)r + (int64_t)cc * mq];
      if (g_is_zero(vc)) continue;
#pragma unroll
      for (int a = 0; a < kNb; ++a)
        if (a < cc) acc[a] = g_mad(Vq[(int64_t)r + (int64_t)a * mq], vc, acc[a]);
    }
#pragma unroll
  for (int a = 0; a < kNb; ++a) {
    part[grp][cc] = acc[a];
    __syncthreads();
    if (tid < kNb) {
      E g;
      g_zero(g);
      for (int p = 0; p < kSyThreads / kNb; ++p) g = g_add(g, part[p][tid]);
      Gm[a][tid] = g;
      for (int b2 = 0; b2 < kNb; ++b2) g_zero(T[a][b2]);
    }
    __syncthreads();
  }
  __syncthreads();
  for (int j = 0; j < nr; ++j) {
    E tj;
    g_cvt(tj, c.tau1[q * kNb + j]);
    if (tid < j) {
      E s;
      g_zero(s);
      for (int p = tid; p < j; ++p) s = g_mad(T[tid][p], Gm[p][j], s);
      E m;
      g_zero(m);
      T[tid][j] = g_mad(g_neg(tj), s, m);
    }
    if (tid == 0) T[j][j] = tj;
    __syncthreads();
  }
  E* Tq = reinterpret_cast<E*>(c.T1) + (int64_t)q * kNb * kNb;
  for (int e = tid; e < kNb * kNb; e += kSyThreads) {
    const int a = e % kNb, b2 = e / kNb;
    Tq[a + b2 * kNb] = T[a][b2];
  }
}

__global__ void __launch_bounds__(kSyThreads) larft1_kernel(const ConeDev* __restrict__ cones,
                                                            const int* __restrict__ blk_cone,
                                                            const int* __restrict__ blk_index) {
  // 8-byte elements either way (FP64, or an FP32 pair)
  __shared__ double Gm[kNb][kNb + 1];
  __shared__ double T[kNb][kNb + 1];
  __shared__ double part[kSyThreads / kNb][kNb];
  const ConeDev& c = cones[blk_cone[blockIdx.x]];
  if (*c.status != 0) return;
  const int q = blk_index[blockIdx.x];
  if (!c.kinfo[7]) {
    // FP64 reflectors (columns in L2): this block becomes FP32 pairs in
    // place (|v| <= 1), so the fused back-transformation runs in
    // double-float for every one-stage cone
    const int n = (int)c.n;
    const int mq = n - (q * kNb + 1);
    const int nr = min(kNb, n - 2 - q * kNb);
    double* Vd = c.V1 + (int64_t)q * n * kNb;
    for (int64_t e = threadIdx.x; e < (int64_t)mq * nr; e += kSyThreads) {
      const double v = Vd[e];
      reinterpret_cast<dfl*>(Vd)[e] = df_from_d_int(v);
    }
    __syncthreads();
  }
  larft1_body<dfl>(c, q, reinterpret_cast<dfl(*)[kNb + 1]>(Gm), reinterpret_cast<dfl(*)[kNb + 1]>(T),
                   reinterpret_cast<dfl(*)[kNb]>(part));
}

}  // namespace

size_t sytrd1_smem_bytes(int n, int G, bool resident) { return sytrd1_bytes(n, G, resident); }

int sytrd1_max_ctas_for(size_t smem) {
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(sytrd1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSyResidentMax);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sytrd1_kernel, kSyThreads, smem);
  return per_sm * sms;
}

int sytrd1_max_ctas(int maxn) { return sytrd1_max_ctas_for(sytrd1_bytes(maxn, 1, false)); }

size_t sytrd1_glb_smem_bytes(int n) { return sytrd1_glb_bytes(n); }

int launch_sytrd1(const ConeDev* cones, const int* cta_cone, const int* cta_rank, const int* cta_count, int nctas,
                  int maxn, size_t smem, int glb, long long wait_limit, cudaStream_t s) {
  if (nctas <= 0) return 0;
  if (smem < sytrd1_bytes(maxn, 1, false)) smem = sytrd1_bytes(maxn, 1, false);
  if (glb && smem < sytrd1_glb_bytes(maxn)) smem = sytrd1_glb_bytes(maxn);
  // co-resident CTAs (they wait on one another); the attribute also survives graph recording
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nctas);
  cfg.blockDim = dim3(kSyThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, sytrd1_kernel, cones, cta_cone, cta_rank, cta_count, wait_limit, (int)smem,
                                glb);
}

void launch_larft1(const ConeDev* cones, const int* blk_cone, const int* blk_index, int nblocks, cudaStream_t s) {
  if (nblocks <= 0) return;
  larft1_kernel<<<nblocks, kSyThreads, 0, s>>>(cones, blk_cone, blk_index);
}

}  // namespace scs
