// One-stage Householder tridiagonalisation for cones whose trailing matrix
// stays in L2 (the medium sizes of the paper's process-matrix step), in a
// single persistent cooperative kernel.
//
// CTA r of a cone's group of G CTAs owns the columns i with i mod G = r for
// the whole reduction (both triangles are kept, so a column is contiguous).
// Column j (m = n - j - 1 rows below the diagonal):
//   A: every CTA waits until the owner of column j has published it (a
//      single-producer flag), reads its rows j+1 .. n-1 and forms the
//      reflector H = I - tau v v^T (v_0 = 1, LAPACK convention) redundantly;
//   B: each CTA computes p_i = tau A(j+1:, i)^T v for its columns and the
//      partial sum of p_i v_i;                               -- group barrier
//   C: every CTA forms w = p - (tau/2)(p^T v) v and applies the rank-2 update
//      A <- A - v w^T - w v^T to its own columns; the owner of column j+1
//      updates it first and publishes it.
// Work items are (column, 256-row chunk) pairs spread over all warps, each
// lane keeping 8 loads in flight (the loop is bound by L2 latency otherwise).
// The diagonal d, off-diagonal e, tau and the reflectors (packed into
// 32-column blocks with their unit diagonal and zeros, ready for the blocked
// back-transformation) are written by the group's first CTA.  Group barriers
// are counters in global memory with release/acquire ordering and a bounded
// wait (ST_TIMEOUT on expiry); the launch is cooperative, so every CTA is
// resident.  Data written by other CTAs is read with ld.global.cg (L2).
//
// larft1_kernel then forms, for every 32-reflector block, the triangular
// factor T of H_0 ... H_31 = I - V T V^T.
#include <math.h>

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

__device__ double block_sum256(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int q = 0; q < kSyThreads / 32; ++q) t += red[q];
  return t;
}

// Barrier over the G CTAs of one cone; returns false when the wait ran out.
__device__ bool group_barrier(int* counter, int target, long long limit, int* flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1);
    int ok = 1;
    if (ld_acquire(counter) < target) {
      const long long t0 = clock64();
      while (ld_acquire(counter) < target) {
        if (clock64() - t0 > limit) { ok = 0; break; }
      }
    }
    __threadfence();
    *flag = ok;
  }
  __syncthreads();
  return *flag != 0;
}

constexpr int kChunk = 256;   // rows per work item (32 lanes x 8 loads in flight)
constexpr int kPartMax = 2048; // work items per round (shared-memory partial sums)

__global__ void __launch_bounds__(kSyThreads) sytrd1_kernel(const ConeDev* __restrict__ cones,
                                                            const int* __restrict__ cta_cone,
                                                            const int* __restrict__ cta_rank,
                                                            const int* __restrict__ cta_count,
                                                            long long wait_limit) {
  extern __shared__ double sy_smem[];
  __shared__ double red[kSyThreads / 32];
  __shared__ double sh_beta, sh_tau, sh_scal, sh_K;
  __shared__ int sh_flag;
  const ConeDev& c = cones[cta_cone[blockIdx.x]];
  const int rank = cta_rank[blockIdx.x], G = cta_count[blockIdx.x];
  const int n = (int)c.n;
  if (*c.status != 0) return;
  double* A = c.A;
  double* v = sy_smem;               // m values of the current reflector
  double* w = sy_smem + n;           // p, then w
  double* psum = sy_smem + 2 * n;    // kPartMax partial dot products
  // p_i (absolute column index) and the partial sums p^T v, double-buffered by
  // step parity: a CTA writes step j+2's values only after every CTA has
  // passed step j+1's barrier, i.e. finished reading step j's values
  double* pbuf2 = c.X;               // 2 x n
  double* part2 = c.X + 2 * n;       // 2 x G
  int* bar = c.prog;                 // barrier counter
  int* ready = c.prog + 1;           // last column whose update is complete
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int bstep = 0;

  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    double* pbuf = pbuf2 + (j & 1) * n;
    double* part = part2 + (j & 1) * G;
    // ---- A: wait until column j is up to date (single producer), then the
    // reflector from its rows j+1 .. n-1, in every CTA
    if (j > 0 && ((j % G) != rank)) {
      if (tid == 0) {
        int ok = 1;
        if (ld_acquire(ready) < j) {
          const long long t0 = clock64();
          while (ld_acquire(ready) < j) {
            if (clock64() - t0 > wait_limit) { ok = 0; break; }
          }
        }
        sh_flag = ok;
      }
      __syncthreads();
      if (!sh_flag) {
        if (tid == 0) atomicOr(c.status, ST_TIMEOUT);
        return;
      }
    }
    for (int t = tid; t < m; t += kSyThreads) v[t] = __ldcg(A + (int64_t)(j + 1 + t) + (int64_t)j * n);
    __syncthreads();
    double ps = 0.0;
    for (int t = 1 + tid; t < m; t += kSyThreads) ps = fma(v[t], v[t], ps);
    const double sigma = block_sum256(ps, red);
    if (tid == 0) {
      const double alpha = v[0];
      double beta = alpha, tau = 0.0, scal = 0.0;
      if (sigma != 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, sigma));
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      sh_beta = beta; sh_tau = tau; sh_scal = scal;
    }
    __syncthreads();
    const double tau = sh_tau, scal = sh_scal;
    for (int t = 1 + tid; t < m; t += kSyThreads) v[t] *= scal;
    if (tid == 0) v[0] = 1.0;
    __syncthreads();
    if (rank == 0) {
      // outputs: d_j, e_j, tau_j and the reflector in its 32-column block
      const int q = j / kNb, col = j % kNb;
      const int r0 = q * kNb + 1;               // first row of block q
      const int mq = n - r0;                    // rows of block q
      double* Vq = c.V1 + (int64_t)q * n * kNb;  // mq x 32, ld mq
      for (int r = tid; r < mq; r += kSyThreads) {
        const int row = r0 + r;
        double val = 0.0;
        if (row == j + 1) val = 1.0;
        else if (row > j + 1) val = v[row - j - 1];
        Vq[(int64_t)r + (int64_t)col * mq] = val;
      }
      if (tid == 0) {
        c.d[j] = __ldcg(A + (int64_t)j + (int64_t)j * n);
        c.e[j] = sh_beta;
        c.rho[j] = tau;  // tau of reflector j (the divide and conquer reuses rho later)
      }
    }
    // my columns: i = first + G * k, i > j (absolute ownership: i mod G == rank)
    const int first = j + 1 + ((rank - (j + 1) % G) + G) % G;
    const int ncol = first < n ? (n - 1 - first) / G + 1 : 0;
    const int nch = (m + kChunk - 1) / kChunk;
    if (tau == 0.0) {
      // H = I (same decision in every CTA): column j+1 is already current
      if (((j + 1) % G) == rank && tid == 0) {
        __threadfence();
        asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(ready), "r"(j + 1) : "memory");
      }
      continue;
    }
    // ---- B: p_i = tau A(j+1:, i)^T v for my columns; items (column, row chunk)
    double mypv = 0.0;
    for (int k0 = 0; k0 < ncol; k0 += kPartMax / nch) {
      const int kc = min(ncol - k0, kPartMax / nch);
      for (int it = warp; it < kc * nch; it += kSyThreads / 32) {
        const int k = k0 + it / nch, ch = it % nch;
        const double* col = A + (int64_t)(first + G * k) * n + (j + 1);
        const int t0 = ch * kChunk + lane;
        double a[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int t = t0 + 32 * r;
          a[r] = t < m ? __ldcg(col + t) : 0.0;
        }
        double acc = 0.0;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int t = t0 + 32 * r;
          if (t < m) acc = fma(a[r], v[t], acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) psum[it] = acc;
      }
      __syncthreads();
      for (int kk = tid; kk < kc; kk += kSyThreads) {
        double p = 0.0;
        for (int ch = 0; ch < nch; ++ch) p += psum[kk * nch + ch];
        p *= tau;
        const int i = first + G * (k0 + kk);
        __stcg(pbuf + i, p);
        mypv = fma(p, v[i - j - 1], mypv);
      }
      __syncthreads();
    }
    const double pv = block_sum256(mypv, red);
    if (tid == 0) __stcg(part + rank, pv);
    if (!group_barrier(bar, (++bstep) * G, wait_limit, &sh_flag)) {
      if (tid == 0) atomicOr(c.status, ST_TIMEOUT);
      return;
    }
    // ---- C: w = p - K v, then the rank-2 update of my columns (column j+1 first)
    double pt = 0.0;
    for (int r = tid; r < G; r += kSyThreads) pt += __ldcg(part + r);
    const double K = 0.5 * tau * block_sum256(pt, red);
    for (int t = tid; t < m; t += kSyThreads) w[t] = fma(-K, v[t], __ldcg(pbuf + j + 1 + t));
    __syncthreads();
    for (int it = warp; it < ncol * nch; it += kSyThreads / 32) {
      const int k = it / nch, ch = it % nch;
      const int i = first + G * k;
      double* col = A + (int64_t)i * n + (j + 1);
      const double vi = v[i - j - 1], wi = w[i - j - 1];
      const int t0 = ch * kChunk + lane;
      double a[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int t = t0 + 32 * r;
        a[r] = t < m ? __ldcg(col + t) : 0.0;
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int t = t0 + 32 * r;
        if (t < m) __stcg(col + t, a[r] - fma(v[t], wi, w[t] * vi));
      }
    }
    // the owner of column j+1 publishes it (its first column, updated above)
    __syncthreads();
    if (((j + 1) % G) == rank && tid == 0) {
      __threadfence();
      asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(ready), "r"(j + 1) : "memory");
    }
  }
  // the last 2 x 2 block: wait for its columns, then d and e
  if (rank == 0) {
    if (tid == 0) {
      int ok = 1;
      if (n >= 3 && ld_acquire(ready) < n - 2) {
        const long long t0 = clock64();
        while (ld_acquire(ready) < n - 2) {
          if (clock64() - t0 > wait_limit) { ok = 0; break; }
        }
      }
      if (!ok) atomicOr(c.status, ST_TIMEOUT);
    }
    // every column of the last block is owned and updated before the final barrier of step n-3
    if (!group_barrier(bar, (++bstep) * G, wait_limit, &sh_flag)) {
      if (tid == 0) atomicOr(c.status, ST_TIMEOUT);
      return;
    }
    if (tid == 0) {
      if (n >= 2) {
        c.d[n - 2] = __ldcg(A + (int64_t)(n - 2) + (int64_t)(n - 2) * n);
        c.e[n - 2] = __ldcg(A + (int64_t)(n - 1) + (int64_t)(n - 2) * n);
      }
      c.d[n - 1] = __ldcg(A + (int64_t)(n - 1) + (int64_t)(n - 1) * n);
      c.e[n - 1] = 0.0;
    }
  } else {
    if (!group_barrier(bar, (++bstep) * G, wait_limit, &sh_flag)) {
      if (tid == 0) atomicOr(c.status, ST_TIMEOUT);
      return;
    }
  }
}

// T factor of each 32-reflector block (one CTA per block): G = V^T V, then
// T(a, j) = -tau_j sum_{q=a}^{j-1} T(a, q) G(q, j), T(j, j) = tau_j.
__global__ void __launch_bounds__(kSyThreads) larft1_kernel(const ConeDev* __restrict__ cones,
                                                            const int* __restrict__ blk_cone,
                                                            const int* __restrict__ blk_index) {
  __shared__ double Gm[kNb][kNb + 1];
  __shared__ double T[kNb][kNb + 1];
  __shared__ double part[kSyThreads / kNb][kNb];
  const ConeDev& c = cones[blk_cone[blockIdx.x]];
  if (*c.status != 0) return;
  const int q = blk_index[blockIdx.x];
  const int n = (int)c.n;
  const int r0 = q * kNb + 1, mq = n - r0;
  const int nr = min(kNb, n - 2 - q * kNb);  // reflectors in the block
  const double* Vq = c.V1 + (int64_t)q * n * kNb;
  const int tid = threadIdx.x;
  // partial Grams: thread = (row group, column cc); 8 row groups of 32 lanes
  const int cc = tid % kNb, grp = tid / kNb;
  double acc[kNb];
#pragma unroll
  for (int a = 0; a < kNb; ++a) acc[a] = 0.0;
  if (cc < nr)
    for (int r = grp; r < mq; r += kSyThreads / kNb) {
      const double vc = Vq[(int64_t)r + (int64_t)cc * mq];
      if (vc == 0.0) continue;
#pragma unroll
      for (int a = 0; a < kNb; ++a)
        if (a < cc) acc[a] = fma(Vq[(int64_t)r + (int64_t)a * mq], vc, acc[a]);
    }
#pragma unroll
  for (int a = 0; a < kNb; ++a) {
    part[grp][cc] = acc[a];
    __syncthreads();
    if (tid < kNb) {
      double g = 0.0;
      for (int p = 0; p < kSyThreads / kNb; ++p) g += part[p][tid];
      Gm[a][tid] = g;
      for (int b2 = 0; b2 < kNb; ++b2) T[a][b2] = 0.0;
    }
    __syncthreads();
  }
  __syncthreads();
  for (int j = 0; j < nr; ++j) {
    const double tj = c.rho[q * kNb + j];
    if (tid < j) {
      double s = 0.0;
      for (int p = tid; p < j; ++p) s = fma(T[tid][p], Gm[p][j], s);
      T[tid][j] = -tj * s;
    }
    if (tid == 0) T[j][j] = tj;
    __syncthreads();
  }
  double* Tq = c.T1 + (int64_t)q * kNb * kNb;
  for (int e = tid; e < kNb * kNb; e += kSyThreads) {
    const int a = e % kNb, b2 = e / kNb;
    Tq[a + b2 * kNb] = T[a][b2];
  }
}

}  // namespace

int sytrd1_max_ctas(int maxn) {
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = ((size_t)2 * maxn + kPartMax) * sizeof(double);
  cudaFuncSetAttribute(sytrd1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sytrd1_kernel, kSyThreads, smem);
  return per_sm * sms;
}

int launch_sytrd1(const ConeDev* cones, const int* cta_cone, const int* cta_rank, const int* cta_count, int nctas,
                  int maxn, long long wait_limit, cudaStream_t s) {
  if (nctas <= 0) return 0;
  const size_t smem = ((size_t)2 * maxn + kPartMax) * sizeof(double);
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
  return (int)cudaLaunchKernelEx(&cfg, sytrd1_kernel, cones, cta_cone, cta_rank, cta_count, wait_limit);
}

void launch_larft1(const ConeDev* cones, const int* blk_cone, const int* blk_index, int nblocks, cudaStream_t s) {
  if (nblocks <= 0) return;
  larft1_kernel<<<nblocks, kSyThreads, 0, s>>>(cones, blk_cone, blk_index);
}

}  // namespace scs
