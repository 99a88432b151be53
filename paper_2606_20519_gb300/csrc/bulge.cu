// Band -> tridiagonal reduction by bulge chasing (second stage of the
// two-stage symmetric eigensolver).
//
// Sweep i removes column i of the band below the subdiagonal with a
// Householder reflector of length <= b and chases the bulge it creates down
// the band: task k of sweep i
//   - builds a reflector from column gc, rows r0 .. r1 (r0 = i+1+k*b,
//     r1 = min(r0+b-1, n-1); gc = i for k = 0, else the first row of the
//     previous task's diagonal block),
//   - applies it from the left to the rest of the bulge (columns gc+1 .. lc),
//   - two-sided to the diagonal block rows/cols r0 .. r1,
//   - from the right to the block below (rows r1+1 .. r1+b), creating the
//     next bulge.
// The fill never reaches further than 2b-1 below the diagonal, so the band is
// stored with 2b diagonals: band[col * 2b + (row - col)].
//
// Parallelism: task (i+1, k) touches only entries that task (i, k+2) and its
// predecessors have finished with, so sweeps run as a pipeline.  Each CTA
// owns the sweeps i = rank, rank + G, ... of one cone and waits on a
// per-sweep progress counter of the previous sweep before each task.  Every
// wait is bounded (clock64 budget); on expiry the cone is flagged
// ST_TIMEOUT and the CTA returns, so no launch can hang.  The launch is
// cooperative, which guarantees that all CTAs are resident together.
#include <cooperative_groups.h>

#include "internal.cuh"

namespace scs {

namespace {

constexpr int kBulgeThreads = 128;
constexpr int KB = kMaxBand;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct BulgeSmem {
  double x[KB];
  double v[KB];
  double w[KB];
  double p[KB];
  double Lb[KB][KB + 1];
  double D[KB][KB + 1];
  double E[KB][KB + 1];
  double beta, tau, kk;
  int abort;
};

__device__ __forceinline__ double* bp(double* band, int ldb, int r, int c) {
  return band + (int64_t)c * ldb + (r - c);
}

// One task: reflector from column gc rows r0..r1, left block columns
// gc+1..lc, diagonal block r0..r1, block below rows r1+1..e2.
__device__ void bulge_task(BulgeSmem& sm, double* band, int ldb, int gc, int r0, int r1, int lc, int e2,
                           double* refl_slot) {
  const int tid = threadIdx.x;
  const int L = r1 - r0 + 1;
  const int nl = lc - gc;
  const int ne = e2 - r1;
  // ---- load the window (bypassing L1: other SMs wrote these lines)
  for (int t = tid; t < L; t += kBulgeThreads) sm.x[t] = __ldcg(bp(band, ldb, r0 + t, gc));
  for (int e = tid; e < L * nl; e += kBulgeThreads) {
    const int t = e % L, q = e / L;
    sm.Lb[t][q] = __ldcg(bp(band, ldb, r0 + t, gc + 1 + q));
  }
  for (int e = tid; e < L * L; e += kBulgeThreads) {
    const int t = e % L, u = e / L;
    if (t >= u) {
      const double val = __ldcg(bp(band, ldb, r0 + t, r0 + u));
      sm.D[t][u] = val;
      sm.D[u][t] = val;
    }
  }
  for (int e = tid; e < ne * L; e += kBulgeThreads) {
    const int q = e % ne, u = e / ne;
    sm.E[q][u] = __ldcg(bp(band, ldb, r1 + 1 + q, r0 + u));
  }
  __syncthreads();
  // ---- reflector (warp 0)
  if (tid < 32) {
    double ps = 0.0;
    for (int t = 1 + tid; t < L; t += 32) ps = fma(sm.x[t], sm.x[t], ps);
    for (int o = 16; o > 0; o >>= 1) ps += __shfl_xor_sync(0xffffffffu, ps, o);
    const double alpha = sm.x[0];
    double beta, tau, scal;
    if (ps == 0.0) {
      beta = alpha; tau = 0.0; scal = 0.0;
    } else {
      const double nrm = sqrt(fma(alpha, alpha, ps));
      beta = alpha >= 0.0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    for (int t = tid; t < L; t += 32) sm.v[t] = (t == 0) ? 1.0 : sm.x[t] * scal;
    if (tid == 0) { sm.beta = beta; sm.tau = tau; }
  }
  __syncthreads();
  const double tau = sm.tau;
  if (tau != 0.0) {
    // ---- left block: Lb <- H Lb ; diag block p = tau D v
    if (tid < nl) {
      double acc = 0.0;
      for (int t = 0; t < L; ++t) acc = fma(sm.v[t], sm.Lb[t][tid], acc);
      sm.w[tid] = acc;
    }
    if (tid >= 32 && tid - 32 < L) {
      const int t = tid - 32;
      double acc = 0.0;
      for (int u = 0; u < L; ++u) acc = fma(sm.D[t][u], sm.v[u], acc);
      sm.p[t] = tau * acc;
    }
    __syncthreads();
    for (int e = tid; e < L * nl; e += kBulgeThreads) {
      const int t = e % L, q = e / L;
      sm.Lb[t][q] = fma(-tau * sm.v[t], sm.w[q], sm.Lb[t][q]);
    }
    if (tid < 32) {
      double acc = 0.0;
      for (int t = tid; t < L; t += 32) acc = fma(sm.p[t], sm.v[t], acc);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (tid == 0) sm.kk = 0.5 * tau * acc;
    }
    __syncthreads();
    // w = p - kk v (reuse x as w for the diagonal block)
    for (int t = tid; t < L; t += kBulgeThreads) sm.x[t] = fma(-sm.kk, sm.v[t], sm.p[t]);
    // below block: row dots
    if (tid < ne) {
      double acc = 0.0;
      for (int u = 0; u < L; ++u) acc = fma(sm.E[tid][u], sm.v[u], acc);
      sm.p[tid] = tau * acc;  // p is free again after kk
    }
    __syncthreads();
    for (int e = tid; e < L * L; e += kBulgeThreads) {
      const int t = e % L, u = e / L;
      if (t >= u) sm.D[t][u] -= sm.v[t] * sm.x[u] + sm.x[t] * sm.v[u];
    }
    for (int e = tid; e < ne * L; e += kBulgeThreads) {
      const int q = e % ne, u = e / ne;
      sm.E[q][u] = fma(-sm.p[q], sm.v[u], sm.E[q][u]);
    }
    __syncthreads();
  }
  // ---- store back
  for (int t = tid; t < L; t += kBulgeThreads) __stcg(bp(band, ldb, r0 + t, gc), t == 0 ? sm.beta : 0.0);
  if (tau != 0.0) {
    for (int e = tid; e < L * nl; e += kBulgeThreads) {
      const int t = e % L, q = e / L;
      __stcg(bp(band, ldb, r0 + t, gc + 1 + q), sm.Lb[t][q]);
    }
    for (int e = tid; e < L * L; e += kBulgeThreads) {
      const int t = e % L, u = e / L;
      if (t >= u) __stcg(bp(band, ldb, r0 + t, r0 + u), sm.D[t][u]);
    }
    for (int e = tid; e < ne * L; e += kBulgeThreads) {
      const int q = e % ne, u = e / ne;
      __stcg(bp(band, ldb, r1 + 1 + q, r0 + u), sm.E[q][u]);
    }
  }
  for (int t = tid; t < L; t += kBulgeThreads) refl_slot[t] = (t == 0) ? tau : sm.v[t];
}

__global__ void __launch_bounds__(kBulgeThreads) bulge_kernel(const ConeDev* __restrict__ cones,
                                                              const int* __restrict__ cta_cone,
                                                              const int* __restrict__ cta_rank,
                                                              const int* __restrict__ cta_count, int b,
                                                              long long wait_limit) {
  __shared__ BulgeSmem sm;
  const ConeDev& c = cones[cta_cone[blockIdx.x]];
  const int rank = cta_rank[blockIdx.x], G = cta_count[blockIdx.x];
  const int n = (int)c.n;
  const int ldb = 2 * b;
  if (*c.status != 0) return;
  const int nsw = c.nsweeps;
  for (int i = rank; i < nsw; i += G) {
    const int Ki = (n - 3 - i) / b + 1;
    const int Kprev = (i > 0) ? (n - 2 - i) / b + 1 : 0;
    for (int k = 0; k < Ki; ++k) {
      if (i > 0) {
        const int need = min(k + 3, Kprev);
        if (threadIdx.x == 0) {
          int abort = 0;
          if (ld_acquire(c.prog + i - 1) < need) {
            const long long t0 = clock64();
            while (ld_acquire(c.prog + i - 1) < need) {
              if (clock64() - t0 > wait_limit) { abort = 1; break; }
              __nanosleep(64);
            }
          }
          if (abort) atomicOr(c.status, ST_TIMEOUT);
          sm.abort = abort;
        }
        __syncthreads();
        if (sm.abort) return;
      }
      const int r0 = i + 1 + k * b;
      const int r1 = min(r0 + b - 1, n - 1);
      const int gc = (k == 0) ? i : r0 - b;
      const int lc = (k == 0) ? i : r0 - 1;
      const int e2 = min(r1 + b, n - 1);
      bulge_task(sm, c.band, ldb, gc, r0, r1, lc, e2, c.refl + ((int64_t)i * c.kmax + k) * (b + 1));
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        st_release(c.prog + i, k + 1);
      }
    }
  }
}

}  // namespace

int bulge_max_ctas(int b) {
  (void)b;
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bulge_kernel, kBulgeThreads, 0);
  return per_sm * sms;
}

int launch_bulge(const ConeDev* cones, int ncones, const int* cta_cone, const int* cta_rank, const int* cta_count,
                 int nctas, int b, long long wait_limit, cudaStream_t s) {
  if (ncones <= 0 || nctas <= 0) return 0;
  void* args[] = {(void*)&cones, (void*)&cta_cone, (void*)&cta_rank, (void*)&cta_count, (void*)&b,
                  (void*)&wait_limit};
  return (int)cudaLaunchCooperativeKernel((void*)bulge_kernel, dim3(nctas), dim3(kBulgeThreads), args, 0, s);
}

}  // namespace scs
