// Band -> tridiagonal reduction by bulge chasing (second stage of the
// two-stage symmetric eigensolver).
//
// Sweep i removes column i of the band below the subdiagonal with a
// Householder reflector of length <= b and chases the bulge it creates down
// the band.  Task k of sweep i
//   - builds a reflector H = I - c u u^T from column gc, rows r0 .. r1
//     (r0 = i+1+k*b, r1 = min(r0+b-1, n-1); gc = i for k = 0, else the first
//     row of the previous task's diagonal block), with u = x - beta e_1 and
//     c = 2 / ||u||^2 = 1 / (||x|| (||x|| + |x_0|)),
//   - applies it from the left to the rest of the bulge (columns gc+1 .. lc),
//   - two-sided to the diagonal block rows/cols r0 .. r1,
//   - from the right to the block below (rows r1+1 .. r1+b), which becomes
//     the bulge of task k+1.
// The fill never reaches further than 2b-1 below the diagonal, so the band is
// stored with 2b diagonals: band[col * 2b + (row - col)].
//
// Parallelism: task (i+1, k) touches only entries that task (i, k+2) and its
// predecessors have finished with, so sweeps run as a pipeline.  Each CTA
// owns the sweeps i = rank, rank + G, ... of one cone and waits on a
// per-sweep progress counter of the previous sweep before each task.  The
// block below of task k is touched by nobody else until task k+1 of the same
// sweep has run, so it stays in shared memory, and the reflector of task k+1
// is formed while the CTA waits for the previous sweep.  On this GPU an FP64
// instruction costs a full warp slot whatever the number of active lanes, so
// every product and update is spread over all 256 threads (one element per
// thread, 16-lane shuffle reductions).  Every wait is bounded (clock64
// budget); on expiry the cone is flagged ST_TIMEOUT and the CTA returns, so
// no launch can hang.  The launch is cooperative, which guarantees that all
// CTAs are resident together.
#include "internal.cuh"

namespace scs {

namespace {

constexpr int kBulgeThreads = 256;
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
  double Bk[2][KB][KB + 1];  // bulge block of the current task (x = column 0) / block below
  double D[KB][KB + 1];
  double u[KB];
  double pD[KB], wL[KB], qE[KB];
  double c, beta;
  int abort;
  unsigned short tri[KB * (KB + 1) / 2];  // lower-triangle index -> (row << 8) | col
};

__device__ __forceinline__ double* bp(double* band, int ldb, int r, int c) {
  return band + (int64_t)c * ldb + (r - c);
}

// Reflector from column 0 of blk (L rows), by one warp: u, c, beta.
__device__ __forceinline__ void householder_warp(BulgeSmem& sm, const double (*blk)[KB + 1], int L, int lane) {
  double ps = 0.0;
  for (int t = 1 + lane; t < L; t += 32) ps = fma(blk[t][0], blk[t][0], ps);
  for (int o = 16; o > 0; o >>= 1) ps += __shfl_xor_sync(0xffffffffu, ps, o);
  const double alpha = blk[0][0];
  double beta = alpha, c = 0.0;
  if (ps != 0.0) {
    const double nrm = sqrt(fma(alpha, alpha, ps));
    beta = alpha >= 0.0 ? -nrm : nrm;
    c = 1.0 / (nrm * (nrm + fabs(alpha)));
  }
  for (int t = lane; t < L; t += 32) sm.u[t] = (t == 0) ? alpha - beta : blk[t][0];
  if (lane == 0) {
    sm.c = c;
    sm.beta = beta;
  }
}

__global__ void __launch_bounds__(kBulgeThreads) bulge_kernel(const ConeDev* __restrict__ cones,
                                                              const int* __restrict__ cta_cone,
                                                              const int* __restrict__ cta_rank,
                                                              const int* __restrict__ cta_count, int b,
                                                              long long wait_limit) {
  __shared__ BulgeSmem sm;
  const ConeDev& cn = cones[cta_cone[blockIdx.x]];
  const int rank = cta_rank[blockIdx.x], G = cta_count[blockIdx.x];
  const int n = (int)cn.n;
  const int ldb = 2 * b;
  if (*cn.status != 0) return;
  double* band = cn.band;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nsw = cn.nsweeps;
  for (int t = tid; t < KB; t += kBulgeThreads)
    for (int v = 0; v <= t; ++v) sm.tri[t * (t + 1) / 2 + v] = (unsigned short)((t << 8) | v);
  __syncthreads();

  for (int i = rank; i < nsw; i += G) {
    const int Ki = (n - 3 - i) / b + 1;
    const int Kprev = (i > 0) ? (n - 2 - i) / b + 1 : 0;
    for (int k = 0; k < Ki; ++k) {
      const int r0 = i + 1 + k * b;
      const int r1 = min(r0 + b - 1, n - 1);
      const int L = r1 - r0 + 1;
      const int gc = (k == 0) ? i : r0 - b;
      const int nl = (k == 0) ? 0 : b - 1;  // bulge columns after gc
      const int e2 = min(r1 + b, n - 1);
      const int ne = e2 - r1;
      double (*B)[KB + 1] = sm.Bk[k & 1];       // bulge block (column 0 = x)
      double (*E)[KB + 1] = sm.Bk[(k + 1) & 1];  // block below -> next bulge
      // ---- wait for the previous sweep (warp 1); for k = 0 the column comes from it
      if (i > 0 && tid == 32) {
        const int need = min(k + 3, Kprev);
        int abort = 0;
        if (ld_acquire(cn.prog + i - 1) < need) {
          const long long t0 = clock64();
          while (ld_acquire(cn.prog + i - 1) < need) {
            if (clock64() - t0 > wait_limit) { abort = 1; break; }
            __nanosleep(32);
          }
        }
        if (abort) atomicOr(cn.status, ST_TIMEOUT);
        sm.abort = abort;
      }
      __syncthreads();
      if (i > 0 && sm.abort) return;
      // ---- loads: column (k = 0), diagonal block, block below
      if (k == 0)
        for (int t = tid; t < L; t += kBulgeThreads) B[t][0] = __ldcg(bp(band, ldb, r0 + t, gc));
      for (int e = tid; e < L * L; e += kBulgeThreads) {
        const int t = e % L, v = e / L;
        if (t >= v) {
          const double val = __ldcg(bp(band, ldb, r0 + t, r0 + v));
          sm.D[t][v] = val;
          sm.D[v][t] = val;
        }
      }
      for (int e = tid; e < ne * L; e += kBulgeThreads) {
        const int q = e % ne, v = e / ne;
        E[q][v] = __ldcg(bp(band, ldb, r1 + 1 + q, r0 + v));
      }
      __syncthreads();
      if (k == 0) {
        if (warp == 0) householder_warp(sm, B, L, lane);
        __syncthreads();
      }
      const double c = sm.c;
      if (c != 0.0) {
        // ---- products, 32/RB lanes per dot product (RB = 16 or 32 rows per
        // warp): warp 0 pD = c D u and w = pD - K u, warp 1 wL = c Lb^T u,
        // warp 2 qE = c E u.  Few FP64 instructions: a lane-sequential dot
        // product beats a shuffle tree on this part.
        if (warp < 3) {
          const int RB = (b <= 16) ? 16 : 32;
          const int lpr = 32 / RB;
          const int row = lane / lpr, part = lane % lpr;
          const int nrows = warp == 0 ? L : (warp == 1 ? nl : ne);
          double acc = 0.0;
          if (row < nrows)
            for (int v = part; v < L; v += lpr) {
              const double m = warp == 0 ? sm.D[row][v] : (warp == 1 ? B[v][1 + row] : E[row][v]);
              acc = fma(m, sm.u[v], acc);
            }
          if (lpr == 2) acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          acc *= c;
          if (warp == 0) {
            double kv = (row < L && part == 0) ? acc * sm.u[row] : 0.0;
            for (int o = 16; o > 0; o >>= 1) kv += __shfl_xor_sync(0xffffffffu, kv, o);
            const double K = 0.5 * c * kv;
            if (row < L && part == 0) sm.pD[row] = fma(-K, sm.u[row], acc);  // w
          } else if (row < nrows && part == 0) {
            if (warp == 1) sm.wL[row] = acc; else sm.qE[row] = acc;
          }
        }
        __syncthreads();
        // ---- updates: one element per thread, D lower (2 FMA), bulge (1), below (1)
        const int nD = L * (L + 1) / 2, nLb = L * nl, nE = ne * L;
        for (int e = tid; e < nD + nLb + nE; e += kBulgeThreads) {
          if (e < nD) {
            const int t = sm.tri[e] >> 8, v = sm.tri[e] & 255;
            const double val = fma(-sm.u[t], sm.pD[v], fma(-sm.pD[t], sm.u[v], sm.D[t][v]));
            __stcg(bp(band, ldb, r0 + t, r0 + v), val);
          } else if (e < nD + nLb) {
            const int f = e - nD, t = f % L, q = f / L;
            __stcg(bp(band, ldb, r0 + t, gc + 1 + q), fma(-sm.u[t], sm.wL[q], B[t][1 + q]));
          } else {
            const int f = e - nD - nLb, q = f % ne, v = f / ne;
            E[q][v] = fma(-sm.qE[q], sm.u[v], E[q][v]);
          }
        }
      } else {
        for (int e = tid; e < L * nl; e += kBulgeThreads) {
          const int t = e % L, q = e / L;
          __stcg(bp(band, ldb, r0 + t, gc + 1 + q), B[t][1 + q]);
        }
      }
      // (the bulge columns gc+1..lc lived only in shared memory since the previous task)
      for (int t = tid; t < L; t += kBulgeThreads) __stcg(bp(band, ldb, r0 + t, gc), t == 0 ? sm.beta : 0.0);
      // reflector for the back-transformation: c, u_0 .. u_{L-1}
      double* slot = cn.refl + ((int64_t)i * cn.kmax + k) * (b + 1);
      for (int t = tid; t <= L; t += kBulgeThreads) slot[t] = (t == 0) ? c : sm.u[t - 1];
      const bool last = (k + 1 == Ki);
      if (last)
        for (int e = tid; e < ne * L; e += kBulgeThreads) {
          const int q = e % ne, v = e / ne;
          __stcg(bp(band, ldb, r1 + 1 + q, r0 + v), E[q][v]);
        }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(cn.prog + i, k + 1);
      }
      // reflector of the next task from the block below, while warp 1 waits
      if (!last && warp == 0) householder_warp(sm, E, ne, lane);
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
  // co-resident CTAs (they wait on one another); the attribute also survives graph recording
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nctas);
  cfg.blockDim = dim3(kBulgeThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, bulge_kernel, cones, cta_cone, cta_rank, cta_count, b, wait_limit);
}

}  // namespace scs
