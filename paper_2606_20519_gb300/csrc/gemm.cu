// Grouped FP64 GEMM used by every dense contraction of the FP64 path:
// the two-sided trailing update of the dense->band stage, the stage-1
// back-transformation, and the eigenvector updates of the divide and conquer.
//
// FP64 on GB300 runs at about 2 DFMA per clock per SM, so the kernel is bound
// by the FP64 pipe, not by memory: a 64x64 tile, 256 threads each owning a
// 4x4 block of independent accumulators, operands staged through shared
// memory.  Problems of different sizes share one launch (a tile prefix sum
// maps blockIdx.x to a problem), and sizes that are only known on the device
// (number of kept eigenvectors, non-deflated poles) are read from device
// memory so that the launch sequence is static and can be captured in a graph.
#include "internal.cuh"

namespace scs {

namespace {

__device__ __forceinline__ int find_problem(const int* prefix, int count, int tile) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(prefix + mid) <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int BM = kGemmBM, BN = kGemmBN, BK = kGemmBK;

__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmDesc* __restrict__ descs,
                                                       const int* __restrict__ prefix, int count) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];

  const int tile = blockIdx.x;
  const int p = find_problem(prefix, count, tile);
  const GemmDesc& g = descs[p];
  if (g.skip && *g.skip) return;
  int N = g.N, K = g.K;
  if (g.dynN) N = min(N, *g.dynN);
  if (g.dynK) K = min(K, *g.dynK);
  const int M = g.M;
  const int tiles_m = (M + BM - 1) / BM;
  const int local = tile - prefix[p];
  const int tm = local % tiles_m, tn = local / tiles_m;
  const int i0 = tm * BM, j0 = tn * BN;
  if (j0 >= N || i0 >= M) return;
  const int flags = g.flags;
  if ((flags & GF_LOWER_C) && tn > tm) return;

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

  const double* __restrict__ A = g.A;
  const double* __restrict__ B = g.B;
  const int lda = g.lda, ldb = g.ldb;
  const bool ta = flags & GF_TRANS_A, tb = flags & GF_TRANS_B, sa = flags & GF_SYM_A;
  const bool scl = flags & GF_SCALE_B;

  for (int k0 = 0; k0 < K; k0 += BK) {
    // ---- A tile: op(A)(i0 + ii, k0 + kk)
#pragma unroll
    for (int q = 0; q < (BM * BK) / 256; ++q) {
      const int e = tid + q * 256;
      int ii, kk;
      if (ta) { kk = e % BK; ii = e / BK; } else { ii = e % BM; kk = e / BM; }
      const int i = i0 + ii, k = k0 + kk;
      double v = 0.0;
      if (i < M && k < K) {
        if (sa) v = (i >= k) ? A[(int64_t)i + (int64_t)k * lda] : A[(int64_t)k + (int64_t)i * lda];
        else if (ta) v = A[(int64_t)k + (int64_t)i * lda];
        else v = A[(int64_t)i + (int64_t)k * lda];
      }
      As[kk][ii] = v;
    }
    // ---- B tile: op(B)(k0 + kk, j0 + jj)
#pragma unroll
    for (int q = 0; q < (BN * BK) / 256; ++q) {
      const int e = tid + q * 256;
      int jj, kk;
      if (tb) { jj = e % BN; kk = e / BN; } else { kk = e % BK; jj = e / BK; }
      const int j = j0 + jj, k = k0 + kk;
      double v = 0.0;
      if (j < N && k < K) {
        v = tb ? B[(int64_t)j + (int64_t)k * ldb] : B[(int64_t)k + (int64_t)j * ldb];
        if (scl) v *= g.bscale[k];
      }
      Bs[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }

  double* __restrict__ C = g.C;
  const int ldc = g.ldc;
  const double alpha = g.alpha, beta = g.beta;
  const bool lowc = flags & GF_LOWER_C;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = j0 + ty + 16 * c;
    if (j >= N) continue;
    const int jc = g.colmap ? g.colmap[j] : j;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + tx + 16 * r;
      if (i >= M) continue;
      if (lowc && i < j) continue;
      double* cp = C + (int64_t)i + (int64_t)jc * ldc;
      double v = alpha * acc[r][c];
      if (beta != 0.0) v = fma(beta, *cp, v);
      *cp = v;
    }
  }
}

}  // namespace

void launch_gemm(const GemmDesc* descs, const int* tile_prefix, int count, int total_tiles, cudaStream_t s) {
  if (count <= 0 || total_tiles <= 0) return;
  gemm_f64_kernel<<<total_tiles, 256, 0, s>>>(descs, tile_prefix, count);
}

}  // namespace scs
