// Grouped FP64 GEMM used by every dense contraction of the FP64 path:
// the two-sided trailing update of the dense->band stage, the stage-1
// back-transformation, the eigenvector updates of the divide and conquer and
// the derivative contractions.
//
// FP64 on GB300 runs at about 2 DFMA per clock per SM, so the kernel is bound
// by the FP64 pipe, not by memory: the goal is to keep every SM's FP64 pipe
// busy with no wasted lanes.  256 threads form a 16 x 16 grid, each owning a
// (BM/16) x (BN/16) block of independent accumulators; operands are staged
// through shared memory.  Four tile shapes cover the shapes of this
// pipeline: 64x64 (square-ish), 128x16 (tall, N = band width), 16x128
// (short, M = band width) and 16x16 (band-width squares).  Long reductions
// with few output tiles are split along K (split-K): each slice writes its partial product to scratch and a
// second kernel sums the slices in a fixed order, so results are
// bit-for-bit repeatable.  Problems of different sizes share one launch (a
// tile prefix sum maps blockIdx.x to a problem), and sizes that are only
// known on the device (kept eigenvectors, non-deflated poles) are read from
// device memory so that the launch sequence is static.
#include "dfloat.cuh"
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

constexpr int BK = kGemmBK;

template <int BM, int BN, typename T>
__device__ __forceinline__ void gemm_body(const GemmDesc* __restrict__ descs, const int* __restrict__ prefix,
                                          int count) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];

  const int tile = blockIdx.x;
  const int p = find_problem(prefix, count, tile);
  const GemmDesc& g = descs[p];
  if (g.skip && *g.skip) return;
  int N = g.N, K = g.K;
  if (g.dynN) N = min(N, *g.dynN);
  if (g.dynK) K = min(K, *g.dynK);
  const int Ms = g.M;
  const int M = g.dynM ? min(Ms, *g.dynM) : Ms;
  const int S = g.splitk;
  const int tiles_m = (Ms + BM - 1) / BM;
  int local = tile - prefix[p];
  const int kb = local % S;
  local /= S;
  const int tm = local % tiles_m, tn = local / tiles_m;
  const int i0 = tm * BM, j0 = tn * BN;
  const int flags = g.flags;
  const bool lowc = flags & GF_LOWER_C;
  if (j0 >= N || i0 >= M) return;
  if (lowc && j0 > i0 + BM - 1) return;
  const int kchunk = ((g.K + S - 1) / S + BK - 1) / BK * BK;
  const int kbeg = kb * kchunk;
  const int kend = min(K, kbeg + kchunk);

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T acc[TM][TN];
#pragma unroll
  for (int r = 0; r < TM; ++r)
#pragma unroll
    for (int c = 0; c < TN; ++c) g_zero(acc[r][c]);

  const double* __restrict__ A = g.A;
  const double* __restrict__ B = g.B;
  const int lda = g.lda, ldb = g.ldb;
  const bool ta = flags & GF_TRANS_A, tb = flags & GF_TRANS_B, sa = flags & GF_SYM_A;
  const bool scl = flags & GF_SCALE_B;

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK + 255) / 256; ++q) {
      const int e = tid + q * 256;
      if ((BM * BK) % 256 == 0 || e < BM * BK) {
        int ii, kk;
        if (ta) { kk = e % BK; ii = e / BK; } else { ii = e % BM; kk = e / BM; }
        const int i = i0 + ii, k = k0 + kk;
        double v = 0.0;
        if (i < M && k < kend) {
          if (sa) v = (i >= k) ? A[(int64_t)i + (int64_t)k * lda] : A[(int64_t)k + (int64_t)i * lda];
          else if (ta) v = A[(int64_t)k + (int64_t)i * lda];
          else v = A[(int64_t)i + (int64_t)k * lda];
        }
        g_cvt(As[kk][ii], v);
      }
    }
#pragma unroll
    for (int q = 0; q < (BN * BK + 255) / 256; ++q) {
      const int e = tid + q * 256;
      if ((BN * BK) % 256 == 0 || e < BN * BK) {
        int jj, kk;
        if (tb) { jj = e % BN; kk = e / BN; } else { kk = e % BK; jj = e / BK; }
        const int j = j0 + jj, k = k0 + kk;
        double v = 0.0;
        if (j < N && k < kend) {
          v = tb ? B[(int64_t)j + (int64_t)k * ldb] : B[(int64_t)k + (int64_t)j * ldb];
          if (scl) v *= g.bscale[k];
        }
        g_cvt(Bs[kk][jj], v);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bv[TN];
#pragma unroll
      for (int r = 0; r < TM; ++r) a[r] = As[kk][tx + 16 * r];
#pragma unroll
      for (int c = 0; c < TN; ++c) bv[c] = Bs[kk][ty + 16 * c];
#pragma unroll
      for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = g_mad(a[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }

  if (S > 1) {
    // partial product of slice kb: scratch[kb][i + j * M] (static N)
    double* part = g.partial + (int64_t)kb * Ms * g.N;
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const int j = j0 + ty + 16 * c;
      if (j >= N) continue;
#pragma unroll
      for (int r = 0; r < TM; ++r) {
        const int i = i0 + tx + 16 * r;
        if (i < M) part[(int64_t)i + (int64_t)j * Ms] = g_val(acc[r][c]);
      }
    }
    return;
  }
  double* C = g.C;
  const int ldc = g.ldc;
  const double alpha = g.alpha, beta = g.beta;
#pragma unroll
  for (int c = 0; c < TN; ++c) {
    const int j = j0 + ty + 16 * c;
    if (j >= N) continue;
    const int jc = g.colmap ? g.colmap[j] : j;
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      const int i = i0 + tx + 16 * r;
      if (i >= M) continue;
      if (lowc && i < j) continue;
      double* cp = (flags & GF_TRANS_C) ? C + (int64_t)jc + (int64_t)i * ldc : C + (int64_t)i + (int64_t)jc * ldc;
      double v = alpha * g_val(acc[r][c]);
      if (beta != 0.0) v = fma(beta, (flags & GF_BETA_B) ? g.B[(int64_t)i + (int64_t)j * g.ldb] : *cp, v);
      *cp = v;
    }
  }
}

template <int BM, int BN>
__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmDesc* __restrict__ descs,
                                                       const int* __restrict__ prefix, int count) {
  gemm_body<BM, BN, double>(descs, prefix, count);
}

template <int BM, int BN>
__global__ void __launch_bounds__(256) gemm_df_kernel(const GemmDesc* __restrict__ descs,
                                                      const int* __restrict__ prefix, int count) {
  gemm_body<BM, BN, dfl>(descs, prefix, count);
}

// Sums the split-K slices of every problem with splitk > 1 (blockIdx.y).
__global__ void gemm_reduce_kernel(const GemmDesc* __restrict__ descs) {
  const GemmDesc& g = descs[blockIdx.y];
  if (g.splitk <= 1) return;
  if (g.skip && *g.skip) return;
  int N = g.N;
  if (g.dynN) N = min(N, *g.dynN);
  const int Ms = g.M, S = g.splitk;
  const int M = g.dynM ? min(Ms, *g.dynM) : Ms;
  const bool lowc = g.flags & GF_LOWER_C;
  const int64_t total = (int64_t)Ms * N;
  const int64_t slice = (int64_t)Ms * g.N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % Ms), j = (int)(e / Ms);
    if (i >= M) continue;
    if (lowc && i < j) continue;
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += g.partial[q * slice + e];
    const int jc = g.colmap ? g.colmap[j] : j;
    double* cp = (g.flags & GF_TRANS_C) ? g.C + (int64_t)jc + (int64_t)i * g.ldc : g.C + (int64_t)i + (int64_t)jc * g.ldc;
    double v = g.alpha * s;
    if (g.beta != 0.0) v = fma(g.beta, (g.flags & GF_BETA_B) ? g.B[(int64_t)i + (int64_t)j * g.ldb] : *cp, v);
    *cp = v;
  }
}

}  // namespace

void gemm_tile_shape(int variant, int* bm, int* bn) {
  switch (variant) {
    case GEMM_TALL: *bm = 128; *bn = 16; break;
    case GEMM_SHORT: *bm = 16; *bn = 128; break;
    case GEMM_SMALL: *bm = 16; *bn = 16; break;
    default: *bm = 64; *bn = 64; break;  // GEMM_SQUARE, GEMM_SQUARE_DF
  }
}

void launch_gemm(const GemmDesc* descs, const int* tile_prefix, int count, int total_tiles, int variant,
                 int needs_reduce, int64_t max_mn, cudaStream_t s) {
  if (count <= 0 || total_tiles <= 0) return;
  if (variant == GEMM_SQUARE_DF) {
    gemm_df_kernel<64, 64><<<total_tiles, 256, 0, s>>>(descs, tile_prefix, count);
    if (needs_reduce) launch_gemm_reduce(descs, count, max_mn, s);
    return;
  }
  switch (variant) {
    case GEMM_TALL: gemm_f64_kernel<128, 16><<<total_tiles, 256, 0, s>>>(descs, tile_prefix, count); break;
    case GEMM_SHORT: gemm_f64_kernel<16, 128><<<total_tiles, 256, 0, s>>>(descs, tile_prefix, count); break;
    case GEMM_SMALL: gemm_f64_kernel<16, 16><<<total_tiles, 256, 0, s>>>(descs, tile_prefix, count); break;
    default: gemm_f64_kernel<64, 64><<<total_tiles, 256, 0, s>>>(descs, tile_prefix, count); break;
  }
  if (needs_reduce) launch_gemm_reduce(descs, count, max_mn, s);
}

void launch_gemm_reduce(const GemmDesc* descs, int count, int64_t max_mn, cudaStream_t s) {
  int gx = (int)((max_mn + 255) / 256);
  if (gx > 512) gx = 512;
  if (gx < 1) gx = 1;
  gemm_reduce_kernel<<<dim3(gx, count), 256, 0, s>>>(descs);
}

}  // namespace scs
