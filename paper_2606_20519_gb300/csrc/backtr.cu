// Back-transformation through the stage-2 (bulge-chasing) reflectors:
// Z <- Q2 Z with Q2 = H(0,0) H(0,1) ... H(nsweeps-1, last), i.e. the
// reflectors are applied in reverse order of generation.  The reflectors of
// one sweep act on disjoint row blocks, so a whole sweep is applied at once
// (one thread per reflector and column), sweeps one after the other.  Each
// CTA holds a slab of columns of Z in shared memory for the whole pass.
#include "dfloat.cuh"
#include "internal.cuh"

namespace scs {

namespace {

constexpr int kBtThreads = 256;

// Shared-memory slab: row r of the slab lives at row r + r / b, so the rows of
// neighbouring reflectors (b apart) fall in different banks.
template <int B>
__device__ __forceinline__ int srow(int r) { return r + r / B; }

template <int B>
__global__ void __launch_bounds__(kBtThreads) backtr2_kernel(const ConeDev* __restrict__ cones, int cs) {
  const ConeDev& c = cones[blockIdx.y];
  if (*c.status != 0 || c.nsweeps == 0) return;
  const int n = (int)c.n;
  const int kcols = c.kinfo[0];
  const int j0 = blockIdx.x * cs;
  if (j0 >= kcols) return;
  const int nc = min(cs, kcols - j0);
  constexpr int b = B;
  extern __shared__ double zs[];  // zs[srow(r) * nc + col]
  double* Z = c.Z;
  for (int e = threadIdx.x; e < n * nc; e += kBtThreads) {
    const int r = e % n, col = e / n;
    zs[srow<B>(r) * nc + col] = Z[(int64_t)r + (int64_t)(j0 + col) * n];
  }
  __syncthreads();
  // The reflectors of one sweep are contiguous in memory: stage them into
  // shared memory with one coalesced copy, so the dot-product chains below
  // never wait on L2.  job = (reflector kq, column), column fastest; each
  // thread runs up to 4 jobs at once (4 independent FP64 chains).
  double* rs = zs + (size_t)(n + n / B + 1) * nc;  // staged reflectors (kmax * (B + 1))
  for (int i = c.nsweeps - 1; i >= 0; --i) {
    const int Ki = (n - 3 - i) / b + 1;
    const double* sw = c.refl + (int64_t)i * c.kmax * (b + 1);
    for (int e = threadIdx.x; e < Ki * (b + 1); e += kBtThreads) rs[e] = __ldg(sw + e);
    __syncthreads();
    const int jobs = Ki * nc;
    for (int base = threadIdx.x; base < jobs; base += 4 * kBtThreads) {
      int r0[4], L[4];
      const double* slot[4];
      double* zc[4];
      double cr[4], dot[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int job = base + q * kBtThreads;
        L[q] = 0;
        cr[q] = 0.0;
        dot[q] = 0.0;
        r0[q] = 0;
        slot[q] = rs;
        zc[q] = zs;
        if (job < jobs) {
          const int kq = job / nc, col = job % nc;
          r0[q] = i + 1 + kq * b;
          L[q] = min(r0[q] + b - 1, n - 1) - r0[q] + 1;
          slot[q] = rs + kq * (b + 1);
          cr[q] = slot[q][0];
          zc[q] = zs + col;
          if (cr[q] == 0.0) L[q] = 0;
        }
      }
      const int Lmax = max(max(L[0], L[1]), max(L[2], L[3]));
      for (int t = 0; t < Lmax; ++t) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (t < L[q]) dot[q] = fma(slot[q][1 + t], zc[q][srow<B>(r0[q] + t) * nc], dot[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) dot[q] *= cr[q];
      for (int t = 0; t < Lmax; ++t) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (t < L[q]) {
            double* z = zc[q] + srow<B>(r0[q] + t) * nc;
            *z = fma(-dot[q], slot[q][1 + t], *z);
          }
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * nc; e += kBtThreads) {
    const int r = e % n, col = e / n;
    Z[(int64_t)r + (int64_t)(j0 + col) * n] = zs[srow<B>(r) * nc + col];
  }
}

}  // namespace

// Columns per CTA: small enough for about two CTAs per SM at the expected
// number of kept columns, and within the shared-memory budget.
static size_t backtr2_refl_doubles(int n, int band) { return (size_t)((n >= 3 ? (n - 3) / band + 1 : 0) + 1) * (band + 1); }

static int backtr2_cols(int n, int band, int kexp, int sms) {
  const int rows = n + n / band + 1;  // padded rows
  // every CTA streams all reflectors once, so wide slabs save L2 traffic,
  // but the slabs must also give about two CTAs per SM
  const long long avail = 200 * 1024 - 8 * (long long)backtr2_refl_doubles(n, band);
  int cs = (int)(avail / (8 * (rows > 0 ? rows : 1)));
  const int want = (kexp + 2 * sms - 1) / (2 * sms);
  if (cs > want) cs = want;
  if (cs > 32) cs = 32;
  if (cs < 1) cs = 1;
  return cs;
}

template <int B>
static void launch_bt2(const ConeDev* cones, int ncones, int maxn, int maxk, int cs, cudaStream_t s) {
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(backtr2_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
  }
  const int gx = (maxk + cs - 1) / cs;
  const size_t rows = (size_t)maxn + maxn / B + 1;
  const size_t smem = (rows * cs + backtr2_refl_doubles(maxn, B)) * sizeof(double);
  backtr2_kernel<B><<<dim3(gx, ncones), kBtThreads, smem, s>>>(cones, cs);
}

void launch_backtr2(const ConeDev* cones, int ncones, int maxn, int maxk, int kexp, int band, cudaStream_t s) {
  if (ncones <= 0 || maxk <= 0) return;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int cs = backtr2_cols(maxn, band, kexp, sms);
  switch (band) {
    case 2: launch_bt2<2>(cones, ncones, maxn, maxk, cs, s); break;
    case 4: launch_bt2<4>(cones, ncones, maxn, maxk, cs, s); break;
    case 8: launch_bt2<8>(cones, ncones, maxn, maxk, cs, s); break;
    case 16: launch_bt2<16>(cones, ncones, maxn, maxk, cs, s); break;
    default: launch_bt2<32>(cones, ncones, maxn, maxk, cs, s); break;
  }
}

// ------------------------------------------------------------------------
// Stage-1 back-transformation in one launch: Z <- Q1 Z with
// Q1 = (I - V_0 T_0 V_0^T) ... (I - V_{B-1} T_{B-1} V_{B-1}^T), the blocks of
// the one-stage tridiagonalisation (32 reflectors each) or the band
// reduction's panels, applied last block first.  A CTA holds a slab of up to
// KC kept columns in shared memory for the whole pass; per block it forms
// W = V^T Z (lanes over rows, four reflectors per warp, then a warp
// reduce-scatter), W' = T W and Z -= V W'.  When the slab and the widest
// block fit in shared memory together (sides up to about 830), each block is
// first copied there by the whole CTA with every copy in flight at once
// (staged); beyond, the warps stream the blocks from L2 inside their loops.
// The slab never leaves the SM.  CTA ->
// (cone, rank in the cone's group, group size) comes from tables, so big
// cones get many CTAs and small ones one.
namespace {

constexpr int kB1Threads = 256;
constexpr int kB1MaxCols = 8;
constexpr size_t kB1SmemMax = 200 * 1024;
constexpr size_t kB1StagedMax = 220 * 1024;  // dynamic shared memory of a staged launch, at most

template <typename E>
struct Stage1Block {
  int r0, mq, bb, wb;
  const E* V;
  const E* T;
};

__device__ __forceinline__ int stage1_nblocks(const ConeDev& c) {
  const int n = (int)c.n;
  if (c.path == 0) return c.npanels;
  return n >= 3 ? (n - 2 + kSy1Block - 1) / kSy1Block : 0;
}

template <typename E>
__device__ __forceinline__ Stage1Block<E> stage1_block(const ConeDev& c, int q) {
  const int n = (int)c.n;
  const E* V1 = reinterpret_cast<const E*>(c.V1);
  const E* T1 = reinterpret_cast<const E*>(c.T1);
  Stage1Block<E> k;
  if (c.path == 0) {
    k.wb = c.b;
    k.r0 = (q + 1) * c.b;
    k.mq = n - k.r0;
    k.bb = min(c.b, k.mq);
    k.V = V1 + (int64_t)q * n * c.b;
    k.T = T1 + (int64_t)q * c.b * c.b;
  } else {
    k.wb = kSy1Block;
    k.r0 = q * kSy1Block + 1;
    k.mq = n - k.r0;
    k.bb = min(kSy1Block, n - 2 - q * kSy1Block);
    k.V = V1 + (int64_t)q * n * kSy1Block;
    k.T = T1 + (int64_t)q * kSy1Block * kSy1Block;
  }
  return k;
}

// Sum of v over the warp, recursive halving: on return lane l holds the sum
// of element (l >> (5 - log2 NV)) of v.
template <int NV, typename E>
__device__ __forceinline__ E warp_reduce_scatter(E (&v)[NV]) {
  const int lane = threadIdx.x & 31;
  int cnt = NV;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    if (cnt > 1) {
      const int half = cnt / 2;
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int i = 0; i < NV / 2; ++i) {
        if (i < half) {
          const E send = up ? v[i] : v[i + half];
          const E keep = up ? v[i + half] : v[i];
          v[i] = g_add(keep, g_shfl_xor(send, off));
        }
      }
      cnt = half;
    } else {
      v[0] = g_add(v[0], g_shfl_xor(v[0], off));
    }
  }
  return v[0];
}

// cnt 8-byte elements from global to shared memory: 16-byte asynchronous
// copies when both addresses allow them (every thread issues its share at
// once), element copies otherwise.  The caller waits (cp_async_wait_all) and
// synchronises the CTA.
template <typename E>
__device__ __forceinline__ void stage_copy(E* dst, const E* src, int cnt) {
  static_assert(sizeof(E) == 8, "8-byte elements");
  const uint32_t sd = (uint32_t)__cvta_generic_to_shared(dst);
  if (((reinterpret_cast<uintptr_t>(src) | (uintptr_t)sd) & 15u) == 0) {
    const int pairs = cnt / 2;
    for (int e = threadIdx.x; e < pairs; e += kB1Threads)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sd + 16u * (uint32_t)e), "l"(src + 2 * e)
                   : "memory");
    if ((cnt & 1) && threadIdx.x == 0) dst[cnt - 1] = src[cnt - 1];
  } else {
    for (int e = threadIdx.x; e < cnt; e += kB1Threads) dst[e] = src[e];
  }
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// A reflector-block element: from shared memory (ST, the block staged there)
// or through the read-only cache.
template <bool ST, typename E>
__device__ __forceinline__ E ld_blk(const E* p) {
  if constexpr (ST) return *p;
  else return g_ldg(p);
}

// One slab of KC columns through every block, in element type E (FP64, or
// double-float when the reflectors and T factors were stored as FP32 pairs).
// ST: each block's reflectors V (bb x mq) and T factor are first copied into
// shared memory (Vs, Ts) by the whole CTA, with every copy in flight at once,
// and the products read them there; otherwise every warp streams them from
// L2 inside its loops, one dependent round of loads after another.
template <int KC, typename E, bool ST>
__device__ void bt1_slab(const ConeDev& c, int j0, int ncols, E* zs, E* Wsm, E* Wt, E* Vs, E* Ts) {
  const int n = (int)c.n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double* Z = c.Z;
  // rows 1 .. n-1 of the slab (row 0 is untouched: Q1 = diag(1, Q1'))
  for (int e = tid; e < KC * n; e += kB1Threads) {
    const int col = e / n, r = e - col * n;
    g_cvt(zs[e], col < ncols ? Z[(int64_t)r + (int64_t)(j0 + col) * n] : 0.0);
  }
  __syncthreads();
  const int nblk = stage1_nblocks(c);
  for (int q = nblk - 1; q >= 0; --q) {
    Stage1Block<E> B = stage1_block<E>(c, q);
    if constexpr (ST) {
      stage_copy(Vs, B.V, B.bb * B.mq);
      stage_copy(Ts, B.T, B.bb * B.wb);
      cp_async_wait_all();
      __syncthreads();
      B.V = Vs;
      B.T = Ts;
    }
    // ---- W = V^T Z(r0:, slab): warp w takes reflectors 4w .. 4w+3
    {
      E acc[4 * KC];
#pragma unroll
      for (int i = 0; i < 4 * KC; ++i) g_zero(acc[i]);
      const int a0 = warp * 4;
      if (a0 < B.bb) {
        const E* zr = zs + B.r0;
#pragma unroll 2
        for (int r = lane; r < B.mq; r += 32) {
          E z[KC];
#pragma unroll
          for (int col = 0; col < KC; ++col) z[col] = zr[col * n + r];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            E v;
            if (a0 + i < B.bb) v = ld_blk<ST>(B.V + r + (int64_t)(a0 + i) * B.mq);
            else g_zero(v);
#pragma unroll
            for (int col = 0; col < KC; ++col) acc[i * KC + col] = g_mad(v, z[col], acc[i * KC + col]);
          }
        }
      }
      const E s = warp_reduce_scatter<4 * KC>(acc);
      constexpr int kShift = (4 * KC == 32) ? 0 : (4 * KC == 16) ? 1 : (4 * KC == 8) ? 2 : 3;
      if ((lane & ((1 << kShift) - 1)) == 0) {
        const int idx = lane >> kShift;  // i * KC + col
        Wsm[(a0 + idx / KC) * KC + (idx % KC)] = s;
      }
    }
    __syncthreads();
    // ---- W' = T W (T upper triangular)
    if (tid < kSy1Block * KC) {
      const int a = tid / KC, col = tid % KC;
      E s0, s1;
      g_zero(s0);
      g_zero(s1);
      if (a < B.bb) {
        int bq = a;
        for (; bq + 1 < B.bb; bq += 2) {
          s0 = g_mad(ld_blk<ST>(B.T + a + (int64_t)bq * B.wb), Wsm[bq * KC + col], s0);
          s1 = g_mad(ld_blk<ST>(B.T + a + (int64_t)(bq + 1) * B.wb), Wsm[(bq + 1) * KC + col], s1);
        }
        if (bq < B.bb) s0 = g_mad(ld_blk<ST>(B.T + a + (int64_t)bq * B.wb), Wsm[bq * KC + col], s0);
      }
      Wt[a * KC + col] = g_add(s0, s1);
    }
    __syncthreads();
    // ---- Z(r0:, slab) -= V W'
    for (int r = tid; r < B.mq; r += kB1Threads) {
      E s0[KC], s1[KC];
#pragma unroll
      for (int col = 0; col < KC; ++col) { g_zero(s0[col]); g_zero(s1[col]); }
#pragma unroll 8
      for (int a = 0; a < kSy1Block; a += 2) {
        if (a < B.bb) {
          const E v0 = ld_blk<ST>(B.V + r + (int64_t)a * B.mq);
          E v1;
          if (a + 1 < B.bb) v1 = ld_blk<ST>(B.V + r + (int64_t)(a + 1) * B.mq);
          else g_zero(v1);
#pragma unroll
          for (int col = 0; col < KC; ++col) {
            s0[col] = g_mad(v0, Wt[a * KC + col], s0[col]);
            s1[col] = g_mad(v1, Wt[(a + 1) * KC + col], s1[col]);
          }
        }
      }
#pragma unroll
      for (int col = 0; col < KC; ++col)
        zs[col * n + B.r0 + r] = g_add(zs[col * n + B.r0 + r], g_neg(g_add(s0[col], s1[col])));
    }
    __syncthreads();
  }
  for (int e = tid; e < KC * n; e += kB1Threads) {
    const int col = e / n, r = e - col * n;
    if (col < ncols && r >= 1) Z[(int64_t)r + (int64_t)(j0 + col) * n] = g_val(zs[e]);
  }
  __syncthreads();
}

template <typename E, bool ST>
__device__ void bt1_cols(const ConeDev& c, int lo, int hi, int kcmax, E* smem, E* Wsm, E* Wt, E* Vs, E* Ts) {
  for (int j0 = lo; j0 < hi;) {
    const int left = hi - j0;
    if (left > 4 && kcmax >= 8) {
      bt1_slab<8, E, ST>(c, j0, min(left, 8), smem, Wsm, Wt, Vs, Ts);
      j0 += min(left, 8);
    } else if (left > 2 && kcmax >= 4) {
      bt1_slab<4, E, ST>(c, j0, min(left, 4), smem, Wsm, Wt, Vs, Ts);
      j0 += min(left, 4);
    } else if (left >= 2 && kcmax >= 2) {
      bt1_slab<2, E, ST>(c, j0, 2, smem, Wsm, Wt, Vs, Ts);
      j0 += 2;
    } else {
      bt1_slab<1, E, ST>(c, j0, 1, smem, Wsm, Wt, Vs, Ts);
      j0 += 1;
    }
  }
}

// Shared memory of a staged launch: the slabs (kcmax x maxn, rounded to an
// even count so that the block copies start on 16 bytes), then the widest
// reflector block (32 x maxn) and its T factor (32 x 32).
__host__ __device__ inline size_t bt1_slab_elems(int kcmax, int maxn) { return ((size_t)kcmax * maxn + 1) / 2 * 2; }
__host__ __device__ inline size_t bt1_staged_bytes(int kcmax, int maxn) {
  return (bt1_slab_elems(kcmax, maxn) + (size_t)kMaxBand * maxn + (size_t)kMaxBand * kMaxBand) * 8;
}

__global__ void __launch_bounds__(kB1Threads) bt1_kernel(const ConeDev* __restrict__ cones,
                                                         const int* __restrict__ cta_cone,
                                                         const int* __restrict__ cta_rank,
                                                         const int* __restrict__ cta_count, int kcmax,
                                                         int maxn, int staged) {
  extern __shared__ __align__(16) double b1_smem[];
  // 8-byte elements either way (FP64, or an FP32 pair)
  __shared__ double Wsm[kSy1Block * kB1MaxCols];
  __shared__ double Wt[kSy1Block * kB1MaxCols];
  const ConeDev& c = cones[cta_cone[blockIdx.x]];
  if (*c.status != 0) return;
  const int rank = cta_rank[blockIdx.x], G = cta_count[blockIdx.x];
  const int k = c.kinfo[0];
  // columns [lo, hi) of this CTA
  const int base = k / G, extra = k % G;
  const int lo = rank * base + min(rank, extra);
  const int hi = lo + base + (rank < extra ? 1 : 0);
  // one-stage reflectors and T factors are FP32 pairs (written so by the
  // shared-memory reduction, or converted by larft1_kernel)
  double* Vs = b1_smem + bt1_slab_elems(kcmax, maxn);
  double* Ts = Vs + (size_t)kMaxBand * maxn;
  if (c.path == 1) {
    dfl* sm = reinterpret_cast<dfl*>(b1_smem);
    dfl* w0 = reinterpret_cast<dfl*>(Wsm);
    dfl* w1 = reinterpret_cast<dfl*>(Wt);
    if (staged)
      bt1_cols<dfl, true>(c, lo, hi, kcmax, sm, w0, w1, reinterpret_cast<dfl*>(Vs), reinterpret_cast<dfl*>(Ts));
    else
      bt1_cols<dfl, false>(c, lo, hi, kcmax, sm, w0, w1, nullptr, nullptr);
  } else {
    if (staged) bt1_cols<double, true>(c, lo, hi, kcmax, b1_smem, Wsm, Wt, Vs, Ts);
    else bt1_cols<double, false>(c, lo, hi, kcmax, b1_smem, Wsm, Wt, nullptr, nullptr);
  }
}

}  // namespace

int bt1_max_side() { return (int)(kB1SmemMax / sizeof(double)); }

bool bt1_stages(int maxn) { return bt1_staged_bytes(1, maxn) <= kB1StagedMax; }

void launch_bt1(const ConeDev* cones, const int* cta_cone, const int* cta_rank, const int* cta_count, int nctas,
                int maxn, cudaStream_t s) {
  if (nctas <= 0 || maxn <= 0) return;
  int kcmax = kB1MaxCols;
  while (kcmax > 1 && (size_t)kcmax * maxn * sizeof(double) > kB1SmemMax) kcmax /= 2;
  size_t smem = (size_t)kcmax * maxn * sizeof(double);
  // staged reflector blocks when a slab and the widest block fit (sides up to
  // about 830): the widest slab that leaves room for them
  // staged CTAs take most of an SM's shared memory (one per SM): only launches
  // of at most one wave
  int staged = 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (nctas <= sms) {
    int kc = kB1MaxCols;
    while (kc > 1 && bt1_staged_bytes(kc, maxn) > kB1StagedMax) kc /= 2;
    if (bt1_staged_bytes(kc, maxn) <= kB1StagedMax) {
      staged = 1;
      kcmax = kc;
      smem = bt1_staged_bytes(kc, maxn);
    }
  }
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(bt1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kB1StagedMax);
  }
  bt1_kernel<<<nctas, kB1Threads, smem, s>>>(cones, cta_cone, cta_rank, cta_count, kcmax, maxn, staged);
}

}  // namespace scs
