// Split-TF32 GEMM on the 5th-generation tensor cores (tcgen05), FP64 in and out.
//
// C = alpha op(A) op(B) + beta C with FP64 operands in global memory.  Each
// operand element x is rounded to FP32 and split exactly into three TF32
// values x32 = hi + mid + lo, and the product is formed from the six part
// products whose orders sum to at most 2 (hh, hm, mh, hl, mm, lh), each a
// tcgen05.mma of kind::tf32 with FP32 accumulation in tensor memory.  The
// dropped products are below 2^-33 of the result; the operand rounding
// (2^-24) and the FP32 accumulation bound the accuracy.  The FP64 parts of
// the eigensolver (Householder panels, bulge chasing, secular equations,
// sign decisions) stay FP64.
//
// Tile 128 x BN (BN = 16 or 64), K-stage 32, two shared-memory stages.  The
// 128 threads load FP64, split and store the three TF32 parts into the
// K-major, no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix,
// K-direction core stride 128 B, 8-row-group stride 1024 B); thread 0 issues
// the MMAs and a tcgen05.commit per stage to that stage's mbarrier, so the
// next stage loads while the tensor core works.  The epilogue reads the
// accumulator with tcgen05.ld (warp w owns rows 32w .. 32w+31).  Every
// mbarrier wait is bounded; on expiry the cone is flagged ST_TIMEOUT and the
// tile is skipped, and tensor memory is always released.
#include <stdint.h>

#include "internal.cuh"

namespace scs {

namespace {

constexpr int TBM = 128, TBK = 32;
constexpr int KG = TBK / 4;  // 16-byte K groups per row
constexpr long long kTcWaitIters = 4000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;   // K-direction core-matrix stride
  d |= (uint64_t)((1024u >> 4) & 0x3FFF) << 32;  // 8-row-group stride
  d |= (uint64_t)1 << 46;                        // descriptor version for tcgen05
  return d;                                      // no swizzle, base offset 0
}

__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return ((r >> 3) * KG + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// FP64 -> FP32 with round-to-nearest-even by integer operations, so that the
// conversion of every operand element does not occupy the FP64 pipe (on this
// part a conversion costs as much as an FP64 FMA); magnitudes below 2^-126
// become zero (far below the split's resolution).
__device__ __forceinline__ float f64_to_f32(double v) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7FF) - 896;
  if (e <= 0) return 0.0f;
  // 52-bit mantissa -> 23 bits, rounding on the 29 dropped bits (ties to even);
  // a carry out of the mantissa correctly bumps the exponent field
  uint32_t bits = ((uint32_t)min(e, 254) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1FFFFFFFu, half = 0x10000000u;
  if (rest > half || (rest == half && (bits & 1u))) ++bits;
  return __uint_as_float((hi & 0x80000000u) | bits);
}

// x ~ hi + mid + lo, three TF32 values that reproduce the FP32 rounding of x
// exactly (11 + 11 + 2 significant bits).
__device__ __forceinline__ void split_store(uint8_t* const* parts, uint32_t off, double v) {
  const float x = f64_to_f32(v);
  const uint32_t h = to_tf32(x);
  const float r1 = x - __uint_as_float(h);
  const uint32_t m = to_tf32(r1);
  const uint32_t l = to_tf32(r1 - __uint_as_float(m));
  *(uint32_t*)(parts[0] + off) = h;
  *(uint32_t*)(parts[1] + off) = m;
  *(uint32_t*)(parts[2] + off) = l;
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (long long it = 0; it < kTcWaitIters; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ int find_problem(const int* prefix, int count, int tile) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(prefix + mid) <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int NSPLIT = 3;

template <int BN>
struct TcSmem {
  uint8_t a[2][NSPLIT][TBM * TBK * 4];  // [stage][hi/mid/lo]
  uint8_t b[2][NSPLIT][BN * TBK * 4];
  uint64_t mbar[2];
  uint32_t tmem;
  int fail;
};

template <int BN>
__global__ void __launch_bounds__(128) tc_gemm_kernel(const GemmDesc* __restrict__ descs,
                                                      const int* __restrict__ prefix, int count) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  TcSmem<BN>& sm = *reinterpret_cast<TcSmem<BN>*>(smem_raw);
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
  const int tiles_m = (Ms + TBM - 1) / TBM;
  int local = tile - prefix[p];
  const int kb = local % S;
  local /= S;
  const int tm = local % tiles_m, tn = local / tiles_m;
  const int i0 = tm * TBM, j0 = tn * BN;
  const int flags = g.flags;
  const bool lowc = flags & GF_LOWER_C;
  if (j0 >= N || i0 >= M) return;
  if (lowc && j0 > i0 + TBM - 1) return;
  const int kchunk = ((g.K + S - 1) / S + TBK - 1) / TBK * TBK;
  const int kbeg = kb * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int nk = kend > kbeg ? (kend - kbeg + TBK - 1) / TBK : 0;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* __restrict__ A = g.A;
  const double* __restrict__ B = g.B;
  const int lda = g.lda, ldb = g.ldb;
  const bool ta = flags & GF_TRANS_A, tb = flags & GF_TRANS_B, sa = flags & GF_SYM_A;
  const bool scl = flags & GF_SCALE_B;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    sm.fail = 0;
  }
  // one accumulator per 8-wide K-step and stage: 2 stages x 4 K-steps x BN columns
  constexpr int NACC = 2 * (TBK / 8);
  constexpr int TCOLS = (NACC * BN) < 32 ? 32 : NACC * BN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sm.tmem;
  // idesc: D f32, A/B tf32, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);

  // Short accumulations: the MMAs of K-step ks of stage kt write accumulator
  // (kt & 1, ks), fresh each time; two stages later all threads read the
  // stage's four accumulators and add them into compensated FP32 register
  // sums (TwoSum), so the tensor core's FP32 accumulation never spans more
  // than 8 products of the leading parts.
  float acc_hi[BN], acc_lo[BN];
#pragma unroll
  for (int q = 0; q < BN; ++q) { acc_hi[q] = 0.0f; acc_lo[q] = 0.0f; }
  bool ok = true;
  auto drain = [&](int stage) {
#pragma unroll
    for (int ks = 0; ks < TBK / 8; ++ks) {
    const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(((stage & 1) * (TBK / 8) + ks) * BN);
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(base + c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float a = acc_hi[c0 + q], b = __uint_as_float(r[q]);
        const float s = a + b;
        const float bp = s - a;
        const float e = (a - (s - bp)) + (b - bp);
        acc_hi[c0 + q] = s;
        acc_lo[c0 + q] += e;
      }
    }
    }
  };
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    if (kt >= 2) {
      if (!mbar_wait(smem_u32(&sm.mbar[s]), ((kt - 2) >> 1) & 1)) ok = false;
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (ok) drain(kt - 2);
    }
    const int k0 = kbeg + kt * TBK;
    // ---- A tile: op(A)(i0 + r, k0 + k), 128 x 32
#pragma unroll 4
    for (int q = 0; q < (TBM * TBK) / 128; ++q) {
      const int e = tid + q * 128;
      int r, k;
      if (ta) { k = e % TBK; r = e / TBK; } else { r = e % TBM; k = e / TBM; }
      const int i = i0 + r, kk = k0 + k;
      double v = 0.0;
      if (i < M && kk < kend) {
        if (sa) v = (i >= kk) ? A[(int64_t)i + (int64_t)kk * lda] : A[(int64_t)kk + (int64_t)i * lda];
        else if (ta) v = A[(int64_t)kk + (int64_t)i * lda];
        else v = A[(int64_t)i + (int64_t)kk * lda];
      }
      uint8_t* pa[3] = {sm.a[s][0], sm.a[s][1], sm.a[s][2]};
      split_store(pa, tile_off(r, k), v);
    }
    // ---- B tile: op(B)(k0 + k, j0 + c) stored as BN rows (c) x 32 (k), K-major
#pragma unroll 4
    for (int q = 0; q < (BN * TBK + 127) / 128; ++q) {
      const int e = tid + q * 128;
      if ((BN * TBK) % 128 == 0 || e < BN * TBK) {
        int c, k;
        if (tb) { c = e % BN; k = e / BN; } else { k = e % TBK; c = e / TBK; }
        const int j = j0 + c, kk = k0 + k;
        double v = 0.0;
        if (j < N && kk < kend) {
          v = tb ? B[(int64_t)j + (int64_t)kk * ldb] : B[(int64_t)kk + (int64_t)j * ldb];
          if (scl) v *= g.bscale[kk];
        }
        uint8_t* pb[3] = {sm.b[s][0], sm.b[s][1], sm.b[s][2]};
        split_store(pb, tile_off(c, k), v);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      // products with i + j <= 2 of the three parts: hh, hm, mh, hl, mm, lh
      constexpr int PA[6] = {0, 0, 1, 0, 1, 2};
      constexpr int PB[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
      for (int ks = 0; ks < TBK / 8; ++ks) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint64_t da = make_desc(smem_u32(sm.a[s][PA[q]]) + ks * 256);
          const uint64_t db = make_desc(smem_u32(sm.b[s][PB[q]]) + ks * 256);
          const uint32_t acc = (q > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                  tmem + (uint32_t)((s * (TBK / 8) + ks) * BN)),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&sm.mbar[s])));
    }
  }
  // drain the last one or two stages
  for (int kt = max(0, nk - 2); kt < nk; ++kt) {
    if (!mbar_wait(smem_u32(&sm.mbar[kt & 1]), (kt >> 1) & 1)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) drain(kt);
  }
  if (!ok) sm.fail = 1;
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool fail = sm.fail != 0;
  if (fail && tid == 0 && g.skip) atomicOr(const_cast<int*>(g.skip), ST_TIMEOUT);

  if (!fail) {
    const int row = i0 + warp * 32 + lane;
    double* part = (S > 1) ? g.partial + (int64_t)kb * Ms * g.N : nullptr;
    if (row < M) {
#pragma unroll
      for (int q = 0; q < BN; ++q) {
        const int j = j0 + q;
        if (j >= N) continue;
        const double acc = (double)acc_hi[q] + (double)acc_lo[q];
        if (part) {
          part[(int64_t)row + (int64_t)j * Ms] = acc;
          continue;
        }
        if (lowc && row < j) continue;
        const int jc = g.colmap ? g.colmap[j] : j;
        double* cp = (flags & GF_TRANS_C) ? g.C + (int64_t)jc + (int64_t)row * g.ldc
                                          : g.C + (int64_t)row + (int64_t)jc * g.ldc;
        double v = g.alpha * acc;
        if (g.beta != 0.0) v = fma(g.beta, *cp, v);
        *cp = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

template <int BN>
void launch_tc(const GemmDesc* descs, const int* prefix, int count, int tiles, cudaStream_t s) {
  static bool attr = false;
  const size_t smem = sizeof(TcSmem<BN>) + 1024;
  if (!attr) {
    cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  tc_gemm_kernel<BN><<<tiles, 128, smem, s>>>(descs, prefix, count);
}

}  // namespace

void tc_tile_shape(int variant, int* bm, int* bn) {
  *bm = TBM;
  *bn = (variant == TC_N16) ? 16 : 64;
}

void launch_tc_gemm(const GemmDesc* descs, const int* tile_prefix, int count, int total_tiles, int variant,
                    cudaStream_t s) {
  if (count <= 0 || total_tiles <= 0) return;
  if (variant == TC_N16) launch_tc<16>(descs, tile_prefix, count, total_tiles, s);
  else launch_tc<64>(descs, tile_prefix, count, total_tiles, s);
}

}  // namespace scs
