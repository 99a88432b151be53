// Split-TF32 GEMM on the 5th-generation tensor cores (tcgen05), FP64 in and out.
//
// C = alpha op(A) op(B) + beta C with FP64 operands in global memory.
//
// Operand split on a common grid (the Ozaki idea of error-free slicing):
// the elements of one row of op(A) (one column of op(B)) within a 16-wide
// K chunk share the exponent 2^T of their largest magnitude, and each
// element x is rounded to the 32-bit fixed-point grid 2^(T-32) and cut into
// three integer slices of 10, 11 and 11 bits,
//     x ~ hi + mid + lo,  hi on 2^(T-10), mid on 2^(T-21), lo on 2^(T-32),
// each exactly a TF32 value.  Then every hi*hi product of a chunk is an
// integer multiple of one unit with at most 20 bits, so a chunk's 16 of them
// sum EXACTLY in the tensor core's FP32 accumulator (at most 2^24 units).
// The other retained products (hm, mh, hl, mm, lh) are at most 2^-10 of
// those and go to a second accumulator, whose FP32 rounding costs 2^-34.
// The dropped products (ml, lm, ll) and the grid rounding leave an error of
// about 2^-30 of max|a| max|b| per term, against 2^-24 when the operands
// were rounded to FP32.  Accumulators are drained per stage into
// compensated FP32 sums (TwoSum).  The FP64 parts of the eigensolver
// (Householder panels, bulge chasing, secular equations, sign decisions)
// stay FP64.
//
// Tile 128 x BN (BN = 16 or 64), K-stage 16, two shared-memory stages (about
// 100 KB of shared memory, so two CTAs share an SM).  The
// 128 threads load FP64 into a staging buffer while taking the chunk
// exponents (shared-memory atomicMax), then slice and store the three TF32
// parts into the K-major, no-swizzle core-matrix layout (8 rows x 16 bytes
// per core matrix, K-direction core stride 128 B, 8-row-group stride
// 1024 B); thread 0 issues the MMAs and a tcgen05.commit per stage to that
// stage's mbarrier, so the next stage loads while the tensor core works.
// The epilogue reads tensor memory with tcgen05.ld (warp w owns rows
// 32w .. 32w+31).  Every mbarrier wait is bounded; on expiry the cone is
// flagged ST_TIMEOUT and the tile is skipped, and tensor memory is always
// released.
#include <stdint.h>

#include "internal.cuh"

namespace scs {

namespace {

constexpr int TBM = 128, TBK = 16;
constexpr int KG = TBK / 4;  // 16-byte K groups per row
constexpr long long kTcWaitIters = 4000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;             // K-direction core-matrix stride
  d |= (uint64_t)(((uint32_t)(KG * 128) >> 4) & 0x3FFF) << 32;  // 8-row-group stride
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

// v * 2^p for an integer 0 <= v < 2^12 (exact unless the result leaves the
// normal FP32 range, far below the slices' resolution in this solver).
__device__ __forceinline__ float scaled_int(uint32_t v, int p) {
  if (v == 0u) return 0.0f;
  const float f = (float)v;
  if (p >= -126 && p <= 127) return f * __int_as_float((p + 127) << 23);
  if (p < -126 && p >= -252) return (f * __int_as_float((p + 126 + 127) << 23)) * __int_as_float(1 << 23);
  return p > 0 ? __int_as_float(0x7f800000) : 0.0f;
}

// Slices of v on the grid of its chunk (largest biased exponent eg): v ~
// sign (qh 2^(T-10) + qm 2^(T-21) + ql 2^(T-32)), T = eg - 1022, with
// q = round(|v| 2^(32-T)) < 2^32 + 1 taken from the FP64 bits by integer
// operations only (nothing here occupies the FP64 pipe).
__device__ __forceinline__ void split_grid(uint8_t* const* parts, uint32_t off, double v, int eg) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7FF);
  float fh = 0.0f, fm = 0.0f, fl = 0.0f;
  if (e != 0 && eg != 0) {
    const int sh = 21 + (eg - e);  // >= 21
    const uint64_t mant = ((uint64_t)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
    const uint64_t q = sh >= 64 ? 0ull : (((mant >> (sh - 1)) + 1ull) >> 1);
    const int T = eg - 1022;
    fh = scaled_int((uint32_t)(q >> 22), T - 10);
    fm = scaled_int((uint32_t)(q >> 11) & 0x7FFu, T - 21);
    fl = scaled_int((uint32_t)q & 0x7FFu, T - 32);
    if (hi >> 31) { fh = -fh; fm = -fm; fl = -fl; }
  }
  *(float*)(parts[0] + off) = fh;
  *(float*)(parts[1] + off) = fm;
  *(float*)(parts[2] + off) = fl;
}

// FP32 -> FP64 by integer operations (exact; FP32 subnormals become zero,
// below 2^-126 of nothing that matters here), so that the epilogue does not
// spend FP64-pipe conversions.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0u) return 0.0;
  const uint32_t m = u & 0x7FFFFFu;
  const uint32_t ex = (e == 0xFFu) ? 0x7FFu : e + 896u;
  const uint32_t hi = (u & 0x80000000u) | (ex << 20) | (m >> 3);
  return __hiloint2double((int)hi, (int)(m << 29));
}

__device__ __forceinline__ int exp_field(double v) { return (int)(((uint32_t)__double2hiint(v) >> 20) & 0x7FF); }

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

constexpr int KCH = 16;  // K chunk sharing one exponent (16 hi*hi products sum exactly)

template <int BN>
struct TcSmem {
  uint8_t a[2][NSPLIT][TBM * TBK * 4];  // [stage][hi/mid/lo]
  uint8_t b[2][NSPLIT][BN * TBK * 4];
  double sta[TBM * TBK];                // FP64 staging of the stage being loaded
  double stb[BN * TBK];
  int ema[2][TBM][TBK / KCH];           // [stage][row][chunk] largest exponent field
  int emb[2][BN][TBK / KCH];
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
  for (int q = tid; q < 2 * (TBM + BN) * (TBK / KCH); q += 128) {
    if (q < 2 * TBM * (TBK / KCH)) (&sm.ema[0][0][0])[q] = 0;
    else (&sm.emb[0][0][0])[q - 2 * TBM * (TBK / KCH)] = 0;
  }
  // per stage: one exact accumulator per 16-wide K chunk (hi*hi) and one for
  // the smaller products: 2 stages x 3 accumulators x BN columns
  constexpr int NACC = 2 * (TBK / KCH + 1);
  constexpr int ACC_PER_STAGE = TBK / KCH + 1;
  constexpr int TCOLS = (NACC * BN) <= 32 ? 32 : (NACC * BN) <= 64 ? 64 : (NACC * BN) <= 128 ? 128
                        : (NACC * BN) <= 256 ? 256 : 512;
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

  // Accumulators of stage kt: (kt & 1, chunk) for the exact hi*hi sums and
  // (kt & 1, rest) for the others, fresh each time; two stages later all
  // threads read them and add them into compensated FP32 register sums
  // (TwoSum).
  float acc_hi[BN], acc_lo[BN];
#pragma unroll
  for (int q = 0; q < BN; ++q) { acc_hi[q] = 0.0f; acc_lo[q] = 0.0f; }
  bool ok = true;
  auto drain = [&](int stage) {
#pragma unroll
    for (int ks = 0; ks < ACC_PER_STAGE; ++ks) {
    const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(((stage & 1) * ACC_PER_STAGE + ks) * BN);
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
  // Raw FP64 tile kt into the staging buffer with cp.async (every element of
  // the tile in flight at once; out-of-range elements are zero-filled).
  auto issue_tile = [&](int kt) {
    const int k0 = kbeg + kt * TBK;
    const bool kfast = ta || (sa && i0 + TBM <= k0);
#pragma unroll
    for (int q = 0; q < (TBM * TBK) / 128; ++q) {
      const int e = tid + q * 128;
      int r, k;
      if (kfast) { k = e % TBK; r = e / TBK; } else { r = e % TBM; k = e / TBM; }
      const int i = i0 + r, kk = k0 + k;
      if (i < M && kk < kend) {
        const double* src = sa ? ((i >= kk) ? A + (int64_t)i + (int64_t)kk * lda : A + (int64_t)kk + (int64_t)i * lda)
                               : (ta ? A + (int64_t)kk + (int64_t)i * lda : A + (int64_t)i + (int64_t)kk * lda);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(&sm.sta[e])), "l"(src) : "memory");
      } else {
        sm.sta[e] = 0.0;
      }
    }
#pragma unroll
    for (int q = 0; q < (BN * TBK + 127) / 128; ++q) {
      const int e = tid + q * 128;
      if ((BN * TBK) % 128 == 0 || e < BN * TBK) {
        int c, k;
        if (tb) { c = e % BN; k = e / BN; } else { k = e % TBK; c = e / TBK; }
        const int j = j0 + c, kk = k0 + k;
        if (j < N && kk < kend) {
          const double* src = tb ? B + (int64_t)j + (int64_t)kk * ldb : B + (int64_t)kk + (int64_t)j * ldb;
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(&sm.stb[e])), "l"(src) : "memory");
        } else {
          sm.stb[e] = 0.0;
        }
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (nk > 0) issue_tile(0);
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    if (kt >= 2) {
      if (!mbar_wait(smem_u32(&sm.mbar[s]), ((kt - 2) >> 1) & 1)) ok = false;
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (ok) drain(kt - 2);
    }
    const int k0 = kbeg + kt * TBK;
    // element -> (r, k) so that consecutive threads read consecutive memory:
    // k fastest for op(A) = A^T and for a symmetric tile wholly above the
    // diagonal (read from the lower triangle, i.e. transposed)
    const bool kfast = ta || (sa && i0 + TBM <= k0);
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // ---- pass 1: chunk exponents of the staged values (B scaled first if asked)
#pragma unroll 4
    for (int q = 0; q < (TBM * TBK) / 128; ++q) {
      const int e = tid + q * 128;
      int r, k;
      if (kfast) { k = e % TBK; r = e / TBK; } else { r = e % TBM; k = e / TBM; }
      const int ex = exp_field(sm.sta[e]);
      if (ex) atomicMax(&sm.ema[s][r][k / KCH], ex);
    }
#pragma unroll 4
    for (int q = 0; q < (BN * TBK + 127) / 128; ++q) {
      const int e = tid + q * 128;
      if ((BN * TBK) % 128 == 0 || e < BN * TBK) {
        int c, k;
        if (tb) { c = e % BN; k = e / BN; } else { k = e % TBK; c = e / TBK; }
        double v = sm.stb[e];
        if (scl && v != 0.0) {
          v *= g.bscale[k0 + k];
          sm.stb[e] = v;
        }
        const int ex = exp_field(v);
        if (ex) atomicMax(&sm.emb[s][c][k / KCH], ex);
      }
    }
    __syncthreads();
    // ---- pass 2: slices on the chunk grids; clear the other stage's exponents
    {
      uint8_t* pa[3] = {sm.a[s][0], sm.a[s][1], sm.a[s][2]};
#pragma unroll 4
      for (int q = 0; q < (TBM * TBK) / 128; ++q) {
        const int e = tid + q * 128;
        int r, k;
        if (kfast) { k = e % TBK; r = e / TBK; } else { r = e % TBM; k = e / TBM; }
        split_grid(pa, tile_off(r, k), sm.sta[e], sm.ema[s][r][k / KCH]);
      }
      uint8_t* pb[3] = {sm.b[s][0], sm.b[s][1], sm.b[s][2]};
#pragma unroll 4
      for (int q = 0; q < (BN * TBK + 127) / 128; ++q) {
        const int e = tid + q * 128;
        if ((BN * TBK) % 128 == 0 || e < BN * TBK) {
          int c, k;
          if (tb) { c = e % BN; k = e / BN; } else { k = e % TBK; c = e / TBK; }
          split_grid(pb, tile_off(c, k), sm.stb[e], sm.emb[s][c][k / KCH]);
        }
      }
      for (int q = tid; q < (TBM + BN) * (TBK / KCH); q += 128) {
        if (q < TBM * (TBK / KCH)) (&sm.ema[s ^ 1][0][0])[q] = 0;
        else (&sm.emb[s ^ 1][0][0])[q - TBM * (TBK / KCH)] = 0;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      // products with i + j <= 2 of the three parts: hh (exact, per 16-wide
      // chunk), then hm, mh, hl, mm, lh (one accumulator per stage)
      constexpr int PA[6] = {0, 0, 1, 0, 1, 2};
      constexpr int PB[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
      for (int ks = 0; ks < TBK / 8; ++ks) {
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const uint64_t da = make_desc(smem_u32(sm.a[s][PA[q]]) + ks * 256);
          const uint64_t db = make_desc(smem_u32(sm.b[s][PB[q]]) + ks * 256);
          const int slot = (q == 0) ? (ks * 8) / KCH : TBK / KCH;
          const uint32_t acc = (q == 0) ? (((ks * 8) % KCH) != 0 ? 1u : 0u) : ((ks == 0 && q == 1) ? 0u : 1u);
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                  tmem + (uint32_t)((s * ACC_PER_STAGE + slot) * BN)),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&sm.mbar[s])));
    }
    // the next tile's copies fly while the next iteration waits for and drains stage kt-1
    if (kt + 1 < nk) issue_tile(kt + 1);
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
    const bool alpha_one = g.alpha == 1.0, alpha_mone = g.alpha == -1.0, beta_one = g.beta == 1.0;
    const int row = i0 + warp * 32 + lane;
    double* part = (S > 1) ? g.partial + (int64_t)kb * Ms * g.N : nullptr;
    if (row < M) {
#pragma unroll
      for (int q = 0; q < BN; ++q) {
        const int j = j0 + q;
        if (j >= N) continue;
        if (lowc && !part && row < j) continue;
        double acc = f32_to_f64(acc_hi[q]) + f32_to_f64(acc_lo[q]);
        if (part) {
          part[(int64_t)row + (int64_t)j * Ms] = acc;
          continue;
        }
        const int jc = g.colmap ? g.colmap[j] : j;
        double* cp = (flags & GF_TRANS_C) ? g.C + (int64_t)jc + (int64_t)row * g.ldc
                                          : g.C + (int64_t)row + (int64_t)jc * g.ldc;
        // alpha = +-1 and beta in {0, 1} (every contraction of the solver) without extra FP64 work
        double v;
        if (alpha_one) v = acc;
        else if (alpha_mone) v = __longlong_as_double(__double_as_longlong(acc) ^ (long long)0x8000000000000000ULL);
        else v = g.alpha * acc;
        if (g.beta != 0.0) {
          const double cv = (flags & GF_BETA_B) ? g.B[(int64_t)row + (int64_t)j * ldb] : *cp;
          v = beta_one ? cv + v : fma(g.beta, cv, v);
        }
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
  static std::atomic<unsigned long long> attr{0};
  const size_t smem = sizeof(TcSmem<BN>) + 1024;
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
