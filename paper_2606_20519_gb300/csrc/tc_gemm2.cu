// Split-TF32 GEMM for long contractions on the 5th-generation tensor cores
// (tcgen05), FP64 in and out: C = alpha op(A) op(B) + beta C.
//
// Operands are sliced ONCE per product (tc2_slice_kernel), not per tile:
// the elements of one row of op(A) (one column of op(B)) within a 64-wide
// K group share the exponent 2^T of their largest magnitude; each element is
// rounded to the 31-bit fixed-point grid 2^(T-31) and cut into integer
// slices of 9, 11 and 11 bits,
//     x ~ hi + mid + lo,  hi on 2^(T-9), mid on 2^(T-20), lo on 2^(T-31),
// each exactly a TF32 value (hi <= 2^9).  Every hi*hi product of a group is
// then an integer multiple of one unit with at most 18 bits, so the group's
// 64 of them sum EXACTLY in an FP32 accumulator (at most 2^24 units).  The
// products hm, mh, hl, mm, lh, ml, lm (at most 2^-9 of those) share a second
// accumulator, whose FP32 rounding costs about 2^-33; only lo*lo (2^-40) is
// dropped, and the grid rounding leaves 2^-32 of max|a| max|b| per term.
// The slices are written tile by tile in the K-major, no-swizzle
// core-matrix layout that the MMA descriptors read (8 rows x 16 bytes per
// core matrix), 128 rows x 16 K x 3 slices per block, so that the GEMM
// moves each block into shared memory with one bulk asynchronous copy.
//
// GEMM: tile 128 x 128, K-stage 16, four shared-memory stages (192 KB, one
// CTA per SM).  Warp 8 (one thread) issues the bulk copies and the MMAs
// (8 products x 2 K-steps of 8 per stage) into a pair of tensor-memory
// accumulators per 64-wide K group, double-buffered by group (512 columns);
// warps 0-7 drain a finished group (tcgen05.ld) into compensated FP32 sums
// (TwoSum), 64 columns each, while the next group runs, and write the
// result.  Every mbarrier wait is bounded; on expiry the cone is flagged
// ST_TIMEOUT and the tile is skipped, and tensor memory is always released.
#include <stdint.h>

#include "internal.cuh"

namespace scs {

namespace {

constexpr int M2 = 128, N2 = 128, K2 = 16, G2 = 64, ST2 = 4;
constexpr int GS2 = G2 / K2;   // stages per exponent group
constexpr int BLK = M2 * K2;   // floats per slice block (= N2 * K2)
constexpr int BLK_BYTES = BLK * 4;
constexpr long long kWait2 = 4000000LL;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row r, k) in a 128 x 16 block: core matrices of 8 rows x 4 K,
// K-direction stride 128 B, 8-row-group stride 512 B
__device__ __forceinline__ uint32_t boff(int r, int k) {
  return ((r >> 3) * 4 + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t mdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;  // K-direction core-matrix stride
  d |= (uint64_t)((512u >> 4) & 0x3FFF) << 32;  // 8-row-group stride
  d |= (uint64_t)1 << 46;                       // descriptor version for tcgen05
  return d;
}

__device__ __forceinline__ int expf64(double v) { return (int)(((uint32_t)__double2hiint(v) >> 20) & 0x7FF); }

// v * 2^p for an integer 0 <= v < 2^12 (exact in the normal FP32 range).
__device__ __forceinline__ float sc_int(uint32_t v, int p) {
  if (v == 0u) return 0.0f;
  const float f = (float)v;
  if (p >= -126 && p <= 127) return f * __int_as_float((p + 127) << 23);
  if (p < -126 && p >= -252) return (f * __int_as_float((p + 126 + 127) << 23)) * __int_as_float(1 << 23);
  return p > 0 ? __int_as_float(0x7f800000) : 0.0f;
}

// 9/11/11-bit slices of v on the grid of its group (largest biased exponent
// eg): q = round(|v| 2^(31-T)), T = eg - 1022, from the FP64 bits by integer
// operations only.
__device__ __forceinline__ void slice3(float* b0, float* b1, float* b2, uint32_t off, double v, int eg) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7FF);
  float fh = 0.0f, fm = 0.0f, fl = 0.0f;
  if (e != 0 && eg != 0) {
    const int sh = 22 + (eg - e);  // >= 22
    const uint64_t mant = ((uint64_t)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
    const uint64_t q = sh >= 64 ? 0ull : (((mant >> (sh - 1)) + 1ull) >> 1);
    const int T = eg - 1022;
    fh = sc_int((uint32_t)(q >> 22), T - 9);
    fm = sc_int((uint32_t)(q >> 11) & 0x7FFu, T - 20);
    fl = sc_int((uint32_t)q & 0x7FFu, T - 31);
    if (hi >> 31) { fh = -fh; fm = -fm; fl = -fl; }
  }
  *(float*)((uint8_t*)b0 + off) = fh;
  *(float*)((uint8_t*)b1 + off) = fm;
  *(float*)((uint8_t*)b2 + off) = fl;
}

__device__ __forceinline__ double f32_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0u) return 0.0;
  const uint32_t m = u & 0x7FFFFFu;
  const uint32_t ex = (e == 0xFFu) ? 0x7FFu : e + 896u;
  const uint32_t hi = (u & 0x80000000u) | (ex << 20) | (m >> 3);
  return __hiloint2double((int)hi, (int)(m << 29));
}

__device__ __forceinline__ int find_item(const int* prefix, int count, int x) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(prefix + mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ double job_load(const SliceJob& J, int i, int k) {
  const double* p = J.p;
  double v;
  if (J.mode == 0) v = p[(int64_t)i + (int64_t)k * J.ld];
  else if (J.mode == 1) v = p[(int64_t)k + (int64_t)i * J.ld];
  else v = (i >= k) ? p[(int64_t)i + (int64_t)k * J.ld] : p[(int64_t)k + (int64_t)i * J.ld];
  if (J.scale) v *= J.scale[k];
  return v;
}

// One CTA per (job, 64-row half of a 128-row tile, 64-wide K group): the
// 64 x 64 piece is read once into shared memory (all loads independent),
// then the rows' exponents are taken, and the three slices of each 16-wide K
// tile are staged in shared memory and copied out; the 64 rows of a half
// fill a contiguous half of every 8 KB block.
constexpr int SR = 64;       // rows per slicing CTA
constexpr int SLD = G2 + 1;  // row stride of the staged piece (doubles)
constexpr int HBLK = BLK / 2;
constexpr size_t kSliceSmem = sizeof(double) * SR * SLD + sizeof(float) * 3 * HBLK + sizeof(int) * SR;

__global__ void __launch_bounds__(256) tc2_slice_kernel(const SliceJob* __restrict__ jobs,
                                                        const int* __restrict__ prefix, int njobs) {
  extern __shared__ __align__(16) uint8_t sraw[];
  float* blk = reinterpret_cast<float*>(sraw);                                    // [3][HBLK]
  double* tile = reinterpret_cast<double*>(sraw + sizeof(float) * 3 * HBLK);       // [SR][SLD]
  int* em = reinterpret_cast<int*>(sraw + sizeof(float) * 3 * HBLK + sizeof(double) * SR * SLD);
  const int b = blockIdx.x;
  const int jid = find_item(prefix, njobs, b);
  const SliceJob& J = jobs[jid];
  const int local = b - prefix[jid];
  const int ngrp = (J.K + G2 - 1) / G2;
  const int th = local / ngrp, g = local % ngrp;  // th: 64-row half index
  const int tb = th >> 1, half = th & 1;
  const int rows = J.dynRows ? min(J.rows, *J.dynRows) : J.rows;
  const int Keff = J.dynK ? min(J.K, *J.dynK) : J.K;
  const int r0 = th * SR, k0 = g * G2, k1 = min(Keff, k0 + G2);
  const int KT = (J.K + K2 - 1) / K2;
  const int tid = threadIdx.x;
  // row-fast reads when consecutive rows are contiguous, K-fast otherwise
  const bool kfast = (J.mode == 1) || (J.mode == 2 && r0 + SR <= k0);
#pragma unroll 8
  for (int q = 0; q < (SR * G2) / 256; ++q) {
    const int e = tid + q * 256;
    int r, k;
    if (kfast) { k = e % G2; r = e / G2; } else { r = e % SR; k = e / SR; }
    const int i = r0 + r, kk = k0 + k;
    tile[r * SLD + k] = (i < rows && kk < k1) ? job_load(J, i, kk) : 0.0;
  }
  __syncthreads();
  // exponents: four threads per row, 16 columns each
  {
    const int r = tid >> 2, h = tid & 3;
    int m = 0;
#pragma unroll
    for (int k = h * 16; k < h * 16 + 16; ++k) m = max(m, expf64(tile[r * SLD + k]));
    m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = max(m, __shfl_xor_sync(0xffffffffu, m, 2));
    if (h == 0) em[r] = m;
  }
  __syncthreads();
  const int kt0 = k0 / K2, kt_end = min(KT, (k0 + G2) / K2);
  const uint32_t hoff = (uint32_t)half * (BLK_BYTES / 2);
  for (int kt = kt0; kt < kt_end; ++kt) {
#pragma unroll 4
    for (int q = 0; q < HBLK / 256; ++q) {
      const int e = tid + q * 256;
      const int r = e % SR, k = e / SR;  // shared memory: any order
      slice3(blk, blk + HBLK, blk + 2 * HBLK, boff(half * SR + r, k) - hoff, tile[r * SLD + (kt - kt0) * K2 + k],
             em[r]);
    }
    __syncthreads();
    float* base = J.out + (int64_t)(tb * KT + kt) * 3 * BLK + half * HBLK;
    for (int q = tid; q < 3 * HBLK / 4; q += 256) {
      const int sl = q / (HBLK / 4), w = q % (HBLK / 4);
      reinterpret_cast<float4*>(base + sl * BLK)[w] = reinterpret_cast<const float4*>(blk + sl * HBLK)[w];
    }
    __syncthreads();
  }
}

struct Tc2Smem {
  uint8_t a[ST2][3][BLK_BYTES];
  uint8_t b[ST2][3][BLK_BYTES];
  uint64_t full[ST2], empty[ST2], gdone[2], gfree[2], fin;
  uint32_t tmem;
  int fail;
};

__device__ __forceinline__ bool wait_parity(uint32_t addr, uint32_t parity) {
  for (long long it = 0; it < kWait2; ++it) {
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

// Stage t of the tile: the six slice blocks (3 of op(A), 3 of op(B)) by bulk
// asynchronous copies into slot t % ST2, completing on its "full" barrier.
__device__ __forceinline__ void bulk_stage(Tc2Smem& sm, int t, const float* pa0, const float* pb0, int& loaded) {
  ++loaded;
  const int s = t % ST2;
  const uint32_t fb = su32(&sm.full[s]);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(6 * BLK_BYTES) : "memory");
  const float* pa = pa0 + (int64_t)t * 3 * BLK;
  const float* pb = pb0 + (int64_t)t * 3 * BLK;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(sm.a[s][sl])),
                 "l"(pa + sl * BLK), "r"(BLK_BYTES), "r"(fb)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(sm.b[s][sl])),
                 "l"(pb + sl * BLK), "r"(BLK_BYTES), "r"(fb)
                 : "memory");
  }
}

__global__ void __launch_bounds__(288, 1) tc2_gemm_kernel(const GemmDesc* __restrict__ descs,
                                                          const int* __restrict__ prefix, int count) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Tc2Smem& sm = *reinterpret_cast<Tc2Smem*>(smem_raw);
  const int tile = blockIdx.x;
  const int p = find_item(prefix, count, tile);
  const GemmDesc& g = descs[p];
  if (g.skip && *g.skip) return;
  const int Ms = g.M, S = g.splitk;
  const int M = g.dynM ? min(Ms, *g.dynM) : Ms;
  const int N = g.dynN ? min(g.N, *g.dynN) : g.N;
  const int Kst = g.K, K = g.dynK ? min(Kst, *g.dynK) : Kst;
  const int tiles_m = (Ms + M2 - 1) / M2;
  int local = tile - prefix[p];
  const int kb = local % S;
  local /= S;
  const int tm = local % tiles_m, tn = local / tiles_m;
  const int i0 = tm * M2, j0 = tn * N2;
  const int flags = g.flags;
  const bool lowc = flags & GF_LOWER_C;
  if (j0 >= N || i0 >= M) return;
  if (lowc && j0 > i0 + M2 - 1) return;
  const int KT = (Kst + K2 - 1) / K2;
  const int kchunk = ((Kst + S - 1) / S + G2 - 1) / G2 * G2;
  const int kbeg = kb * kchunk, kend = min(K, kbeg + kchunk);
  const int nk = kend > kbeg ? (kend - kbeg + K2 - 1) / K2 : 0;
  const int ngrp = (nk + GS2 - 1) / GS2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < ST2; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sm.full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sm.empty[s])));
    }
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sm.gdone[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 256;" ::"r"(su32(&sm.gfree[q])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&sm.fin)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    sm.fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sm.tmem)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = sm.tmem;
  // idesc: D f32, A/B tf32, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N2 >> 3) << 17) | ((uint32_t)(M2 >> 4) << 24);

  float acc_hi[64], acc_lo[64];
  bool ok = true;
  if (warp == 8) {
    if (lane == 0) {
      const float* As = g.As;
      const float* Bs = g.Bs;
      int loaded = 0, consumed = 0;
      const float* pa0 = As + (int64_t)(tm * KT + kbeg / K2) * 3 * BLK;
      const float* pb0 = Bs + (int64_t)(tn * KT + kbeg / K2) * 3 * BLK;
      const int pre = nk < ST2 ? nk : ST2;
      for (int t = 0; t < pre; ++t) bulk_stage(sm, t, pa0, pb0, loaded);
      // products: hh (its own accumulator), then hm, mh, hl, mm, lh, ml, lm
      constexpr int PA[8] = {0, 0, 1, 0, 1, 2, 1, 2};
      constexpr int PB[8] = {0, 1, 0, 2, 1, 0, 2, 1};
      for (int t = 0; t < nk; ++t) {
        const int s = t % ST2, gi = t / GS2, gb = gi & 1;
        const bool gfirst = (t % GS2) == 0;
        if (gfirst && gi >= 2 && !wait_parity(su32(&sm.gfree[gb]), ((gi >> 1) - 1) & 1)) { ok = false; break; }
        if (!wait_parity(su32(&sm.full[s]), (t / ST2) & 1)) { ok = false; break; }
        consumed = t + 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int ks = 0; ks < K2 / 8; ++ks) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const uint64_t da = mdesc(su32(sm.a[s][PA[q]]) + ks * 256);
            const uint64_t db = mdesc(su32(sm.b[s][PB[q]]) + ks * 256);
            const uint32_t col = (uint32_t)(gb * 2 * N2 + (q == 0 ? 0 : N2));
            const uint32_t acc = (gfirst && ks == 0 && q <= 1) ? 0u : 1u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + col),
                "l"(da), "l"(db), "r"(idesc), "r"(acc));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(&sm.empty[s])));
        if ((t % GS2) == GS2 - 1 || t == nk - 1)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              su32(&sm.gdone[gb])));
        // refill the slot of the previous stage once its products are done
        if (t >= 1 && t - 1 + ST2 < nk) {
          const int sp = (t - 1) % ST2;
          if (!wait_parity(su32(&sm.empty[sp]), ((t - 1) / ST2) & 1)) { ok = false; break; }
          bulk_stage(sm, t - 1 + ST2, pa0, pb0, loaded);
        }
      }
      if (!ok) {
        // before the tile is abandoned: the copies still in flight land
        // (bounded waits), and every product issued so far completes
        for (int u = consumed; u < loaded; ++u) (void)wait_parity(su32(&sm.full[u % ST2]), (u / ST2) & 1);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(&sm.fin)));
        (void)wait_parity(su32(&sm.fin), 0);
        atomicExch(&sm.fail, 1);
      }
    }
  } else {
    const int qd = warp & 3, half = warp >> 2;
#pragma unroll
    for (int q = 0; q < 64; ++q) { acc_hi[q] = 0.0f; acc_lo[q] = 0.0f; }
    for (int gi = 0; gi < ngrp; ++gi) {
      const int gb = gi & 1;
      if (!wait_parity(su32(&sm.gdone[gb]), (gi >> 1) & 1)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int which = 0; which < 2; ++which) {
        const uint32_t base = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(gb * 2 * N2 + which * N2 + half * 64);
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
          uint32_t r[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(base + c0));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float a = acc_hi[c0 + q], bv = __uint_as_float(r[q]);
            const float s2 = a + bv;
            const float bp = s2 - a;
            const float er = (a - (s2 - bp)) + (bv - bp);
            acc_hi[c0 + q] = s2;
            acc_lo[c0 + q] += er;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&sm.gfree[gb])) : "memory");
    }
    if (!ok) atomicExch(&sm.fail, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const bool fail = sm.fail != 0;
  if (fail && tid == 0 && g.skip) atomicOr(const_cast<int*>(g.skip), ST_TIMEOUT);

  if (!fail && warp < 8) {
    const int qd = warp & 3, half = warp >> 2;
    const int row = i0 + qd * 32 + lane;
    double* part = (S > 1) ? g.partial + (int64_t)kb * Ms * g.N : nullptr;
    if (row < M) {
#pragma unroll
      for (int q = 0; q < 64; ++q) {
        const int j = j0 + half * 64 + q;
        if (j >= N) continue;
        if (lowc && !part && row < j) continue;
        const double acc = f32_f64(acc_hi[q]) + f32_f64(acc_lo[q]);
        if (part) {
          part[(int64_t)row + (int64_t)j * Ms] = acc;
          continue;
        }
        const int jc = g.colmap ? g.colmap[j] : j;
        double* cp = (flags & GF_TRANS_C) ? g.C + (int64_t)jc + (int64_t)row * g.ldc
                                          : g.C + (int64_t)row + (int64_t)jc * g.ldc;
        double v = g.alpha == 1.0 ? acc : g.alpha * acc;
        if (g.beta != 0.0) {
          const double cv = (flags & GF_BETA_B) ? g.B[(int64_t)row + (int64_t)j * g.ldb] : *cp;
          v = fma(g.beta, cv, v);
        }
        *cp = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace

void launch_tc2_slice(const SliceJob* jobs, const int* prefix, int njobs, int total, cudaStream_t s) {
  if (njobs <= 0 || total <= 0) return;
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(tc2_slice_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSliceSmem);
  }
  tc2_slice_kernel<<<total, 256, kSliceSmem, s>>>(jobs, prefix, njobs);
}

void launch_tc2_gemm(const GemmDesc* descs, const int* tile_prefix, int count, int total_tiles, cudaStream_t s) {
  if (count <= 0 || total_tiles <= 0) return;
  static std::atomic<unsigned long long> attr{0};
  const size_t smem = sizeof(Tc2Smem) + 1024;
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(tc2_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  tc2_gemm_kernel<<<total_tiles, 288, smem, s>>>(descs, tile_prefix, count);
}

int64_t tc2_slice_floats(int rows, int K) {
  const int64_t tiles = (rows + M2 - 1) / M2, KT = (K + K2 - 1) / K2;
  return tiles * KT * 3 * BLK;
}

int tc2_slice_ctas(int rows, int K) { return 2 * ((rows + M2 - 1) / M2) * ((K + G2 - 1) / G2); }

}  // namespace scs
