// Complex Hermitian cones without the real embedding (the paper's cones are
// complex Hermitian: App. D.1's vec map carries sqrt(2) Re X_ij and
// sqrt(2) Im X_ij; App. D.2 times complex eigendecompositions).
//
//   hetrd1_kernel  one-stage Householder reduction X = Q T Q^H, T real
//                  symmetric tridiagonal: complex reflectors H_j = I - tau_j
//                  u_j u_j^H, u_j(0) = 1, that also leave every off-diagonal
//                  real (beta real in the reflector of a complex alpha).  Its
//                  structure is the real one-stage kernel's (sytrd1.cu): CTA
//                  r of a cone's group owns the columns i mod G = r in shared
//                  memory, each step's p = tau A v and next column are
//                  published into write-once slabs and polled by value, one
//                  warp per column forms the rank-2 update and the column's
//                  whole dot product; the arithmetic is complex double-float.
//   hlarft_kernel  the triangular factor of every block of 32 reflectors,
//                  H_0 .. H_31 = I - V T V^H.
//   hbt_kernel     Q Z for the kept eigenvectors Z of T (real, from the
//                  divide and conquer of the real path), block by block.
//   hrecon_kernel  the clipped reconstruction V_k diag(l_k) V_k^H (positive
//                  part, or X minus the negative part) written straight into
//                  the Hermitian svec.
//
// For the step j reflector v (v_0 = 1) and p = tau A22 v, K = (tau/2) p^H v
// is real (p^H v = conj(tau) v^H A v), w = p - K v, and the update
// A -= v w^H + w v^H reads, per element of column i (stored as A(r, i)):
//     A(r, i) -= v_r conj(p_i - 2K v_i) + p_r conj(v_i);
// the next column becomes (a_t - p_t) - v_t (conj(p_0) - 2K); and with the
// next reflector u = scal x (u_0 = 1), p_i = tau (conj(a_0) + scal sum_{t>=1}
// conj(a_t) x_t) since A(i, r) = conj(A(r, i)).
#include <limits.h>
#include <math.h>

#include "dfloat.cuh"
#include "internal.cuh"

namespace scs {

namespace {

constexpr int kHThreads = 256;
constexpr int kHNb = 32;  // reflectors per block of the back-transformation

// published words (one double-float each: re and im apart), sentinel as the real kernel's
constexpr unsigned long long kHSentinel = 0xA5A5A5A5FFA5A5A5ull;
__device__ __forceinline__ void hst_pub(dfl* p, dfl v) {
  const unsigned long long bits =
      ((unsigned long long)__float_as_uint(v.lo) << 32) | (unsigned long long)__float_as_uint(v.hi);
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(bits) : "memory");
}
__device__ __forceinline__ unsigned long long hld_pub(const dfl* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ dfl hbits(unsigned long long b) {
  return df_make(__uint_as_float((unsigned)(b & 0xffffffffull)), __uint_as_float((unsigned)(b >> 32)));
}
__device__ __forceinline__ int h_ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int64_t hcol_off(int64_t n, int64_t j) { return j * (2 * n - j); }
// slab of step j: 4 m_j words (p re/im interleaved, then the column re/im)
__device__ __forceinline__ int64_t hslab(int64_t n, int64_t j) { return 4 * (j * (n - 1) - (j * (j - 1)) / 2); }

// one barrier over the group (its 8 counters as the real kernel's), once per call
__device__ bool h_group_barrier(int* counters, int rank, int G, long long limit) {
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(counters + 32 * (rank % 8)), "r"(1) : "memory");
  int ok = 1;
  const int t = threadIdx.x;
  if (t < 8 && t < G) {
    const int target = (G - 1 - t) / 8 + 1;
    const int* cnt = counters + 32 * t;
    if (h_ld_acquire(cnt) < target) {
      const long long t0 = clock64();
      while (h_ld_acquire(cnt) < target) {
        if (clock64() - t0 > limit) { ok = 0; break; }
      }
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

__device__ dfl h_block_sum(dfl v, dfl* red, int& parity) {
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  dfl* r = red + 8 * parity;
  parity ^= 1;
  if (lane == 0) r[w] = v;
  __syncthreads();
  return df_add(df_add(df_add(r[0], r[1]), df_add(r[2], r[3])), df_add(df_add(r[4], r[5]), df_add(r[6], r[7])));
}

// Complex reflector (LAPACK convention) for (alpha, x) with sigma = ||x||^2:
// beta real, H^H (alpha; x) = (beta; 0), tau = (beta - alpha) / beta,
// scal = 1 / (alpha - beta); tau = 0 (H = I) when x = 0 and alpha is real.
__device__ void h_reflector(cdf alpha, dfl sigma, dfl* beta, cdf* tau, cdf* scal) {
  const bool trivial = sigma.hi == 0.0f && sigma.lo == 0.0f && alpha.im.hi == 0.0f && alpha.im.lo == 0.0f;
  if (trivial) {
    *beta = alpha.re;
    *tau = c_zero();
    *scal = c_zero();
    return;
  }
  const dfl nrm = df_sqrt(df_fma(alpha.re, alpha.re, df_fma(alpha.im, alpha.im, sigma)));
  const dfl b = alpha.re.hi >= 0.0f ? df_neg(nrm) : nrm;
  *beta = b;
  *tau = c_make(df_div(df_add(b, df_neg(alpha.re)), b), df_div(df_neg(alpha.im), b));
  // 1 / (alpha - beta) = conj(d) / |d|^2
  const cdf d = c_make(df_add(alpha.re, df_neg(b)), alpha.im);
  const dfl inv = df_div(df_make(1.0f, 0.0f), df_fma(d.re, d.re, df_mul(d.im, d.im)));
  *scal = c_make(df_mul(d.re, inv), df_neg(df_mul(d.im, inv)));
}

// Reflector j (u = scal x for rows > j+1, u(j+1) = 1) into its block of V:
// block q = j / 32 holds rows r0 = 32 q + 1 .. n-1 (mq of them), column
// j mod 32, with the unit diagonal and zeros above; rows spread over the group.
__device__ void h_store_reflector(cdf* V, int n, int j, const cdf* x, cdf scal, bool scaled, int rank, int G) {
  const int q = j / kHNb, col = j % kHNb;
  const int r0 = q * kHNb + 1, mq = n - r0;
  cdf* Vq = V + (int64_t)q * n * kHNb;
  for (int r = rank + G * threadIdx.x; r < mq; r += G * kHThreads) {
    const int row = r0 + r;
    cdf val = c_zero();
    if (row == j + 1) val = c_one();
    else if (row > j + 1) val = scaled ? c_mul(scal, x[row - j - 1]) : x[row - j - 1];
    Vq[(int64_t)r + (int64_t)col * mq] = val;
  }
}

__device__ __forceinline__ void h_wait_tag(const int* tag_p, int tag, int* status) {
  if (*(volatile const int*)tag_p != tag) {
    long long spins = 0;
    while (*(volatile const int*)tag_p != tag) {
      if (++spins > (1ll << 30)) { atomicOr(status, ST_TIMEOUT); break; }
    }
  }
  __threadfence_block();
}

// One warp per own column i >= r0: the step's update (UPDATE), the column's
// conj dot product with x, p_i = tau (conj(a_0) + scal dot) published to Pn
// (re, im) once the scalars are announced; the owner of column r0 publishes
// its rows to Cn.
// With at most NW / 2 columns, two warps share each column (interleaved
// chunks of rows); the second hands its part of the dot product to the first
// through half_part[k], announced by half_tag[k] = tag.
template <bool UPDATE>
__device__ void h_column_pass(cdf* __restrict__ cols, int n, int r0, const cdf* __restrict__ x, const cdf* coef,
                              const int* tag_p, int tag, const cdf* __restrict__ vu, const cdf* __restrict__ pu,
                              dfl K2, dfl* Pn, dfl* Cn, int rank, int G, int* status, int* half_tag,
                              cdf* half_part) {
  constexpr int U = 2;
  constexpr int NW = kHThreads / 32;
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
    cdf* col = cols + (int64_t)((i - rank) / G) * n + r0;
    const bool pub_col = i == r0;
    cdf nai = c_zero(), ncvi = c_zero();
    if (UPDATE) {
      const cdf vi = vu[i - r0 + 1];
      const cdf pi = pu[i - r0 + 1];
      // -conj(p_i - 2K v_i) and -conj(v_i)
      const cdf t2 = c_make(df_fma(df_neg(K2), vi.re, pi.re), df_fma(df_neg(K2), vi.im, pi.im));
      nai = c_neg(c_conj(t2));
      ncvi = c_neg(c_conj(vi));
    }
    c_dot acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = c_dot_zero();
    for (int t0 = lane + half * 32 * U; t0 < L; t0 += tstride) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int t = t0 + 32 * u;
        if (t < L) {
          cdf a = col[t];
          if (UPDATE) {
            a = c_add2prod(a, vu[t + 1], nai, pu[t + 1], ncvi);
            col[t] = a;
          }
          if (pub_col) {
            hst_pub(Cn + 2 * t, a.re);
            hst_pub(Cn + 2 * t + 1, a.im);
          }
          if (t > 0) acc[u] = c_dot_add(acc[u], a, x[t]);
        }
      }
    }
    cdf sdot = c_add(c_dot_value(acc[0]), c_dot_value(acc[1]));
    for (int o = 16; o > 0; o >>= 1) sdot = c_add(sdot, c_shfl_xor(sdot, o));
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
        h_wait_tag(half_tag + k, tag, status);
        sdot = c_add(sdot, half_part[k]);
      }
      h_wait_tag(tag_p, tag, status);
      const cdf tau = coef[0], scal = coef[1];
      const cdf pv = c_mul(tau, c_fma(scal, sdot, c_conj(col[0])));
      hst_pub(Pn + 2 * (i - r0), pv.re);
      hst_pub(Pn + 2 * (i - r0) + 1, pv.im);
    }
  }
}

// p (m values) and column (m values) of a step as they arrive: p into ps,
// a - p into bs; this warp's part of p^H v into red[warp] (complex: 2 slots of 8).
__device__ bool h_poll(const dfl* P, const dfl* C, int m, const cdf* v, cdf* ps, cdf* bs, long long limit,
                       cdf* red) {
  cdf pt = c_zero();
  int ok = 1;
  for (int base = 0; base < m && ok; base += 2 * kHThreads) {
    unsigned long long w[2][4];  // [q][p re, p im, c re, c im]
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int t = base + q * kHThreads + threadIdx.x;
      if (t < m) {
        w[q][0] = hld_pub(P + 2 * t);
        w[q][1] = hld_pub(P + 2 * t + 1);
        w[q][2] = hld_pub(C + 2 * t);
        w[q][3] = hld_pub(C + 2 * t + 1);
      } else {
        w[q][0] = w[q][1] = w[q][2] = w[q][3] = 0ull;
      }
    }
    bool miss = false;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) miss = miss || w[q][e] == kHSentinel;
    if (miss) {
      const long long t0 = clock64();
      while (true) {
        miss = false;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int t = base + q * kHThreads + threadIdx.x;
          const dfl* src[4] = {P + 2 * t, P + 2 * t + 1, C + 2 * t, C + 2 * t + 1};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (w[q][e] == kHSentinel) {
              w[q][e] = hld_pub(src[e]);
              miss = miss || w[q][e] == kHSentinel;
            }
        }
        if (!miss) break;
        if (clock64() - t0 > limit) { ok = 0; break; }
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int t = base + q * kHThreads + threadIdx.x;
      if (t < m) {
        const cdf p = c_make(hbits(w[q][0]), hbits(w[q][1]));
        const cdf a = c_make(hbits(w[q][2]), hbits(w[q][3]));
        ps[t] = p;
        bs[t] = c_add(a, c_neg(p));
        pt = c_cfma(p, v[t], pt);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) pt = c_add(pt, c_shfl_xor(pt, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pt;
  return __syncthreads_and(ok) != 0;
}

__device__ void hetrd1_body(const HConeDev& c, const double* __restrict__ xs, int rank, int G, long long wait_limit,
                            double* smem, dfl* red, cdf* redc, cdf* shc, dfl* shb, int* tag_p, int* half_tag,
                            cdf* half_part) {
  const int n = (int)c.n;
  cdf* base = reinterpret_cast<cdf*>(smem);
  cdf* vc = base;
  cdf* vn = base + n;
  cdf* ps = base + 2 * n;
  cdf* bs = base + 3 * n;
  cdf* cols = base + 4 * n;
  double* colsd = smem + 8 * n;  // the same storage, first loaded as FP64 (re, im)
  dfl* pub = c.pub;
  const int tid = threadIdx.x;
  const double* x = xs + c.xoff;
  int parity = 0;
  if (n == 1) {
    if (rank == 0 && tid == 0) { c.d[0] = x[0]; c.e[0] = 0.0; }
    return;
  }
  // ---- own columns as FP64 from the Hermitian svec, the largest exponent
  int emax = 0;
  for (int i = rank; i < n; i += G) {
    double* dst = colsd + 2 * (int64_t)((i - rank) / G) * n;
    for (int r = tid; r < n; r += kHThreads) {
      double re, im;
      if (r == i) { re = x[hcol_off(n, i)]; im = 0.0; }
      else if (r > i) {
        const int64_t o = hcol_off(n, i) + 1 + 2 * (r - i - 1);
        re = x[o] * M_SQRT1_2; im = x[o + 1] * M_SQRT1_2;
      } else {
        const int64_t o = hcol_off(n, r) + 1 + 2 * (i - r - 1);
        re = x[o] * M_SQRT1_2; im = -x[o + 1] * M_SQRT1_2;
      }
      dst[2 * r] = re;
      dst[2 * r + 1] = im;
      emax = max(emax, max((int)((__double2hiint(re) >> 20) & 0x7FF), (int)((__double2hiint(im) >> 20) & 0x7FF)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if ((tid & 31) == 0 && emax > 0) atomicMax(c.prog + 1, emax);
  {
    const int64_t total = 2 * (int64_t)n * (n - 1);
    const dfl sent = hbits(kHSentinel);
    for (int64_t e = (int64_t)rank * kHThreads + tid; e < total; e += (int64_t)G * kHThreads) pub[e] = sent;
  }
  if (!h_group_barrier(c.prog, rank, G, wait_limit)) {
    if (tid == 0) atomicOr(c.status, ST_TIMEOUT);
    return;
  }
  int eb = *((volatile int*)(c.prog + 1));
  eb = min(max(eb, 1), 2045);
  const double s_in = __longlong_as_double((long long)(2046 - eb) << 52);
  const double s_out = __longlong_as_double((long long)eb << 52);
  for (int i = rank; i < n; i += G) {
    cdf* dst = cols + (int64_t)((i - rank) / G) * n;
    const double* srcd = colsd + 2 * (int64_t)((i - rank) / G) * n;
    for (int r = tid; r < n; r += kHThreads) dst[r] = c_from_d(srcd[2 * r] * s_in, srcd[2 * r + 1] * s_in);
  }
  // ---- prologue: reflector 0 from column 0 (rows 1 ..), every CTA
  dfl ss = df_zero();
  for (int t = tid; t < n - 1; t += kHThreads) {
    const int64_t o = hcol_off(n, 0) + 1 + 2 * t;
    const cdf v = c_from_d(x[o] * M_SQRT1_2 * s_in, x[o + 1] * M_SQRT1_2 * s_in);
    vc[t] = v;
    if (t >= 1) ss = df_fma(v.re, v.re, df_fma(v.im, v.im, ss));
  }
  __syncthreads();
  {
    const dfl sig = h_block_sum(ss, red, parity);
    if (tid == 0) {
      dfl beta;
      h_reflector(vc[0], sig, &beta, shc, shc + 1);
      shb[0] = beta;
    }
    __syncthreads();
    const cdf scal = shc[1];
    for (int t = 1 + tid; t < n - 1; t += kHThreads) vc[t] = c_mul(scal, vc[t]);
    __syncthreads();
    if (tid == 0) vc[0] = c_one();
    if (rank == 0 && tid == 0) {
      c.d[0] = x[0];
      c.e[0] = df_to_d(shb[0]) * s_out;
      c.tau[0] = shc[0];
    }
    h_store_reflector(c.V, n, 0, vc, c_zero(), false, rank, G);
    if (tid == 0) {
      shc[1] = c_one();  // coefficients (tau, 1): v_0 is scaled already
      *tag_p = -1;
    }
    __syncthreads();
  }
  h_column_pass<false>(cols, n, 1, vc, shc, tag_p, -1, nullptr, nullptr, df_zero(), pub + hslab(n, 0),
                       pub + hslab(n, 0) + 2 * (n - 1), rank, G, c.status, half_tag, half_part);
  cdf tau = shc[0];
  __syncthreads();
  for (int j = 0; j + 1 < n; ++j) {
    const int m = n - j - 1;
    dfl* P = pub + hslab(n, j);
    cdf* rp = redc + 8 * parity;
    parity ^= 1;
    if (!h_poll(P, P + 2 * m, m, vc, ps, bs, wait_limit, rp)) {
      if (tid == 0) atomicOr(c.status, ST_TIMEOUT);
      return;
    }
    const cdf S = c_add(c_add(c_add(rp[0], rp[1]), c_add(rp[2], rp[3])), c_add(c_add(rp[4], rp[5]), c_add(rp[6], rp[7])));
    // K = Re(tau S) / 2 (real in exact arithmetic)
    const dfl K = df_mul(df_make(0.5f, 0.0f), df_fma(tau.re, S.re, df_mul(df_neg(tau.im), S.im)));
    const dfl K2 = df_make(2.0f * K.hi, 2.0f * K.lo);
    // c0 = conj(p_0) - 2K; nc_t = b_t - v_t c0
    const cdf nc0 = c_neg(c_make(df_add(ps[0].re, df_neg(K2)), df_neg(ps[0].im)));
    dfl sq = df_zero();
    for (int t = tid; t < m; t += kHThreads) {
      const cdf nc = c_fma(vc[t], nc0, bs[t]);
      bs[t] = nc;
      if (t >= 2) sq = df_fma(nc.re, nc.re, df_fma(nc.im, nc.im, sq));
    }
    if (j + 2 < n) {
      const dfl sig = h_block_sum(sq, red, parity);
      if (tid == 0) {
        dfl beta1;
        h_reflector(bs[1], sig, &beta1, shc, shc + 1);
        shb[0] = beta1;
        __threadfence_block();
        *(volatile int*)tag_p = j;
      }
      dfl* Pn = pub + hslab(n, j + 1);
      h_column_pass<true>(cols, n, j + 2, bs + 1, shc, tag_p, j, vc, ps, K2, Pn, Pn + 2 * (m - 1), rank, G,
                          c.status, half_tag, half_part);
      h_wait_tag(tag_p, j, c.status);
      const cdf tau1 = shc[0], scal1 = shc[1];
      if (rank == 0 && tid == 0) {
        c.d[j + 1] = df_to_d(bs[0].re) * s_out;
        c.e[j + 1] = df_to_d(shb[0]) * s_out;
        c.tau[j + 1] = tau1;
      }
      h_store_reflector(c.V, n, j + 1, bs + 1, scal1, true, rank, G);
      for (int t = tid; t < m - 1; t += kHThreads) vn[t] = t == 0 ? c_one() : c_mul(scal1, bs[1 + t]);
      tau = tau1;
      __syncthreads();
      cdf* tmp = vc;
      vc = vn;
      vn = tmp;
    } else {
      __syncthreads();
      if (rank == 0 && tid == 0) {
        c.d[n - 1] = df_to_d(bs[0].re) * s_out;
        c.e[n - 1] = 0.0;
      }
    }
  }
}

__global__ void __launch_bounds__(kHThreads) hetrd1_kernel(const HConeDev* __restrict__ cones,
                                                           const int* __restrict__ cta_cone,
                                                           const int* __restrict__ cta_rank,
                                                           const int* __restrict__ cta_count, const IoSlot* io,
                                                           long long wait_limit) {
  extern __shared__ double h_smem[];
  __shared__ dfl red[16];
  __shared__ cdf redc[16];
  __shared__ cdf shc[2];
  __shared__ dfl shb[1];
  __shared__ int tag;
  __shared__ int half_tag[kHThreads / 64];
  __shared__ cdf half_part[kHThreads / 64];
  const HConeDev& c = cones[cta_cone[blockIdx.x]];
  if (*c.status != 0) return;
  // no pass has announced a part yet (the body's first CTA barrier orders this)
  if (threadIdx.x < kHThreads / 64) half_tag[threadIdx.x] = INT_MIN;
  hetrd1_body(c, io->x, cta_rank[blockIdx.x], cta_count[blockIdx.x], wait_limit, h_smem, red, redc, shc, shb, &tag,
              half_tag, half_part);
}

// ---------------------------------------------------------------- T factors
// Block q: G = V^H V, then T(a, j) = -tau_j sum_{b=a}^{j-1} T(a, b) G(b, j),
// T(j, j) = tau_j (forward, columnwise).  One CTA per block.
__global__ void __launch_bounds__(kHThreads) hlarft_kernel(const HConeDev* __restrict__ cones,
                                                           const int* __restrict__ blk_cone,
                                                           const int* __restrict__ blk_index) {
  __shared__ cdf Gm[kHNb][kHNb + 1];
  __shared__ cdf T[kHNb][kHNb + 1];
  const HConeDev& c = cones[blk_cone[blockIdx.x]];
  if (*c.status != 0) return;
  const int q = blk_index[blockIdx.x];
  const int n = (int)c.n;
  const int r0 = q * kHNb + 1, mq = n - r0;
  const int nr = min(kHNb, n - 1 - q * kHNb);
  const cdf* Vq = c.V + (int64_t)q * n * kHNb;
  const int tid = threadIdx.x;
  // Gram entries (a, b), a < b: one warp per entry, lanes over rows
  const int warp = tid >> 5, lane = tid & 31;
  for (int e = warp; e < kHNb * kHNb; e += kHThreads / 32) {
    const int a = e % kHNb, b = e / kHNb;
    if (a >= b || b >= nr) continue;
    cdf acc = c_zero();
    for (int r = lane; r < mq; r += 32) acc = c_cfma(Vq[(int64_t)r + (int64_t)a * mq], Vq[(int64_t)r + (int64_t)b * mq], acc);
    for (int o = 16; o > 0; o >>= 1) acc = c_add(acc, c_shfl_xor(acc, o));
    if (lane == 0) Gm[a][b] = acc;
  }
  for (int e = tid; e < kHNb * kHNb; e += kHThreads) T[e % kHNb][e / kHNb] = c_zero();
  __syncthreads();
  for (int j = 0; j < nr; ++j) {
    const cdf tj = c.tau[q * kHNb + j];
    cdf s = c_zero();
    if (tid < j)
      for (int b = tid; b < j; ++b) s = c_fma(T[tid][b], Gm[b][j], s);
    __syncthreads();
    if (tid < j) T[tid][j] = c_neg(c_mul(tj, s));
    if (tid == 0) T[j][j] = tj;
    __syncthreads();
  }
  cdf* Tq = c.T + (int64_t)q * kHNb * kHNb;
  for (int e = tid; e < kHNb * kHNb; e += kHThreads) Tq[e] = T[e % kHNb][e / kHNb];  // column-major
}

// ---------------------------------------------------------------- back-transformation
// W = Q Z for the kept columns of Z (real, n x k, ld n): Q = H_0 .. H_{n-2}
// = Q_0 Q_1 .. (blocks of 32), applied to a slab of KC columns in shared
// memory, last block first: Z -= V (T (V^H Z)).  Row 0 is unchanged.
template <int KC>
__device__ void hbt_slab(const HConeDev& c, int j0, int ncols, cdf* zs, cdf* Ws, cdf* Wt) {
  const int n = (int)c.n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < KC * n; e += kHThreads) {
    const int col = e / n, r = e - col * n;
    const double z = col < ncols ? c.Z[(int64_t)r + (int64_t)(j0 + col) * n] : 0.0;
    zs[e] = c_make(df_from_d_int(z), df_zero());  // eigenvector entries, |z| <= 1
  }
  __syncthreads();
  const int nblk = (n - 2) / kHNb + 1;
  for (int q = nblk - 1; q >= 0; --q) {
    const int r0 = q * kHNb + 1, mq = n - r0;
    const int bb = min(kHNb, n - 1 - q * kHNb);
    const cdf* Vq = c.V + (int64_t)q * n * kHNb;
    const cdf* Tq = c.T + (int64_t)q * kHNb * kHNb;
    // W(a, col) = sum_r conj(V(r, a)) z(r0 + r, col): warp w takes reflectors w, w + 8, ..
    for (int a = warp; a < kHNb; a += kHThreads / 32) {
      c_dot acc[KC];
#pragma unroll
      for (int col = 0; col < KC; ++col) acc[col] = c_dot_zero();
      if (a < bb)
        for (int r = lane + a; r < mq; r += 32) {  // rows above a are zero
          const cdf v = Vq[(int64_t)r + (int64_t)a * mq];
#pragma unroll
          for (int col = 0; col < KC; ++col) acc[col] = c_dot_add(acc[col], v, zs[col * n + r0 + r]);
        }
#pragma unroll
      for (int col = 0; col < KC; ++col) {
        cdf s = c_dot_value(acc[col]);
        for (int o = 16; o > 0; o >>= 1) s = c_add(s, c_shfl_xor(s, o));
        if (lane == 0) Ws[a * KC + col] = s;
      }
    }
    __syncthreads();
    // W' = T W (T upper triangular)
    for (int e = tid; e < kHNb * KC; e += kHThreads) {
      const int a = e / KC, col = e % KC;
      cdf s = c_zero();
      if (a < bb)
        for (int b = a; b < bb; ++b) s = c_fma(Tq[a + b * kHNb], Ws[b * KC + col], s);
      Wt[a * KC + col] = s;
    }
    __syncthreads();
    // z(r0 + r, col) -= sum_a V(r, a) W'(a, col)
    for (int r = tid; r < mq; r += kHThreads) {
      c_dot s[KC];
#pragma unroll
      for (int col = 0; col < KC; ++col) s[col] = c_dot_zero();
      const int amax = min(bb, r + 1);  // V(r, a) = 0 for a > r
      for (int a = 0; a < amax; ++a) {
        const cdf v = Vq[(int64_t)r + (int64_t)a * mq];
#pragma unroll
        for (int col = 0; col < KC; ++col) s[col] = c_dotn_add(s[col], v, Wt[a * KC + col]);
      }
#pragma unroll
      for (int col = 0; col < KC; ++col) zs[col * n + r0 + r] = c_add(zs[col * n + r0 + r], c_neg(c_dot_value(s[col])));
    }
    __syncthreads();
  }
  for (int e = tid; e < KC * n; e += kHThreads) {
    const int col = e / n, r = e - col * n;
    if (col < ncols) c.W[(int64_t)r + (int64_t)(j0 + col) * n] = zs[e];
  }
  __syncthreads();
}

constexpr int kHbtCols = 4;

__global__ void __launch_bounds__(kHThreads) hbt_kernel(const HConeDev* __restrict__ cones,
                                                        const int* __restrict__ cta_cone,
                                                        const int* __restrict__ cta_rank,
                                                        const int* __restrict__ cta_count) {
  extern __shared__ cdf hb_smem[];
  __shared__ cdf Ws[kHNb * kHbtCols];
  __shared__ cdf Wt[kHNb * kHbtCols];
  const HConeDev& c = cones[cta_cone[blockIdx.x]];
  if (*c.status != 0) return;
  const int rank = cta_rank[blockIdx.x], G = cta_count[blockIdx.x];
  const int k = c.kinfo[0];
  const int basek = k / G, extra = k % G;
  const int lo = rank * basek + min(rank, extra);
  const int hi = lo + basek + (rank < extra ? 1 : 0);
  for (int j0 = lo; j0 < hi;) {
    const int left = hi - j0;
    if (left >= 3) { hbt_slab<4>(c, j0, min(left, 4), hb_smem, Ws, Wt); j0 += min(left, 4); }
    else if (left == 2) { hbt_slab<2>(c, j0, 2, hb_smem, Ws, Wt); j0 += 2; }
    else { hbt_slab<1>(c, j0, 1, hb_smem, Ws, Wt); j0 += 1; }
  }
}

// ---------------------------------------------------------------- reconstruction
// Lower triangle of S = W diag(l) W^H (k kept pairs; W complex n x k) in 32 x
// 32 tiles (blockIdx.x), written into the Hermitian svec: positive part
// y = svec(S), or y = x - svec(S) (Moreau) for route 1.
constexpr int kRT = 32;
__global__ void __launch_bounds__(kHThreads) hrecon_kernel(const HConeDev* __restrict__ cones,
                                                           const IoSlot* __restrict__ io) {
  __shared__ cdf As[8][kRT];
  __shared__ cdf Bs[8][kRT];
  const HConeDev& c = cones[blockIdx.y];
  const int n = (int)c.n;
  const int tiles = (n + kRT - 1) / kRT;
  const int t = blockIdx.x;
  if (t >= tiles * (tiles + 1) / 2) return;
  int tm = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
  while (tm * (tm + 1) / 2 > t) --tm;
  const int tn = t - tm * (tm + 1) / 2;
  const int i0 = tm * kRT, j0 = tn * kRT;
  const bool bad = *c.status != 0;
  const int kk = bad ? 0 : c.kinfo[0];
  const int route = c.kinfo[1];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;  // 32 x 8 threads, 4 rows of j each
  cdf acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = c_zero();
  for (int k0 = 0; k0 < kk; k0 += 8) {
    {
      const int l = ty, k = k0 + l;
      cdf a = c_zero(), b = c_zero();
      if (k < kk) {
        // the kept side's eigenvalues, clipped to it
        const dfl lam = df_from_d(route == 0 ? fmax(c.lamk[k], 0.0) : fmin(c.lamk[k], 0.0));
        if (i0 + tx < n) a = c.W[(int64_t)(i0 + tx) + (int64_t)k * n];
        if (j0 + tx < n) {
          const cdf w = c.W[(int64_t)(j0 + tx) + (int64_t)k * n];
          b = c_make(df_mul(lam, w.re), df_mul(lam, w.im));
        }
      }
      As[l][tx] = a;
      Bs[l][tx] = b;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const cdf a = As[l][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = c_fma(a, c_conj(Bs[l][ty + 8 * q]), acc[q]);
    }
    __syncthreads();
  }
  const double* x = io->x + c.xoff;
  double* y = io->y + c.xoff;
  const int i = i0 + tx;
  if (i >= n) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = j0 + ty + 8 * q;
    if (j >= n || j > i) continue;
    if (bad) {
      if (i == j) y[hcol_off(n, j)] = nan("");
      else { y[hcol_off(n, j) + 1 + 2 * (i - j - 1)] = nan(""); y[hcol_off(n, j) + 2 + 2 * (i - j - 1)] = nan(""); }
      continue;
    }
    const double sr = df_to_d(acc[q].re), si = df_to_d(acc[q].im);
    if (i == j) {
      const int64_t o = hcol_off(n, j);
      y[o] = route ? x[o] - sr : sr;
    } else {
      const int64_t o = hcol_off(n, j) + 1 + 2 * (i - j - 1);
      const double yr = M_SQRT2 * sr, yi = M_SQRT2 * si;
      y[o] = route ? x[o] - yr : yr;
      y[o + 1] = route ? x[o + 1] - yi : yi;
    }
  }
}

}  // namespace

size_t hetrd1_smem_bytes(int n, int G) {
  return ((size_t)4 * n + (size_t)((n + G - 1) / G) * n) * sizeof(cdf);
}

int hetrd1_max_ctas_for(size_t smem) {
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(hetrd1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHetrdSmemMax);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hetrd1_kernel, kHThreads, smem);
  return per_sm * sms;
}

size_t hcone_pub_doubles(int64_t n) { return (size_t)(2 * n * (n - 1) + 1); }
size_t hcone_v_elems(int64_t n) { return (size_t)(((n - 2) / kHNb + 1) * n * kHNb); }
size_t hcone_t_elems(int64_t n) { return (size_t)(((n - 2) / kHNb + 1) * kHNb * kHNb); }
int hcone_blocks(int64_t n) { return n >= 2 ? (int)((n - 2) / kHNb + 1) : 0; }

int launch_hetrd1(const HConeDev* cones, const int* cta_cone, const int* cta_rank, const int* cta_count, int nctas,
                  size_t smem, const IoSlot* io, long long wait_limit, cudaStream_t s) {
  if (nctas <= 0) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nctas);
  cfg.blockDim = dim3(kHThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, hetrd1_kernel, cones, cta_cone, cta_rank, cta_count, io, wait_limit);
}

void launch_hlarft(const HConeDev* cones, const int* blk_cone, const int* blk_index, int nblocks, cudaStream_t s) {
  if (nblocks <= 0) return;
  hlarft_kernel<<<nblocks, kHThreads, 0, s>>>(cones, blk_cone, blk_index);
}

void launch_hbt(const HConeDev* cones, const int* cta_cone, const int* cta_rank, const int* cta_count, int nctas,
                int maxn, cudaStream_t s) {
  if (nctas <= 0) return;
  const size_t smem = (size_t)kHbtCols * maxn * sizeof(cdf);
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(hbt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  hbt_kernel<<<nctas, kHThreads, smem, s>>>(cones, cta_cone, cta_rank, cta_count);
}

void launch_hrecon(const HConeDev* cones, int ncones, int maxn, const IoSlot* io, cudaStream_t s) {
  if (ncones <= 0) return;
  const int tiles = (maxn + kRT - 1) / kRT;
  hrecon_kernel<<<dim3(tiles * (tiles + 1) / 2, ncones), kHThreads, 0, s>>>(cones, io);
}

}  // namespace scs
