// Divide and conquer for the symmetric tridiagonal eigenproblem (Cuppen),
// with Dongarra-Sorensen deflation and the Gu-Eisenstat (Loewner) correction
// that keeps the computed eigenvectors orthogonal.
//
// Tearing: every off-diagonal e_m couples rows m and m+1 as |e_m| v v^T with
// v = e_m + sign(e_m) e_{m+1}; the leaves are 1x1 blocks with diagonal
// d_i - |e_{i-1}| - |e_i|.  Level l merges adjacent blocks of size 2^l: with
// Q = diag(Q1, Q2) the children's eigenvectors and D their eigenvalues,
//     T = Q (D + rho z z^T) Q^T,  z = Q^T v / ||Q^T v||,  rho = |e_m| ||Q^T v||^2.
// A merge node
//   prepare : sorts D (merge of two sorted lists), deflates z_j with
//             rho |z_j| <= tol and pairs of close poles by a Givens rotation,
//             tol = 8 eps max(max|d|, rho), and forms the permuted, rotated
//             eigenvector block [kept | deflated];
//   secular : solves 1 + rho sum z_j^2 / (d_j - x) = 0 for each root, one
//             thread per root, in coordinates shifted to the nearer pole
//             (two-pole rational model with a bisection safeguard);
//   loewner : recomputes z from the roots so that the vectors are exact
//             eigenvectors of a nearby problem;
//   select  : places roots and deflated values in sorted order (for the
//             cone's final merge: chooses the side -- positive part, or X minus
//             the negative part -- and keeps only those eigenpairs);
//   vectors : u_i = zhat / (d - lambda_i), normalised;
//   GEMM    : new block = [kept columns] * U^T (grouped GEMM, separate file).
#include <math.h>

#include "internal.cuh"

namespace scs {

namespace {

constexpr int kDcThreads = 256;
constexpr int kQinCols = 4;  // columns per CTA of dc_build_qin
constexpr double kEps = 1.1102230246251565e-16;  // 2^-53

__device__ __forceinline__ long long dkey(double x) {
  long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// 1/x by Newton's iteration for the reciprocal, r <- r + r (1 - x r), from
// the hardware's FP64 reciprocal approximation: two steps take its relative
// error below FP64 rounding (a quotient a * rcp_nr(b) is within about 1.5 ulp
// of a / b) in five FP64-pipe instructions, a fraction of an IEEE division.
// Used where the quotients only feed sums and products (the secular
// function, the Loewner products, the vector components).  Magnitudes
// outside [2^-1000, 2^1000] take the exact division.
__device__ __forceinline__ double rcp_nr(double x) {
  const int ex = (__double2hiint(x) >> 20) & 0x7FF;
  if (ex < 23 || ex > 2023) return 1.0 / x;
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// x > 0 and x < 0 for finite x from its bit pattern (no FP64 instruction)
__device__ __forceinline__ bool d_pos(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool d_neg(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 && (b & 0x7fffffffffffffffLL) != 0;
}

__device__ __forceinline__ double* qin_buf(const ConeDev& c, int level) { return (level & 1) ? c.QB : c.QA; }
__device__ __forceinline__ double* qout_buf(const ConeDev& c, int level) { return (level & 1) ? c.QA : c.QB; }
__device__ __forceinline__ double* lin_buf(const ConeDev& c, int level) { return (level & 1) ? c.lamB : c.lamA; }
__device__ __forceinline__ double* lout_buf(const ConeDev& c, int level) { return (level & 1) ? c.lamA : c.lamB; }

// Leaves.  Sides n >= 3 tear only the off-diagonals e_m with m odd, so the
// leaves are the 2 x 2 blocks [[d_2i - |e_2i-1|, e_2i], [e_2i, d_2i+1 -
// |e_2i+1|]] (and a 1 x 1 block last for odd n), solved in closed form by one
// Jacobi rotation (t the smaller root of t^2 + 2 theta t - 1 = 0,
// theta = (c - a) / 2b: eigenvalues a - t b and c + t b, eigenvectors (cs,
// -sn) and (sn, cs)); they stand in for level 0's merges and feed level 1.
// Side 2 keeps the 1 x 1 leaves (its level-0 merge is the root).
__global__ void dc_leaves_kernel(const ConeDev* __restrict__ cones) {
  const ConeDev& c = cones[blockIdx.y];
  const int64_t n = c.n;
  if (n < 3) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      double di = c.d[i];
      if (i > 0) di -= fabs(c.e[i - 1]);
      if (i + 1 < n) di -= fabs(c.e[i]);
      c.lamA[i] = di;
      c.QA[i + i * n] = 1.0;
    }
    return;
  }
  double* Q = qin_buf(c, 1);
  double* lam = lin_buf(c, 1);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 2 * p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = 2 * p;
    double a = c.d[i];
    if (i > 0) a -= fabs(c.e[i - 1]);
    if (i + 1 == n) {  // the last 1 x 1 leaf of an odd side
      lam[i] = a;
      Q[i + i * n] = 1.0;
      continue;
    }
    double b = c.e[i];
    double cc = c.d[i + 1];
    if (i + 2 < n) cc -= fabs(c.e[i + 1]);
    double l1, l2, cs, sn;
    if (b == 0.0) {
      l1 = a; l2 = cc; cs = 1.0; sn = 0.0;
    } else {
      const double theta = (cc - a) / (2.0 * b);
      const double at = fabs(theta);
      const double t = at > 1e150 ? copysign(0.5 / at, theta)
                                  : copysign(1.0 / (at + sqrt(fma(theta, theta, 1.0))), theta);
      cs = 1.0 / sqrt(fma(t, t, 1.0));
      sn = t * cs;
      l1 = a - t * b;
      l2 = cc + t * b;
    }
    // columns (cs, -sn) for l1 and (sn, cs) for l2, in ascending order
    double q00 = cs, q10 = -sn, q01 = sn, q11 = cs;
    if (l1 > l2) {
      const double tl = l1; l1 = l2; l2 = tl;
      q00 = sn; q10 = cs; q01 = cs; q11 = -sn;
    }
    lam[i] = l1;
    lam[i + 1] = l2;
    Q[i + i * n] = q00;
    Q[(i + 1) + i * n] = q10;
    Q[i + (i + 1) * n] = q01;
    Q[(i + 1) + (i + 1) * n] = q11;
  }
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
  return t;
}

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = red[0];
  for (int q = 1; q < (int)(blockDim.x >> 5); ++q) t = fmax(t, red[q]);
  return t;
}

// ---------------------------------------------------------------- prepare
__global__ void __launch_bounds__(kDcThreads) dc_prepare_kernel(const ConeDev* __restrict__ cones,
                                                                const MergeNode* __restrict__ nodes) {
  const MergeNode nd = nodes[blockIdx.x];
  const ConeDev& c = cones[nd.cone];
  if (*c.status != 0) return;
  const int64_t n = c.n;
  const int s = nd.s, n1 = nd.n1, n2 = nd.n2, K = n1 + n2;
  const double* Qi = qin_buf(c, nd.level);
  const double* li = lin_buf(c, nd.level);
  const int tid = threadIdx.x;
  int* cnt = c.icnt + 4 * s;

  if (n2 == 0) {  // a lone block moves up one level unchanged
    double* Qo = qout_buf(c, nd.level);
    double* lo = lout_buf(c, nd.level);
    for (int64_t e = tid; e < (int64_t)K * K; e += kDcThreads) {
      const int r = (int)(e % K), q = (int)(e / K);
      Qo[(s + r) + (int64_t)(s + q) * n] = Qi[(s + r) + (int64_t)(s + q) * n];
    }
    for (int t = tid; t < K; t += kDcThreads) lo[s + t] = li[s + t];
    if (tid == 0) { cnt[0] = 0; cnt[1] = 0; cnt[2] = 0; }
    return;
  }

  extern __shared__ double dsm[];
  double* dv = dsm;                 // K sorted poles
  double* zv = dv + K;              // K sorted z
  int* perm = (int*)(zv + K);       // K: sorted position -> child column
  int* fp = perm + K;               // K: sorted position -> final column
  __shared__ double red[kDcThreads / 32];
  __shared__ double sh_rho;
  __shared__ int sh_kk, sh_nrot;

  const double beta = c.e[s + n1 - 1];
  const double sgn = beta >= 0.0 ? 1.0 : -1.0;
  // z in child order (stored at the sorted position below)
  // rank by a stable merge of the two sorted child lists
  for (int t = tid; t < K; t += kDcThreads) {
    double val, zval;
    int rnk;
    if (t < n1) {
      val = li[s + t];
      zval = Qi[(s + n1 - 1) + (int64_t)(s + t) * n];
      const long long kv = dkey(val);
      int lo = 0, hi = n2;  // count of child-2 values < val
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (dkey(li[s + n1 + mid]) < kv) lo = mid + 1; else hi = mid;
      }
      rnk = t + lo;
    } else {
      const int u = t - n1;
      val = li[s + t];
      zval = sgn * Qi[(s + n1) + (int64_t)(s + t) * n];
      const long long kv = dkey(val);
      int lo = 0, hi = n1;  // count of child-1 values <= val
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (dkey(li[s + mid]) <= kv) lo = mid + 1; else hi = mid;
      }
      rnk = u + lo;
    }
    dv[rnk] = val;
    zv[rnk] = zval;
    perm[rnk] = t;
  }
  __syncthreads();
  double ss = 0.0, dm = 0.0;
  for (int t = tid; t < K; t += kDcThreads) {
    ss = fma(zv[t], zv[t], ss);
    dm = fmax(dm, fabs(dv[t]));
  }
  const double nrm2 = block_sum(ss, red);
  const double dmax = block_max(dm, red);
  const double inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
  for (int t = tid; t < K; t += kDcThreads) zv[t] *= inv;
  __syncthreads();

  // ---- deflation scan.  Sequential by nature (a rotation changes the pole
  // and z of the survivor, which the next test reads), but almost every
  // test is negative: warp 0 takes 32 positions at a time, evaluates their
  // tests against the current predecessors in parallel and walks a chunk
  // one position at a time only from its first positive test on.
  // Close-pole test |gap c s| <= tol with c = z_j / t, s = z_p / t,
  // t = hypot(z_j, z_p), written without the division: |gap z_j z_p| <= tol t^2.
  double* rot = c.rot + 2 * s;
  int* irot = c.irot + 2 * s;
  const double rho = fabs(beta) * nrm2;
  const double tol = 8.0 * kEps * fmax(dmax, rho);
  if (tid < 32) {
    const int lane = tid;
    int last = -1, nrot = 0;
    for (int base = 0; base < K; base += 32) {
      const int j = base + lane;
      const bool keep = j < K && !(rho * fabs(zv[j]) <= tol);
      const unsigned km = __ballot_sync(0xffffffffu, keep);
      const unsigned below = km & ((1u << lane) - 1u);
      const int p = below ? base + 31 - __clz(below) : last;
      bool trig = false;
      if (keep && p >= 0) {
        const double zp = zv[p], zj = zv[j];
        trig = fabs((dv[j] - dv[p]) * zj * zp) <= tol * fma(zj, zj, zp * zp);
      }
      const unsigned tm = __ballot_sync(0xffffffffu, trig);
      if (tm == 0u) {
        if (j < K) fp[j] = keep ? 1 : 0;
        if (km) last = base + 31 - __clz(km);
        continue;
      }
      const int first = __ffs(tm) - 1;
      if (j < K && lane < first) fp[j] = keep ? 1 : 0;
      const unsigned pre = km & ((1u << first) - 1u);
      if (pre) last = base + 31 - __clz(pre);
      __syncwarp();
      if (lane == 0) {
        const int jend = min(K, base + 32);
        for (int jj = base + first; jj < jend; ++jj) {
          if (rho * fabs(zv[jj]) <= tol) { fp[jj] = 0; continue; }
          if (last >= 0) {
            const double sp = zv[last], cj = zv[jj];
            const double gap = dv[jj] - dv[last];
            const double t2 = fma(cj, cj, sp * sp);
            if (fabs(gap * cj * sp) <= tol * t2) {
              const double tt = sqrt(t2);
              const double cc = cj / tt, sn = sp / tt;
              const double dp = dv[last], dj = dv[jj];
              dv[last] = dp * cc * cc + dj * sn * sn;
              dv[jj] = dp * sn * sn + dj * cc * cc;
              zv[jj] = tt;
              zv[last] = 0.0;
              fp[last] = 0;
              rot[2 * nrot] = cc;
              rot[2 * nrot + 1] = sn;
              irot[2 * nrot] = last;  // sorted indices for now
              irot[2 * nrot + 1] = jj;
              ++nrot;
            }
          }
          fp[jj] = 1;
          last = jj;
        }
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      nrot = __shfl_sync(0xffffffffu, nrot, 0);
      __syncwarp();
    }
    if (lane == 0) {
      sh_rho = rho;
      sh_nrot = nrot;
    }
  }
  __syncthreads();
  // final columns: kept first, deflated after, each in sorted order (block scan of the flags)
  {
    __shared__ int wsum[kDcThreads / 32];
    __shared__ int sh_total;
    const int per = (K + kDcThreads - 1) / kDcThreads;
    const int a0 = min(K, tid * per), a1 = min(K, a0 + per);
    int mine = 0;
    for (int j = a0; j < a1; ++j) mine += fp[j];
    const int lane = tid & 31, wid = tid >> 5;
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (tid == 0) {
      int run = 0;
      for (int q = 0; q < kDcThreads / 32; ++q) { const int v = wsum[q]; wsum[q] = run; run += v; }
      sh_total = run;
    }
    __syncthreads();
    const int kkept = sh_total;
    int kb = wsum[wid] + incl - mine;  // kept positions before mine
    for (int j = a0; j < a1; ++j) {
      if (fp[j]) fp[j] = kb++;
      else fp[j] = kkept + (j - kb);  // deflated: after all kept, in order
    }
    if (tid == 0) sh_kk = kkept;
  }
  __syncthreads();
  for (int r = tid; r < sh_nrot; r += kDcThreads) {
    irot[2 * r] = fp[irot[2 * r]];
    irot[2 * r + 1] = fp[irot[2 * r + 1]];
  }
  __syncthreads();
  const int kk = sh_kk;
  for (int j = tid; j < K; j += kDcThreads) {
    const int f = fp[j];
    if (f < kk) {
      c.dsrt[s + f] = dv[j];
      c.zk[s + f] = zv[j];
    } else {
      c.dval[s + f - kk] = dv[j];
    }
    c.iperm[s + j] = perm[j];
    c.ifp[s + j] = f;
  }
  if (tid == 0) {
    c.rho[s] = sh_rho;
    cnt[0] = kk;
    cnt[1] = K - kk;
    cnt[2] = sh_nrot;
  }
  if (K <= kDcFuseK) {
    // a small merge also builds its permuted block and applies the deflation's
    // rotations here (the separate kernels skip it; two launches fewer per level)
    __syncthreads();
    const double* Qsrc = qin_buf(c, nd.level);
    double* Qb = c.Qin;
    for (int e = tid; e < K * K; e += kDcThreads) {
      const int j = e / K, r = e - j * K;
      const int src = perm[j], dst = fp[j];
      const bool same = (src < n1) == (r < n1);
      Qb[(s + r) + (int64_t)(s + dst) * n] = same ? Qsrc[(s + r) + (int64_t)(s + src) * n] : 0.0;
    }
    __syncthreads();
    const int nr = sh_nrot;
    for (int r = tid; r < K && nr > 0; r += kDcThreads) {
      double* row = Qb + (s + r) + (int64_t)s * n;
      for (int q = 0; q < nr; ++q) {
        const int a = irot[2 * q], bcol = irot[2 * q + 1];
        const double cc = rot[2 * q], sn = rot[2 * q + 1];
        double* pa = row + (int64_t)a * n;
        double* pb = row + (int64_t)bcol * n;
        const double x = *pa, y = *pb;
        *pa = cc * x - sn * y;
        *pb = sn * x + cc * y;
      }
    }
  }
}

// Permuted eigenvector block Qin(:, fp[j]) = Q(:, perm[j]) of each merge node;
// the source is block diagonal (child 1 rows x child 1 columns, child 2 rows x
// child 2 columns).  blockIdx.x = node, blockIdx.y = chunk of kQinCols columns
// (few columns per CTA: the copy is bound by load latency, not bandwidth).
__global__ void dc_build_qin_kernel(const ConeDev* __restrict__ cones, const MergeNode* __restrict__ nodes) {
  const MergeNode nd = nodes[blockIdx.x];
  if (nd.n2 == 0) return;
  const ConeDev& c = cones[nd.cone];
  if (*c.status != 0) return;
  const int64_t n = c.n;
  const int s = nd.s, n1 = nd.n1, K = nd.n1 + nd.n2;
  if (K <= kDcFuseK) return;  // built by dc_prepare_kernel
  const int j0 = blockIdx.y * kQinCols;
  if (j0 >= K) return;
  const double* Qi = qin_buf(c, nd.level);
  double* Qb = c.Qin;
  const int jend = min(K, j0 + kQinCols);
  for (int j = j0; j < jend; ++j) {
    const int src = c.iperm[s + j];
    const int dst = c.ifp[s + j];
    const bool first = src < n1;
    for (int r = threadIdx.x; r < K; r += blockDim.x) {
      const bool same = first == (r < n1);
      Qb[(s + r) + (int64_t)(s + dst) * n] = same ? Qi[(s + r) + (int64_t)(s + src) * n] : 0.0;
    }
  }
}

// Givens rotations of the deflation, in order; one thread per row.
__global__ void dc_apply_rot_kernel(const ConeDev* __restrict__ cones, const MergeNode* __restrict__ nodes,
                                    const int* __restrict__ pos_node, int64_t total) {
  const int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gp >= total) return;
  const int ni = pos_node[total + gp];
  if (ni < 0) return;
  const MergeNode nd = nodes[ni];
  if (nd.n2 == 0) return;
  const ConeDev& c = cones[nd.cone];
  if (*c.status != 0) return;
  const int s = nd.s;
  if (nd.n1 + nd.n2 <= kDcFuseK) return;  // applied by dc_prepare_kernel
  const int nrot = c.icnt[4 * s + 2];
  if (nrot == 0) return;
  const int r = pos_node[gp];
  const int64_t n = c.n;
  const double* rot = c.rot + 2 * s;
  const int* irot = c.irot + 2 * s;
  double* row = c.Qin + (s + r) + (int64_t)s * n;
  for (int q = 0; q < nrot; ++q) {
    const int a = irot[2 * q], bcol = irot[2 * q + 1];
    const double cc = rot[2 * q], sn = rot[2 * q + 1];
    double* pa = row + (int64_t)a * n;
    double* pb = row + (int64_t)bcol * n;
    const double x = *pa, y = *pb;
    *pa = cc * x - sn * y;
    *pb = sn * x + cc * y;
  }
}

// ---------------------------------------------------------------- secular
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_prod_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP64 -> FP32, round to nearest even, by integer operations (a conversion
// instruction would occupy the FP64 pipe); |v| < 2^-126 gives 0.
__device__ __forceinline__ float f64_to_f32_rn(double v) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7FF) - 896;
  if (e <= 0) return 0.0f;
  if (e >= 255) return __uint_as_float((hi & 0x80000000u) | 0x7f800000u);
  uint32_t bits = ((uint32_t)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1FFFFFFFu, half = 0x10000000u;
  if (rest > half || (rest == half && (bits & 1u))) ++bits;
  return __uint_as_float((hi & 0x80000000u) | bits);
}

// Root i of f(x) = 1 + rho sum_j z_j^2 / (d_j - x), d strictly increasing,
// ||z|| = 1, solved by one warp (the sums are split over the lanes; every
// lane ends with the same values).  Returns the origin pole and the offset
// tau = x - d_org; false if the iteration cap was reached.
__device__ bool secular_root_warp(const double* __restrict__ dk, const double* __restrict__ zk, int K, double rho,
                                  int i, int lane, float* dif, double* difd, int* org_out, double* tau_out) {
  int org;
  double lo, hi;
  if (i < K - 1) {
    const double di = dk[i];
    const double mid = 0.5 * (dk[i + 1] - di);
    // f at the midpoint decides the origin pole.  First in FP32 from the FP64
    // pole differences: |d_j - d_i - mid| >= mid for every j, so each term is
    // within a few FP32 roundings, and the sign is taken when |f| clears that
    // bound; otherwise in FP64.
    const float mid32 = f64_to_f32_rn(mid), rho32 = f64_to_f32_rn(rho);
    float f32 = 0.0f, a32 = 0.0f;
    for (int j = lane; j < K; j += 32) {
      const float zz = f64_to_f32_rn(zk[j]);
      const float term = zz * __fdividef(zz, f64_to_f32_rn(dk[j] - di) - mid32);
      f32 += term;
      a32 += fabsf(term);
    }
    f32 = 1.0f + rho32 * warp_sum_f(f32);
    a32 = warp_sum_f(a32);
    const float bound32 = (2.0f * (float)K + 32.0f) * 5.9604645e-8f * (1.0f + rho32 * a32);
    bool right;  // f(mid) >= 0: the root lies left of the midpoint
    if (fabsf(f32) > bound32 && isfinite(f32)) {
      right = f32 >= 0.0f;
    } else {
      double f = 0.0;
      for (int j = lane; j < K; j += 32) f += zk[j] * zk[j] * rcp_nr((dk[j] - di) - mid);
      f = 1.0 + rho * warp_sum_d(f);
      right = f >= 0.0;
    }
    if (right) { org = i; lo = 0.0; hi = mid; }
    else { org = i + 1; lo = -mid; hi = 0.0; }
  } else {
    org = i;
    lo = 0.0;
    hi = rho;
  }
  const double dorg = dk[org];
  double tau = 0.5 * (lo + hi);
  const int li = i, ri = i + 1;
  bool conv = false;
  // ---- FP32 phase: the same bracketed rational iteration with the sums in
  // FP32 (64x the FP64 rate on this part), while the sign of f is certain
  // beyond its FP32 error bound; the FP64 loop below then polishes from the
  // narrowed bracket.  Only the differences d_j - d_org are formed in FP64.
  {
    // d_j - d_org, formed in FP64 once per root (difd: this warp's 2K
    // doubles, the differences then z_j^2) and rounded to FP32 (dif: K floats)
    if (dif)
      for (int j = lane; j < K; j += 32) {
        const double dd = dk[j] - dorg;
        difd[j] = dd;
        dif[j] = f64_to_f32_rn(dd);
        const double zj = zk[j];
        difd[K + j] = zj * zj;
      }
    __syncwarp();
    const float rho32 = f64_to_f32_rn(rho);
    const float p32 = f64_to_f32_rn(dk[li] - dorg);
    const float q32 = ri < K ? f64_to_f32_rn(dk[ri] - dorg) : 0.0f;
    for (int it = 0; it < 40; ++it) {
      const float t32 = f64_to_f32_rn(tau);
      float psi = 0.0f, phi = 0.0f, dpsi = 0.0f, dphi = 0.0f, aerr = 0.0f;
      for (int j = lane; j < K; j += 32) {
        const float del = (dif ? dif[j] : f64_to_f32_rn(dk[j] - dorg)) - t32;
        const float zz = f64_to_f32_rn(zk[j]);
        const float t = __fdividef(zz, del);  // within 2 ulp: inside the bound below
        const float term = zz * t;
        if (j < ri) { psi += term; dpsi = fmaf(t, t, dpsi); }
        else { phi += term; dphi = fmaf(t, t, dphi); }
        aerr += fabsf(term);
      }
      psi = rho32 * warp_sum_f(psi);
      phi = rho32 * warp_sum_f(phi);
      dpsi = rho32 * warp_sum_f(dpsi);
      dphi = rho32 * warp_sum_f(dphi);
      aerr = warp_sum_f(aerr);
      const float g = 1.0f + psi + phi;
      // rounding of the K terms and of their sums: (2K + 16) 2^-24 (1 + rho sum |term|)
      const float bound = (2.0f * (float)K + 16.0f) * 5.9604645e-8f * (1.0f + rho32 * aerr);
      if (!(fabsf(g) > bound) || !isfinite(dpsi + dphi)) break;
      if (g > 0.0f) hi = tau; else lo = tau;
      if (hi - lo <= 4.0 * kEps * fmax(fabs(lo), fabs(hi))) break;
      // two-pole model psi(x) ~ a + sl / (p - x) matching psi and psi' at tau:
      // sl = psi' dl^2, a = psi - sl / dl = psi - psi' dl
      const float dl = p32 - t32;
      const float sl = dpsi * dl * dl;
      const float a = fmaf(-dpsi, dl, psi);
      float x = 0.0f;
      bool okx = false;
      if (ri < K) {
        const float dr = q32 - t32;
        const float sr = dphi * dr * dr;
        const float bq = fmaf(-dphi, dr, phi);
        const float C = 1.0f + a + bq;
        const float B2 = -(C * (p32 + q32) + sl + sr);
        const float C2 = C * p32 * q32 + sl * q32 + sr * p32;
        if (C != 0.0f) {
          const float disc = B2 * B2 - 4.0f * C * C2;
          if (disc >= 0.0f) {
            const float qq = -0.5f * (B2 + copysignf(sqrtf(disc), B2));
            const double x1 = (double)(qq / C);
            if (x1 > lo && x1 < hi) { x = qq / C; okx = true; }
            else if (qq != 0.0f) {
              const double x2 = (double)(C2 / qq);
              if (x2 > lo && x2 < hi) { x = C2 / qq; okx = true; }
            }
          }
        }
      } else {
        const float C = 1.0f + a;
        if (C > 0.0f) {
          const double x1 = (double)(p32 + sl / C);
          if (x1 > lo && x1 < hi) { x = p32 + sl / C; okx = true; }
        }
      }
      tau = okx ? (double)x : 0.5 * (lo + hi);
    }
  }
  const double p = dk[li] - dorg;
  const double q = ri < K ? dk[ri] - dorg : 0.0;
  for (int it = 0; it < 100; ++it) {
    double psi = 0.0, phi = 0.0, dpsi = 0.0, dphi = 0.0;
    for (int j = lane; j < K; j += 32) {
      const double del = (dif ? difd[j] : dk[j] - dorg) - tau;
      const double r = rcp_nr(del);
      double zz2;
      if (dif) {
        zz2 = difd[K + j];
      } else {
        const double zj = zk[j];
        zz2 = zj * zj;
      }
      const double term = zz2 * r;  // z_j^2 / del; its derivative term z_j^2 / del^2 = term r
      if (j < ri) { psi += term; dpsi = fma(term, r, dpsi); }
      else { phi += term; dphi = fma(term, r, dphi); }
    }
    psi = warp_sum_d(psi);
    phi = warp_sum_d(phi);
    // sum |term|: d_j - lambda is formed exactly enough to carry its sign (the
    // pole differences in FP64, tau inside the bracket), so the terms left of
    // the root (j < ri) are negative and the others positive
    const double aerr = phi - psi;
    psi *= rho;
    phi *= rho;
    dpsi = rho * warp_sum_d(dpsi);
    dphi = rho * warp_sum_d(dphi);
    const double g = 1.0 + psi + phi;
    if (fabs(g) <= 8.0 * kEps * K * (1.0 + rho * aerr)) { conv = true; break; }
    if (g > 0.0) hi = tau; else lo = tau;
    if (hi - lo <= 4.0 * kEps * fmax(fabs(lo), fabs(hi))) { conv = true; break; }
    const double dl = p - tau;
    const double sl = dpsi * dl * dl;
    const double a = fma(-dpsi, dl, psi);  // psi - sl / dl
    double x = 0.0;
    bool okx = false;
    if (ri < K) {
      const double dr = q - tau;
      const double sr = dphi * dr * dr;
      const double bq = fma(-dphi, dr, phi);  // phi - sr / dr
      const double C = 1.0 + a + bq;
      const double A2 = C;
      const double B2 = -(C * (p + q) + sl + sr);
      const double C2 = C * p * q + sl * q + sr * p;
      if (A2 != 0.0) {
        const double disc = B2 * B2 - 4.0 * A2 * C2;
        if (disc >= 0.0) {
          const double sq = sqrt(disc);
          const double qq = -0.5 * (B2 + copysign(sq, B2));
          const double x1 = qq / A2;
          if (x1 > lo && x1 < hi) { x = x1; okx = true; }
          else if (qq != 0.0) {
            const double x2 = C2 / qq;
            if (x2 > lo && x2 < hi) { x = x2; okx = true; }
          }
        }
      } else if (B2 != 0.0) {
        const double x1 = -C2 / B2;
        if (x1 > lo && x1 < hi) { x = x1; okx = true; }
      }
    } else {
      const double C = 1.0 + a;
      if (C > 0.0) {
        const double x1 = p + sl / C;
        if (x1 > lo && x1 < hi) { x = x1; okx = true; }
      }
    }
    if (!okx) x = 0.5 * (lo + hi);
    tau = x;
  }
  *org_out = org;
  *tau_out = tau;
  return conv;
}

// Warp-per-position kernels: warp w handles position w of the level's
// position map (a root index or a pole index within its node).
struct WarpPos {
  MergeNode nd;
  int idx;
  bool ok;
};

__device__ __forceinline__ WarpPos warp_pos(const MergeNode* nodes, const int* pos_node, int64_t total) {
  WarpPos w;
  w.ok = false;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= total) return w;
  const int ni = pos_node[total + gw];
  if (ni < 0) return w;
  w.nd = nodes[ni];
  if (w.nd.n2 == 0) return w;
  w.idx = pos_node[gw];
  w.ok = true;
  return w;
}

__global__ void dc_secular_kernel(const ConeDev* __restrict__ cones, const MergeNode* __restrict__ nodes,
                                  const int* __restrict__ pos_node, int64_t total, int difmax) {
  const WarpPos w = warp_pos(nodes, pos_node, total);
  if (!w.ok) return;
  const ConeDev& c = cones[w.nd.cone];
  if (*c.status != 0) return;
  const int s = w.nd.s, i = w.idx;
  const int kk = c.icnt[4 * s];
  if (i >= kk) return;
  const int lane = threadIdx.x & 31;
  // per warp: 2 difmax doubles (pole differences, z^2), then (after the four
  // warps' doubles) difmax floats
  extern __shared__ double sec_difd[];
  const int wq = threadIdx.x >> 5;
  double* difd = difmax >= kk ? sec_difd + 2 * wq * difmax : nullptr;
  float* dif = difmax >= kk ? reinterpret_cast<float*>(sec_difd + 8 * difmax) + wq * difmax : nullptr;
  int org;
  double tau;
  const bool ok = secular_root_warp(c.dsrt + s, c.zk + s, kk, c.rho[s], i, lane, dif, difd, &org, &tau);
  if (lane == 0) {
    c.iorg[s + i] = org;
    c.tau[s + i] = tau;
    if (!ok) atomicOr(c.status, ST_NOCONV);
  }
}

// lambda_i - d_j, accurate: (d_org(i) - d_j) + tau_i
__device__ __forceinline__ double lam_minus_d(const double* dk, const int* org, const double* tau, int i, int j) {
  return (dk[org[i]] - dk[j]) + tau[i];
}

// Loewner (Gu-Eisenstat) z: zhat_j^2 = prod_i (lambda_i - d_j) / (rho prod_{i != j} (d_i - d_j)),
// evaluated as a product of ratios that are all in (0, 1].
__global__ void dc_loewner_kernel(const ConeDev* __restrict__ cones, const MergeNode* __restrict__ nodes,
                                  const int* __restrict__ pos_node, int64_t total) {
  const WarpPos w = warp_pos(nodes, pos_node, total);
  if (!w.ok) return;
  const ConeDev& c = cones[w.nd.cone];
  if (*c.status != 0) return;
  const int s = w.nd.s, j = w.idx;
  const int kk = c.icnt[4 * s];
  if (j >= kk) return;
  const int lane = threadIdx.x & 31;
  const double* dk = c.dsrt + s;
  const int* org = c.iorg + s;
  const double* tau = c.tau + s;
  const double dj = dk[j];
  double prod = 1.0;
  for (int i = lane; i < kk; i += 32) {
    if (i < j) prod *= lam_minus_d(dk, org, tau, i, j) * rcp_nr(dk[i] - dj);
    else if (i > j) prod *= lam_minus_d(dk, org, tau, i - 1, j) * rcp_nr(dk[i] - dj);
  }
  prod = warp_prod_d(prod) * (lam_minus_d(dk, org, tau, kk - 1, j) / c.rho[s]);
  if (lane == 0) c.zhat[s + j] = copysign(sqrt(fabs(prod)), c.zk[s + j]);
}

// ---------------------------------------------------------------- select
__global__ void __launch_bounds__(kDcThreads) dc_select_kernel(const ConeDev* __restrict__ cones,
                                                               const MergeNode* __restrict__ nodes) {
  const MergeNode nd = nodes[blockIdx.x];
  if (nd.n2 == 0) return;
  const ConeDev& c = cones[nd.cone];
  if (*c.status != 0) return;
  const int s = nd.s, K = nd.n1 + nd.n2;
  const int* cnt = c.icnt + 4 * s;
  const int kk = cnt[0], ndf = cnt[1];
  extern __shared__ double dsm[];
  double* lam = dsm;               // kk roots (increasing)
  double* dfs = lam + K;           // ndf deflated values, sorted
  int* dord = (int*)(dfs + K);     // sorted rank -> deflated index
  const int tid = threadIdx.x;
  const double* dk = c.dsrt + s;
  for (int i = tid; i < kk; i += kDcThreads) lam[i] = dk[c.iorg[s + i]] + c.tau[s + i];
  // rank the deflated values (they may be slightly out of order after rotations)
  for (int q = tid; q < ndf; q += kDcThreads) {
    const double v = c.dval[s + q];
    const long long kv = dkey(v);
    int r = 0;
    for (int u = 0; u < ndf; ++u) {
      const long long ku = dkey(c.dval[s + u]);
      r += (ku < kv) || (ku == kv && u < q);
    }
    dfs[r] = v;
    dord[r] = q;
  }
  __syncthreads();
  if (!nd.root) {
    double* lo = lout_buf(c, nd.level);
    int* imap = c.imap + s;
    for (int i = tid; i < kk; i += kDcThreads) {
      const long long kv = dkey(lam[i]);
      int a = 0, b = ndf;  // deflated < lam_i
      while (a < b) { const int m = (a + b) >> 1; if (dkey(dfs[m]) < kv) a = m + 1; else b = m; }
      const int pos = i + a;
      lo[s + pos] = lam[i];
      imap[i] = s + pos;
    }
    for (int r = tid; r < ndf; r += kDcThreads) {
      const long long kv = dkey(dfs[r]);
      int a = 0, b = kk;  // roots <= value
      while (a < b) { const int m = (a + b) >> 1; if (dkey(lam[m]) <= kv) a = m + 1; else b = m; }
      const int pos = r + a;
      lo[s + pos] = dfs[r];
      imap[kk + dord[r]] = s + pos;  // deflated column kk + q -> output column
    }
    return;
  }
  // ---- cone's final merge: choose the side and the kept eigenpairs.  Signs
  // are read from the bit patterns (integer operations: a comparison of
  // doubles would occupy the FP64 pipe), and every scan is spread over the CTA.
  __shared__ int sh_pos, sh_neg, sh_lo, sh_hi, sh_wsum[kDcThreads / 32], sh_kd;
  if (tid == 0) { sh_pos = 0; sh_neg = 0; sh_lo = kk; sh_hi = 0; }
  __syncthreads();
  int np = 0, nn = 0;
  for (int i = tid; i < kk; i += kDcThreads) { np += d_pos(lam[i]); nn += d_neg(lam[i]); }
  for (int r = tid; r < ndf; r += kDcThreads) { np += d_pos(dfs[r]); nn += d_neg(dfs[r]); }
  atomicAdd(&sh_pos, np);
  atomicAdd(&sh_neg, nn);
  __syncthreads();
  const int allv = c.kinfo[3];
  int route;
  const int side = c.kinfo[4];
  if (side == 1) route = 0;
  else if (side == 2) route = 1;
  else route = (sh_pos <= sh_neg) ? 0 : 1;
  // kept roots form a contiguous range [r_lo, r_hi) of the increasing roots
  if (!allv) {
    if (route == 0) {
      for (int i = tid; i < kk; i += kDcThreads)
        if (d_pos(lam[i])) { atomicMin(&sh_lo, i); break; }
    } else {
      for (int i = tid; i < kk; i += kDcThreads)
        if (d_neg(lam[i])) atomicMax(&sh_hi, i + 1);
    }
  }
  __syncthreads();
  const int r_lo = (allv || route == 1) ? 0 : sh_lo;
  const int r_hi = (allv || route == 0) ? kk : sh_hi;
  const int kr = r_hi - r_lo;
  // roots -> Z columns 0..kr-1; kept deflated -> Z columns kr.., in sorted order
  int* imap = c.imap + s;
  for (int i = tid; i < kk; i += kDcThreads) {
    const bool keep = i >= r_lo && i < r_hi;
    imap[i] = keep ? (i - r_lo) : -1;
    if (keep) c.lamk[i - r_lo] = lam[i];
  }
  {
    // exclusive scan of the keep flags over contiguous chunks of the sorted deflated values
    const int per = (ndf + kDcThreads - 1) / kDcThreads;
    const int a0 = min(ndf, tid * per), a1 = min(ndf, a0 + per);
    int mine = 0;
    for (int r = a0; r < a1; ++r) mine += allv || (route == 0 ? d_pos(dfs[r]) : d_neg(dfs[r]));
    const int lane = tid & 31, wid = tid >> 5;
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) sh_wsum[wid] = incl;
    __syncthreads();
    if (tid == 0) {
      int run = 0;
      for (int q = 0; q < kDcThreads / 32; ++q) { const int v = sh_wsum[q]; sh_wsum[q] = run; run += v; }
      sh_kd = run;
    }
    __syncthreads();
    int kb = sh_wsum[wid] + incl - mine;
    for (int r = a0; r < a1; ++r) {
      const double v = dfs[r];
      const bool keep = allv || (route == 0 ? d_pos(v) : d_neg(v));
      if (keep) {
        imap[kk + dord[r]] = kr + kb;
        c.lamk[kr + kb] = v;
        ++kb;
      } else {
        imap[kk + dord[r]] = -1;
      }
    }
  }
  if (tid == 0) {
    c.kinfo[0] = kr + sh_kd;
    c.kinfo[1] = route;
    c.kinfo[2] = kr;
    c.kinfo[5] = r_lo;
    c.kinfo[8] = sh_pos;
    c.kinfo[9] = sh_neg;
  }
}

// ---------------------------------------------------------------- vectors
// U(row, j) = zhat_j / (d_j - lambda_i) / ||.||: one warp per root i forms
// the components (lanes over j) and their norm, then rescales its own stores.
__global__ void dc_vectors_kernel(const ConeDev* __restrict__ cones, const MergeNode* __restrict__ nodes,
                                  const int* __restrict__ pos_node, int64_t total) {
  const WarpPos w = warp_pos(nodes, pos_node, total);
  if (!w.ok) return;
  const ConeDev& c = cones[w.nd.cone];
  if (*c.status != 0) return;
  const int s = w.nd.s, i = w.idx;
  const int kk = c.icnt[4 * s];
  if (i >= kk) return;
  int row = i;
  if (w.nd.root) {
    row = c.imap[s + i];
    if (row < 0) return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t n = c.n;
  const double* dk = c.dsrt + s;
  const double* zh = c.zhat + s;
  const double dorg = dk[c.iorg[s + i]];
  const double tau = c.tau[s + i];
  double* U = c.Ucm + s + row + (int64_t)s * n;  // U[j * n] = component j
  double nrm = 0.0;
  for (int j = lane; j < kk; j += 32) {
    const double u = zh[j] * rcp_nr((dk[j] - dorg) - tau);
    U[(int64_t)j * n] = u;
    nrm = fma(u, u, nrm);
  }
  const double inv = 1.0 / sqrt(warp_sum_d(nrm));
  for (int j = lane; j < kk; j += 32) U[(int64_t)j * n] *= inv;
}

// deflated columns: Qin(:, kk + q) -> output column; blockIdx.x = node,
// blockIdx.y = chunk of 8 deflated columns.
__global__ void dc_copy_deflated_kernel(const ConeDev* __restrict__ cones, const MergeNode* __restrict__ nodes) {
  const MergeNode nd = nodes[blockIdx.x];
  if (nd.n2 == 0) return;
  const ConeDev& c = cones[nd.cone];
  if (*c.status != 0) return;
  const int s = nd.s, K = nd.n1 + nd.n2;
  const int kk = c.icnt[4 * s], ndf = c.icnt[4 * s + 1];
  const int q0 = blockIdx.y * 8;
  if (q0 >= ndf) return;
  const int64_t n = c.n;
  double* out = nd.root ? c.Z : qout_buf(c, nd.level);
  const int64_t roff = nd.root ? 0 : s;
  const int qend = min(ndf, q0 + 8);
  for (int q = q0; q < qend; ++q) {
    const int col = c.imap[s + kk + q];
    if (col < 0) continue;
    const double* src = c.Qin + s + (int64_t)(s + kk + q) * n;
    double* dst = out + roff + (int64_t)col * n;
    for (int r = threadIdx.x; r < K; r += blockDim.x) dst[r] = src[r];
  }
}

}  // namespace

void launch_dc_leaves(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)((maxn + 255) / 256);
  if (gx > 64) gx = 64;
  dc_leaves_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones);
}

void launch_dc_prepare(const ConeDev* cones, const MergeNode* nodes, int nnodes, int maxK, cudaStream_t s) {
  if (nnodes <= 0) return;
  const size_t smem = (size_t)maxK * (2 * sizeof(double) + 2 * sizeof(int));
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(dc_prepare_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(dc_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  }
  dc_prepare_kernel<<<nnodes, kDcThreads, smem, s>>>(cones, nodes);
}

void launch_dc_secular(const ConeDev* cones, const MergeNode* nodes, const int* pos_node, int64_t total, int maxK,
                       cudaStream_t s) {
  if (total <= 0) return;
  // four warps per CTA, each with maxK doubles and maxK floats of shared
  // memory (none when that would not fit)
  constexpr size_t kSecSmemMax = 160 * 1024;
  static std::atomic<unsigned long long> attr{0};
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(dc_secular_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSecSmemMax);
  }
  const size_t smem = (size_t)4 * maxK * (2 * sizeof(double) + sizeof(float));
  const int difmax = smem <= kSecSmemMax ? maxK : 0;
  dc_secular_kernel<<<(unsigned)((total * 32 + 127) / 128), 128, difmax ? smem : 0, s>>>(cones, nodes, pos_node,
                                                                                         total, difmax);
}

void launch_dc_loewner(const ConeDev* cones, const MergeNode* nodes, const int* pos_node, int64_t total,
                       cudaStream_t s) {
  if (total <= 0) return;
  dc_loewner_kernel<<<(unsigned)((total * 32 + 127) / 128), 128, 0, s>>>(cones, nodes, pos_node, total);
}

void launch_dc_build_qin(const ConeDev* cones, const MergeNode* nodes, int nnodes, int maxK, cudaStream_t s) {
  if (nnodes <= 0) return;
  dc_build_qin_kernel<<<dim3(nnodes, (maxK + kQinCols - 1) / kQinCols), 256, 0, s>>>(cones, nodes);
}

void launch_dc_apply_rot(const ConeDev* cones, const MergeNode* nodes, const int* pos_node, int64_t total,
                         cudaStream_t s) {
  if (total <= 0) return;
  dc_apply_rot_kernel<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(cones, nodes, pos_node, total);
}

void launch_dc_select(const ConeDev* cones, const MergeNode* nodes, int nnodes, int maxK, cudaStream_t s) {
  if (nnodes <= 0) return;
  const size_t smem = (size_t)maxK * (2 * sizeof(double) + sizeof(int));
  dc_select_kernel<<<nnodes, kDcThreads, smem, s>>>(cones, nodes);
}

void launch_dc_vectors(const ConeDev* cones, const MergeNode* nodes, const int* pos_node, int64_t total, int maxK,
                       cudaStream_t s) {
  (void)maxK;
  if (total <= 0) return;
  dc_vectors_kernel<<<(unsigned)((total * 32 + 127) / 128), 128, 0, s>>>(cones, nodes, pos_node, total);
}

void launch_dc_copy_deflated(const ConeDev* cones, const MergeNode* nodes, int nnodes, int maxK, cudaStream_t s) {
  if (nnodes <= 0) return;
  dc_copy_deflated_kernel<<<dim3(nnodes, (maxK + 7) / 8), 256, 0, s>>>(cones, nodes);
}

}  // namespace scs
