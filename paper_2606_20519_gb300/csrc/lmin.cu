// Positivity post-processing of the paper's instrument and process steps
// (App. C: mixing the outcome blocks of one input with white noise; App. D:
// mixing a process matrix with the trivial process).  Both need only the
// smallest eigenvalue of each block and then a convex combination with a
// multiple of the identity:
//   lambda_a = lambda_min(C_a);  p = 1 if min_a lambda_a >= 0, else
//   p = min over lambda_a < eps of (nu - eps) / (nu - lambda_a);
//   C~_a = p C_a + (1 - p) nu 1.
// lambda_min comes from the tridiagonal form the projection's reduction
// already produces (one-stage or two-stage), by multisection on Sturm counts:
// a warp tests 32 points of the current interval at once, so each round
// narrows it 33-fold and eleven rounds reach FP64 resolution.
#include <float.h>
#include <math.h>

#include "internal.cuh"

namespace scs {

namespace {

__device__ __forceinline__ int64_t lcol(int64_t n, int64_t j) { return j * n - (j * (j - 1)) / 2; }

// Number of eigenvalues of the tridiagonal (d, e) below x (Sturm sequence of
// the LDL^T factorization of T - x I; tiny pivots replaced by -pivmin).
__device__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e, int n, double x,
                           double pivmin) {
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int cnt = q < 0.0 ? 1 : 0;
  for (int i = 1; i < n; ++i) {
    const double ei = e[i - 1];
    q = (d[i] - x) - ei * ei / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0 ? 1 : 0;
  }
  return cnt;
}

// One warp per cone: lambda_min of its tridiagonal form into io->lam[cidx].
__global__ void lmin_kernel(const ConeDev* __restrict__ cones, const IoSlot* __restrict__ io) {
  const ConeDev& c = cones[blockIdx.x];
  const int lane = threadIdx.x;
  const int n = (int)c.n;
  if (*c.status) {
    if (lane == 0) io->lam[c.cidx] = nan("");
    return;
  }
  const double* __restrict__ d = c.d;
  const double* __restrict__ e = c.e;
  // Gershgorin interval and the largest squared off-diagonal
  double lo = DBL_MAX, hi = -DBL_MAX, emax = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double el = i > 0 ? fabs(e[i - 1]) : 0.0, er = i + 1 < n ? fabs(e[i]) : 0.0;
    lo = fmin(lo, d[i] - el - er);
    hi = fmax(hi, d[i] + el + er);
    emax = fmax(emax, er * er);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
  const double pivmin = DBL_MIN * fmax(1.0, emax);
  // absolute resolution eps ||T|| (what the Sturm count resolves anyway);
  // widen slightly so that the interval surely brackets the spectrum
  const double tnorm = fmax(fabs(lo), fabs(hi));
  const double tol = 2.0 * DBL_EPSILON * tnorm + pivmin;
  lo -= tol;
  hi += tol;
  for (int round = 0; round < 64; ++round) {
    if (hi - lo <= tol) break;
    const double w = (hi - lo) / 33.0;
    const double x = lo + (lane + 1) * w;
    const unsigned below = __ballot_sync(0xffffffffu, sturm_count(d, e, n, x, pivmin) >= 1);
    if (below) {
      const int j = __ffs(below) - 1;
      const double nhi = lo + (j + 1) * w;
      lo = j > 0 ? lo + j * w : lo;
      hi = nhi;
    } else {
      lo = lo + 32 * w;
    }
  }
  if (lane == 0) io->lam[c.cidx] = 0.5 * (lo + hi);
}

// p of every group from its blocks' lambda_min (NaN if any is NaN).
__global__ void mix_weight_kernel(const int* __restrict__ groups, const double* __restrict__ nu,
                                  const double* __restrict__ lam, double eps, int ngroups, double* __restrict__ p) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroups) return;
  const int a0 = groups[g], a1 = groups[g + 1];
  double mn = DBL_MAX;
  bool bad = false;
  for (int a = a0; a < a1; ++a) {
    const double l = lam[a];
    if (isnan(l)) bad = true;
    mn = fmin(mn, l);
  }
  double w = 1.0;
  if (bad) {
    w = nan("");
  } else if (mn < 0.0) {
    const double v = nu[g];
    for (int a = a0; a < a1; ++a)
      if (lam[a] < eps) w = fmin(w, (v - eps) / (v - lam[a]));
  }
  p[g] = w;
}

// y = p x + (1 - p) nu svec(1) for every block (meta: offset, side, group).
__global__ void mix_apply_kernel(const int64_t* __restrict__ meta, const double* __restrict__ x,
                                 double* __restrict__ y, const double* __restrict__ p,
                                 const double* __restrict__ nu) {
  const int64_t o = meta[3 * blockIdx.y], n = meta[3 * blockIdx.y + 1];
  const int g = (int)meta[3 * blockIdx.y + 2];
  const double w = p[g], t = (1.0 - w) * nu[g];
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const int64_t cj = o + lcol(n, j);
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) {
      double v = w * x[cj + (i - j)];
      if (i == j) v += t;
      y[cj + (i - j)] = v;
    }
  }
}

}  // namespace

void launch_lmin(const ConeDev* cones, int ncones, const IoSlot* io, cudaStream_t s) {
  if (ncones <= 0) return;
  lmin_kernel<<<ncones, 32, 0, s>>>(cones, io);
}

void launch_mix_weight(const int* groups, const double* nu, const double* lam, double eps, int ngroups, double* p,
                       cudaStream_t s) {
  if (ngroups <= 0) return;
  mix_weight_kernel<<<(ngroups + 127) / 128, 128, 0, s>>>(groups, nu, lam, eps, ngroups, p);
}

void launch_mix_apply(const int64_t* meta, int count, int64_t maxn, const double* x, double* y, const double* p,
                      const double* nu, cudaStream_t s) {
  if (count <= 0) return;
  int gx = (int)(maxn < 256 ? maxn : 256);
  if (gx < 1) gx = 1;
  mix_apply_kernel<<<dim3(gx, count), 64, 0, s>>>(meta, x, y, p, nu);
}

}  // namespace scs
