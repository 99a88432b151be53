// Daleckii-Krein vector-Jacobian product of the PSD projection.
//
// With X = V diag(l) V^T (all n eigenpairs) and G = smat(g),
//     DPi(X)[G] = V (L o (V^T G V)) V^T,
//     L_ij = 1 (l_i > 0, l_j > 0), 0 (l_i <= 0, l_j <= 0),
//            max(l_i, l_j) / |l_i - l_j| otherwise (opposite signs: no
//            cancellation in the divided difference of max(., 0)).
// The derivative map is self-adjoint and svec is an isometry (App. D.1), so
// the svec VJP equals svec(DPi(X)[smat(g)]).  The contractions run in the
// grouped GEMM; this file holds the elementwise Loewner scaling and the
// final svec packing.
#include <math.h>

#include "internal.cuh"

namespace scs {

namespace {

__device__ __forceinline__ double loewner(double a, double b) {
  const bool pa = a > 0.0, pb = b > 0.0;
  if (pa && pb) return 1.0;
  if (!pa && !pb) return 0.0;
  return (pa ? a : b) / fabs(a - b);
}

// M(i, j) *= L(l_i, l_j) on an n x n column-major block (M = QB).
__global__ void loewner_scale_kernel(const ConeDev* __restrict__ cones) {
  const ConeDev& c = cones[blockIdx.y];
  if (*c.status != 0) return;
  const int64_t n = c.n;
  const int64_t nn = n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    c.QB[e] *= loewner(c.lamk[i], c.lamk[j]);
  }
}

// Stored eigendecomposition out: V block = Z (all n columns), lam = lamk;
// NaN for a cone whose status is bad.
__global__ void export_eig_kernel(const ConeDev* __restrict__ cones, const IoSlot* __restrict__ io) {
  const ConeDev& c = cones[blockIdx.y];
  const int64_t n = c.n, nn = n * n;
  const bool bad = *c.status != 0;
  double* V = io->V + c.voff;
  double* lam = io->lam + c.loff;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    V[e] = bad ? nan("") : c.Z[e];
    if (e < n) lam[e] = bad ? nan("") : c.lamk[e];
  }
}

// Stored eigendecomposition in, in place of the eigensolver's output.
__global__ void import_eig_kernel(const ConeDev* __restrict__ cones, const IoSlot* __restrict__ io) {
  const ConeDev& c = cones[blockIdx.y];
  const int64_t n = c.n, nn = n * n;
  const double* V = io->V + c.voff;
  const double* lam = io->lam + c.loff;
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = V[e];
    bad |= !isfinite(v);
    c.Z[e] = v;
    if (e < n) {
      const double l = lam[e];
      bad |= !isfinite(l);
      c.lamk[e] = l;
    }
  }
  if (bad) atomicOr(c.status, ST_NONFINITE);
}

// xbar = svec of the lower triangle of H (H = QB here), NaN on a bad cone.
__global__ void pack_lower_kernel(const ConeDev* __restrict__ cones, const IoSlot* __restrict__ io) {
  const ConeDev& c = cones[blockIdx.y];
  double* xbar = io->xbar;
  const int64_t n = c.n;
  const int64_t len = n * (n + 1) / 2;
  const bool bad = *c.status != 0;
  double* out = xbar + c.xoff;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x) {
    // invert t -> (i, j), column j starts at j*n - j(j-1)/2
    double jd = ((2.0 * n + 1.0) - sqrt((2.0 * n + 1.0) * (2.0 * n + 1.0) - 8.0 * (double)t)) * 0.5;
    int64_t j = (int64_t)jd;
    if (j < 0) j = 0;
    if (j > n - 1) j = n - 1;
    while (j > 0 && j * n - (j * (j - 1)) / 2 > t) --j;
    while (j + 1 < n && (j + 1) * n - ((j + 1) * j) / 2 <= t) ++j;
    const int64_t i = j + (t - (j * n - (j * (j - 1)) / 2));
    const double sc = (i == j) ? 1.0 : M_SQRT2;
    out[t] = bad ? nan("") : sc * c.QB[i + j * n];
  }
}

}  // namespace

void launch_loewner_scale(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)((maxn * maxn + 255) / 256);
  if (gx > 2048) gx = 2048;
  loewner_scale_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones);
}

void launch_export_eig(const ConeDev* cones, int ncones, int64_t maxn, const IoSlot* io, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)((maxn * maxn + 255) / 256);
  if (gx > 2048) gx = 2048;
  export_eig_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones, io);
}

void launch_import_eig(const ConeDev* cones, int ncones, int64_t maxn, const IoSlot* io, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)((maxn * maxn + 255) / 256);
  if (gx > 2048) gx = 2048;
  import_eig_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones, io);
}

void launch_pack_lower(const ConeDev* cones, int ncones, int64_t maxn, const IoSlot* io, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)((maxn * (maxn + 1) / 2 + 255) / 256);
  if (gx > 2048) gx = 2048;
  pack_lower_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones, io);
}

}  // namespace scs
