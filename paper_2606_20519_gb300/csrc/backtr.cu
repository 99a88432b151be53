// Back-transformation through the stage-2 (bulge-chasing) reflectors:
// Z <- Q2 Z with Q2 = H(0,0) H(0,1) ... H(nsweeps-1, last), i.e. the
// reflectors are applied in reverse order of generation.  The reflectors of
// one sweep act on disjoint row blocks, so a whole sweep is applied at once
// (one thread per reflector and column), sweeps one after the other.  Each
// CTA holds a slab of columns of Z in shared memory for the whole pass.
#include "internal.cuh"

namespace scs {

namespace {

constexpr int kBtThreads = 256;

__global__ void __launch_bounds__(kBtThreads) backtr2_kernel(const ConeDev* __restrict__ cones, int cs) {
  const ConeDev& c = cones[blockIdx.y];
  if (*c.status != 0) return;
  const int n = (int)c.n;
  const int kcols = c.kinfo[0];
  const int j0 = blockIdx.x * cs;
  if (j0 >= kcols) return;
  const int nc = min(cs, kcols - j0);
  const int b = c.b;
  extern __shared__ double zs[];  // zs[r * nc + col]
  double* Z = c.Z;
  for (int e = threadIdx.x; e < n * nc; e += kBtThreads) {
    const int r = e % n, col = e / n;
    zs[r * nc + col] = Z[(int64_t)r + (int64_t)(j0 + col) * n];
  }
  __syncthreads();
  for (int i = c.nsweeps - 1; i >= 0; --i) {
    const int Ki = (n - 3 - i) / b + 1;
    const int jobs = Ki * nc;
    for (int job = threadIdx.x; job < jobs; job += kBtThreads) {
      const int kq = job / nc, col = job % nc;
      const int r0 = i + 1 + kq * b;
      const int r1 = min(r0 + b - 1, n - 1);
      const double* slot = c.refl + ((int64_t)i * c.kmax + kq) * (b + 1);
      const double tau = __ldg(slot);
      if (tau == 0.0) continue;
      double dot = zs[r0 * nc + col];
      for (int r = r0 + 1; r <= r1; ++r) dot = fma(__ldg(slot + (r - r0)), zs[r * nc + col], dot);
      dot *= tau;
      zs[r0 * nc + col] -= dot;
      for (int r = r0 + 1; r <= r1; ++r) zs[r * nc + col] = fma(-dot, __ldg(slot + (r - r0)), zs[r * nc + col]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * nc; e += kBtThreads) {
    const int r = e % n, col = e / n;
    Z[(int64_t)r + (int64_t)(j0 + col) * n] = zs[r * nc + col];
  }
}

}  // namespace

int backtr2_cols(int n) {
  int cs = (200 * 1024) / (8 * (n > 0 ? n : 1));
  if (cs > 32) cs = 32;
  if (cs < 1) cs = 1;
  return cs;
}

void launch_backtr2(const ConeDev* cones, int ncones, int maxn, int maxk, cudaStream_t s) {
  if (ncones <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(backtr2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    attr = true;
  }
  const int cs = backtr2_cols(maxn);
  const int gx = (maxk + cs - 1) / cs;
  if (gx <= 0) return;
  backtr2_kernel<<<dim3(gx, ncones), kBtThreads, (size_t)maxn * cs * sizeof(double), s>>>(cones, cs);
}

}  // namespace scs
