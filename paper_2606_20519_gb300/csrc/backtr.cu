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
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(backtr2_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    attr = true;
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

}  // namespace scs
