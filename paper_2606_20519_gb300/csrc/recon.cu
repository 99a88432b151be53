// Clipped reconstruction straight into svec.
//
// With Z the k kept eigenvectors and l their eigenvalues (all positive, or
// all negative when the cone's final merge chose the Moreau side), the
// kernel forms the lower triangle of S = Z diag(l) Z^T tile by tile (SYRK:
// only tiles on or below the diagonal) and writes, for i >= j,
//     y[svec(i, j)] = s_ij * S(i, j)              (positive part), or
//     y[svec(i, j)] = x[svec(i, j)] - s_ij * S(i, j)   (X - negative part),
// with s_ij = 1 on the diagonal and sqrt(2) off it (the vec_R map, App. D.1).
// Each svec entry is read and written by one thread, so y may alias x.
// A cone whose status is not clean is filled with NaN.
#include <math.h>

#include "dfloat.cuh"
#include "internal.cuh"

namespace scs {

namespace {

constexpr int BK = 16;

// The products run in double-float (FP32 pairs): Z's entries are bounded by
// one and the eigenvalues are scaled by 2^-s, s the exponent of the largest
// |l_k| (integer operations on the exponent field); the sum is scaled back in
// FP64 in the epilogue.
template <int BM>
__global__ void __launch_bounds__(256, 2) recon_kernel(const ConeDev* __restrict__ cones, const IoSlot* __restrict__ io) {
  const double* x = io->x;
  double* y = io->y;
  __shared__ dfl As[BK][BM + 1];
  __shared__ dfl Bs[BK][BM + 1];
  __shared__ int s_exp;
  const ConeDev& c = cones[blockIdx.y];
  const int n = (int)c.n;
  const int tiles = (n + BM - 1) / BM;
  const int t = blockIdx.x;
  if (t >= tiles * (tiles + 1) / 2) return;
  int tm = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
  while (tm * (tm + 1) / 2 > t) --tm;
  const int tn = t - tm * (tm + 1) / 2;
  const int i0 = tm * BM, j0 = tn * BM;
  const bool bad = *c.status != 0;
  // all-pairs mode: the route's side comes first, kinfo[6] of them
  const int kk = bad ? 0 : (c.kinfo[3] ? c.kinfo[6] : c.kinfo[0]);
  const int route = c.kinfo[1];
  const double* Z = c.Z;
  const double* lam = c.lamk;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // the largest biased exponent of the kept eigenvalues
  if (tid == 0) s_exp = 0;
  __syncthreads();
  {
    int m = 0;
    for (int k = tid; k < kk; k += 256) m = max(m, (int)((__double2hiint(lam[k]) >> 20) & 0x7FF));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((tid & 31) == 0 && m > 0) atomicMax(&s_exp, m);
  }
  __syncthreads();
  const int es = min(max(s_exp, 1), 2045);  // l 2^-(es - 1023) lies within [-2, 2]
  constexpr int R = BM / 16;  // rows (and columns) per thread
  dfl acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < R; ++q) acc[r][q] = df_zero();
  for (int k0 = 0; k0 < kk; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / 256; ++q) {
      const int e = tid + q * 256;
      const int ii = e % BM, l = e / BM;
      const int i = i0 + ii, j = j0 + ii, k = k0 + l;
      dfl a = df_zero(), bv = df_zero();
      if (k < kk) {
        if (i < n) a = df_from_d_int(Z[(int64_t)i + (int64_t)k * n]);
        if (j < n) {
          // all eigenpairs are present when the derivative is needed: clip by side
          const double lk = route == 0 ? fmax(lam[k], 0.0) : fmin(lam[k], 0.0);
          bv = df_mul(df_from_d_int(Z[(int64_t)j + (int64_t)k * n]), df_from_d_scaled(lk, es - 1023));
        }
      }
      As[l][ii] = a;
      Bs[l][ii] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < BK; ++l) {
      dfl a[R], bv[R];
#pragma unroll
      for (int r = 0; r < R; ++r) a[r] = As[l][tx + 16 * r];
#pragma unroll
      for (int q = 0; q < R; ++q) bv[q] = Bs[l][ty + 16 * q];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < R; ++q) acc[r][q] = df_fma(a[r], bv[q], acc[r][q]);
    }
    __syncthreads();
  }
  const double up = __longlong_as_double((long long)es << 52);  // 2^(es - 1023)
  const double* xs = x + c.xoff;
  double* ys = y + c.xoff;
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = j0 + ty + 16 * q;
    if (j >= n) continue;
    const int64_t colo = (int64_t)j * n - ((int64_t)j * (j - 1)) / 2;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + tx + 16 * r;
      if (i >= n || i < j) continue;
      const int64_t idx = colo + (i - j);
      const double sc = (i == j) ? up : M_SQRT2 * up;
      const double sv = df_to_d(acc[r][q]);
      double v;
      if (bad) v = nan("");
      else if (route == 0) v = sc * sv;
      else v = fma(-sc, sv, xs[idx]);
      ys[idx] = v;
    }
  }
}

// Split mode: S = Z diag(l) Z^T was formed (lower triangle) in QA by the
// tensor-core GEMM; write svec(S) (positive part) or x - svec(S).
__global__ void pack_recon_kernel(const ConeDev* __restrict__ cones, const IoSlot* __restrict__ io) {
  const double* x = io->x;
  double* y = io->y;
  const ConeDev& c = cones[blockIdx.y];
  const int64_t n = c.n;
  const int64_t len = n * (n + 1) / 2;
  const bool bad = *c.status != 0;
  const int route = c.kinfo[1];
  const double* xs = x + c.xoff;
  double* ys = y + c.xoff;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const int64_t colo = j * n - (j * (j - 1)) / 2;
    const int kk = c.kinfo[0];
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) {
      const int64_t idx = colo + (i - j);
      if (idx >= len) continue;
      const double s = kk > 0 ? c.QA[i + j * n] : 0.0;
      const double sc = (i == j) ? 1.0 : M_SQRT2;
      double v;
      if (bad) v = nan("");
      else if (route == 0) v = sc * s;
      else v = fma(-sc, s, xs[idx]);
      ys[idx] = v;
    }
  }
}

}  // namespace

void launch_pack_recon(const ConeDev* cones, int ncones, int64_t maxn, const IoSlot* io, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)(maxn < 2048 ? maxn : 2048);
  pack_recon_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones, io);
}

void launch_recon(const ConeDev* cones, int ncones, int maxn, const IoSlot* io, cudaStream_t s) {
  if (ncones <= 0) return;
  // 64-row tiles, or 32-row tiles when those would leave most SMs idle
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int t64 = (maxn + 63) / 64;
  if ((int64_t)t64 * (t64 + 1) / 2 * ncones < sms) {
    const int t32 = (maxn + 31) / 32;
    recon_kernel<32><<<dim3(t32 * (t32 + 1) / 2, ncones), 256, 0, s>>>(cones, io);
  } else {
    recon_kernel<64><<<dim3(t64 * (t64 + 1) / 2, ncones), 256, 0, s>>>(cones, io);
  }
}

}  // namespace scs
