// Factorization-free approximate projection (Conclusions, "Approximate
// semidefinite-cone projections"): on the spectrum, max(t, 0) = t (1 + sign t) / 2,
// and sign is replaced by a composite of odd cubics evaluated by matrix
// products alone (scaled Newton-Schulz, the closed-form scaling of
// Chen & Chow 2014 capped so that the top of the interval stays above 1/2):
//   S_0 = X / ||X||_F,   S_{k+1} = a_k S_k + b_k S_k^3,   Y = (X + S_K X) / 2.
// The products are grouped GEMMs (FP64 or split-TF32 tensor cores) that
// write lower triangles.  The kernels here give each cone's norm (the 2-norm
// of its svec, svec being an isometry, App. D.1), the dense X and S_0, the
// upper triangle of each new iterate (so that it is exactly symmetric), and
// the svec of Y's lower triangle.
#include <math.h>

#include "internal.cuh"

namespace scs {

namespace {

__device__ __forceinline__ int64_t pcol(int64_t n, int64_t j) { return j * n - (j * (j - 1)) / 2; }

// Fixed-order block sum (warp shuffles, then warp 0 over the warp sums).
__device__ double block_sum_fixed(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < nw; ++q) s += sh[q];
  return s;
}

// Partial sums of squares of each cone's svec, kPolyChunk entries per block.
__global__ void poly_norm_kernel(const PolyConeDev* __restrict__ cones, const int* __restrict__ part_cone,
                                 const IoSlot* __restrict__ io, double* __restrict__ part) {
  __shared__ double sh[32];
  const int b = blockIdx.x;
  const PolyConeDev& c = cones[part_cone[b]];
  const int64_t len = c.n * (c.n + 1) / 2;
  const int64_t q0 = (int64_t)(b - c.part0) * kPolyChunk;
  const int64_t q1 = q0 + kPolyChunk < len ? q0 + kPolyChunk : len;
  const double* __restrict__ x = io->x + c.xoff;
  double s = 0.0;
  for (int64_t e = q0 + threadIdx.x; e < q1; e += blockDim.x) {
    const double v = x[e];
    s = fma(v, v, s);
  }
  s = block_sum_fixed(s, sh);
  if (threadIdx.x == 0) part[b] = s;
}

// One warp per cone: ||X||_F^2 = nsq ||svec||^2 from the partial sums (fixed
// order; nsq = 1/2 for the real embedding of a Hermitian cone), then
// 1 / ||X||_F (0 for X = 0); a non-finite sum marks the cone.
__global__ void poly_sigma_kernel(const PolyConeDev* __restrict__ cones, const double* __restrict__ part,
                                  double* __restrict__ inv, double nsq) {
  const PolyConeDev& c = cones[blockIdx.x];
  double s = 0.0;
  for (int q = threadIdx.x; q < c.nparts; q += 32) s += part[c.part0 + q];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) {
    double r = 0.0;
    if (!isfinite(s)) atomicOr(c.status, ST_NONFINITE);
    else if (s > 0.0) r = 1.0 / sqrt(s * nsq);
    inv[blockIdx.x] = r;
  }
}

// Dense X and S_0 = X / ||X||_F (both triangles, column-major, ld = n).
// Block (bi, bj) with bi >= bj reads the lower 32 x 32 tile from the svec
// (contiguous along a column) and writes it and its mirror image.
__global__ void poly_unpack_kernel(const PolyConeDev* __restrict__ cones, const IoSlot* __restrict__ io,
                                   const double* __restrict__ inv) {
  __shared__ double t[32][33];
  const PolyConeDev& c = cones[blockIdx.z];
  const int64_t n = c.n;
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bj > bi || (int64_t)bi * 32 >= n) return;
  const double* __restrict__ x = io->x + c.xoff;
  const double r = inv[blockIdx.z];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t ib = (int64_t)bi * 32, jb = (int64_t)bj * 32;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = ib + tx, j = jb + ty + 8 * k;
    double v = 0.0;
    if (i < n && j < n && i >= j) {
      v = x[pcol(n, j) + (i - j)];
      if (i != j) v *= M_SQRT1_2;
    }
    t[tx][ty + 8 * k] = v;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = ib + tx, j = jb + ty + 8 * k;
    if (i < n && j < n) {
      const double v = (i >= j) ? t[tx][ty + 8 * k] : t[ty + 8 * k][tx];
      c.X[i + j * n] = v;
      c.S0[i + j * n] = v * r;
    }
  }
  if (bi == bj) return;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = jb + tx, j = ib + ty + 8 * k;  // upper tile (bj, bi): X(i, j) = X(j, i)
    if (i < n && j < n) {
      const double v = t[ty + 8 * k][tx];
      c.X[i + j * n] = v;
      c.S0[i + j * n] = v * r;
    }
  }
}

// Upper triangle of an iterate from its lower triangle, 32 x 32 tiles:
// block (bi, bj), bi >= bj, reads tile (bi, bj) down its columns and writes
// its transpose into tile (bj, bi).
__global__ void poly_mirror_kernel(const PolyConeDev* __restrict__ cones, int which) {
  __shared__ double t[32][33];
  const PolyConeDev& c = cones[blockIdx.z];
  const int64_t n = c.n;
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bj > bi || (int64_t)bi * 32 >= n) return;
  if (!c.mirror || *c.status) return;
  double* __restrict__ S = which ? c.S0 : c.S1;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t ib = (int64_t)bi * 32, jb = (int64_t)bj * 32;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = ib + tx, j = jb + ty + 8 * k;
    t[tx][ty + 8 * k] = (i < n && j < n && i >= j) ? S[i + j * n] : 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t i = jb + tx, j = ib + ty + 8 * k;  // upper entry (i, j), i < j, takes S(j, i)
    if (i < n && j < n && i < j) S[i + j * n] = t[ty + 8 * k][tx];
  }
}

// svec of the lower triangle of Y (NaN for a marked cone).
__global__ void poly_pack_kernel(const PolyConeDev* __restrict__ cones, const IoSlot* __restrict__ io) {
  const PolyConeDev& c = cones[blockIdx.y];
  const int64_t n = c.n;
  const bool bad = *c.status != 0;
  double* __restrict__ y = io->y + c.xoff;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const int64_t o = pcol(n, j);
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) {
      double v = c.Y[i + j * n];
      if (i != j) v *= M_SQRT2;
      y[o + (i - j)] = bad ? nan("") : v;
    }
  }
}

}  // namespace

void launch_poly_prepare(const PolyConeDev* cones, int ncones, const int* part_cone, int nparts, int64_t maxn,
                         const IoSlot* io, double* part, double* inv, double nsq, cudaStream_t s) {
  if (ncones <= 0 || nparts <= 0) return;
  poly_norm_kernel<<<nparts, 256, 0, s>>>(cones, part_cone, io, part);
  poly_sigma_kernel<<<ncones, 32, 0, s>>>(cones, part, inv, nsq);
  const int tiles = (int)((maxn + 31) / 32);
  poly_unpack_kernel<<<dim3(tiles, tiles, ncones), dim3(32, 8), 0, s>>>(cones, io, inv);
}

void launch_poly_mirror(const PolyConeDev* cones, int ncones, int64_t maxn, int which, cudaStream_t s) {
  if (ncones <= 0) return;
  const int tiles = (int)((maxn + 31) / 32);
  poly_mirror_kernel<<<dim3(tiles, tiles, ncones), dim3(32, 8), 0, s>>>(cones, which);
}

void launch_poly_pack(const PolyConeDev* cones, int ncones, int64_t maxn, const IoSlot* io, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)maxn;
  if (gx > 1024) gx = 1024;
  if (gx < 1) gx = 1;
  poly_pack_kernel<<<dim3(gx, ncones), 128, 0, s>>>(cones, io);
}

}  // namespace scs
