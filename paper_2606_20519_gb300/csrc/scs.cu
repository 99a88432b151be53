// The SCS iteration around the PSD projection (App. D.1, final iterates):
//   u~ = (I + Q)^{-1} (u + v),  u = Pi_C(u~ - v),  v = v - u~ + u,
// with u = (x, y, tau), Q = [[0, A^T, c], [-A, 0, b], [-c^T, -b^T, 0]] and an
// A with orthonormal columns, so that M = [[I, A^T], [-A, I]] has the closed
// inverse z_x = (a_x - A^T a_y) / 2, z_y = a_y + A z_x (one product with A^T,
// one with A), and (I + Q)^{-1} follows from z = M^{-1} w and p = M^{-1}(c, b):
//   tau~ = (w_tau + c.z_x + b.z_y) / (1 + c.p_x + b.p_y),  (x~, y~) = z - tau~ p.
// A dense A (column-major, m x k) is streamed from HBM once per product (both
// products are FP64-pipe-bound on this part: m k FMAs against 8 m k bytes); a
// structured A is applied by the contractions of kron.cu; the rest are short
// vector kernels; the cone projection of the y block is the library's own
// launch sequence.
#include <algorithm>

#include "internal.cuh"

namespace scs {

namespace {

// A^T (a1 + a2) in two launches with a fixed summation order: block (g, r)
// forms, for the kGtCols columns of group g and the rows of chunk r, the
// partial dot products part[r * k + j] (each thread kGtCols independent FMA
// chains, the vector element read once for all of them); then
// out[j] = sum_r part[r * k + j] in increasing r.
constexpr int kGtCols = 8;
__global__ void __launch_bounds__(256) gemv_t_part_kernel(const double* __restrict__ A, int64_t m, int64_t k,
                                                          const double* __restrict__ a1,
                                                          const double* __restrict__ a2, int chunks,
                                                          double* __restrict__ part) {
  __shared__ double sh[8][kGtCols];
  const int64_t j0 = (int64_t)blockIdx.x * kGtCols;
  const int64_t rows = (m + chunks - 1) / chunks;
  const int64_t r0 = (int64_t)blockIdx.y * rows, r1 = r0 + rows < m ? r0 + rows : m;
  const int nc = k - j0 < kGtCols ? (int)(k - j0) : kGtCols;
  double acc[kGtCols];
#pragma unroll
  for (int c = 0; c < kGtCols; ++c) acc[c] = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += 256) {
    const double a = a2 ? a1[i] + a2[i] : a1[i];
#pragma unroll
    for (int c = 0; c < kGtCols; ++c)
      if (c < nc) acc[c] = fma(A[(j0 + c) * m + i], a, acc[c]);
  }
#pragma unroll
  for (int c = 0; c < kGtCols; ++c) {
    double s = acc[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][c] = s;
  }
  __syncthreads();
  if (threadIdx.x < nc) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sh[q][threadIdx.x];
    part[(int64_t)blockIdx.y * k + j0 + threadIdx.x] = t;
  }
}

__global__ void gemv_t_sum_kernel(const double* __restrict__ part, int chunks, int64_t k, double* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double t = 0.0;
  for (int r = 0; r < chunks; ++r) t += part[(int64_t)r * k + j];
  out[j] = t;
}

// out[i] = a1[i] + a2[i] + A(i, :) . x: threads over rows (coalesced down the
// columns), x staged in shared memory in chunks; four independent FMA chains
// per thread (columns q mod 4), summed in a fixed order.
__global__ void __launch_bounds__(256) gemv_n_kernel(const double* __restrict__ A, int64_t m, int64_t k,
                                                     const double* __restrict__ x, const double* __restrict__ a1,
                                                     const double* __restrict__ a2, double* __restrict__ out) {
  __shared__ double xs[1024];
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int64_t j0 = 0; j0 < k; j0 += 1024) {
    const int64_t nj = k - j0 < 1024 ? k - j0 : 1024;
    __syncthreads();
    for (int q = threadIdx.x; q < nj; q += 256) xs[q] = x[j0 + q];
    __syncthreads();
    if (i < m) {
      const double* __restrict__ p = A + i + j0 * m;
      int64_t q = 0;
#pragma unroll 2
      for (; q + 3 < nj; q += 4) {
        s0 = fma(p[q * m], xs[q], s0);
        s1 = fma(p[(q + 1) * m], xs[q + 1], s1);
        s2 = fma(p[(q + 2) * m], xs[q + 2], s2);
        s3 = fma(p[(q + 3) * m], xs[q + 3], s3);
      }
      for (; q < nj; ++q) s0 = fma(p[q * m], xs[q], s0);
    }
  }
  if (i < m) out[i] = (a2 ? a1[i] + a2[i] : a1[i]) + ((s0 + s1) + (s2 + s3));
}

// out[j] = (a1[j] + a2[j] - t[j]) / 2  (a2 may be null)
__global__ void half_diff_kernel(const double* __restrict__ a1, const double* __restrict__ a2,
                                 const double* __restrict__ t, int64_t k, double* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) out[j] = 0.5 * ((a2 ? a1[j] + a2[j] : a1[j]) - t[j]);
}

// partial sums of c . zx + b . zy over fixed chunks (one per block)
__global__ void __launch_bounds__(256) dot2_kernel(const double* __restrict__ c, const double* __restrict__ zx,
                                                   int64_t k, const double* __restrict__ b,
                                                   const double* __restrict__ zy, int64_t m,
                                                   double* __restrict__ part) {
  __shared__ double sh[8];
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < k + m; e += (int64_t)gridDim.x * 256)
    s = e < k ? fma(c[e], zx[e], s) : fma(b[e - k], zy[e - k], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sh[q];
    part[blockIdx.x] = t;
  }
}

// setup (tau_in null): hp = sum(part); iteration: tau~ = (u_tau + v_tau + sum(part)) / (1 + hp)
__global__ void finish_kernel(const double* __restrict__ part, int nparts, const double* __restrict__ u_tau,
                              const double* __restrict__ v_tau, double* __restrict__ hp, double* __restrict__ tau) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += part[q];
  if (!u_tau) *hp = s;
  else *tau = (*u_tau + *v_tau + s) / (1.0 + *hp);
}

// u~ = z - tau~ p (tau~ itself in the last coordinate); t = u~ - v;
// x: u = t; y: t goes to the projection input, u~_y is kept; tau: u = max(t, 0);
// v = v - u~ + u for x and tau (the y part after the projection).
__global__ void update_kernel(const double* __restrict__ z, const double* __restrict__ p,
                              const double* __restrict__ tau, int64_t k, int64_t m, double* __restrict__ u,
                              double* __restrict__ v, double* __restrict__ tin, double* __restrict__ uty) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double tt = *tau;
  if (e < k) {
    const double ut = z[e] - tt * p[e];
    const double t = ut - v[e];
    u[e] = t;
    v[e] = v[e] - ut + t;
  } else if (e < k + m) {
    const double ut = z[e] - tt * p[e];
    tin[e - k] = ut - v[e];
    uty[e - k] = ut;
  } else if (e == k + m) {
    const double t = tt - v[e];
    const double un = t > 0.0 ? t : 0.0;
    u[e] = un;
    v[e] = v[e] - tt + un;
  }
}

// v_y = v_y - u~_y + u_y
__global__ void vy_kernel(double* __restrict__ vy, const double* __restrict__ uty, const double* __restrict__ uy,
                          int64_t m) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) vy[i] = vy[i] - uty[i] + uy[i];
}

}  // namespace

// Row chunks of the A^T product: about four blocks per SM over all column groups
// (eight measured the same).
int scs_gemv_t_chunks(int64_t m, int64_t k) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t groups = (k + kGtCols - 1) / kGtCols;
  int64_t r = (4 * (int64_t)sms + groups - 1) / std::max<int64_t>(1, groups);
  r = std::min<int64_t>(r, std::max<int64_t>(1, m / 1024));
  return (int)std::max<int64_t>(1, std::min<int64_t>(r, 64));
}

int scs_dot_parts(int64_t len) {
  int64_t g = (len + 255) / 256;
  return (int)(g < 512 ? (g < 1 ? 1 : g) : 512);
}

// out = A^T (a1 + a2), k entries
void op_t(const ScsOp& op, int64_t m, int64_t k, const double* a1, const double* a2, double* out, cudaStream_t s) {
  if (k <= 0) return;
  if (op.A) {
    const int chunks = op.tchunks;
    gemv_t_part_kernel<<<dim3((unsigned)((k + kGtCols - 1) / kGtCols), (unsigned)chunks), 256, 0, s>>>(
        op.A, m, k, a1, a2, chunks, op.tpart);
    gemv_t_sum_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(op.tpart, chunks, k, out);
  } else {
    launch_kron_apply_t(op.kron, a1, a2, out, op.t0, op.t1, op.status, s);
  }
}

// out = a1 + a2 + A x, m entries
void op_n(const ScsOp& op, int64_t m, int64_t k, const double* x, const double* a1, const double* a2, double* out,
          cudaStream_t s) {
  if (op.A || k == 0) gemv_n_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(op.A, m, k, x, a1, a2, out);
  else launch_kron_apply(op.kron, x, a1, a2, out, op.t0, op.t1, op.status, s);
}

void launch_scs_setup(const ScsOp& op, const double* b, const double* c, int64_t m, int64_t k, double* p,
                      double* hp, double* tk, double* part, cudaStream_t s) {
  // p_x = (c - A^T b) / 2, p_y = b + A p_x, hp = c . p_x + b . p_y
  if (k > 0) {
    op_t(op, m, k, b, nullptr, tk, s);
    half_diff_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(c, nullptr, tk, k, p);
  }
  op_n(op, m, k, p, b, nullptr, p + k, s);
  const int np = scs_dot_parts(k + m);
  dot2_kernel<<<np, 256, 0, s>>>(c, p, k, b, p + k, m, part);
  finish_kernel<<<1, 32, 0, s>>>(part, np, nullptr, nullptr, hp, nullptr);
}

void launch_scs_affine(const ScsOp& op, const double* b, const double* c, int64_t m, int64_t k, const double* p,
                       const double* hp, double* u, double* v, double* z, double* tk, double* part, double* tau,
                       double* tin, double* uty, cudaStream_t s) {
  // w = u + v; z_x = (w_x - A^T w_y) / 2; z_y = w_y + A z_x
  if (k > 0) {
    op_t(op, m, k, u + k, v + k, tk, s);
    half_diff_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(u, v, tk, k, z);
  }
  op_n(op, m, k, z, u + k, v + k, z + k, s);
  const int np = scs_dot_parts(k + m);
  dot2_kernel<<<np, 256, 0, s>>>(c, z, k, b, z + k, m, part);
  finish_kernel<<<1, 32, 0, s>>>(part, np, u + k + m, v + k + m, const_cast<double*>(hp), tau);
  update_kernel<<<(unsigned)((k + m + 1 + 255) / 256), 256, 0, s>>>(z, p, tau, k, m, u, v, tin, uty);
}

void launch_scs_vy(double* vy, const double* uty, const double* uy, int64_t m, cudaStream_t s) {
  vy_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(vy, uty, uy, m);
}

}  // namespace scs
