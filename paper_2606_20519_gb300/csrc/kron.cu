// The structured affine operator of the SCS iteration (App. D.2): A x and
// A^T y as contractions over local bases, the Kronecker products
//     F_mu = F1[mu_1] (x) F2[mu_2] (x) ... (x) FS[mu_S]
// never formed.  Column j of A is svec(F_mu) for the multi-index mu of the
// flat index index[j] (C order over the local basis sizes k_1 .. k_S).
//
// A x: the coefficients are scattered into a k_1 x .. x k_S tensor; mode s
// is then replaced by the d_s x d_s entries of the local matrices (one
// contraction per mode with the d_s^2 x k_s matrix M_s[(i, j), b] =
// F_s[b](i, j)), which leaves W with the mode-s index (i_s, j_s); W(r, c),
// r = (i_1 .. i_S), c = (j_1 .. j_S) in np.kron's order, is packed into svec.
// A^T y runs the same steps backwards: smat(y) into the (i_s, j_s) modes, the
// contractions with M_s^T, the gather of the listed coefficients.
//
// The local bases the paper uses (generalized Gell-Mann matrices and their
// real forms) have at most d_s nonzeros per position, so every contraction
// skips the zero entries of M_s; a warp works on 32 fibres with one output
// index, which keeps that test uniform across the warp.
#include "internal.cuh"

namespace scs {

namespace {

constexpr int kKrThreads = 256;
constexpr int kFib = 32;  // fibres per CTA

// x -> coefficient tensor (zeroed first); flat indices out of range are
// reported in *status and skipped.
__global__ void kron_zero_kernel(double* __restrict__ t, int64_t len) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
    t[e] = 0.0;
}

__global__ void kron_scatter_kernel(const int64_t* __restrict__ index, int64_t k, int64_t kt,
                                    const double* __restrict__ x, double* __restrict__ t, int* status) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const int64_t f = index[j];
  if (f < 0 || f >= kt) { atomicOr(status, ST_BADARG); return; }
  t[f] = x[j];
}

// out[j] = t[index[j]]
__global__ void kron_gather_kernel(const int64_t* __restrict__ index, int64_t k, int64_t kt,
                                   const double* __restrict__ t, double* __restrict__ out, int* status) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const int64_t f = index[j];
  if (f < 0 || f >= kt) { atomicOr(status, ST_BADARG); out[j] = 0.0; return; }
  out[j] = t[f];
}

// One contraction: the tensor viewed as (P, kin, Q) becomes (P, kout, Q).
// Forward (trans = 0): kin = k_s, kout = d^2, out[p, i d + j, q] =
//   sum_b F[b](i, j) in[p, b, q].
// Backward (trans = 1): kin = d^2, kout = k_s, out[p, b, q] =
//   sum_{i, j} F[b](i, j) in[p, i d + j, q].
// F[b](i, j) = basis[b d^2 + i + j d] (column-major local matrices).
// CTA: kFib consecutive fibres f = p Q + q; the input tile (kin x kFib) in
// shared memory; warp w forms outputs w, w + 8, ...
__global__ void __launch_bounds__(kKrThreads) kron_mode_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                               const double* __restrict__ basis, int d, int ks,
                                                               int trans, int64_t P, int64_t Q) {
  extern __shared__ double kr_smem[];
  const int d2 = d * d;
  const int kin = trans ? d2 : ks, kout = trans ? ks : d2;
  double* M = kr_smem;                  // kout x kin, row-major
  double* tile = kr_smem + kout * kin;  // kin x kFib
  for (int e = threadIdx.x; e < kout * kin; e += kKrThreads) {
    const int a = e / kin, b = e % kin;  // output a, input b
    // forward: a = i d + j, b = basis index; backward: a = basis index, b = i d + j
    const int bi = trans ? a : b, pos = trans ? b : a;
    const int i = pos / d, j = pos % d;
    M[e] = basis[(int64_t)bi * d2 + i + (int64_t)j * d];
  }
  const int64_t nf = P * Q;
  const int64_t f0 = (int64_t)blockIdx.x * kFib;
  for (int e = threadIdx.x; e < kin * kFib; e += kKrThreads) {
    const int b = e / kFib, l = e % kFib;
    const int64_t f = f0 + l;
    double v = 0.0;
    if (f < nf) {
      const int64_t p = f / Q, q = f % Q;
      v = in[(p * kin + b) * Q + q];
    }
    tile[b * kFib + l] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t f = f0 + lane;
  const bool live = f < nf;
  const int64_t p = live ? f / Q : 0, q = live ? f % Q : 0;
  for (int a = warp; a < kout; a += kKrThreads / 32) {
    const double* Ma = M + a * kin;
    double acc = 0.0;
    for (int b = 0; b < kin; ++b) {
      const double mv = Ma[b];
      if (mv != 0.0) acc = fma(mv, tile[b * kFib + lane], acc);
    }
    if (live) out[(p * kout + a) * Q + q] = acc;
  }
}

__device__ __forceinline__ int64_t svec_off(int64_t n, int64_t j) { return j * n - (j * (j - 1)) / 2; }

// W (modes (i_s, j_s), a_s = i_s d_s + j_s, C order) <-> matrix indices:
// r = sum_s i_s R_s, c = sum_s j_s R_s with R_s = prod_{t > s} d_t.
__device__ __forceinline__ int64_t w_index(const KronDev& op, int64_t r, int64_t c) {
  int64_t idx = 0, stride = 1;
  for (int s = op.S - 1; s >= 0; --s) {
    const int d = op.d[s];
    const int64_t is = r % d, js = c % d;
    r /= d;
    c /= d;
    idx += (is * d + js) * stride;
    stride *= (int64_t)d * d;
  }
  return idx;
}

// out = a1 (+ a2) + svec(W): one CTA per column c of the lower triangle
__global__ void kron_pack_kernel(KronDev op, const double* __restrict__ w, const double* __restrict__ a1,
                                 const double* __restrict__ a2, double* __restrict__ out) {
  const int64_t n = op.N, c = blockIdx.x;
  const int64_t base = svec_off(n, c);
  for (int64_t r = c + threadIdx.x; r < n; r += blockDim.x) {
    const int64_t e = base + (r - c);
    double v = w[w_index(op, r, c)];
    if (r != c) v *= M_SQRT2;
    double acc = a1 ? a1[e] : 0.0;
    if (a2) acc += a2[e];
    out[e] = acc + v;
  }
}

// W(r, c) = smat(a1 + a2)(r, c) for every (r, c)
__global__ void kron_unpack_kernel(KronDev op, const double* __restrict__ a1, const double* __restrict__ a2,
                                   double* __restrict__ w) {
  const int64_t n = op.N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n, c = e % n;
    const int64_t lo = r >= c ? r : c, hi = r >= c ? c : r;
    const int64_t s = svec_off(n, hi) + (lo - hi);
    double v = a1[s];
    if (a2) v += a2[s];
    if (r != c) v *= M_SQRT1_2;
    w[w_index(op, r, c)] = v;
  }
}

int grid_for(int64_t len) {
  int64_t g = (len + kKrThreads - 1) / kKrThreads;
  return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

// the contractions in order; returns the buffer holding the result
double* contract_all(const KronDev& op, int trans, double* t0, double* t1, cudaStream_t s) {
  int64_t cur[kKronMaxModes];
  for (int q = 0; q < op.S; ++q) cur[q] = trans ? (int64_t)op.d[q] * op.d[q] : op.kb[q];
  double* src = t0;
  double* dst = t1;
  for (int q = 0; q < op.S; ++q) {
    int64_t P = 1, Q = 1;
    for (int t = 0; t < q; ++t) P *= cur[t];
    for (int t = q + 1; t < op.S; ++t) Q *= cur[t];
    const int d = op.d[q], ks = op.kb[q];
    const int kin = trans ? d * d : ks, kout = trans ? ks : d * d;
    const size_t smem = sizeof(double) * ((size_t)kin * kout + (size_t)kin * kFib);
    const int64_t nf = P * Q;
    kron_mode_kernel<<<(unsigned)((nf + kFib - 1) / kFib), kKrThreads, smem, s>>>(src, dst, op.basis[q], d, ks, trans,
                                                                                  P, Q);
    cur[q] = kout;
    double* tmp = src;
    src = dst;
    dst = tmp;
  }
  return src;
}

}  // namespace

size_t kron_mode_smem_max() {
  // kin, kout <= 64 (local sides up to 8)
  return sizeof(double) * (64 * 64 + 64 * kFib);
}

void kron_prepare() {
  cudaFuncSetAttribute(kron_mode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kron_mode_smem_max());
}

int kron_launches(const KronDev& op) { return op.S + 3; }

// out = a1 + a2 + A x (svec, m entries); x has k entries
void launch_kron_apply(const KronDev& op, const double* x, const double* a1, const double* a2, double* out,
                       double* t0, double* t1, int* status, cudaStream_t s) {
  kron_zero_kernel<<<grid_for(op.Kt), kKrThreads, 0, s>>>(t0, op.Kt);
  if (op.k > 0)
    kron_scatter_kernel<<<(unsigned)((op.k + kKrThreads - 1) / kKrThreads), kKrThreads, 0, s>>>(op.index, op.k,
                                                                                                 op.Kt, x, t0, status);
  double* w = contract_all(op, 0, t0, t1, s);
  kron_pack_kernel<<<(unsigned)op.N, 128, 0, s>>>(op, w, a1, a2, out);
}

// out = A^T (a1 + a2) (k entries); a1, a2 svec (a2 may be null)
void launch_kron_apply_t(const KronDev& op, const double* a1, const double* a2, double* out, double* t0, double* t1,
                         int* status, cudaStream_t s) {
  if (op.k <= 0) return;
  kron_unpack_kernel<<<grid_for(op.N * op.N), kKrThreads, 0, s>>>(op, a1, a2, t0);
  double* t = contract_all(op, 1, t0, t1, s);
  kron_gather_kernel<<<(unsigned)((op.k + kKrThreads - 1) / kKrThreads), kKrThreads, 0, s>>>(op.index, op.k, op.Kt,
                                                                                             t, out, status);
}

}  // namespace scs
