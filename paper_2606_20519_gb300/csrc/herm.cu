// Complex Hermitian cones through the real symmetric embedding.
//
// The paper's cones are complex Hermitian (its vec map of App. D.1 carries
// sqrt(2) Re X_ij and sqrt(2) Im X_ij).  For X = A + iB (A symmetric, B
// antisymmetric) the real matrix
//     M = [[A, -B], [B, A]]   (side 2n, symmetric)
// has every eigenvalue of X twice, and since the embedding respects sums,
// products and adjoints, Pi(M) is the embedding of Pi(X): the real solver on
// M gives Pi(X) exactly (up to rounding).  These kernels move between the
// Hermitian svec (per column j the diagonal entry, then sqrt(2) Re X_ij,
// sqrt(2) Im X_ij for i > j; n^2 reals, column j starting at j(2n - j)) and
// the real svec of M; every entry of one is +-1 times an entry of the other,
// or zero.
#include "internal.cuh"

namespace scs {

namespace {

// meta per cone: n, offset in the Hermitian buffer, offset in the real buffer
__device__ __forceinline__ int64_t hcol(int64_t n, int64_t j) { return j * (2 * n - j); }
__device__ __forceinline__ int64_t rcol(int64_t N, int64_t c) { return c * N - (c * (c - 1)) / 2; }

// real svec of M from the Hermitian svec; blockIdx.y = cone, columns of M over blockIdx.x
__global__ void herm_embed_kernel(const int64_t* __restrict__ meta, const double* __restrict__ hs,
                                  double* __restrict__ ms) {
  const int64_t n = meta[3 * blockIdx.y], ho = meta[3 * blockIdx.y + 1], ro = meta[3 * blockIdx.y + 2];
  const int64_t N = 2 * n;
  const double* h = hs + ho;
  double* m = ms + ro;
  for (int64_t c = blockIdx.x; c < N; c += gridDim.x) {
    for (int64_t r = c + threadIdx.x; r < N; r += blockDim.x) {
      double v;
      if (r < n || c >= n) {
        // a diagonal block: A (top-left or bottom-right)
        const int64_t i = r < n ? r : r - n, j = c < n ? c : c - n;
        v = (i == j) ? h[hcol(n, j)] : h[hcol(n, j) + 1 + 2 * (i - j - 1)];
      } else {
        // bottom-left block: B(i, j) = Im X_ij, an off-diagonal entry of M
        const int64_t i = r - n, j = c;
        if (i > j) v = h[hcol(n, j) + 2 + 2 * (i - j - 1)];
        else if (i < j) v = -h[hcol(n, i) + 2 + 2 * (j - i - 1)];
        else v = 0.0;
      }
      m[rcol(N, c) + (r - c)] = v;
    }
  }
}

// Hermitian svec of Pi(X) from the real svec of Pi(M) (top-left and bottom-left blocks)
__global__ void herm_extract_kernel(const int64_t* __restrict__ meta, const double* __restrict__ ms,
                                    double* __restrict__ hs) {
  const int64_t n = meta[3 * blockIdx.y], ho = meta[3 * blockIdx.y + 1], ro = meta[3 * blockIdx.y + 2];
  const int64_t N = 2 * n;
  const double* m = ms + ro;
  double* h = hs + ho;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const int64_t hc = hcol(n, j), rc = rcol(N, j);
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) {
      if (i == j) {
        h[hc] = m[rc];
      } else {
        h[hc + 1 + 2 * (i - j - 1)] = m[rc + (i - j)];      // sqrt(2) Re X_ij
        h[hc + 2 + 2 * (i - j - 1)] = m[rc + (n + i - j)];  // sqrt(2) Im X_ij
      }
    }
  }
}

}  // namespace

void launch_herm_embed(const int64_t* meta, int count, int64_t maxn, const double* hs, double* ms, cudaStream_t s) {
  if (count <= 0 || maxn <= 0) return;
  int gx = (int)(2 * maxn);
  if (gx > 1024) gx = 1024;
  herm_embed_kernel<<<dim3(gx, count), 128, 0, s>>>(meta, hs, ms);
}

void launch_herm_extract(const int64_t* meta, int count, int64_t maxn, const double* ms, double* hs, cudaStream_t s) {
  if (count <= 0 || maxn <= 0) return;
  int gx = (int)maxn;
  if (gx > 1024) gx = 1024;
  herm_extract_kernel<<<dim3(gx, count), 128, 0, s>>>(meta, ms, hs);
}

}  // namespace scs
