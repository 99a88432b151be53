// svec <-> dense maps and small data-movement kernels.
//
// svec is the real symmetric case of the vec_R map of App. D.1: the lower
// triangle column by column, diagonal entries as they are, off-diagonal
// entries times sqrt(2).  Column j starts at offset j*n - j*(j-1)/2.
#include <math.h>

#include "internal.cuh"

namespace scs {

namespace {

__device__ __forceinline__ int64_t svec_col_offset(int64_t n, int64_t j) { return j * n - (j * (j - 1)) / 2; }

// Dense symmetric A (column-major, both triangles) from the svec input.
__global__ void unpack_kernel(const ConeDev* __restrict__ cones, const IoSlot* __restrict__ io, int which) {
  const ConeDev& c = cones[blockIdx.y];
  const double* __restrict__ x = which ? io->g : io->x;
  const int64_t n = c.n;
  const int64_t nn = n * n;
  const double* xs = x + c.xoff;
  // the derivative's input enters scaled by a power of two (kinfo[10])
  const double down = which ? vjp_gscale_down(c.kinfo[10]) : 1.0;
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    const int64_t lo = i >= j ? i : j, hi = i >= j ? j : i;  // (row, col) in the lower triangle
    double v = xs[svec_col_offset(n, hi) + (lo - hi)];
    v *= (lo != hi) ? M_SQRT1_2 * down : down;
    if (!isfinite(v)) bad = true;
    c.A[e] = v;
  }
  if (bad) atomicOr(c.status, ST_NONFINITE);
}

// Cones of side 1: X = (x) has V = (1), l = x, so Pi(x) = max(x, 0) and
// DPi(x)[g] = g for x > 0, 0 otherwise (the derivative taken as 0 at 0).
// offs: [0, count) svec offsets, [count, 2 count) V offsets, [2 count, 3 count) lam offsets,
// [3 count, 4 count) the cone's position in the call (MODE_LMIN: lambda_min = x).
__global__ void trivial_kernel(const int64_t* __restrict__ offs, int count, const IoSlot* __restrict__ io, int mode,
                               int* status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t o = offs[t], ov = offs[count + t], ol = offs[2 * count + t];
  const double v = (mode & MODE_IMPORT) ? io->lam[ol] : io->x[o];
  const bool bad = !isfinite(v) || ((mode & MODE_IMPORT) && !isfinite(io->V[ov]));
  if (bad) atomicOr(status, ST_NONFINITE);
  if (mode & MODE_Y) io->y[o] = bad ? nan("") : (v > 0.0 ? v : 0.0);
  if (mode & MODE_VJP) io->xbar[o] = bad ? nan("") : (v > 0.0 ? io->g[o] : 0.0);
  if (mode & MODE_EXPORT) {
    io->V[ov] = bad ? nan("") : 1.0;
    io->lam[ol] = bad ? nan("") : v;
  }
  if (mode & MODE_LMIN) io->lam[offs[3 * count + t]] = bad ? nan("") : v;
}

// Lower band (bandwidth b) of A into band storage with 2b diagonals; the
// extra diagonals hold the bulge fill and start at zero.
__global__ void band_extract_kernel(const ConeDev* __restrict__ cones) {
  const ConeDev& c = cones[blockIdx.y];
  if (c.path != 0) return;
  const int64_t n = c.n;
  const int ldb = 2 * c.b;
  const int64_t total = n * ldb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / ldb;
    const int d = (int)(e % ldb);
    double v = 0.0;
    if (d <= c.b && col + d < n) v = c.A[(col + d) + col * n];
    c.band[e] = v;
  }
}

__global__ void tridiag_extract_kernel(const ConeDev* __restrict__ cones) {
  const ConeDev& c = cones[blockIdx.y];
  if (c.path != 0) return;
  const int64_t n = c.n;
  const int ldb = 2 * c.b;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    c.d[j] = c.band[j * ldb];
    c.e[j] = (j + 1 < n) ? c.band[j * ldb + 1] : 0.0;
  }
}

__global__ void set_io_kernel(IoSlot* slot, IoSlot v) { *slot = v; }

__global__ void status_reduce_kernel(const int* __restrict__ status, int count, int* out) {
  int v = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) v |= status[i];
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicOr(out, v);
}

}  // namespace

void launch_set_io(IoSlot* slot, const IoSlot& v, cudaStream_t s) { set_io_kernel<<<1, 1, 0, s>>>(slot, v); }

void launch_unpack(const ConeDev* cones, int ncones, int64_t maxn2, const IoSlot* io, int which, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)((maxn2 + 255) / 256);
  if (gx > 1024) gx = 1024;
  unpack_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones, io, which);
}

void launch_trivial(const int64_t* offs, int count, const IoSlot* io, int mode, int* status, cudaStream_t s) {
  if (count <= 0) return;
  trivial_kernel<<<(count + 255) / 256, 256, 0, s>>>(offs, count, io, mode, status);
}

void launch_band_extract(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)((maxn * 2 * kMaxBand + 255) / 256);
  if (gx > 1024) gx = 1024;
  band_extract_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones);
}

void launch_tridiag_extract(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)((maxn + 255) / 256);
  if (gx > 64) gx = 64;
  tridiag_extract_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones);
}

void launch_status_reduce(const int* status, int count, int* out, cudaStream_t s) {
  if (count <= 0) return;
  int g = (count + 255) / 256;
  if (g > 64) g = 64;
  status_reduce_kernel<<<g, 256, 0, s>>>(status, count, out);
}

}  // namespace scs
