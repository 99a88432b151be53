// Per-cone statistics of a projection call: the counts of positive and
// negative eigenvalues, the route taken, the device status, and an FP64
// a-posteriori residual of the result.
//
// The residual is the complementarity term of the optimality conditions of
// the projection.  Y = Pi(X) exactly when Y >= 0, Y - X >= 0 and
// <Y, Y - X> = 0 (the PSD cone is self-dual; App. D.1 states the Moreau
// decomposition this follows from).  The two cone memberships hold by
// construction up to the eigensolver's backward error (Y is formed from the
// kept eigenpairs of one sign), so the statistic reported for every result is
//     c = <Y, Y - X> / (||Y||_F ||X||_F),
// computed in FP64 on the svec buffers, which carry the trace inner product
// (the vec_R map is an isometry).  Writing Y = Pi(X) + E, c equals
// <E, |X|> / (||Y|| ||X||) + ||E||^2 / (||Y|| ||X||), with |X| = 2 Pi(X) - X: to
// first order the error's component along |X|.
//
// x may be overwritten by the call (y may alias x), so the input is copied
// at the start of a call that asks for statistics and the sums read the copy.
#include <math.h>

#include "internal.cuh"

namespace scs {

namespace {

constexpr int kStThreads = 256;

__global__ void stats_save_x_kernel(const IoSlot* __restrict__ io, double* __restrict__ xs, int64_t total) {
  const double* x = io->x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    xs[e] = x[e];
}

// One CTA per (cone, chunk): sums of y (y - x), y y and x x over the chunk,
// combined in a fixed order (the result does not depend on scheduling).
__global__ void __launch_bounds__(kStThreads) stats_part_kernel(const StatsCone* __restrict__ sc,
                                                                const int* __restrict__ part_cone,
                                                                const double* __restrict__ xs,
                                                                const IoSlot* __restrict__ io,
                                                                double* __restrict__ part) {
  __shared__ double red[3][kStThreads / 32];
  const int p = blockIdx.x;
  const StatsCone& c = sc[part_cone[p]];
  const int64_t lo = c.off + (int64_t)(p - c.part0) * kStatsChunk;
  const int64_t hi = min(c.off + c.len, lo + (int64_t)kStatsChunk);
  const double* y = io->y;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t e = lo + threadIdx.x; e < hi; e += kStThreads) {
    const double yv = y[e], xv = xs[e];
    s0 = fma(yv, yv - xv, s0);
    s1 = fma(yv, yv, s1);
    s2 = fma(xv, xv, s2);
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { red[0][w] = s0; red[1][w] = s1; red[2][w] = s2; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int q = 0; q < kStThreads / 32; ++q) t += red[threadIdx.x][q];
    part[3 * (int64_t)p + threadIdx.x] = t;
  }
}

__device__ int status_code(int bits) {
  if (bits & ST_TIMEOUT) return 4;    // SCS_PSD_ETIMEOUT
  if (bits & ST_NOCONV) return 5;     // SCS_PSD_ENOCONV
  if (bits & ST_NONFINITE) return 6;  // SCS_PSD_ENONFINITE
  return bits ? 1 : 0;
}

// One thread per cone of the call: the partial sums in order, the counts and
// route from the cone's final merge (side-1 cones: the sign of x), the status.
__global__ void stats_final_kernel(const StatsCone* __restrict__ sc, int count, const ConeDev* __restrict__ cones,
                                   const int* __restrict__ triv_status, const double* __restrict__ part,
                                   const double* __restrict__ xs, ConeStats* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const StatsCone& c = sc[i];
  double yz = 0.0, yy = 0.0, xx = 0.0;
  for (int q = 0; q < c.nparts; ++q) {
    yz += part[3 * (int64_t)(c.part0 + q)];
    yy += part[3 * (int64_t)(c.part0 + q) + 1];
    xx += part[3 * (int64_t)(c.part0 + q) + 2];
  }
  ConeStats r;
  r.k_pos = 0; r.k_neg = 0; r.route = 0; r.status = 0;
  if (c.cone >= 0) {
    const ConeDev& d = cones[c.cone];
    const int bits = *d.status;
    r.status = status_code(bits);
    if (!bits) {
      r.k_pos = d.kinfo[8];
      r.k_neg = d.kinfo[9];
      r.route = d.kinfo[1];
    }
  } else if (c.side == 1) {
    const double v = xs[c.off];
    r.k_pos = v > 0.0;
    r.k_neg = v < 0.0;
    r.status = isfinite(v) ? 0 : status_code(*triv_status);
  }
  const double ny = sqrt(yy), nx = sqrt(xx);
  r.norm_y = ny;
  r.norm_x = nx;
  r.complementarity = (ny > 0.0 && nx > 0.0) ? yz / (ny * nx) : (isfinite(yz) ? 0.0 : yz);
  r.reserved = 0.0;
  out[i] = r;
}

}  // namespace

void launch_stats_save_x(const IoSlot* io, double* xs, int64_t total, cudaStream_t s) {
  if (total <= 0) return;
  int g = (int)((total + 255) / 256);
  if (g > 1024) g = 1024;
  stats_save_x_kernel<<<g, 256, 0, s>>>(io, xs, total);
}

void launch_stats(const StatsCone* sc, int count, const int* part_cone, int nparts, const ConeDev* cones,
                  const int* triv_status, const double* xs, const IoSlot* io, double* part, ConeStats* out,
                  cudaStream_t s) {
  if (count <= 0) return;
  if (nparts > 0) stats_part_kernel<<<nparts, kStThreads, 0, s>>>(sc, part_cone, xs, io, part);
  stats_final_kernel<<<(count + 127) / 128, 128, 0, s>>>(sc, count, cones, triv_status, part, xs, out);
}

}  // namespace scs
