// Daleckii-Krein vector-Jacobian product of the PSD projection.
//
// With X = V diag(l) V^T (all n eigenpairs) and G = smat(g),
//     DPi(X)[G] = V (L o (V^T G V)) V^T,
//     L_ij = 1 (l_i > 0, l_j > 0), 0 (l_i <= 0, l_j <= 0),
//            max(l_i, l_j) / |l_i - l_j| otherwise (opposite signs: no
//            cancellation in the divided difference of max(., 0)).
// The derivative map is self-adjoint and svec is an isometry (App. D.1), so
// the svec VJP equals svec(DPi(X)[smat(g)]).
//
// L is constant on blocks: with S the positive eigenpairs and R the rest,
// L = [[1, C], [C^T, 0]], C_ij = l_i / (l_i - l_j).  So with M = V^T G V,
//     DPi(X)[G] = Z1 + Z1^T,  Z1 = V_S X V^T,  X = [M_SS / 2, C o M_SR],
// and only the k_S rows of M and X are formed: 8 k_S n^2 flops instead of
// the 7 n^3 of the dense formula.  When the non-positive pairs are fewer,
// the same holds for 1 - L (1 on their block, 0 on the positive block):
//     DPi(X)[G] = G - (Z1 + Z1^T),  S = {l <= 0}, C_ij = |l_i| / (l_j - l_i).
// The eigenpairs are first reordered so that S comes first (route 0: S =
// {l > 0}; route 1: S = {l <= 0}; the route is the projection's side).  The
// contractions run in the grouped GEMM; this file holds the reordering, the
// elementwise scaling and the final svec packing.  G enters the contractions
// scaled by 2^-s, s the exponent of its largest entry (exact), so that every
// operand lies within FP32's exponent range and the FP64 path may run them
// in double-float arithmetic; the packing scales back.
#include <math.h>

#include "internal.cuh"

namespace scs {

namespace {


// Route and S-first order of the n eigenpairs (one CTA per cone): route 0
// when the positive pairs are at most the negative ones (or opts->side asks
// for it), S = {l > 0}; route 1: S = {l <= 0}.  perm (iperm) gives every
// column its place, S first, each part in its old order; kinfo[6] = |S|.
__global__ void __launch_bounds__(256) vjp_partition_kernel(const ConeDev* __restrict__ cones) {
  const ConeDev& c = cones[blockIdx.x];
  if (*c.status != 0) return;
  const int n = (int)c.n;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  __shared__ int wsum[8], wpos[8], wneg[8];
  __shared__ int sh_route, sh_ks;
  int np = 0, nn = 0;
  for (int j = tid; j < n; j += 256) { np += c.lamk[j] > 0.0; nn += c.lamk[j] < 0.0; }
  for (int o = 16; o > 0; o >>= 1) {
    np += __shfl_xor_sync(0xffffffffu, np, o);
    nn += __shfl_xor_sync(0xffffffffu, nn, o);
  }
  if (lane == 0) { wpos[wid] = np; wneg[wid] = nn; }
  __syncthreads();
  if (tid == 0) {
    int p = 0, q = 0;
    for (int w = 0; w < 8; ++w) { p += wpos[w]; q += wneg[w]; }
    const int side = c.kinfo[4];
    sh_route = side == 1 ? 0 : side == 2 ? 1 : (p <= q ? 0 : 1);
  }
  __syncthreads();
  const int route = sh_route;
  // stable partition by a block scan over contiguous segments
  const int per = (n + 255) / 256;
  const int a0 = min(n, tid * per), a1 = min(n, a0 + per);
  int mine = 0;
  for (int j = a0; j < a1; ++j) {
    const double l = c.lamk[j];
    mine += route == 0 ? (l > 0.0) : (l <= 0.0);
  }
  int incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int w = 0; w < 8; ++w) { const int v = wsum[w]; wsum[w] = run; run += v; }
    sh_ks = run;
  }
  __syncthreads();
  const int ks = sh_ks;
  int sb = wsum[wid] + incl - mine;  // S members before my segment
  for (int j = a0; j < a1; ++j) {
    const double l = c.lamk[j];
    const bool inS = route == 0 ? (l > 0.0) : (l <= 0.0);
    if (inS) c.iperm[j] = sb++;
    else c.iperm[j] = ks + (j - sb);
  }
  if (tid == 0) {
    c.kinfo[1] = route;
    c.kinfo[6] = ks;
  }
}

// Z, lamk -> QA, lamA in the S-first order (pass 1 of the reordering).
__global__ void vjp_permute_kernel(const ConeDev* __restrict__ cones) {
  const ConeDev& c = cones[blockIdx.y];
  if (*c.status != 0) return;
  const int64_t n = c.n, nn = n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    const int64_t d = c.iperm[j];
    c.QA[i + d * n] = c.Z[e];
    if (i == 0) c.lamA[d] = c.lamk[j];
  }
}

// QA, lamA -> Z, lamk (pass 2).
__global__ void vjp_copyback_kernel(const ConeDev* __restrict__ cones) {
  const ConeDev& c = cones[blockIdx.y];
  if (*c.status != 0) return;
  const int64_t n = c.n, nn = n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    c.Z[e] = c.QA[e];
    if (e < n) c.lamk[e] = c.lamA[e];
  }
}

// X = factor o M on the k_S x n block of QB (ld n): factor 1/2 on S x S,
// L (route 0) or 1 - L (route 1) on S x R.
__global__ void vjp_scale_kernel(const ConeDev* __restrict__ cones) {
  const ConeDev& c = cones[blockIdx.y];
  if (*c.status != 0) return;
  const int64_t n = c.n;
  const int ks = c.kinfo[6], route = c.kinfo[1];
  const int64_t tot = (int64_t)ks * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % ks, j = e / ks;
    double f;
    if (j < ks) {
      f = 0.5;
    } else {
      const double li = c.lamk[i], lj = c.lamk[j];
      f = route == 0 ? li / (li - lj) : fabs(li) / (lj - li);
    }
    c.QB[i + j * n] *= f;
  }
}

// kinfo[10] = the largest biased exponent of the cone's g (one CTA per cone).
__global__ void vjp_gexp_kernel(const ConeDev* __restrict__ cones, const IoSlot* __restrict__ io) {
  const ConeDev& c = cones[blockIdx.x];
  const int64_t len = c.n * (c.n + 1) / 2;
  const double* g = io->g + c.xoff;
  int m = 0;
  for (int64_t e = threadIdx.x; e < len; e += blockDim.x) m = max(m, (__double2hiint(g[e]) >> 20) & 0x7FF);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ int wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, wm[w]);
    c.kinfo[10] = m;
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

// xbar = svec(Z1 + Z1^T) (route 0) or svec(G - Z1 - Z1^T) (route 1), with
// Z1 in QB and G in A; NaN on a bad cone.
__global__ void pack_lower_kernel(const ConeDev* __restrict__ cones, const IoSlot* __restrict__ io) {
  const ConeDev& c = cones[blockIdx.y];
  double* xbar = io->xbar;
  const int64_t n = c.n;
  const int64_t len = n * (n + 1) / 2;
  const bool bad = *c.status != 0;
  double* out = xbar + c.xoff;
  const double up = vjp_gscale_up(c.kinfo[10]);  // G was scaled by 1 / up
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x) {
    // invert t -> (i, j), column j starts at j*n - j(j-1)/2
    double jd = ((2.0 * n + 1.0) - sqrt((2.0 * n + 1.0) * (2.0 * n + 1.0) - 8.0 * (double)t)) * 0.5;
    int64_t j = (int64_t)jd;
    if (j < 0) j = 0;
    if (j > n - 1) j = n - 1;
    while (j > 0 && j * n - (j * (j - 1)) / 2 > t) --j;
    while (j + 1 < n && (j + 1) * n - ((j + 1) * j) / 2 <= t) ++j;
    const int64_t i = j + (t - (j * n - (j * (j - 1)) / 2));
    const double sc = (i == j) ? up : M_SQRT2 * up;
    double h = c.QB[i + j * n] + c.QB[j + i * n];
    if (c.kinfo[1] == 1) h = c.A[i + j * n] - h;
    out[t] = bad ? nan("") : sc * h;
  }
}

}  // namespace

void launch_vjp_reorder(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)((maxn * maxn + 255) / 256);
  if (gx > 2048) gx = 2048;
  vjp_partition_kernel<<<ncones, 256, 0, s>>>(cones);
  vjp_permute_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones);
  vjp_copyback_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones);
}

void launch_vjp_gexp(const ConeDev* cones, int ncones, const IoSlot* io, cudaStream_t s) {
  if (ncones <= 0) return;
  vjp_gexp_kernel<<<ncones, 1024, 0, s>>>(cones, io);
}

void launch_vjp_scale(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s) {
  if (ncones <= 0) return;
  int gx = (int)((maxn * maxn / 2 + 255) / 256);
  if (gx > 2048) gx = 2048;
  if (gx < 1) gx = 1;
  vjp_scale_kernel<<<dim3(gx, ncones), 256, 0, s>>>(cones);
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
