// Householder QR of one tall panel of the dense->band reduction, factored by
// a thread-block cluster.
//
// Panel p of a side-n cone covers columns c0 = p*b .. c0+b-1 and rows
// r0 = c0+b .. n-1 (m = n - r0 rows).  Its QR factorisation P = Q R,
// Q = I - V T V^T (compact WY, V unit lower trapezoidal), reduces the panel
// to an upper triangle R, which lands inside the band of width b.
//
// The m x b panel is split by rows over the CTAs of a cluster; each CTA keeps
// its rows in shared memory for the whole factorisation.  Per column the
// norm and the b dot products with the reflector are reduced across the
// cluster through distributed shared memory (each CTA sums the partial sums
// of all ranks in the same order, so every CTA holds bit-identical values).
// Reflectors follow the LAPACK convention: H = I - tau v v^T, v(0) = 1,
// H x = beta e_1 with beta = -sign(alpha) ||x||.  T is accumulated from the
// Gram matrix V^T V by the forward recurrence T(0:j, j) = -tau_j T(0:j,0:j) (V^T v_j).
#include <cooperative_groups.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace scs {

namespace {

constexpr int kPanelThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kPanelThreads) panel_kernel(const ConeDev* __restrict__ cones,
                                                              const int* __restrict__ cone_ids, int panel,
                                                              int b, int R) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int job = blockIdx.x / C;
  const ConeDev& cn = cones[cone_ids[job]];
  const int64_t n = cn.n;
  const int c0 = panel * b;
  const int r0 = c0 + b;
  const int m = (int)n - r0;
  const int bb = min(b, m);
  const bool skip = (*cn.status != 0) || m < 2;  // identical in every CTA of the cluster

  extern __shared__ double smem[];
  const int bp = b + 1;
  double* S = smem;                      // R x bp, row-major (row = panel row)
  double* red1 = S + (size_t)R * bp;     // [2][2]: partial sigma, alpha
  double* red2 = red1 + 4;               // [2][kMaxBand] partial dots
  double* part = red2 + 2 * kMaxBand;    // [8][kMaxBand] per-row-group partials
  double* taus = part + 8 * kMaxBand;    // [kMaxBand]
  double* Gp = taus + kMaxBand;          // [kMaxBand][kMaxBand] partial Gram
  double* Ts = Gp + kMaxBand * kMaxBand; // [kMaxBand][kMaxBand] T (rank 0)
  double* Gw = Ts + kMaxBand * kMaxBand; // [8 warps][kMaxBand][kMaxBand] per-warp Gram partials
  __shared__ double wsum[kPanelThreads / 32];
  __shared__ double sh_beta, sh_tau, sh_scal;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int g0 = rank * R;
  const int BP = (b <= 16) ? 16 : 32;       // lanes per panel row
  const int tc = lane % BP;                 // column of this lane
  const int roff = warp * (32 / BP) + lane / BP;
  const int rstep = (kPanelThreads / 32) * (32 / BP);
  const int nr = skip ? 0 : max(0, min(m - g0, R));
  double* A = cn.A;

  // load my rows of the panel
  for (int c = 0; c < b; ++c)
    for (int i = tid; i < nr; i += kPanelThreads)
      S[i * bp + c] = A[(int64_t)(r0 + g0 + i) + (int64_t)(c0 + c) * n];
  __syncthreads();

  if (!skip) {
    for (int j = 0; j < bb; ++j) {
      const int slot = j & 1;
      // ---- norm of column j below row j, and alpha = P(j, j)
      double ps = 0.0;
      for (int i = tid; i < nr; i += kPanelThreads) {
        const int gi = g0 + i;
        if (gi > j) {
          const double v = S[i * bp + j];
          ps = fma(v, v, ps);
        }
      }
      ps = warp_sum(ps);
      if (lane == 0) wsum[warp] = ps;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kPanelThreads / 32; ++w) t += wsum[w];
        red1[slot * 2 + 0] = t;
        const int jl = j - g0;
        red1[slot * 2 + 1] = (jl >= 0 && jl < nr) ? S[jl * bp + j] : 0.0;
      }
      cluster.sync();
      if (tid == 0) {
        double sigma = 0.0, alpha = 0.0;
        const int owner = j / R;
        for (int r = 0; r < C; ++r) {
          const double* rr = cluster.map_shared_rank(red1, r);
          sigma += rr[slot * 2 + 0];
          if (r == owner) alpha = rr[slot * 2 + 1];
        }
        double beta, tau, scal;
        if (sigma == 0.0) {
          beta = alpha; tau = 0.0; scal = 0.0;
        } else {
          const double nrm = sqrt(fma(alpha, alpha, sigma));
          beta = alpha >= 0.0 ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        sh_beta = beta; sh_tau = tau; sh_scal = scal;
        taus[j] = tau;
      }
      __syncthreads();
      const double tau = sh_tau, scal = sh_scal, beta = sh_beta;
      // ---- v: scale column j below row j; row j keeps beta (R_jj), v_j = 1
      for (int i = tid; i < nr; i += kPanelThreads) {
        const int gi = g0 + i;
        if (gi > j) S[i * bp + j] *= scal;
        else if (gi == j) S[i * bp + j] = beta;
      }
      __syncthreads();
      // ---- w_c = sum_{gi >= j} v_gi P(gi, c), c > j.  Lanes map to columns
      // (BP = 16 or 32 lanes per row), so a warp covers 32/BP rows at a time
      // and every lane issues useful FP64 work.
      const bool colok = tc > j && tc < b;
      if (tau != 0.0) {
        double pd = 0.0;
        if (colok)
          for (int i = roff; i < nr; i += rstep) {
            const int gi = g0 + i;
            if (gi < j) continue;
            const double v = (gi == j) ? 1.0 : S[i * bp + j];
            pd = fma(v, S[i * bp + tc], pd);
          }
        if (BP == 16) pd += __shfl_xor_sync(0xffffffffu, pd, 16);
        if (lane < BP) part[warp * kMaxBand + lane] = pd;
      }
      __syncthreads();
      if (tau != 0.0 && tid < BP) {
        double t = 0.0;
        for (int q = 0; q < kPanelThreads / 32; ++q) t += part[q * kMaxBand + tid];
        red2[slot * kMaxBand + tid] = t;
      }
      cluster.sync();
      if (tau != 0.0) {
        double w = 0.0;
        if (colok)
          for (int r = 0; r < C; ++r) w += cluster.map_shared_rank(red2, r)[slot * kMaxBand + tc];
        const double tw = tau * w;
        if (colok)
          for (int i = roff; i < nr; i += rstep) {
            const int gi = g0 + i;
            if (gi < j) continue;
            const double v = (gi == j) ? 1.0 : S[i * bp + j];
            S[i * bp + tc] = fma(-tw, v, S[i * bp + tc]);
          }
      }
      __syncthreads();
    }
  }

  // ---- outputs: V (m x bb, ld m), R into A, partial Gram V^T V
  double* V = cn.V1 + (int64_t)panel * n * b;
  double* U3 = cn.U3;  // [V | W | V] for the rank-2b trailing update
  if (!skip) {
    for (int c = 0; c < bb; ++c)
      for (int i = tid; i < nr; i += kPanelThreads) {
        const int gi = g0 + i;
        const double v = gi > c ? S[i * bp + c] : (gi == c ? 1.0 : 0.0);
        V[(int64_t)gi + (int64_t)c * m] = v;
        U3[(int64_t)gi + (int64_t)c * m] = v;
        U3[(int64_t)gi + (int64_t)(2 * bb + c) * m] = v;
      }
    for (int c = 0; c < b; ++c)
      for (int i = tid; i < nr; i += kPanelThreads) {
        const int gi = g0 + i;
        const double v = (gi <= c || c >= bb) ? S[i * bp + c] : 0.0;
        A[(int64_t)(r0 + gi) + (int64_t)(c0 + c) * n] = v;
      }
    // partial Gram G(a, c) = sum_rows V(i, a) V(i, c): thread = (row subset, column c)
    double acc[kMaxBand];
#pragma unroll
    for (int a = 0; a < kMaxBand; ++a) acc[a] = 0.0;
    if (tc < bb)
      for (int i = roff; i < nr; i += rstep) {
        const int gi = g0 + i;
        if (gi < tc) continue;  // v_c is zero above row c
        const double vc = gi == tc ? 1.0 : S[i * bp + tc];
#pragma unroll
        for (int a = 0; a < kMaxBand; ++a) {
          if (a < tc) {
            const double va = gi == a ? 1.0 : (gi > a ? S[i * bp + a] : 0.0);
            acc[a] = fma(va, vc, acc[a]);
          }
        }
      }
#pragma unroll
    for (int a = 0; a < kMaxBand; ++a) {
      double v = acc[a];
      if (BP == 16) v += __shfl_xor_sync(0xffffffffu, v, 16);
      acc[a] = v;
    }
    __syncthreads();
    // per-warp partials into Ts (free until rank 0 forms T), then sum over warps
    if (lane < BP) {
#pragma unroll
      for (int a = 0; a < kMaxBand; ++a)
        if (a < bb) Gw[(warp * kMaxBand + a) * kMaxBand + lane] = acc[a];
    }
    __syncthreads();
    for (int e = tid; e < bb * bb; e += kPanelThreads) {
      const int a = e % bb, c = e / bb;
      double g = 0.0;
      if (a < c)
        for (int q = 0; q < kPanelThreads / 32; ++q) g += Gw[(q * kMaxBand + a) * kMaxBand + c];
      Gp[a * kMaxBand + c] = g;
    }
  }
  cluster.sync();
  if (!skip && rank == 0) {
    // G = sum of partial Grams; T by the forward recurrence
    for (int e = tid; e < bb * bb; e += kPanelThreads) {
      const int a = e % bb, c = e / bb;
      double g = 0.0;
      if (a < c)
        for (int r = 0; r < C; ++r) g += cluster.map_shared_rank(Gp, r)[a * kMaxBand + c];
      Gp[a * kMaxBand + c] = g;  // only a < c is used below (own slot, read after sync)
    }
    __syncthreads();
    for (int j = 0; j < bb; ++j) {
      // T(a, j) = -tau_j sum_{q=a}^{j-1} T(a, q) G(q, j)   for a < j
      if (tid < j) {
        double acc = 0.0;
        for (int q = tid; q < j; ++q) acc = fma(Ts[tid * kMaxBand + q], Gp[q * kMaxBand + j], acc);
        Ts[tid * kMaxBand + j] = -taus[j] * acc;
      }
      if (tid == 0) Ts[j * kMaxBand + j] = taus[j];
      for (int a = j + 1 + tid; a < bb; a += kPanelThreads) Ts[a * kMaxBand + j] = 0.0;
      __syncthreads();
    }
    double* T = cn.T1 + (int64_t)panel * b * b;
    for (int e = tid; e < b * b; e += kPanelThreads) {
      const int a = e % b, c = e / b;
      T[a + c * b] = (a < bb && c < bb) ? Ts[a * kMaxBand + c] : 0.0;
    }
  }
  // no CTA may leave while another can still read its shared memory
  cluster.sync();
}

}  // namespace

size_t panel_smem_bytes(int b, int R) {
  return sizeof(double) * ((size_t)R * (b + 1) + 4 + 2 * kMaxBand + 8 * kMaxBand + kMaxBand +
                           2 * kMaxBand * kMaxBand + 8 * kMaxBand * kMaxBand);
}

void launch_panel(const ConeDev* cones, const int* cone_ids, int njobs, int panel, int b, int cluster, int R,
                  cudaStream_t s) {
  if (njobs <= 0) return;
  static std::atomic<unsigned long long> attr_done{0};
  if (first_on_device(attr_done)) {
    cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * cluster, 1, 1);
  cfg.blockDim = dim3(kPanelThreads, 1, 1);
  cfg.dynamicSmemBytes = panel_smem_bytes(b, R);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, panel_kernel, cones, cone_ids, panel, b, R);
}

}  // namespace scs
