// C-ABI of the scs_psd library: handles, plans, workspace and the launch
// sequence of the projection pipeline (see internal.cuh for the steps).
//
// A plan is built once per list of cone sides (and options): it lays out the
// device workspace, precomputes every launch's work list (panel jobs, GEMM
// descriptors with device-side sizes, bulge-chasing CTA assignment, merge
// nodes of each divide-and-conquer level) and uploads them.  Later calls with
// the same shapes replay the same launch sequence; the sequence is recorded as
// a CUDA graph the first time and updated in place when the data pointers
// change.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/scs_psd.h"
#include "internal.cuh"

using namespace scs;

namespace {

constexpr int kDefaultBand = 16;
// auto: one-stage tridiagonalisation up to this side (measured faster than the
// two-stage route at every side up to 4096 on this part, FP64 and split)
constexpr int64_t kOneStageMax = 6144;
constexpr long long kDefaultWaitCycles = 4000000000LL;  // ~2 s at 2 GHz
constexpr int64_t kMaxSide = 8192;

struct GemmLaunch {
  int desc_off = 0, count = 0, prefix_off = 0, tiles = 0;
  int variant = GEMM_SQUARE, needs_reduce = 0;
  int tc = 0;  // 1: split-TF32 tensor-core kernel
  int tc2 = 0;  // 1: long-contraction split-TF32 kernel (operands sliced once per launch)
  int sjob_off = 0, njobs = 0, sprefix_off = 0, sctas = 0;  // its slice jobs
  int64_t max_mn = 0;
};

// One launch of the long-contraction kernel's slicing step over a list of operands.
struct SliceLaunch {
  int sjob_off = 0, njobs = 0, sprefix_off = 0, sctas = 0;
};

struct PanelStep {
  int panel = 0, njobs = 0, cluster = 1, R = 0;
  int ids_off = 0;  // offset into the int metadata
  GemmLaunch g[6];
};

struct BulgeLaunch {
  int nctas = 0, ncones = 0;
  int cone_off = 0, rank_off = 0, count_off = 0;
};

struct Sytrd1Launch {
  int nctas = 0, maxn = 0;
  size_t smem = 0;
  int glb = 0;  // columns in L2 computed in double-float (else FP64)
  int cone_off = 0, rank_off = 0, count_off = 0;
};

struct Level {
  int nnodes = 0, maxK = 0;
  int nodes_off = 0;  // into MergeNode metadata
  int pos_off = 0;    // into int metadata (2 * total)
  GemmLaunch g;
};

// Launch-shape choices of a plan: the ones the autotuner searches.
struct Tuning {
  int band = 0;       // 0: automatic path (one-stage up to kOneStageMax), 1: one-stage, 2..32: two-stage width
  int gemm_ctas = 2;  // grouped GEMMs: split K until a launch has about this many CTAs per SM
  int bt1_cols = 8;   // fused stage-1 back-transformation: columns per CTA slab, at most
  int sy_share = 1;   // one-stage tridiagonalisation: a large cone's group has at most SMs / sy_share CTAs
  std::string str() const {
    char b[64];
    snprintf(b, sizeof(b), "t%d,%d,%d,%d", band, gemm_ctas, bt1_cols, sy_share);
    return b;
  }
};

struct Plan {
  std::string key;
  Tuning tune;
  int b = kDefaultBand;
  int allv = 0, side = 0, precision = SCS_PSD_FP64;
  GemmLaunch recon_tc;  // split mode: S = Z diag(l) Z^T on the tensor cores
  // shapes
  std::vector<int32_t> sides;
  std::vector<int64_t> offsets;
  int ncones = 0;  // cones with n >= 2
  int64_t maxn = 0;
  int ntriv = 0;
  int64_t total_pos = 0;
  // device memory
  void* cone_mem = nullptr;
  void* meta_mem = nullptr;
  ConeDev* cones_d = nullptr;
  int* ints_d = nullptr;
  GemmDesc* descs_d = nullptr;
  SliceJob* sjobs_d = nullptr;  // slice jobs of the long-contraction products (split mode)
  MergeNode* nodes_d = nullptr;
  int64_t* triv_offs_d = nullptr;  // 4 * ntriv: svec, V and lam offsets and call positions of the side-1 cones
  int64_t vtotal = 0, ltotal = 0;   // doubles of a stored eigendecomposition (sum n^2, sum n)
  int* status_d = nullptr;  // ncones + 1 (last: trivial cones)
  int* prog_d = nullptr;
  size_t prog_count = 0;
  // steps
  std::vector<PanelStep> panels;
  std::vector<BulgeLaunch> bulges;
  std::vector<Sytrd1Launch> sytrd1;
  int nlarft = 0, larft_cone_off = 0, larft_idx_off = 0;
  std::vector<Level> levels;
  std::vector<GemmLaunch> bt1;  // 3 per panel, reverse order
  int bt1k_nctas = 0, bt1k_cone_off = 0, bt1k_rank_off = 0, bt1k_count_off = 0, bt1k_maxn = 0;  // fused kernel
  GemmLaunch vjp[4];
  int64_t launches = 0;
  IoSlot* io_d = nullptr;  // the caller's buffers of the current call
  // Recorded launch sequences, one per output mode (MODE_* bits),
  // with the wait limit they were recorded with.
  int64_t eager_runs = 0;
  cudaGraphExec_t gexec[kModes] = {};
  long long gwait[kModes] = {};
  int64_t glaunches[kModes] = {};
  bool gfailed[kModes] = {};
  bool arena_owned = false;  // memory carved from a caller-provided region (not freed here)
  // complex Hermitian cones reduced natively (herm): the cones' complex
  // workspace, the reduction's CTA groups, the T-factor blocks, the
  // back-transformation's CTAs
  bool herm = false;
  void* hmem = nullptr;
  HConeDev* hcones_d = nullptr;
  std::vector<Sytrd1Launch> hetrd;
  int hlarft_n = 0, hlarft_cone_off = 0, hlarft_idx_off = 0;
  int hbt_nctas = 0, hbt_cone_off = 0, hbt_rank_off = 0, hbt_count_off = 0;
  // per-cone statistics (allocated by the first call that asks for them)
  void* stats_mem = nullptr;
  StatsCone* stats_cones_d = nullptr;
  int* stats_part_cone_d = nullptr;
  double* stats_part_d = nullptr;
  double* stats_xs_d = nullptr;
  ConeStats* stats_out_d = nullptr;
  int stats_nparts = 0;
  int64_t stats_total = 0;
  ~Plan() {
    for (cudaGraphExec_t ge : gexec)
      if (ge) cudaGraphExecDestroy(ge);
    if (!arena_owned && cone_mem) cudaFree(cone_mem);
    if (!arena_owned && meta_mem) cudaFree(meta_mem);
    if (stats_mem) cudaFree(stats_mem);
    if (hmem) cudaFree(hmem);
  }
};

// A shape list of complex Hermitian cones: the real side-2n embeddings'
// shapes and a device buffer for their svec.
struct HermPlan {
  std::vector<int64_t> roff;   // real offsets (count + 1)
  std::vector<int32_t> rsides; // 2 n
  int64_t maxn = 0;
  int64_t* meta_d = nullptr;   // per cone: n, Hermitian offset, real offset
  double* buf = nullptr;       // roff[count] doubles
  ~HermPlan() {
    if (meta_d) cudaFree(meta_d);
    if (buf) cudaFree(buf);
  }
};

// Positivity post-processing of a shape list and grouping: device copies of
// the groups, the per-cone (offset, side, group) table, and buffers for the
// blocks' lambda_min, the groups' nu and the mixing weights.
struct MixPlan {
  int count = 0, ngroups = 0;
  int64_t maxn = 0;
  void* mem = nullptr;
  int* groups_d = nullptr;
  int64_t* meta_d = nullptr;
  double* lam_d = nullptr;
  double* nu_d = nullptr;
  double* p_d = nullptr;
  ~MixPlan() {
    if (mem) cudaFree(mem);
  }
};

// Workspace of the SCS iteration for one (m, k): p = M^{-1}(c, b), 1 + h.p,
// z, A^T w, dot partials, tau~, the projection's input and u~_y.
struct ScsPlan {
  int64_t m = 0, k = 0;
  void* mem = nullptr;
  double *p = nullptr, *hp = nullptr, *z = nullptr, *tk = nullptr, *part = nullptr, *tau = nullptr;
  double *tin = nullptr, *uty = nullptr;
  double* tpart = nullptr;  // dense A^T: row-chunk partial dot products
  int tchunks = 1;
  // structured operator: two work tensors of N^2 doubles and a status word
  void* kmem = nullptr;
  int64_t kdoubles = 0;
  double *t0 = nullptr, *t1 = nullptr;
  int* kstatus = nullptr;
  ~ScsPlan() {
    if (mem) cudaFree(mem);
    if (kmem) cudaFree(kmem);
  }
};

// Factorization-free approximate projection of a shape list: the composite's
// coefficients, the per-cone buffers (X, two iterates, S^2 / Y) and the
// grouped GEMMs of every step, in launch order.
struct PolyPlan {
  int precision = SCS_PSD_FP64;
  int steps = 0;
  double nsq = 1.0;  // ||X||_F^2 = nsq * ||svec||^2 (1/2 for the real embedding of a Hermitian cone)
  int ncones = 0, nparts = 0;
  int64_t maxn = 0;
  void* work = nullptr;
  void* meta = nullptr;
  PolyConeDev* cones_d = nullptr;
  int* ints_d = nullptr;  // tile prefixes, partial-sum owners, status
  GemmDesc* descs_d = nullptr;
  int* part_cone_d = nullptr;
  int* status_d = nullptr;
  double* part_d = nullptr;
  double* inv_d = nullptr;
  IoSlot* io_d = nullptr;
  SliceJob* sjobs_d = nullptr;
  std::vector<GemmLaunch> gemms;
  std::vector<SliceLaunch> slices;
  struct Op {
    int kind;  // 0: gemms[idx], 1: slices[idx], 2: mirror of the new iterate (idx: 0 = S1, 1 = S0)
    int idx;
  };
  std::vector<Op> ops;
  int64_t eager_runs = 0, launches = 0, glaunches = 0;
  cudaGraphExec_t gexec = nullptr;
  bool gfailed = false;
  ~PolyPlan() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (work) cudaFree(work);
    if (meta) cudaFree(meta);
  }
};

}  // namespace

struct scs_psd_handle_s {
  int device = 0;
  int sms = 0;
  bool trace = false;
  bool last_replayed = false;
  cudaStream_t capture_stream = nullptr;  // records graphs; never executes work
  // second stream for work that overlaps the divide and conquer (the T factors
  // of the one-stage reflectors); joined back with events before it is needed
  bool use_aux = false;
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> trace_ev;
  int* status_word = nullptr;  // device
  cudaStream_t last_stream = nullptr;
  int64_t last_launches = 0;
  std::string last_stats_key;  // plan of the last call that recorded statistics ("" if none)
  int32_t last_stats_count = 0;
  std::map<std::string, std::unique_ptr<Plan>> plans;
  std::map<std::string, Tuning> tuned;  // autotuner's choices by shapes and precision
  std::map<std::string, std::unique_ptr<HermPlan>> herm;  // Hermitian shape lists
  std::map<std::string, std::unique_ptr<PolyPlan>> poly;  // polynomial projections by shapes and schedule
  std::map<std::string, std::unique_ptr<MixPlan>> mix;    // positivity post-processing by shapes and groups
  std::map<std::pair<int64_t, int64_t>, std::unique_ptr<ScsPlan>> scs;  // SCS iterations by (m, k)
  Tuning last_tune;
  std::mutex mu;
};

namespace {

size_t align_up(size_t v, size_t a = 256) { return (v + a - 1) / a * a; }

int64_t svec_len(int64_t n) { return n * (n + 1) / 2; }

int num_panels(int64_t n, int b) { return n - 2 >= b ? (int)((n - 2) / b) : 0; }

int num_levels(int64_t n) {
  int L = 0;
  while ((int64_t(1) << L) < n) ++L;
  return L;
}

// ---- per-cone workspace layout
struct ConeLayout {
  size_t off[40];
  size_t bytes;
};

enum Field {
  F_A, F_BAND, F_REFL, F_D, F_E, F_V1, F_T1, F_Y, F_X, F_U3, F_MB, F_NB, F_QA, F_QB, F_LAMA, F_LAMB, F_QIN, F_UCM, F_Z,
  F_LAMK, F_DSRT, F_ZK, F_DVAL, F_TAU, F_ZHAT, F_ROT, F_RHO, F_IPERM, F_IFP, F_IROT, F_IORG, F_IMAP, F_ICNT,
  F_KINFO, F_TAU1, F_NFIELDS
};

int num_blocks1(int64_t n) { return n >= 3 ? (int)((n - 2 + kSy1Block - 1) / kSy1Block) : 0; }

ConeLayout cone_layout(int64_t n, int b, int path) {
  ConeLayout L{};
  const int P = path ? 0 : num_panels(n, b);
  const int Q = path ? num_blocks1(n) : 0;
  const int bw = std::max(b, kSy1Block);
  const int64_t nsw = path ? 0 : std::max<int64_t>(0, n - 2);
  const int64_t kmax = (n >= 3 ? (n - 3) / b + 1 : 0) + 1;
  const size_t d = sizeof(double), i4 = sizeof(int);
  const size_t sz[F_NFIELDS] = {
      d * n * n, d * n * 2 * b, d * nsw * kmax * (b + 1), d * n, d * n,
      d * std::max<int64_t>((int64_t)P * n * b, (int64_t)Q * n * kSy1Block),
      d * std::max<int64_t>((int64_t)P * b * b, (int64_t)Q * kSy1Block * kSy1Block),
      d * n * bw, d * n * bw + d * 2048, d * n * 3 * b, d * b * b, d * b * b, d * n * n, d * n * n, d * n, d * n,
      d * n * n, d * n * n, d * n * n, d * n, d * n, d * n, d * n, d * n, d * n, d * 2 * n, d * n,
      i4 * n, i4 * n, i4 * 2 * n, i4 * n, i4 * n, i4 * 4 * n, i4 * 16, d * n};
  size_t o = 0;
  for (int f = 0; f < F_NFIELDS; ++f) {
    o = align_up(o);
    L.off[f] = o;
    o += std::max<size_t>(sz[f], 8);
  }
  L.bytes = align_up(o);
  return L;
}

#define CUDA_TRY(expr)                        \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return SCS_PSD_ECUDA; \
  } while (0)

struct MetaBuilder {
  std::vector<int> ints;
  std::vector<GemmDesc> descs;
  std::vector<int64_t> part_off;  // per descriptor: offset in the split-K scratch (doubles)
  std::vector<MergeNode> nodes;
  int sms = 148;
  int gemm_ctas = 2;   // split-K target, CTAs per SM
  int64_t scratch_doubles = 0;
  bool split = false;  // use the split-TF32 tensor-core kernel where the shape suits it
  bool tc2 = false;    // with split: the long-contraction kernel (operands sliced once per launch)
  std::vector<SliceJob> sjobs;
  std::vector<int64_t> sjob_out;      // per slice job: offset of its output in the slice scratch (floats)
  std::vector<int64_t> desc_as, desc_bs;  // per descriptor: slice-scratch offsets of op(A), op(B) (-1: none)
  int64_t slice_floats = 0;

  // The long-contraction kernel: tiles 128 x 128, one CTA per SM, split K in
  // 64-wide groups; one slice job per operand of every problem.
  // One launch of the slicing kernel over these operands (their outputs set by the caller).
  SliceLaunch add_slices(const std::vector<SliceJob>& jobs) {
    SliceLaunch L;
    L.sjob_off = (int)sjobs.size();
    L.njobs = (int)jobs.size();
    L.sprefix_off = (int)ints.size();
    int sct = 0;
    for (const SliceJob& j : jobs) {
      ints.push_back(sct);
      sjobs.push_back(j);
      sjob_out.push_back(-1);
      sct += tc2_slice_ctas(j.rows, j.K);
    }
    ints.push_back(sct);
    L.sctas = sct;
    return L;
  }

  // make_jobs = false: the descriptors' As / Bs already point at sliced operands.
  GemmLaunch add_gemm_tc2(std::vector<GemmDesc> probs, bool make_jobs = true) {
    GemmLaunch g;
    g.tc2 = 1;
    g.desc_off = (int)descs.size();
    g.count = (int)probs.size();
    g.prefix_off = (int)ints.size();
    int64_t base = 0;
    for (const GemmDesc& p : probs) {
      int64_t tiles = (int64_t)((p.M + 127) / 128) * ((p.N + 127) / 128);
      if (p.flags & GF_LOWER_C) tiles = (tiles + (p.M + 127) / 128) / 2 + 1;
      base += tiles;
    }
    int S = 1;
    const int64_t want = sms;
    if (base > 0 && base < want) S = (int)std::min<int64_t>(64, (want + base - 1) / base);
    int t = 0;
    int64_t off = 0, soff = 0;
    std::vector<int> sprefix;
    int sct = 0;
    g.sjob_off = (int)sjobs.size();
    for (GemmDesc& p : probs) {
      const int Sp = std::max(1, std::min(S, (p.K + 127) / 128));  // at least two 64-wide groups per piece
      p.splitk = Sp;
      ints.push_back(t);
      t += ((p.M + 127) / 128) * ((p.N + 127) / 128) * Sp;
      part_off.push_back(Sp > 1 ? off : -1);
      if (Sp > 1) { off += (int64_t)Sp * p.M * p.N; g.needs_reduce = 1; }
      g.max_mn = std::max<int64_t>(g.max_mn, (int64_t)p.M * p.N);
      if (!make_jobs) {
        desc_as.push_back(-1);
        desc_bs.push_back(-1);
        descs.push_back(p);
        continue;
      }
      const int fl = p.flags;
      SliceJob ja{p.A, nullptr, nullptr, p.lda, p.M, p.K, (fl & GF_SYM_A) ? 2 : ((fl & GF_TRANS_A) ? 1 : 0),
                  p.dynM, p.dynK};
      SliceJob jb{p.B, (fl & GF_SCALE_B) ? p.bscale : nullptr, nullptr, p.ldb, p.N, p.K, (fl & GF_TRANS_B) ? 0 : 1,
                  p.dynN, p.dynK};
      desc_as.push_back(soff);
      sjobs.push_back(ja); sjob_out.push_back(soff); sprefix.push_back(sct);
      soff += tc2_slice_floats(p.M, p.K); sct += tc2_slice_ctas(p.M, p.K);
      desc_bs.push_back(soff);
      sjobs.push_back(jb); sjob_out.push_back(soff); sprefix.push_back(sct);
      soff += tc2_slice_floats(p.N, p.K); sct += tc2_slice_ctas(p.N, p.K);
      descs.push_back(p);
    }
    ints.push_back(t);
    g.tiles = t;
    g.njobs = (int)sjobs.size() - g.sjob_off;
    g.sprefix_off = (int)ints.size();
    ints.insert(ints.end(), sprefix.begin(), sprefix.end());
    ints.push_back(sct);
    g.sctas = sct;
    scratch_doubles = std::max(scratch_doubles, off);
    slice_floats = std::max(slice_floats, soff);
    return g;
  }

  // Picks the engine and tile shape for the launch and a split-K factor per
  // problem so that the launch has about two CTAs per SM.  bounded: every
  // operand lies well inside FP32's exponent range (eigenvector blocks, and
  // their products with a matrix scaled to its largest entry), so the FP64
  // path may run the 64 x 64 tiles in double-float arithmetic.
  GemmLaunch add_gemm(std::vector<GemmDesc> probs, bool bounded = false) {
    if (split && tc2 && !probs.empty()) {
      // long contractions go to the kernel whose operands are sliced once per product
      int maxM = 0, minK = 1 << 30;
      for (const GemmDesc& p : probs) {
        maxM = std::max(maxM, p.M);
        minK = std::min(minK, p.K);
      }
      if (maxM >= 128 && minK >= 256) return add_gemm_tc2(probs);
    }
    GemmLaunch g;
    g.desc_off = (int)descs.size();
    g.count = (int)probs.size();
    g.prefix_off = (int)ints.size();
    int maxM = 0, maxN = 0, minK = 1 << 30;
    double fma_total = 0.0;
    int64_t tiles64 = 0;
    for (const GemmDesc& p : probs) {
      maxM = std::max(maxM, p.M);
      maxN = std::max(maxN, p.N);
      minK = std::min(minK, p.K);
      fma_total += (double)p.M * p.N * p.K;
      tiles64 += (int64_t)((p.M + 63) / 64) * ((p.N + 63) / 64);
    }
    int bm, bn;
    g.tc = (split && maxM >= 64 && minK >= 32 && !probs.empty()) ? 1 : 0;
    if (g.tc) {
      g.variant = (maxN <= 16) ? TC_N16 : TC_N64;
      tc_tile_shape(g.variant, &bm, &bn);
    } else {
      g.variant = (maxM <= 16 && maxN <= 16) ? GEMM_SMALL
                  : (maxN <= 16) ? GEMM_TALL : (maxM <= 16) ? GEMM_SHORT : GEMM_SQUARE;
      // few small products (fewer 64 x 64 tiles than SMs, at most 16M FMA in
      // all): 16 x 16 FP64 tiles spread them over every SM, where 64 x 64
      // tiles left most SMs idle (the divide and conquer's merges of 32 .. 128
      // rows at n = 625 took 37 .. 44 us each in 64 x 64 tiles)
      if (g.variant == GEMM_SQUARE && tiles64 < sms && fma_total <= 16.0 * 1024 * 1024) g.variant = GEMM_SMALL;
      if (bounded && g.variant == GEMM_SQUARE && minK >= 32) g.variant = GEMM_SQUARE_DF;
      gemm_tile_shape(g.variant, &bm, &bn);
    }
    int64_t base = 0;
    for (const GemmDesc& p : probs) {
      int64_t tiles = (int64_t)((p.M + bm - 1) / bm) * ((p.N + bn - 1) / bn);
      if (p.flags & GF_LOWER_C) tiles = (tiles + (p.M + bm - 1) / bm) / 2 + 1;
      base += tiles;
    }
    int S = 1;
    const int64_t want = (int64_t)gemm_ctas * sms;
    if (base > 0 && base < want) S = (int)std::min<int64_t>(64, (want + base - 1) / base);
    int t = 0;
    int64_t off = 0;
    for (GemmDesc& p : probs) {
      const int Sp = std::max(1, std::min(S, p.K / (g.tc ? 128 : 32)));
      p.splitk = Sp;
      ints.push_back(t);
      const int tm = (p.M + bm - 1) / bm, tn = (p.N + bn - 1) / bn;
      t += std::max(0, tm * tn) * Sp;
      part_off.push_back(Sp > 1 ? off : -1);
      if (Sp > 1) { off += (int64_t)Sp * p.M * p.N; g.needs_reduce = 1; }
      g.max_mn = std::max<int64_t>(g.max_mn, (int64_t)p.M * p.N);
      descs.push_back(p);
      desc_as.push_back(-1);
      desc_bs.push_back(-1);
    }
    ints.push_back(t);
    scratch_doubles = std::max(scratch_doubles, off);
    g.tiles = t;
    return g;
  }
};

GemmDesc mk(const double* A, int lda, const double* B, int ldb, double* C, int ldc, int M, int N, int K,
            double alpha, double beta, int flags, const int* skip) {
  GemmDesc g{};
  g.A = A; g.B = B; g.C = C;
  g.lda = lda; g.ldb = ldb; g.ldc = ldc;
  g.M = M; g.N = N; g.K = K;
  g.alpha = alpha; g.beta = beta;
  g.flags = flags;
  g.skip = skip;
  g.splitk = 1;
  return g;
}

// Optional device region to carve the plan's memory from instead of
// cudaMalloc; metadata is then uploaded with cudaMemcpyAsync on `stream`.
struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  cudaStream_t stream = nullptr;
  void* take(size_t bytes) {
    const size_t o = align_up(used);
    if (o + bytes > size) return nullptr;
    used = o + bytes;
    return base + o;
  }
};

int build_plan(scs_psd_handle h, Plan& P, const int32_t* sides, int32_t count, int b, int allv, int side,
               int precision, int onestage, const Tuning& tune, Arena* arena = nullptr, bool herm = false) {
  P.tune = tune;
  P.b = b;
  P.allv = allv;
  P.side = side;
  P.precision = precision;
  P.herm = herm;
  if (herm) onestage = 1;  // the complex reduction hands over a tridiagonal form
  P.sides.assign(sides, sides + count);
  P.offsets.resize(count + 1);
  P.offsets[0] = 0;
  for (int i = 0; i < count; ++i)
    P.offsets[i + 1] = P.offsets[i] + (herm ? (int64_t)sides[i] * sides[i] : svec_len(sides[i]));

  // ---- cones of the main path (n >= 2) and trivial ones
  std::vector<int> big;
  std::vector<int64_t> triv_offs, triv_voff, triv_loff, triv_idx;
  std::vector<int64_t> voff(count + 1, 0), loff(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    voff[i + 1] = voff[i] + (int64_t)sides[i] * sides[i];
    loff[i + 1] = loff[i] + sides[i];
  }
  P.vtotal = voff[count];
  P.ltotal = loff[count];
  for (int i = 0; i < count; ++i) {
    if (sides[i] >= 2) big.push_back(i);
    else if (sides[i] == 1) {
      triv_offs.push_back(P.offsets[i]);
      triv_voff.push_back(voff[i]);
      triv_loff.push_back(loff[i]);
      triv_idx.push_back(i);
    }
  }
  P.ncones = (int)big.size();
  P.ntriv = (int)triv_offs.size();
  triv_offs.insert(triv_offs.end(), triv_voff.begin(), triv_voff.end());
  triv_offs.insert(triv_offs.end(), triv_loff.begin(), triv_loff.end());
  triv_offs.insert(triv_offs.end(), triv_idx.begin(), triv_idx.end());
  std::vector<ConeLayout> lay(P.ncones);
  std::vector<int> path(P.ncones);
  size_t cone_bytes = 0;
  std::vector<size_t> cone_base(P.ncones);
  for (int c = 0; c < P.ncones; ++c) {
    const int64_t n = sides[big[c]];
    P.maxn = std::max(P.maxn, n);
    // one-stage needs its vectors in shared memory: at most about 7600 (else two-stage)
    const bool fits1 = sytrd1_smem_bytes((int)n, 1, false) <= 200 * 1024;
    path[c] = (onestage == 1) ? (fits1 ? 1 : 0) : (onestage == 0 ? 0 : (n <= kOneStageMax ? 1 : 0));
    lay[c] = cone_layout(n, b, path[c]);
    cone_base[c] = cone_bytes;
    cone_bytes += lay[c].bytes;
  }
  if (cone_bytes) {
    if (arena) {
      P.arena_owned = true;
      if (!(P.cone_mem = arena->take(cone_bytes))) return SCS_PSD_ENOMEM;
    } else if (cudaMalloc(&P.cone_mem, cone_bytes) != cudaSuccess) {
      return SCS_PSD_ENOMEM;
    }
  }
  char* base = (char*)P.cone_mem;

  // ---- metadata sizes known up front: status (ncones+1), prog
  MetaBuilder mb;
  mb.sms = h->sms > 0 ? h->sms : 148;
  mb.gemm_ctas = std::max(1, tune.gemm_ctas);
  mb.split = (precision == SCS_PSD_SPLIT_TF32);
  mb.tc2 = mb.split;
  std::vector<ConeDev> cones(P.ncones);
  size_t prog_total = 0;
  std::vector<size_t> prog_off(P.ncones);
  for (int c = 0; c < P.ncones; ++c) {
    prog_off[c] = prog_total;
    // bulge progress counters (n - 2), or the one-stage barrier's 8 counters 32 ints apart
    prog_total += std::max<int64_t>(256, sides[big[c]] - 2);
  }
  // ints layout: [status (ncones+1)] [prog] [rest...]
  const int status_off = 0;
  mb.ints.resize(P.ncones + 1, 0);
  const int prog_base = (int)mb.ints.size();
  mb.ints.resize(mb.ints.size() + prog_total, 0);
  // ConeDev pointers to ints are fixed after the meta allocation; remember offsets
  for (int c = 0; c < P.ncones; ++c) {
    const int64_t n = sides[big[c]];
    char* cb = base + cone_base[c];
    const ConeLayout& L = lay[c];
    ConeDev& d = cones[c];
    d.n = n;
    d.xoff = P.offsets[big[c]];
    d.voff = voff[big[c]];
    d.loff = loff[big[c]];
    d.cidx = big[c];
    d.path = path[c];
    d.b = b;
    d.npanels = path[c] ? 0 : num_panels(n, b);
    d.nsweeps = path[c] ? 0 : (int)std::max<int64_t>(0, n - 2);
    d.kmax = (int)((n >= 3 ? (n - 3) / b + 1 : 0) + 1);
#define FLD(T, f) reinterpret_cast<T*>(cb + L.off[f])
    d.A = FLD(double, F_A); d.band = FLD(double, F_BAND); d.refl = FLD(double, F_REFL);
    d.d = FLD(double, F_D); d.e = FLD(double, F_E); d.V1 = FLD(double, F_V1); d.T1 = FLD(double, F_T1);
    d.Y = FLD(double, F_Y); d.X = FLD(double, F_X); d.U3 = FLD(double, F_U3); d.Mb = FLD(double, F_MB);
    d.Nb = FLD(double, F_NB); d.QA = FLD(double, F_QA); d.QB = FLD(double, F_QB); d.lamA = FLD(double, F_LAMA);
    d.lamB = FLD(double, F_LAMB); d.Qin = FLD(double, F_QIN); d.Ucm = FLD(double, F_UCM); d.Z = FLD(double, F_Z);
    d.lamk = FLD(double, F_LAMK); d.dsrt = FLD(double, F_DSRT); d.zk = FLD(double, F_ZK); d.dval = FLD(double, F_DVAL);
    d.tau = FLD(double, F_TAU); d.zhat = FLD(double, F_ZHAT); d.rot = FLD(double, F_ROT); d.rho = FLD(double, F_RHO);
    d.tau1 = FLD(double, F_TAU1);
    d.ifp = FLD(int, F_IFP);
    d.iperm = FLD(int, F_IPERM); d.irot = FLD(int, F_IROT); d.iorg = FLD(int, F_IORG); d.imap = FLD(int, F_IMAP);
    d.icnt = FLD(int, F_ICNT); d.kinfo = FLD(int, F_KINFO);
#undef FLD
  }
  // The GEMM descriptors need the status pointers (skip), which live in the
  // metadata block: allocate it first with a generous upper bound, then fill.
  // Upper bound: count descriptors/ints/nodes while building with placeholders.
  // We build with a null status base and patch afterwards.
  // encoded as (status slot index + 1) until the metadata block exists
  auto st_ptr = [&](int c) -> const int* { return reinterpret_cast<const int*>((intptr_t)(status_off + c + 1 + 1)); };

  // ---- stage 1: panels
  int maxP = 0;
  for (int c = 0; c < P.ncones; ++c) maxP = std::max(maxP, cones[c].npanels);
  for (int p = 0; p < maxP; ++p) {
    PanelStep ps;
    ps.panel = p;
    std::vector<int> ids;
    int maxm = 0;
    for (int c = 0; c < P.ncones; ++c)
      if (p < cones[c].npanels) {
        ids.push_back(c);
        maxm = std::max<int>(maxm, (int)cones[c].n - (p + 1) * b);
      }
    ps.njobs = (int)ids.size();
    ps.cluster = std::min(16, std::max(1, (maxm + 255) / 256));
    ps.R = (maxm + ps.cluster - 1) / ps.cluster;
    ps.ids_off = (int)mb.ints.size();
    mb.ints.insert(mb.ints.end(), ids.begin(), ids.end());
    std::vector<GemmDesc> g[6];
    for (int c : ids) {
      const ConeDev& d = cones[c];
      const int n = (int)d.n;
      const int r0 = (p + 1) * b, m = n - r0, bb = std::min(b, m);
      double* A22 = d.A + r0 + (int64_t)r0 * n;
      double* V = d.V1 + (int64_t)p * n * b;
      double* T = d.T1 + (int64_t)p * b * b;
      double* Xm = d.U3 + (int64_t)bb * m;
      const int* sk = st_ptr(c);
      g[0].push_back(mk(A22, n, V, m, d.Y, m, m, bb, m, 1.0, 0.0, GF_SYM_A, sk));
      g[1].push_back(mk(d.Y, m, T, b, Xm, m, m, bb, bb, 1.0, 0.0, 0, sk));
      g[2].push_back(mk(V, m, Xm, m, d.Mb, b, bb, bb, m, 1.0, 0.0, GF_TRANS_A, sk));
      g[3].push_back(mk(T, b, d.Mb, b, d.Nb, b, bb, bb, bb, 1.0, 0.0, GF_TRANS_A, sk));
      g[4].push_back(mk(V, m, d.Nb, b, Xm, m, m, bb, bb, -0.5, 1.0, 0, sk));
      g[5].push_back(mk(Xm, m, d.U3, m, A22, n, m, m, 2 * bb, -1.0, 1.0, GF_TRANS_B | GF_LOWER_C, sk));
    }
    for (int q = 0; q < 6; ++q) ps.g[q] = mb.add_gemm(g[q]);
    P.panels.push_back(ps);
  }

  // ---- stage 2: bulge chasing CTA assignment (cooperative launches)
  {
    int cap = bulge_max_ctas(b);
    if (cap <= 0) cap = 1;
    std::vector<int> two;
    for (int c = 0; c < P.ncones; ++c)
      if (cones[c].path == 0 && cones[c].nsweeps > 0) two.push_back(c);
    std::vector<int> want(two.size());
    for (size_t q = 0; q < two.size(); ++q) {
      const int64_t n = cones[two[q]].n;
      const int nsw = cones[two[q]].nsweeps;
      int w = (int)std::max<int64_t>(1, n / (3 * b) + 1);
      w = std::min(w, std::max(1, nsw));
      want[q] = w;
    }
    int c = 0;
    const int ntwo = (int)two.size();
    while (c < ntwo) {
      // pack cones into one launch while the CTA cap allows at least 1 each
      int first = c, total_want = 0;
      while (c < ntwo && (c - first) < cap) { total_want += want[c]; ++c; }
      const int nc = c - first;
      std::vector<int> give(nc);
      if (total_want <= cap) {
        for (int q = 0; q < nc; ++q) give[q] = want[first + q];
      } else {
        int left = cap - nc;  // 1 each guaranteed
        long long extra_want = 0;
        for (int q = 0; q < nc; ++q) extra_want += want[first + q] - 1;
        for (int q = 0; q < nc; ++q) {
          const long long ew = want[first + q] - 1;
          give[q] = 1 + (extra_want > 0 ? (int)(ew * left / extra_want) : 0);
        }
      }
      BulgeLaunch bl;
      bl.ncones = nc;
      std::vector<int> cc, rr, gg;
      for (int q = 0; q < nc; ++q)
        for (int r = 0; r < give[q]; ++r) { cc.push_back(two[first + q]); rr.push_back(r); gg.push_back(give[q]); }
      bl.nctas = (int)cc.size();
      bl.cone_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), cc.begin(), cc.end());
      bl.rank_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), rr.begin(), rr.end());
      bl.count_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), gg.begin(), gg.end());
      P.bulges.push_back(bl);
    }
  }

  // ---- one-stage tridiagonalisation: CTA groups per cone (cooperative launches)
  {
    std::vector<int> one;
    int64_t maxn1 = 0;
    for (int c = 0; c < P.ncones; ++c)
      if (cones[c].path == 1) { one.push_back(c); maxn1 = std::max(maxn1, cones[c].n); }
    if (!one.empty()) {
      // at most one CTA per SM for a cone: a step's work is small and the
      // group barrier's cost grows with the number of CTAs
      const int cap = std::max(1, sytrd1_max_ctas((int)maxn1));
      const int sm_cap = std::max(1, h->sms / std::max(1, tune.sy_share));
      // large cones (n >= 256) share the GPU in one launch, small cones get one CTA each
      std::vector<int> large, small;
      for (int c : one) (cones[c].n >= 256 ? large : small).push_back(c);
      auto emit = [&](const std::vector<int>& list, bool spread) {
        // one-CTA cones keep their matrix in shared memory when it fits:
        // group them by the occupancy of that size
        int gcap = cap;
        if (!spread && !list.empty()) {
          int mx = 0;
          for (int c : list) mx = std::max<int>(mx, (int)cones[c].n);
          const size_t res = sytrd1_smem_bytes(mx, 1, true);
          if (res <= 200 * 1024) gcap = std::max(1, sytrd1_max_ctas_for(res));
        }
        // large cones whose matrices together exceed L2 but each fit it: one
        // launch per L2-sized group (the double-float route with the columns in
        // global memory then applies to each group)
        constexpr double kL2Group = 112.0 * 1024 * 1024;
        bool by_bytes = false;
        if (spread) {
          double total = 0.0, mxb = 0.0;
          for (int c : list) {
            const double b = 8.0 * (double)cones[c].n * (double)cones[c].n;
            total += b;
            mxb = std::max(mxb, b);
          }
          by_bytes = total > kL2Group && mxb <= kL2Group;
        }
        size_t i = 0;
        while (i < list.size()) {
          std::vector<int> grp;
          double work = 0.0, bytes = 0.0;
          while (i < list.size() && (int)grp.size() < gcap) {
            const double b = 8.0 * (double)cones[list[i]].n * (double)cones[list[i]].n;
            if (by_bytes && !grp.empty() && bytes + b > kL2Group) break;
            grp.push_back(list[i]);
            work += std::pow((double)cones[list[i]].n, 3.0);
            bytes += b;
            ++i;
          }
          // CTAs per cone: a share of the co-resident CTAs by work, at least 4
          // columns each
          auto spread_give = [&](int budget) {
            std::vector<int> give(grp.size(), 1);
            if (!spread) return give;
            const int left = budget - (int)grp.size();
            for (size_t q = 0; q < grp.size(); ++q) {
              const double share = std::pow((double)cones[grp[q]].n, 3.0) / work;
              int extra = (int)(share * left);
              extra = std::min<int64_t>(extra, std::max<int64_t>(0, cones[grp[q]].n / 4 - 1));
              extra = std::min(extra, sm_cap - 1);
              give[q] += extra;
            }
            return give;
          };
          std::vector<int> give = spread_give(cap);
          Sytrd1Launch sl;
          sl.maxn = (int)maxn1;
          // shared-memory-resident columns when every cone of the launch fits and
          // the launch stays co-resident
          {
            size_t need = 0;
            for (size_t q = 0; q < grp.size(); ++q)
              need = std::max(need, sytrd1_smem_bytes((int)cones[grp[q]].n, give[q], true));
            int total = 0;
            for (int g : give) total += g;
            if (need <= 200 * 1024 && sytrd1_max_ctas_for(need) >= total) {
              sl.smem = need;
            } else if (spread && tune.sy_share <= 1) {
              // columns in L2: whole waves of r CTAs per SM (an SM with one CTA
              // more than the others sets every step's pace), r near one CTA per
              // 28 columns per SM (measured: 8 cones of side 1296 at 2 per SM,
              // 57 ms; at 4 per SM, 74 ms; 4 cones of side 4096 best at 4)
              double cols = 0.0;
              for (int c : grp) cols += (double)cones[c].n;
              const int sms_all = std::max(1, h->sms);
              int r = (int)std::lround(cols / (28.0 * sms_all));
              r = std::max(1, std::min(r, std::max(1, cap / sms_all)));
              give = spread_give(std::max((int)grp.size(), r * sms_all));
            }
            if (sl.smem == 0) {
              // columns in L2: double-float arithmetic when the launch's matrices
              // stay in L2 (8 cones of side 1296, 107 MB: 45 ms against 58 ms in
              // FP64); beyond that the FP64 route, whose instruction stream keeps
              // more of the stream from HBM in flight (4 cones of side 4096: 0.71 s
              // against 1.43 s)
              double bytes = 0.0;
              int mx = 0, tot = 0;
              for (size_t q = 0; q < grp.size(); ++q) {
                bytes += 8.0 * (double)cones[grp[q]].n * (double)cones[grp[q]].n;
                mx = std::max<int>(mx, (int)cones[grp[q]].n);
                tot += give[q];
              }
              const size_t gb = sytrd1_glb_smem_bytes(mx);
              if (bytes <= 112.0 * 1024 * 1024 && gb <= 200 * 1024 && sytrd1_max_ctas_for(gb) >= tot) {
                sl.glb = 1;
                sl.smem = gb;
              }
            }
          }
          std::vector<int> cc, rr, gg;
          for (size_t q = 0; q < grp.size(); ++q)
            for (int r = 0; r < give[q]; ++r) { cc.push_back(grp[q]); rr.push_back(r); gg.push_back(give[q]); }
          sl.nctas = (int)cc.size();
          sl.cone_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), cc.begin(), cc.end());
          sl.rank_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), rr.begin(), rr.end());
          sl.count_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), gg.begin(), gg.end());
          P.sytrd1.push_back(sl);
        }
      };
      emit(large, true);
      emit(small, false);
      std::vector<int> bc, bi;
      for (int c : one)
        for (int q = 0; q < num_blocks1(cones[c].n); ++q) { bc.push_back(c); bi.push_back(q); }
      P.nlarft = (int)bc.size();
      P.larft_cone_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), bc.begin(), bc.end());
      P.larft_idx_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), bi.begin(), bi.end());
    }
  }

  // ---- complex Hermitian cones: reduction groups, T-factor blocks, back-transformation CTAs
  std::vector<HConeDev> hcones;
  size_t hbytes = 0;
  std::vector<size_t> hoff;
  if (herm) {
    const int sms = std::max(1, h->sms);
    std::vector<int> G(P.ncones);
    size_t maxneed = 0;
    for (int c = 0; c < P.ncones; ++c) {
      const int n = (int)cones[c].n;
      int g = n >= 256 ? std::min(sms, n / 4) : 1;
      while (g < sms && hetrd1_smem_bytes(n, g) > kHetrdSmemMax) ++g;
      if (hetrd1_smem_bytes(n, g) > kHetrdSmemMax) return SCS_PSD_EINVAL;
      G[c] = g;
      maxneed = std::max(maxneed, hetrd1_smem_bytes(n, g));
    }
    int c = 0;
    while (c < P.ncones) {
      // cones of one cooperative launch: every CTA co-resident
      Sytrd1Launch sl;
      size_t need = 0;
      int total = 0;
      std::vector<int> cc, rr, gg;
      while (c < P.ncones) {
        const size_t nd = std::max(need, hetrd1_smem_bytes((int)cones[c].n, G[c]));
        const int cap = std::max(1, hetrd1_max_ctas_for(nd));
        if (total > 0 && total + G[c] > cap) break;
        need = nd;
        for (int r = 0; r < G[c]; ++r) { cc.push_back(c); rr.push_back(r); gg.push_back(G[c]); }
        total += G[c];
        ++c;
      }
      sl.nctas = total;
      sl.smem = need;
      sl.maxn = 0;
      sl.cone_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), cc.begin(), cc.end());
      sl.rank_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), rr.begin(), rr.end());
      sl.count_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), gg.begin(), gg.end());
      P.hetrd.push_back(sl);
    }
    (void)maxneed;
    std::vector<int> bc, bi, tc, tr, tg;
    for (int q = 0; q < P.ncones; ++q) {
      const int64_t n = cones[q].n;
      for (int k = 0; k < hcone_blocks(n); ++k) { bc.push_back(q); bi.push_back(k); }
      // back-transformation: about two kept columns per CTA for half the columns
      // kept (every SM busy at n = 625; each CTA streams the reflector blocks from L2)
      const int g = (int)std::max<int64_t>(1, std::min<int64_t>(2 * sms, (n / 2 + 1) / 2));
      for (int r = 0; r < g; ++r) { tc.push_back(q); tr.push_back(r); tg.push_back(g); }
    }
    P.hlarft_n = (int)bc.size();
    P.hlarft_cone_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), bc.begin(), bc.end());
    P.hlarft_idx_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), bi.begin(), bi.end());
    P.hbt_nctas = (int)tc.size();
    P.hbt_cone_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), tc.begin(), tc.end());
    P.hbt_rank_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), tr.begin(), tr.end());
    P.hbt_count_off = (int)mb.ints.size(); mb.ints.insert(mb.ints.end(), tg.begin(), tg.end());
    // complex workspace per cone: publication slabs, V blocks, T blocks, tau, W
    hoff.resize(P.ncones);
    for (int q = 0; q < P.ncones; ++q) {
      const int64_t n = cones[q].n;
      hoff[q] = hbytes;
      hbytes += align_up(sizeof(double) * hcone_pub_doubles(n)) + align_up(sizeof(cdf) * hcone_v_elems(n)) +
                align_up(sizeof(cdf) * hcone_t_elems(n)) + align_up(sizeof(cdf) * (size_t)n) +
                align_up(sizeof(cdf) * (size_t)(n * n));
    }
  }

  // ---- divide and conquer levels
  {
    std::vector<int64_t> pos_base(P.ncones);
    int64_t tp = 0;
    int maxL = 0;
    for (int c = 0; c < P.ncones; ++c) {
      pos_base[c] = tp;
      tp += cones[c].n;
      maxL = std::max(maxL, num_levels(cones[c].n));
    }
    P.total_pos = tp;
    for (int l = 0; l < maxL; ++l) {
      Level lv;
      lv.nodes_off = (int)mb.nodes.size();
      std::vector<int> loc(tp, -1), nid(tp, -1);
      std::vector<GemmDesc> gd;
      for (int c = 0; c < P.ncones; ++c) {
        const int64_t n = cones[c].n;
        const int L = num_levels(n);
        if (l >= L) continue;
        if (l == 0 && n >= 3) continue;  // 2 x 2 leaves (closed form) stand in for level 0
        const int64_t half = int64_t(1) << l, full = half << 1;
        for (int64_t s = 0; s < n; s += full) {
          MergeNode nd;
          nd.cone = c;
          nd.s = (int)s;
          nd.n1 = (int)std::min(half, n - s);
          nd.n2 = (int)std::max<int64_t>(0, std::min(half, n - s - nd.n1));
          nd.root = (l == L - 1) ? 1 : 0;
          nd.level = l;
          const int K = nd.n1 + nd.n2;
          const int idx = (int)mb.nodes.size() - lv.nodes_off;
          for (int t = 0; t < K; ++t) {
            loc[pos_base[c] + s + t] = t;
            nid[pos_base[c] + s + t] = idx;
          }
          lv.maxK = std::max(lv.maxK, K);
          mb.nodes.push_back(nd);
          if (nd.n2 > 0) {
            const ConeDev& d = cones[c];
            const int ni = (int)n;
            double* Qo = (l & 1) ? d.QA : d.QB;
            GemmDesc g = mk(d.Qin + s + s * n, ni, d.Ucm + s + s * n, ni, nd.root ? d.Z : Qo + s, ni, K, K, K, 1.0,
                            0.0, GF_TRANS_B, st_ptr(c));
            g.dynK = d.icnt + 4 * s;
            g.dynN = nd.root ? d.kinfo + 2 : d.icnt + 4 * s;
            g.colmap = nd.root ? nullptr : d.imap + s;
            gd.push_back(g);
          }
        }
      }
      lv.nnodes = (int)mb.nodes.size() - lv.nodes_off;
      if (lv.nnodes == 0) continue;
      lv.pos_off = (int)mb.ints.size();
      mb.ints.insert(mb.ints.end(), loc.begin(), loc.end());
      mb.ints.insert(mb.ints.end(), nid.begin(), nid.end());
      lv.g = mb.add_gemm(gd, true);
      P.levels.push_back(lv);
    }
  }

  // ---- stage-1 back-transformation (two-stage cones: band-reduction panels;
  // one-stage cones: 32-reflector blocks), last block first.  One-stage cones
  // use the fused FP64 kernel (a slab of columns per CTA, CTAs given to the
  // cones in proportion to their work n^2 k; at these sides it beats the
  // split products, whose K is only 32); the rest use grouped GEMMs.
  auto fused_bt1 = [&](const ConeDev& d) { return d.path == 1 && d.n >= 3 && d.n <= bt1_max_side(); };
  {
    std::vector<int> fc;
    double wsum = 0.0;
    for (int c = 0; c < P.ncones; ++c)
      if (fused_bt1(cones[c])) {
        fc.push_back(c);
        const double n = (double)cones[c].n;
        wsum += n * n * (allv ? n : 0.5 * n);
      }
    if (!fc.empty()) {
      const double budget = std::max<double>(2.0 * mb.sms, (double)fc.size());
      std::vector<int> cc, cr, cn;
      for (int c : fc) {
        const int64_t n = cones[c].n;
        const double w = (double)n * n * (allv ? n : 0.5 * n);
        // columns per CTA: a power of two (the slab widths of the kernel)
        const int bud = std::max(1, (int)(budget * w / wsum));
        const int kest = allv ? (int)n : (int)(n + 1) / 2;
        int per = 1;
        const int per_max = std::max(1, std::min(8, tune.bt1_cols));
        while (per < per_max && (kest + per - 1) / per > bud) per *= 2;
        int g = std::max(1, (kest + per - 1) / per);
        // a lone cone whose reflector blocks are staged in shared memory runs
        // one CTA per SM: keep its launch to one wave
        if (fc.size() == 1 && bt1_stages((int)n)) g = std::min(g, std::max(1, mb.sms));
        for (int r = 0; r < g; ++r) { cc.push_back(c); cr.push_back(r); cn.push_back(g); }
        P.bt1k_maxn = std::max<int>(P.bt1k_maxn, (int)n);
      }
      P.bt1k_nctas = (int)cc.size();
      P.bt1k_cone_off = (int)mb.ints.size();
      mb.ints.insert(mb.ints.end(), cc.begin(), cc.end());
      P.bt1k_rank_off = (int)mb.ints.size();
      mb.ints.insert(mb.ints.end(), cr.begin(), cr.end());
      P.bt1k_count_off = (int)mb.ints.size();
      mb.ints.insert(mb.ints.end(), cn.begin(), cn.end());
    }
  }
  int maxQ = 0;
  for (int c = 0; c < P.ncones; ++c)
    if (cones[c].path == 1 && !fused_bt1(cones[c])) maxQ = std::max(maxQ, num_blocks1(cones[c].n));
  for (int p = std::max(maxP, maxQ) - 1; p >= 0; --p) {
    std::vector<GemmDesc> g[3];
    for (int c = 0; c < P.ncones; ++c) {
      const ConeDev& d = cones[c];
      const int n = (int)d.n;
      int r0, m, bb, wb;
      double *V, *T;
      if (d.path == 0) {
        if (p >= d.npanels) continue;
        r0 = (p + 1) * b; m = n - r0; bb = std::min(b, m); wb = b;
        V = d.V1 + (int64_t)p * n * b;
        T = d.T1 + (int64_t)p * b * b;
      } else {
        if (fused_bt1(d) || p >= num_blocks1(n)) continue;
        r0 = p * kSy1Block + 1; m = n - r0; bb = std::min<int>(kSy1Block, n - 2 - p * kSy1Block);
        wb = kSy1Block;
        V = d.V1 + (int64_t)p * n * kSy1Block;
        T = d.T1 + (int64_t)p * kSy1Block * kSy1Block;
      }
      GemmDesc a1;
      if (mb.split) {
        // (V^T Z)^T = Z^T V: the long dimension (kept columns) becomes M
        a1 = mk(d.Z + r0, n, V, m, d.Y, wb, n, bb, m, 1.0, 0.0, GF_TRANS_A | GF_TRANS_C, st_ptr(c));
        a1.dynM = d.kinfo;
      } else {
        a1 = mk(V, m, d.Z + r0, n, d.Y, wb, bb, n, m, 1.0, 0.0, GF_TRANS_A, st_ptr(c));
        a1.dynN = d.kinfo;
      }
      GemmDesc b2 = mk(T, wb, d.Y, wb, d.X, wb, bb, n, bb, 1.0, 0.0, 0, st_ptr(c));
      b2.dynN = d.kinfo;
      GemmDesc c3 = mk(V, m, d.X, wb, d.Z + r0, n, m, n, bb, -1.0, 1.0, 0, st_ptr(c));
      c3.dynN = d.kinfo;
      g[0].push_back(a1);
      g[1].push_back(b2);
      g[2].push_back(c3);
    }
    for (int q = 0; q < 3; ++q) P.bt1.push_back(mb.add_gemm(g[q]));
  }

  // ---- split mode: reconstruction S = Z diag(l) Z^T (lower) on the tensor cores
  if (mb.split && !allv) {
    std::vector<GemmDesc> g;
    for (int c = 0; c < P.ncones; ++c) {
      const ConeDev& d = cones[c];
      const int n = (int)d.n;
      GemmDesc q = mk(d.Z, n, d.Z, n, d.QA, n, n, n, n, 1.0, 0.0, GF_TRANS_B | GF_SCALE_B | GF_LOWER_C, st_ptr(c));
      q.bscale = d.lamk;
      q.dynK = d.kinfo;
      g.push_back(q);
    }
    P.recon_tc = mb.add_gemm(g);
  }

  // ---- derivative contractions
  if (allv) {
    std::vector<GemmDesc> g[4];
    for (int c = 0; c < P.ncones; ++c) {
      const ConeDev& d = cones[c];
      const int n = (int)d.n;
      // S-first eigenvectors (k_S = kinfo[6]): H = V_S^T G, M = H V, (scale), W = X V^T, Z1 = V_S W
      GemmDesc q0 = mk(d.Z, n, d.A, n, d.QA, n, n, n, n, 1.0, 0.0, GF_TRANS_A, st_ptr(c));
      GemmDesc q1 = mk(d.QA, n, d.Z, n, d.QB, n, n, n, n, 1.0, 0.0, 0, st_ptr(c));
      GemmDesc q2 = mk(d.QB, n, d.Z, n, d.QA, n, n, n, n, 1.0, 0.0, GF_TRANS_B, st_ptr(c));
      GemmDesc q3 = mk(d.Z, n, d.QA, n, d.QB, n, n, n, n, 1.0, 0.0, 0, st_ptr(c));
      q0.dynM = d.kinfo + 6;
      q1.dynM = d.kinfo + 6;
      q2.dynM = d.kinfo + 6;
      q3.dynK = d.kinfo + 6;
      g[0].push_back(q0);
      g[1].push_back(q1);
      g[2].push_back(q2);
      g[3].push_back(q3);
    }
    // operands bounded: eigenvectors, and G scaled by a power of two to its largest entry
    for (int q = 0; q < 4; ++q) P.vjp[q] = mb.add_gemm(g[q], true);
  }

  // ---- allocate and upload metadata
  const size_t cones_b = align_up(sizeof(ConeDev) * std::max(1, P.ncones));
  const size_t ints_b = align_up(sizeof(int) * std::max<size_t>(1, mb.ints.size()));
  const size_t descs_b = align_up(sizeof(GemmDesc) * std::max<size_t>(1, mb.descs.size()));
  const size_t nodes_b = align_up(sizeof(MergeNode) * std::max<size_t>(1, mb.nodes.size()));
  const size_t triv_b = align_up(4 * sizeof(int64_t) * std::max(1, P.ntriv));
  const size_t scratch_b = align_up(sizeof(double) * std::max<int64_t>(1, mb.scratch_doubles));
  const size_t io_b = align_up(sizeof(IoSlot));
  const size_t sjobs_b = mb.sjobs.empty() ? 0 : align_up(sizeof(SliceJob) * mb.sjobs.size());
  const size_t slice_b = mb.slice_floats > 0 ? align_up(sizeof(float) * (size_t)mb.slice_floats) : 0;
  const size_t total = cones_b + ints_b + descs_b + nodes_b + triv_b + scratch_b + io_b + sjobs_b + slice_b;
  if (arena) {
    P.arena_owned = true;
    if (!(P.meta_mem = arena->take(total))) return SCS_PSD_ENOMEM;
  } else if (cudaMalloc(&P.meta_mem, total) != cudaSuccess) {
    return SCS_PSD_ENOMEM;
  }
  char* mbase = (char*)P.meta_mem;
  P.cones_d = (ConeDev*)mbase;
  P.ints_d = (int*)(mbase + cones_b);
  P.descs_d = (GemmDesc*)(mbase + cones_b + ints_b);
  P.nodes_d = (MergeNode*)(mbase + cones_b + ints_b + descs_b);
  P.triv_offs_d = (int64_t*)(mbase + cones_b + ints_b + descs_b + nodes_b);
  double* scratch = (double*)(mbase + cones_b + ints_b + descs_b + nodes_b + triv_b);
  P.io_d = (IoSlot*)(mbase + cones_b + ints_b + descs_b + nodes_b + triv_b + scratch_b);
  P.sjobs_d = sjobs_b ? (SliceJob*)(mbase + cones_b + ints_b + descs_b + nodes_b + triv_b + scratch_b + io_b) : nullptr;
  float* slices = slice_b ? (float*)(mbase + cones_b + ints_b + descs_b + nodes_b + triv_b + scratch_b + io_b + sjobs_b)
                          : nullptr;
  for (size_t q = 0; q < mb.sjobs.size(); ++q)
    if (mb.sjob_out[q] >= 0) mb.sjobs[q].out = slices + mb.sjob_out[q];
  for (size_t q = 0; q < mb.descs.size(); ++q) {
    mb.descs[q].partial = mb.part_off[q] >= 0 ? scratch + mb.part_off[q] : nullptr;
    if (mb.desc_as[q] >= 0) mb.descs[q].As = slices + mb.desc_as[q];
    if (mb.desc_bs[q] >= 0) mb.descs[q].Bs = slices + mb.desc_bs[q];
  }
  P.status_d = P.ints_d + status_off;
  P.prog_d = P.ints_d + prog_base;
  P.prog_count = prog_total;
  // patch pointers that refer to the metadata block
  for (int c = 0; c < P.ncones; ++c) {
    cones[c].status = P.status_d + c + 1;
    cones[c].prog = P.prog_d + prog_off[c];
  }
  for (GemmDesc& g : mb.descs)
    if (g.skip) g.skip = P.ints_d + ((intptr_t)g.skip - 1);
  if (herm && P.ncones) {
    if (cudaMalloc(&P.hmem, hbytes + align_up(sizeof(HConeDev) * P.ncones)) != cudaSuccess) {
      P.hmem = nullptr;
      return SCS_PSD_ENOMEM;
    }
    char* hb = (char*)P.hmem;
    P.hcones_d = (HConeDev*)(hb + hbytes);
    hcones.resize(P.ncones);
    for (int q = 0; q < P.ncones; ++q) {
      const ConeDev& d = cones[q];
      const int64_t n = d.n;
      HConeDev& hc = hcones[q];
      char* o = hb + hoff[q];
      hc.n = n;
      hc.xoff = d.xoff;
      hc.d = d.d;
      hc.e = d.e;
      hc.status = d.status;
      hc.prog = d.prog;
      hc.Z = d.Z;
      hc.lamk = d.lamk;
      hc.kinfo = d.kinfo;
      hc.pub = (dfl*)o; o += align_up(sizeof(double) * hcone_pub_doubles(n));
      hc.V = (cdf*)o; o += align_up(sizeof(cdf) * hcone_v_elems(n));
      hc.T = (cdf*)o; o += align_up(sizeof(cdf) * hcone_t_elems(n));
      hc.tau = (cdf*)o; o += align_up(sizeof(cdf) * (size_t)n);
      hc.W = (cdf*)o;
    }
  }
  // kinfo: [3] all eigenpairs, [4] side option (staged in a host block next to the rest)
  std::vector<int> kin_all((size_t)P.ncones * 8, 0);
  for (int c = 0; c < P.ncones; ++c) {
    kin_all[(size_t)c * 8 + 3] = allv;
    kin_all[(size_t)c * 8 + 4] = side;
  }
  auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (!bytes) return cudaSuccess;
    if (arena) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, arena->stream);
    return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  cudaError_t e = cudaSuccess;
  if (P.ncones) e = up(P.cones_d, cones.data(), sizeof(ConeDev) * P.ncones);
  if (e == cudaSuccess) e = up(P.ints_d, mb.ints.data(), sizeof(int) * mb.ints.size());
  if (e == cudaSuccess) e = up(P.descs_d, mb.descs.data(), sizeof(GemmDesc) * mb.descs.size());
  if (e == cudaSuccess) e = up(P.nodes_d, mb.nodes.data(), sizeof(MergeNode) * mb.nodes.size());
  if (e == cudaSuccess && sjobs_b) e = up(P.sjobs_d, mb.sjobs.data(), sizeof(SliceJob) * mb.sjobs.size());
  if (e == cudaSuccess && P.ntriv) {
    e = up(P.triv_offs_d, triv_offs.data(), sizeof(int64_t) * 4 * P.ntriv);
  }
  for (int c = 0; c < P.ncones && e == cudaSuccess; ++c) e = up(cones[c].kinfo, &kin_all[(size_t)c * 8], 8 * sizeof(int));
  if (e == cudaSuccess && herm && P.ncones) e = up(P.hcones_d, hcones.data(), sizeof(HConeDev) * P.ncones);
  if (e != cudaSuccess) return SCS_PSD_ECUDA;
  (void)h;
  return SCS_PSD_OK;
}

#define LAUNCH_CHECK()                                      \
  do {                                                      \
    ++n_launch;                                             \
    cudaError_t _e = cudaGetLastError();                    \
    if (_e != cudaSuccess) return SCS_PSD_ECUDA;            \
  } while (0)

int run_gemm_at(const GemmDesc* descs_d, const int* ints_d, const GemmLaunch& g, cudaStream_t s,
                int64_t& n_launch, const SliceJob* sjobs_d = nullptr) {
  if (g.count <= 0 || g.tiles <= 0) return SCS_PSD_OK;
  if (g.tc2) {
    if (!sjobs_d) return SCS_PSD_EINVAL;
    if (g.njobs > 0) {
      launch_tc2_slice(sjobs_d + g.sjob_off, ints_d + g.sprefix_off, g.njobs, g.sctas, s);
      ++n_launch;
    }
    launch_tc2_gemm(descs_d + g.desc_off, ints_d + g.prefix_off, g.count, g.tiles, s);
    if (g.needs_reduce) launch_gemm_reduce(descs_d + g.desc_off, g.count, g.max_mn, s);
  } else if (g.tc) {
    launch_tc_gemm(descs_d + g.desc_off, ints_d + g.prefix_off, g.count, g.tiles, g.variant, s);
    if (g.needs_reduce) launch_gemm_reduce(descs_d + g.desc_off, g.count, g.max_mn, s);
  } else {
    launch_gemm(descs_d + g.desc_off, ints_d + g.prefix_off, g.count, g.tiles, g.variant, g.needs_reduce,
                g.max_mn, s);
  }
  if (g.needs_reduce) ++n_launch;
  LAUNCH_CHECK();
  return SCS_PSD_OK;
}

int run_gemm(const Plan& P, const GemmLaunch& g, cudaStream_t s, int64_t& n_launch) {
  return run_gemm_at(P.descs_d, P.ints_d, g, s, n_launch, P.sjobs_d);
}

// Phase timing: an event pair per phase interval when tracing is on.
struct PhaseMark {
  scs_psd_handle h;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  int phase = -1;
  void begin(int ph) {
    if (!h->trace) return;
    end();
    phase = ph;
    cudaEventCreate(&a);
    cudaEventRecord(a, s);
  }
  void end() {
    if (!h->trace || phase < 0) return;
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, s);
    h->trace_ev.push_back({phase, {a, b}});
    phase = -1;
  }
};

// The launch sequence of one call (MODE_* bits) after the caller's buffers
// are in P.io_d.
int run_body(scs_psd_handle h, Plan& P, int mode, long long wait_limit, cudaStream_t s, int64_t& n_launch) {
  int rc;
  const bool want_y = (mode & MODE_Y) != 0, want_vjp = (mode & MODE_VJP) != 0;
  bool joined = true;  // false while work on the second stream is outstanding
  const IoSlot* io = P.io_d;
  PhaseMark pm{h, s};
  CUDA_TRY(cudaMemsetAsync(P.status_d, 0, sizeof(int) * (P.ncones + 1), s));
  if (P.prog_count) CUDA_TRY(cudaMemsetAsync(P.prog_d, 0, sizeof(int) * P.prog_count, s));
  if (mode & MODE_STATS) {
    // the input as it was (y may alias x)
    if (!P.stats_mem) return SCS_PSD_EINVAL;
    launch_stats_save_x(io, P.stats_xs_d, P.stats_total, s);
    LAUNCH_CHECK();
  }
  if (P.ntriv) {
    launch_trivial(P.triv_offs_d, P.ntriv, io, mode, P.status_d, s);
    LAUNCH_CHECK();
  }
  if (P.ncones) {
    const int nc = P.ncones;
    if (mode & MODE_IMPORT) {
      launch_import_eig(P.cones_d, nc, P.maxn, io, s);
      LAUNCH_CHECK();
      launch_vjp_reorder(P.cones_d, nc, P.maxn, s);
      n_launch += 2;
      LAUNCH_CHECK();
    } else {
      if (P.herm) {
        // complex Hermitian cones: reduction straight from the Hermitian svec to
        // the real tridiagonal form, the T factors on the second stream
        pm.begin(1);
        for (const Sytrd1Launch& sl : P.hetrd) {
          if (launch_hetrd1(P.hcones_d, P.ints_d + sl.cone_off, P.ints_d + sl.rank_off, P.ints_d + sl.count_off,
                            sl.nctas, sl.smem, io, wait_limit, s))
            return SCS_PSD_ECUDA;
          LAUNCH_CHECK();
        }
        const bool side = h->use_aux && !h->trace && h->aux_stream && P.hlarft_n > 0;
        if (side) {
          CUDA_TRY(cudaEventRecord(h->ev_fork, s));
          CUDA_TRY(cudaStreamWaitEvent(h->aux_stream, h->ev_fork, 0));
        } else {
          pm.begin(5);
        }
        launch_hlarft(P.hcones_d, P.ints_d + P.hlarft_cone_off, P.ints_d + P.hlarft_idx_off, P.hlarft_n,
                      side ? h->aux_stream : s);
        LAUNCH_CHECK();
        if (side) {
          CUDA_TRY(cudaEventRecord(h->ev_join, h->aux_stream));
          joined = false;
        }
      } else {
        pm.begin(0);
        launch_unpack(P.cones_d, nc, P.maxn * P.maxn, io, 0, s);
        LAUNCH_CHECK();
        if (!P.panels.empty()) pm.begin(1);
        for (const PanelStep& ps : P.panels) {
          launch_panel(P.cones_d, P.ints_d + ps.ids_off, ps.njobs, ps.panel, P.b, ps.cluster, ps.R, s);
          LAUNCH_CHECK();
          for (int q = 0; q < 6; ++q)
            if ((rc = run_gemm(P, ps.g[q], s, n_launch))) return rc;
        }
        if (!P.sytrd1.empty()) {
          pm.begin(1);
          for (const Sytrd1Launch& sl : P.sytrd1) {
            if (launch_sytrd1(P.cones_d, P.ints_d + sl.cone_off, P.ints_d + sl.rank_off, P.ints_d + sl.count_off,
                              sl.nctas, sl.maxn, sl.smem, sl.glb, wait_limit, s))
              return SCS_PSD_ECUDA;
            LAUNCH_CHECK();
          }
          // the T factors need only the reflectors: on the second stream they
          // overlap the divide and conquer (kept on s while tracing phases)
          const bool side = h->use_aux && !h->trace && h->aux_stream && P.nlarft > 0;
          if (mode & MODE_LMIN) {
            // lambda_min stops at the tridiagonal form: no T factors
          } else if (side) {
            CUDA_TRY(cudaEventRecord(h->ev_fork, s));
            CUDA_TRY(cudaStreamWaitEvent(h->aux_stream, h->ev_fork, 0));
          } else {
            pm.begin(5);
          }
          if (!(mode & MODE_LMIN)) {
            launch_larft1(P.cones_d, P.ints_d + P.larft_cone_off, P.ints_d + P.larft_idx_off, P.nlarft,
                          side ? h->aux_stream : s);
            LAUNCH_CHECK();
          }
          if (side && !(mode & MODE_LMIN)) {
            CUDA_TRY(cudaEventRecord(h->ev_join, h->aux_stream));
            joined = false;
          }
        }
        pm.begin(2);
        launch_band_extract(P.cones_d, nc, P.maxn, s);
        LAUNCH_CHECK();
        for (const BulgeLaunch& bl : P.bulges) {
          if (launch_bulge(P.cones_d, bl.ncones, P.ints_d + bl.cone_off, P.ints_d + bl.rank_off,
                           P.ints_d + bl.count_off, bl.nctas, P.b, wait_limit, s))
            return SCS_PSD_ECUDA;
          LAUNCH_CHECK();
        }
        launch_tridiag_extract(P.cones_d, nc, P.maxn, s);
        LAUNCH_CHECK();
        if (mode & MODE_LMIN) {
          launch_lmin(P.cones_d, nc, io, s);
          LAUNCH_CHECK();
          pm.end();
          launch_status_reduce(P.status_d, P.ncones + 1, h->status_word, s);
          LAUNCH_CHECK();
          return SCS_PSD_OK;
        }
      }
      pm.begin(3);
      launch_dc_leaves(P.cones_d, nc, P.maxn, s);
      LAUNCH_CHECK();
      for (const Level& lv : P.levels) {
        const MergeNode* nodes = P.nodes_d + lv.nodes_off;
        const int* pos = P.ints_d + lv.pos_off;
        launch_dc_prepare(P.cones_d, nodes, lv.nnodes, lv.maxK, s);
        LAUNCH_CHECK();
        if (lv.maxK > kDcFuseK) {  // else done inside dc_prepare_kernel
          launch_dc_build_qin(P.cones_d, nodes, lv.nnodes, lv.maxK, s);
          LAUNCH_CHECK();
          launch_dc_apply_rot(P.cones_d, nodes, pos, P.total_pos, s);
          LAUNCH_CHECK();
        }
        launch_dc_secular(P.cones_d, nodes, pos, P.total_pos, lv.maxK, s);
        LAUNCH_CHECK();
        launch_dc_loewner(P.cones_d, nodes, pos, P.total_pos, s);
        LAUNCH_CHECK();
        launch_dc_select(P.cones_d, nodes, lv.nnodes, lv.maxK, s);
        LAUNCH_CHECK();
        launch_dc_vectors(P.cones_d, nodes, pos, P.total_pos, lv.maxK, s);
        LAUNCH_CHECK();
        if ((rc = run_gemm(P, lv.g, s, n_launch))) return rc;
        launch_dc_copy_deflated(P.cones_d, nodes, lv.nnodes, lv.maxK, s);
        LAUNCH_CHECK();
      }
      if (P.herm) {
        pm.begin(5);
        if (!joined) {
          CUDA_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
          joined = true;
        }
        launch_hbt(P.hcones_d, P.ints_d + P.hbt_cone_off, P.ints_d + P.hbt_rank_off, P.ints_d + P.hbt_count_off,
                   P.hbt_nctas, (int)P.maxn, s);
        LAUNCH_CHECK();
        pm.begin(6);
        launch_hrecon(P.hcones_d, nc, (int)P.maxn, io, s);
        LAUNCH_CHECK();
        pm.end();
        launch_status_reduce(P.status_d, P.ncones + 1, h->status_word, s);
        LAUNCH_CHECK();
        return SCS_PSD_OK;
      }
      pm.begin(4);
      launch_backtr2(P.cones_d, nc, (int)P.maxn, (int)P.maxn, P.allv ? (int)P.maxn : (int)(P.maxn + 1) / 2, P.b, s);
      LAUNCH_CHECK();
      pm.begin(5);
      if (!joined) {
        CUDA_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
        joined = true;
      }
      if (P.bt1k_nctas) {
        launch_bt1(P.cones_d, P.ints_d + P.bt1k_cone_off, P.ints_d + P.bt1k_rank_off, P.ints_d + P.bt1k_count_off,
                   P.bt1k_nctas, P.bt1k_maxn, s);
        LAUNCH_CHECK();
      }
      for (const GemmLaunch& gl : P.bt1)
        if ((rc = run_gemm(P, gl, s, n_launch))) return rc;
      if (P.allv) {
        // all eigenpairs: the route's side first (the derivative and the
        // reconstruction use only those k_S columns)
        launch_vjp_reorder(P.cones_d, nc, P.maxn, s);
        n_launch += 2;
        LAUNCH_CHECK();
      }
      if (mode & MODE_EXPORT) {
        launch_export_eig(P.cones_d, nc, P.maxn, io, s);
        LAUNCH_CHECK();
      }
      if (want_y) {
        pm.begin(6);
        if (P.recon_tc.count > 0) {
          if ((rc = run_gemm(P, P.recon_tc, s, n_launch))) return rc;
          launch_pack_recon(P.cones_d, nc, P.maxn, io, s);
        } else {
          launch_recon(P.cones_d, nc, (int)P.maxn, io, s);
        }
        LAUNCH_CHECK();
      }
    }
    if (want_vjp) {
      pm.begin(7);
      launch_vjp_gexp(P.cones_d, nc, io, s);
      LAUNCH_CHECK();
      launch_unpack(P.cones_d, nc, P.maxn * P.maxn, io, 1, s);
      LAUNCH_CHECK();
      if ((rc = run_gemm(P, P.vjp[0], s, n_launch))) return rc;
      if ((rc = run_gemm(P, P.vjp[1], s, n_launch))) return rc;
      launch_vjp_scale(P.cones_d, nc, P.maxn, s);
      LAUNCH_CHECK();
      if ((rc = run_gemm(P, P.vjp[2], s, n_launch))) return rc;
      if ((rc = run_gemm(P, P.vjp[3], s, n_launch))) return rc;
      launch_pack_lower(P.cones_d, nc, P.maxn, io, s);
      LAUNCH_CHECK();
    }
  }
  pm.end();
  if (mode & MODE_STATS) {
    launch_stats(P.stats_cones_d, (int)P.sides.size(), P.stats_part_cone_d, P.stats_nparts, P.cones_d, P.status_d,
                 P.stats_xs_d, io, P.stats_part_d, P.stats_out_d, s);
    n_launch += P.stats_nparts > 0 ? 1 : 0;
    LAUNCH_CHECK();
  }
  launch_status_reduce(P.status_d, P.ncones + 1, h->status_word, s);
  LAUNCH_CHECK();
  return SCS_PSD_OK;
}

// Device buffers of the per-cone statistics of a plan: the call's cone table,
// the partial sums, a copy of the input and the output records.
int ensure_stats(Plan& P) {
  if (P.stats_mem) return SCS_PSD_OK;
  const int count = (int)P.sides.size();
  std::vector<StatsCone> sc(count);
  std::vector<int> pc;
  int big = 0;
  for (int i = 0; i < count; ++i) {
    StatsCone& c = sc[i];
    c.off = P.offsets[i];
    c.len = P.offsets[i + 1] - P.offsets[i];
    c.side = P.sides[i];
    c.cone = P.sides[i] >= 2 ? big++ : -1;
    c.part0 = (int)pc.size();
    c.nparts = (int)((c.len + kStatsChunk - 1) / kStatsChunk);
    for (int q = 0; q < c.nparts; ++q) pc.push_back(i);
  }
  P.stats_nparts = (int)pc.size();
  P.stats_total = P.offsets[count];
  const size_t sc_b = align_up(sizeof(StatsCone) * std::max(1, count));
  const size_t pc_b = align_up(sizeof(int) * std::max<size_t>(1, pc.size()));
  const size_t part_b = align_up(3 * sizeof(double) * std::max<size_t>(1, pc.size()));
  const size_t xs_b = align_up(sizeof(double) * (size_t)std::max<int64_t>(1, P.stats_total));
  const size_t out_b = align_up(sizeof(ConeStats) * std::max(1, count));
  if (cudaMalloc(&P.stats_mem, sc_b + pc_b + part_b + xs_b + out_b) != cudaSuccess) {
    P.stats_mem = nullptr;
    return SCS_PSD_ENOMEM;
  }
  char* b = (char*)P.stats_mem;
  P.stats_cones_d = (StatsCone*)b;
  P.stats_part_cone_d = (int*)(b + sc_b);
  P.stats_part_d = (double*)(b + sc_b + pc_b);
  P.stats_xs_d = (double*)(b + sc_b + pc_b + part_b);
  P.stats_out_d = (ConeStats*)(b + sc_b + pc_b + part_b + xs_b);
  if (cudaMemcpy(P.stats_cones_d, sc.data(), sizeof(StatsCone) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
      (!pc.empty() &&
       cudaMemcpy(P.stats_part_cone_d, pc.data(), sizeof(int) * pc.size(), cudaMemcpyHostToDevice) != cudaSuccess))
    return SCS_PSD_ECUDA;
  return SCS_PSD_OK;
}

// Records the launch sequence of `mode` as a graph on the handle's capture
// stream (recording executes nothing).  A sequence that cannot be recorded
// is marked and stays eager.
void record_graph(scs_psd_handle h, Plan& P, int mode, long long wait_limit) {
  if (P.gexec[mode]) {
    cudaGraphExecDestroy(P.gexec[mode]);
    P.gexec[mode] = nullptr;
  }
  if (!h->capture_stream && cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    h->capture_stream = nullptr;
    P.gfailed[mode] = true;
    return;
  }
  cudaStream_t cs = h->capture_stream;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    P.gfailed[mode] = true;
    return;
  }
  int64_t n_launch = 0;
  const int rc = run_body(h, P, mode, wait_limit, cs, n_launch);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &graph);
  cudaGraphExec_t ge = nullptr;
  if (rc == SCS_PSD_OK && e == cudaSuccess && graph && cudaGraphInstantiate(&ge, graph, 0) == cudaSuccess) {
    P.gexec[mode] = ge;
    P.gwait[mode] = wait_limit;
    P.glaunches[mode] = n_launch;
  } else {
    P.gfailed[mode] = true;
    h->use_aux = false;  // a failed recording may leave the second stream unusable: stay on one stream
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
}

// One call: publish the caller's buffers, then run the launch sequence --
// eagerly on the first call of a plan (and whenever tracing, or when the
// caller's stream is itself being captured), as a recorded graph after that.
int run_plan(scs_psd_handle h, Plan& P, const IoSlot& io, int mode, long long wait_limit, cudaStream_t s,
             bool allow_graph) {
  int64_t n_launch = 0;
  launch_set_io(P.io_d, io, s);
  LAUNCH_CHECK();
  h->last_replayed = false;
  if (allow_graph && !h->trace && P.eager_runs > 0 && !P.gfailed[mode]) {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cst) == cudaSuccess && cst == cudaStreamCaptureStatusNone) {
      if (!P.gexec[mode] || P.gwait[mode] != wait_limit) record_graph(h, P, mode, wait_limit);
      if (P.gexec[mode]) {
        CUDA_TRY(cudaGraphLaunch(P.gexec[mode], s));
        P.launches = n_launch + P.glaunches[mode];
        h->last_replayed = true;
        return SCS_PSD_OK;
      }
    }
    cudaGetLastError();
  }
  const int rc = run_body(h, P, mode, wait_limit, s, n_launch);
  if (rc) return rc;
  ++P.eager_runs;
  P.launches = n_launch;
  return SCS_PSD_OK;
}

std::string plan_key(const int32_t* sides, int32_t count, int b, int allv, int side, int precision) {
  std::string k;
  k.reserve(16 + 4 * (size_t)count);
  char hdr[80];
  snprintf(hdr, sizeof(hdr), "b%d,a%d,s%d,p%d,c%d:", b, allv, side, precision, count);
  k += hdr;
  k.append(reinterpret_cast<const char*>(sides), sizeof(int32_t) * (size_t)count);
  return k;
}

int check_shapes(const int64_t* offsets, const int32_t* sides, int32_t count) {
  if (count < 0) return SCS_PSD_EINVAL;
  if (count == 0) return SCS_PSD_OK;
  if (!offsets || !sides) return SCS_PSD_EINVAL;
  if (offsets[0] != 0) return SCS_PSD_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (sides[i] < 0 || sides[i] > kMaxSide) return SCS_PSD_EINVAL;
    if (offsets[i + 1] - offsets[i] != svec_len(sides[i])) return SCS_PSD_EINVAL;
  }
  return SCS_PSD_OK;
}

std::string tune_key(const int32_t* sides, int32_t count, int precision) {
  return plan_key(sides, count, 0, 0, 0, precision);
}

// The cached plan for these shapes, options and launch shapes (built on first use).
int get_plan(scs_psd_handle h, const int32_t* sides, int32_t count, int allv, int side, int precision,
             const Tuning& tune, Plan** out, bool herm = false) {
  int b = kDefaultBand, onestage = -1;
  if (tune.band == 1) onestage = 1;
  else if (tune.band >= 2) { onestage = 0; b = tune.band; }
  if (b < 2 || b > kMaxBand) return SCS_PSD_EINVAL;
  const std::string key = plan_key(sides, count, b, allv, side, precision) + (char)('A' + onestage + 1) + tune.str() +
                          (herm ? "H" : "");
  auto it = h->plans.find(key);
  if (it != h->plans.end()) {
    *out = it->second.get();
    return SCS_PSD_OK;
  }
  if (h->plans.size() >= 16) {
    cudaDeviceSynchronize();
    h->plans.clear();
  }
  auto np = std::make_unique<Plan>();
  np->key = key;
  const int rc = build_plan(h, *np, sides, count, b, allv, side, precision, onestage, tune, nullptr, herm);
  if (rc) return rc;
  *out = np.get();
  h->plans[key] = std::move(np);
  return SCS_PSD_OK;
}

// One call of any entry point: `mode` (MODE_* bits) says which of io's
// buffers are read and written; every one it names must be non-NULL.
int do_call(scs_psd_handle h, const IoSlot& io, int mode, const int64_t* offsets, const int32_t* sides,
            int32_t count, const scs_psd_opts* opts, void* stream, bool herm = false) {
  if (!h) return SCS_PSD_EINVAL;
  int rc = herm ? SCS_PSD_OK : check_shapes(offsets, sides, count);
  if (rc) return rc;
  if (count == 0 || offsets[count] == 0) return SCS_PSD_OK;
  if (!(mode & MODE_IMPORT) && !io.x) return SCS_PSD_EINVAL;
  if ((mode & MODE_Y) && !io.y) return SCS_PSD_EINVAL;
  if ((mode & MODE_VJP) && (!io.g || !io.xbar)) return SCS_PSD_EINVAL;
  if ((mode & (MODE_EXPORT | MODE_IMPORT)) && (!io.V || !io.lam)) return SCS_PSD_EINVAL;
  if ((mode & MODE_LMIN) && !io.lam) return SCS_PSD_EINVAL;
  // every mode but the plain projection needs all n eigenpairs of each cone
  const int allv = (mode & (MODE_VJP | MODE_EXPORT | MODE_IMPORT)) ? 1 : 0;
  int side = 0, precision = SCS_PSD_FP64;
  long long wait = kDefaultWaitCycles;
  if (opts) {
    if (opts->precision != SCS_PSD_FP64 && opts->precision != SCS_PSD_SPLIT_TF32) return SCS_PSD_EINVAL;
    if (opts->graphs < 0 || opts->graphs > 1 || opts->stats < 0 || opts->stats > 1) return SCS_PSD_EINVAL;
    if (opts->band < 0 || opts->band > kMaxBand) return SCS_PSD_EINVAL;
    if (opts->stats) {
      // statistics describe a projection's result: the call must write y
      if (!(mode & MODE_Y)) return SCS_PSD_EINVAL;
      mode |= MODE_STATS;
    }
    precision = opts->precision;
    side = opts->side;
    if (opts->wait_limit_cycles > 0) wait = opts->wait_limit_cycles;
  }
  if (side < 0 || side > 2) return SCS_PSD_EINVAL;
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return SCS_PSD_ECUDA;
  // launch shapes: an explicit band wins; otherwise the autotuner's choice for
  // these shapes and precision, if it ran; otherwise the defaults
  Tuning tune;
  if (opts && opts->band) {
    tune.band = opts->band;
  } else {
    auto t = h->tuned.find(tune_key(sides, count, precision));
    if (t != h->tuned.end()) tune = t->second;
  }
  Plan* P = nullptr;
  rc = get_plan(h, sides, count, allv, side, precision, tune, &P, herm);
  if (rc) return rc;
  if ((mode & MODE_STATS) && (rc = ensure_stats(*P))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  rc = run_plan(h, *P, io, mode, wait, s, !(opts && opts->graphs == 1));
  h->last_stream = s;
  h->last_launches = P->launches;
  h->last_tune = P->tune;
  if (mode & MODE_STATS) {
    h->last_stats_key = rc == SCS_PSD_OK ? P->key : std::string();
    h->last_stats_count = count;
  }
  return rc;
}

// ---- autotuner: times launch-shape candidates on the caller's input ----
// Coordinate search: first the route and band width (automatic, one-stage,
// two-stage with b = 8, 16, 32), then the GEMM split-K target (1, 2, 4 CTAs
// per SM), then -- when the winner has one-stage cones -- the slab width of
// the fused back-transformation (2, 4, 8 columns) and the group size of the
// one-stage reduction (all SMs, half or a quarter).  Each candidate runs once to warm up
// and three times under CUDA events on `stream`; candidates whose device
// status is not clean are discarded.  The winner is kept in the handle for
// these shapes and precision and used by later calls that leave opts->band 0.
int autotune(scs_psd_handle h, const double* x, const int64_t* offsets, const int32_t* sides, int32_t count,
             const scs_psd_opts* opts, void* stream, int32_t* chosen, double* best_ms_out) {
  if (!h || !x) return SCS_PSD_EINVAL;
  int rc = check_shapes(offsets, sides, count);
  if (rc) return rc;
  if (count == 0 || offsets[count] == 0) return SCS_PSD_OK;
  int side = 0, precision = SCS_PSD_FP64;
  long long wait = kDefaultWaitCycles;
  if (opts) {
    if (opts->precision != SCS_PSD_FP64 && opts->precision != SCS_PSD_SPLIT_TF32) return SCS_PSD_EINVAL;
    precision = opts->precision;
    side = opts->side;
    if (opts->wait_limit_cycles > 0) wait = opts->wait_limit_cycles;
  }
  if (side < 0 || side > 2) return SCS_PSD_EINVAL;
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return SCS_PSD_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  int maxn = 0;
  for (int i = 0; i < count; ++i) maxn = std::max(maxn, (int)sides[i]);
  double* y = nullptr;
  if (cudaMalloc(&y, sizeof(double) * (size_t)offsets[count]) != cudaSuccess) return SCS_PSD_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const IoSlot io{x, y, nullptr, nullptr, nullptr, nullptr};
  const double kInf = 1e300;
  auto measure = [&](const Tuning& t) -> double {
    Plan* P = nullptr;
    if (get_plan(h, sides, count, 0, side, precision, t, &P)) return kInf;
    if (cudaMemsetAsync(h->status_word, 0, sizeof(int), s) != cudaSuccess) return kInf;
    if (run_plan(h, *P, io, MODE_Y, wait, s, false)) return kInf;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r)
      if (run_plan(h, *P, io, MODE_Y, wait, s, false)) return kInf;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return kInf;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    int st = 0;
    if (cudaMemcpy(&st, h->status_word, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || st != 0) return kInf;
    return ms / 3.0;
  };
  Tuning best;
  double best_ms = kInf;
  auto consider = [&](const Tuning& t) {
    const double ms = measure(t);
    if (ms < best_ms) { best_ms = ms; best = t; }
  };
  consider(Tuning());
  if (maxn >= 3) {
    for (int band : {1, 8, 16, 32}) {
      Tuning t;
      t.band = band;
      consider(t);
    }
  }
  const Tuning route = best;
  for (int gc : {1, 4}) {
    Tuning t = route;
    t.gemm_ctas = gc;
    consider(t);
  }
  bool has_one = false;
  for (int i = 0; i < count; ++i) {
    const int n = sides[i];
    if (n >= 3 && (best.band == 1 || (best.band == 0 && n <= kOneStageMax))) has_one = true;
  }
  if (has_one) {
    const Tuning base = best;
    for (int cols : {1, 2, 4}) {
      Tuning t = base;
      t.bt1_cols = cols;
      consider(t);
    }
    const Tuning base2 = best;
    for (int share : {2, 4}) {
      Tuning t = base2;
      t.sy_share = share;
      consider(t);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(y);
  cudaMemset(h->status_word, 0, sizeof(int));
  // keep only the winner's plan among this shape list's candidates
  h->plans.clear();
  if (best_ms >= kInf) return SCS_PSD_ECUDA;
  h->tuned[tune_key(sides, count, precision)] = best;
  if (chosen) {
    chosen[0] = best.band;
    chosen[1] = best.gemm_ctas;
    chosen[2] = best.bt1_cols;
    chosen[3] = best.sy_share;
  }
  if (best_ms_out) *best_ms_out = best_ms;
  return SCS_PSD_OK;
}

// ---- complex Hermitian cones: through the real side-2n embedding ----
int proj_poly(scs_psd_handle h, const double* x, double* y, const int64_t* offsets, const int32_t* sides,
              int32_t count, double lo, int32_t steps, const scs_psd_opts* opts, void* stream, double nsq);

// poly_lo > 0: the factorization-free composite instead of the eigendecomposition,
// with the norm of the Hermitian matrix (half the squared norm of the embedding).
int proj_hermitian(scs_psd_handle h, const double* x, double* y, const int64_t* offsets, const int32_t* sides,
                   int32_t count, const scs_psd_opts* opts, void* stream, double poly_lo = 0.0,
                   int32_t poly_steps = 0) {
  if (!h || count < 0) return SCS_PSD_EINVAL;
  if (opts && opts->stats) return SCS_PSD_EINVAL;  // statistics are kept for real cones only
  if (count == 0) return SCS_PSD_OK;
  if (!offsets || !sides || offsets[0] != 0) return SCS_PSD_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (sides[i] < 0 || 2 * (int64_t)sides[i] > kMaxSide) return SCS_PSD_EINVAL;
    if (offsets[i + 1] - offsets[i] != (int64_t)sides[i] * sides[i]) return SCS_PSD_EINVAL;
  }
  if (offsets[count] == 0) return SCS_PSD_OK;
  if (!x || !y) return SCS_PSD_EINVAL;
  // native complex route: every side within the shared-memory reduction's
  // reach, the eigendecomposition method, the automatic route
  bool native = poly_lo <= 0.0 && !(opts && opts->band);
  for (int i = 0; i < count && native; ++i)
    native = sides[i] <= kHermNativeMax && hetrd1_smem_bytes(sides[i], std::max(1, h->sms)) <= kHetrdSmemMax;
  if (native) {
    const IoSlot io{x, y, nullptr, nullptr, nullptr, nullptr};
    return do_call(h, io, MODE_Y, offsets, sides, count, opts, stream, true);
  }
  HermPlan* hp = nullptr;
  {
    std::lock_guard<std::mutex> lock(h->mu);
    if (cudaSetDevice(h->device) != cudaSuccess) return SCS_PSD_ECUDA;
    const std::string key = plan_key(sides, count, 0, 0, 0, 0);
    auto it = h->herm.find(key);
    if (it == h->herm.end()) {
      auto np = std::make_unique<HermPlan>();
      np->roff.assign(count + 1, 0);
      np->rsides.resize(count);
      std::vector<int64_t> meta(3 * (size_t)count);
      for (int i = 0; i < count; ++i) {
        const int64_t n = sides[i];
        np->rsides[i] = (int32_t)(2 * n);
        np->roff[i + 1] = np->roff[i] + svec_len(2 * n);
        np->maxn = std::max(np->maxn, n);
        meta[3 * i] = n;
        meta[3 * i + 1] = offsets[i];
        meta[3 * i + 2] = np->roff[i];
      }
      if (cudaMalloc(&np->meta_d, sizeof(int64_t) * meta.size()) != cudaSuccess ||
          cudaMalloc(&np->buf, sizeof(double) * (size_t)std::max<int64_t>(1, np->roff[count])) != cudaSuccess)
        return SCS_PSD_ENOMEM;
      if (cudaMemcpy(np->meta_d, meta.data(), sizeof(int64_t) * meta.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return SCS_PSD_ECUDA;
      hp = np.get();
      h->herm[key] = std::move(np);
    } else {
      hp = it->second.get();
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  launch_herm_embed(hp->meta_d, count, hp->maxn, x, hp->buf, s);
  if (cudaGetLastError() != cudaSuccess) return SCS_PSD_ECUDA;
  const IoSlot io{hp->buf, hp->buf, nullptr, nullptr, nullptr, nullptr};
  const int rc = poly_lo > 0.0 ? proj_poly(h, hp->buf, hp->buf, hp->roff.data(), hp->rsides.data(), count, poly_lo,
                                           poly_steps, opts, stream, 0.5)
                               : do_call(h, io, MODE_Y, hp->roff.data(), hp->rsides.data(), count, opts, stream);
  if (rc) return rc;
  launch_herm_extract(hp->meta_d, count, hp->maxn, hp->buf, y, s);
  if (cudaGetLastError() != cudaSuccess) return SCS_PSD_ECUDA;
  h->last_launches += 2;
  return SCS_PSD_OK;
}

// ---- factorization-free approximate projection (Conclusions) ----
// Scaled Newton-Schulz schedule: on [l, 1] the odd cubic
// g(t) = (alpha t / 2)(3 - alpha^2 t^2) peaks at 1 (t = 1/alpha) and maps
// [l, 1] into [g(l), 1] as long as g(l) <= g(1).  alpha is the minimax
// choice alpha^2 = 3 / (1 + l + l^2) of Chen & Chow (2014), where g(l) = g(1),
// capped at 2 cos(2 pi / 9), where g(1) = 1/2: the uncapped cubic sends the
// top of the interval down to the new lower bound, and the rounding of a
// split-precision product there is amplified by about 1 / l.
// steps = 0: the smallest K with 1 - l_K <= 1e-15.
constexpr int kPolyMaxSteps = 200;
constexpr double kPolyAutoTol = 1e-15;

int poly_schedule(double lo, int steps, std::vector<double>* a, std::vector<double>* b, double* lk) {
  if (!(lo > 0.0 && lo < 1.0) || steps < 0 || steps > kPolyMaxSteps) return -1;
  double l = lo;
  int k = 0;
  for (;;) {
    if (steps > 0 && k == steps) break;
    if (steps == 0 && (1.0 - l <= kPolyAutoTol || k == kPolyMaxSteps)) break;
    const double al = std::min(std::sqrt(3.0 / (1.0 + l + l * l)), 2.0 * std::cos(2.0 * M_PI / 9.0));
    if (a) a->push_back(1.5 * al);
    if (b) b->push_back(-0.5 * al * al * al);
    l = 0.5 * al * l * (3.0 - al * al * l * l);
    ++k;
  }
  if (lk) *lk = l;
  return k;
}

// Per cone (side n >= 1) four n x n buffers: X, the even iterates (from S_0),
// the odd iterates, and S^2 (its lower triangle), which the last product
// overwrites with Y.  One step is T = S S (lower triangle), S' = b T S + a S
// (lower triangle; T read as symmetric, a S added from the B operand); the
// end is Y = S_K X / 2 + X / 2 (lower triangle).  Every iterate is used as a
// symmetric matrix (a non-symmetric rounding residue is not a function of X,
// and the iteration amplifies it):
//  * FP64 products read full operands, so each new iterate is mirrored into
//    its upper triangle;
//  * in split-TF32 mode the cones of side >= 64 run on the long-contraction
//    tensor-core kernel, whose operands are sliced from lower triangles: S
//    once per step (it is both operands of S S, by symmetry, and the B
//    operand of T S), T once, X once per call; nothing is mirrored.
//  Smaller cones stay on FP64 products.
int build_poly(scs_psd_handle h, PolyPlan& P, const int64_t* offsets, const int32_t* sides, int32_t count,
               int precision, double lo, int steps, double nsq) {
  std::vector<double> ca, cb;
  const int K = poly_schedule(lo, steps, &ca, &cb, nullptr);
  if (K < 0) return SCS_PSD_EINVAL;
  P.precision = precision;
  P.steps = K;
  P.nsq = nsq;
  const bool split = precision == SCS_PSD_SPLIT_TF32;
  std::vector<PolyConeDev> cones;
  std::vector<int64_t> woff;
  int64_t work = 0;
  for (int i = 0; i < count; ++i) {
    const int64_t n = sides[i];
    if (n < 1) continue;
    PolyConeDev d{};
    d.n = n;
    d.xoff = offsets[i];
    d.part0 = P.nparts;
    d.nparts = (int)((svec_len(n) + kPolyChunk - 1) / kPolyChunk);
    d.mirror = (split && n >= 64) ? 0 : 1;
    P.nparts += d.nparts;
    P.maxn = std::max(P.maxn, n);
    woff.push_back(work);
    work += 4 * (int64_t)align_up((size_t)(n * n), 32);
    if (!d.mirror) work += 3 * (int64_t)align_up((size_t)((tc2_slice_floats((int)n, (int)n) + 1) / 2), 32);
    cones.push_back(d);
  }
  P.ncones = (int)cones.size();
  if (!P.ncones) return SCS_PSD_OK;
  if (cudaMalloc(&P.work, sizeof(double) * (size_t)work) != cudaSuccess) return SCS_PSD_ENOMEM;
  double* wbase = (double*)P.work;
  std::vector<double*> S1(P.ncones), T(P.ncones);
  std::vector<float*> slS(P.ncones, nullptr), slT(P.ncones, nullptr), slX(P.ncones, nullptr);
  bool any_small = false, any_big = false;
  for (int c = 0; c < P.ncones; ++c) {
    const int64_t stride = (int64_t)align_up((size_t)(cones[c].n * cones[c].n), 32);
    cones[c].X = wbase + woff[c];
    cones[c].S0 = cones[c].X + stride;
    S1[c] = cones[c].S0 + stride;
    cones[c].S1 = S1[c];
    T[c] = S1[c] + stride;
    cones[c].Y = T[c];
    if (!cones[c].mirror) {
      const int64_t sst = (int64_t)align_up((size_t)((tc2_slice_floats((int)cones[c].n, (int)cones[c].n) + 1) / 2), 32);
      double* sb = T[c] + stride;
      slS[c] = (float*)sb;
      slT[c] = (float*)(sb + sst);
      slX[c] = (float*)(sb + 2 * sst);
      any_big = true;
    } else {
      any_small = true;
    }
  }
  MetaBuilder mb;
  mb.sms = h->sms;
  mb.split = split;
  // the status word of cone c is encoded as (offset + 1) and patched after upload
  std::vector<int> part_cone(P.nparts);
  for (int c = 0; c < P.ncones; ++c)
    for (int q = 0; q < cones[c].nparts; ++q) part_cone[cones[c].part0 + q] = c;
  auto skip_of = [](int c) { return (const int*)(intptr_t)(c + 1); };
  using Op = PolyPlan::Op;
  // one grouped launch over the cones of one kind (big: tensor-core kernel on sliced operands)
  auto gemm_group = [&](bool big, auto make) {
    std::vector<GemmDesc> g;
    for (int c = 0; c < P.ncones; ++c)
      if ((cones[c].mirror == 0) == big) g.push_back(make(c));
    if (g.empty()) return;
    P.ops.push_back(Op{0, (int)P.gemms.size()});
    P.gemms.push_back(big ? mb.add_gemm_tc2(g, false) : mb.add_gemm(g));
  };
  auto slice_group = [&](auto src, auto dst) {
    std::vector<SliceJob> jobs;
    for (int c = 0; c < P.ncones; ++c) {
      if (cones[c].mirror) continue;
      const int n = (int)cones[c].n;
      jobs.push_back(SliceJob{src(c), nullptr, dst(c), n, n, n, 2});
    }
    if (jobs.empty()) return;
    P.ops.push_back(Op{1, (int)P.slices.size()});
    P.slices.push_back(mb.add_slices(jobs));
  };
  auto tc2_desc = [&](int c, const float* As, const float* Bs, const double* B, double* C, double alpha, double beta,
                      int flags) {
    const int n = (int)cones[c].n;
    GemmDesc g = mk(nullptr, n, B, n, C, n, n, n, n, alpha, beta, flags, skip_of(c));
    g.As = As;
    g.Bs = Bs;
    return g;
  };
  if (any_big) slice_group([&](int c) { return (const double*)cones[c].X; }, [&](int c) { return slX[c]; });
  for (int k = 0; k <= K; ++k) {
    auto Sin = [&](int c) { return (k % 2 == 0) ? cones[c].S0 : S1[c]; };
    auto Sout = [&](int c) { return (k % 2 == 0) ? S1[c] : cones[c].S0; };
    if (any_big) slice_group([&](int c) { return (const double*)Sin(c); }, [&](int c) { return slS[c]; });
    if (k < K) {
      gemm_group(true, [&](int c) { return tc2_desc(c, slS[c], slS[c], nullptr, T[c], 1.0, 0.0, GF_LOWER_C); });
      gemm_group(false, [&](int c) {
        const int n = (int)cones[c].n;
        return mk(Sin(c), n, Sin(c), n, T[c], n, n, n, n, 1.0, 0.0, GF_LOWER_C, skip_of(c));
      });
      if (any_big) slice_group([&](int c) { return (const double*)T[c]; }, [&](int c) { return slT[c]; });
      gemm_group(true, [&](int c) {
        return tc2_desc(c, slT[c], slS[c], Sin(c), Sout(c), cb[k], ca[k], GF_LOWER_C | GF_BETA_B);
      });
      gemm_group(false, [&](int c) {
        const int n = (int)cones[c].n;
        return mk(T[c], n, Sin(c), n, Sout(c), n, n, n, n, cb[k], ca[k], GF_SYM_A | GF_BETA_B | GF_LOWER_C,
                  skip_of(c));
      });
      if (any_small) P.ops.push_back(Op{2, k % 2 == 0 ? 0 : 1});
    } else {
      gemm_group(true, [&](int c) {
        return tc2_desc(c, slS[c], slX[c], cones[c].X, T[c], 0.5, 0.5, GF_LOWER_C | GF_BETA_B);
      });
      gemm_group(false, [&](int c) {
        const int n = (int)cones[c].n;
        return mk(Sin(c), n, cones[c].X, n, T[c], n, n, n, n, 0.5, 0.5, GF_LOWER_C | GF_BETA_B, skip_of(c));
      });
    }
  }
  // metadata: cones | ints (tile prefixes, partial-sum owners, status) | descriptors | partial sums | 1/sigma |
  // split-K scratch | io slot
  const int prefix_n = (int)mb.ints.size();
  std::vector<int> ints = mb.ints;
  const int part_cone_off = (int)ints.size();
  ints.insert(ints.end(), part_cone.begin(), part_cone.end());
  const int status_off = (int)ints.size();
  ints.resize(ints.size() + P.ncones, 0);
  (void)prefix_n;
  const size_t cones_b = align_up(sizeof(PolyConeDev) * P.ncones);
  const size_t ints_b = align_up(sizeof(int) * ints.size());
  const size_t descs_b = align_up(sizeof(GemmDesc) * std::max<size_t>(1, mb.descs.size()));
  const size_t part_b = align_up(sizeof(double) * P.nparts);
  const size_t inv_b = align_up(sizeof(double) * P.ncones);
  const size_t scratch_b = align_up(sizeof(double) * std::max<int64_t>(1, mb.scratch_doubles));
  const size_t io_b = align_up(sizeof(IoSlot));
  const size_t sjobs_b = align_up(sizeof(SliceJob) * std::max<size_t>(1, mb.sjobs.size()));
  const size_t slice_b = align_up(sizeof(float) * (size_t)std::max<int64_t>(1, mb.slice_floats));
  if (cudaMalloc(&P.meta, cones_b + ints_b + descs_b + part_b + inv_b + scratch_b + io_b + sjobs_b + slice_b) !=
      cudaSuccess)
    return SCS_PSD_ENOMEM;
  char* m = (char*)P.meta;
  P.cones_d = (PolyConeDev*)m;
  P.ints_d = (int*)(m + cones_b);
  P.descs_d = (GemmDesc*)(m + cones_b + ints_b);
  P.part_d = (double*)(m + cones_b + ints_b + descs_b);
  P.inv_d = (double*)(m + cones_b + ints_b + descs_b + part_b);
  double* scratch = (double*)(m + cones_b + ints_b + descs_b + part_b + inv_b);
  P.io_d = (IoSlot*)(m + cones_b + ints_b + descs_b + part_b + inv_b + scratch_b);
  P.sjobs_d = (SliceJob*)(m + cones_b + ints_b + descs_b + part_b + inv_b + scratch_b + io_b);
  float* slices = (float*)(m + cones_b + ints_b + descs_b + part_b + inv_b + scratch_b + io_b + sjobs_b);
  for (size_t q = 0; q < mb.sjobs.size(); ++q)
    if (mb.sjob_out[q] >= 0) mb.sjobs[q].out = slices + mb.sjob_out[q];
  P.part_cone_d = P.ints_d + part_cone_off;
  P.status_d = P.ints_d + status_off;
  for (int c = 0; c < P.ncones; ++c) cones[c].status = P.status_d + c;
  for (size_t q = 0; q < mb.descs.size(); ++q) {
    GemmDesc& g = mb.descs[q];
    g.partial = mb.part_off[q] >= 0 ? scratch + mb.part_off[q] : nullptr;
    if (g.skip) g.skip = P.status_d + ((intptr_t)g.skip - 1);
    if (mb.desc_as[q] >= 0) g.As = slices + mb.desc_as[q];
    if (mb.desc_bs[q] >= 0) g.Bs = slices + mb.desc_bs[q];
  }
  if (cudaMemcpy(P.cones_d, cones.data(), sizeof(PolyConeDev) * P.ncones, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(P.ints_d, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(P.descs_d, mb.descs.data(), sizeof(GemmDesc) * mb.descs.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      (!mb.sjobs.empty() &&
       cudaMemcpy(P.sjobs_d, mb.sjobs.data(), sizeof(SliceJob) * mb.sjobs.size(), cudaMemcpyHostToDevice) !=
           cudaSuccess))
    return SCS_PSD_ECUDA;
  return SCS_PSD_OK;
}

int run_poly_body(scs_psd_handle h, PolyPlan& P, cudaStream_t s, int64_t& n_launch) {
  CUDA_TRY(cudaMemsetAsync(P.status_d, 0, sizeof(int) * P.ncones, s));
  launch_poly_prepare(P.cones_d, P.ncones, P.part_cone_d, P.nparts, P.maxn, P.io_d, P.part_d, P.inv_d, P.nsq, s);
  n_launch += 2;
  LAUNCH_CHECK();
  int rc;
  for (const PolyPlan::Op& op : P.ops) {
    if (op.kind == 0) {
      if ((rc = run_gemm_at(P.descs_d, P.ints_d, P.gemms[op.idx], s, n_launch, P.sjobs_d))) return rc;
    } else if (op.kind == 1) {
      const SliceLaunch& L = P.slices[op.idx];
      launch_tc2_slice(P.sjobs_d + L.sjob_off, P.ints_d + L.sprefix_off, L.njobs, L.sctas, s);
      LAUNCH_CHECK();
    } else {
      launch_poly_mirror(P.cones_d, P.ncones, P.maxn, op.idx, s);
      LAUNCH_CHECK();
    }
  }
  launch_poly_pack(P.cones_d, P.ncones, P.maxn, P.io_d, s);
  LAUNCH_CHECK();
  launch_status_reduce(P.status_d, P.ncones, h->status_word, s);
  LAUNCH_CHECK();
  return SCS_PSD_OK;
}

int proj_poly(scs_psd_handle h, const double* x, double* y, const int64_t* offsets, const int32_t* sides,
              int32_t count, double lo, int32_t steps, const scs_psd_opts* opts, void* stream, double nsq = 1.0) {
  if (!h) return SCS_PSD_EINVAL;
  int rc = check_shapes(offsets, sides, count);
  if (rc) return rc;
  if (poly_schedule(lo, steps, nullptr, nullptr, nullptr) < 0) return SCS_PSD_EINVAL;
  if (count == 0 || offsets[count] == 0) return SCS_PSD_OK;
  if (!x || !y) return SCS_PSD_EINVAL;
  int precision = SCS_PSD_FP64;
  bool graphs = true;
  if (opts) {
    if (opts->precision != SCS_PSD_FP64 && opts->precision != SCS_PSD_SPLIT_TF32) return SCS_PSD_EINVAL;
    if (opts->graphs < 0 || opts->graphs > 1 || opts->stats != 0) return SCS_PSD_EINVAL;
    precision = opts->precision;
    graphs = opts->graphs == 0;
  }
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return SCS_PSD_ECUDA;
  char hdr[96];
  snprintf(hdr, sizeof(hdr), "p%d,l%.17g,k%d,q%.17g:", precision, lo, steps, nsq);
  const std::string key = std::string(hdr) + plan_key(sides, count, 0, 0, 0, 0);
  PolyPlan* P = nullptr;
  auto it = h->poly.find(key);
  if (it != h->poly.end()) {
    P = it->second.get();
  } else {
    if (h->poly.size() >= 8) {
      cudaDeviceSynchronize();
      h->poly.clear();
    }
    auto np = std::make_unique<PolyPlan>();
    if ((rc = build_poly(h, *np, offsets, sides, count, precision, lo, steps, nsq))) return rc;
    P = np.get();
    h->poly[key] = std::move(np);
  }
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  if (!P->ncones) return SCS_PSD_OK;
  int64_t n_launch = 0;
  launch_set_io(P->io_d, IoSlot{x, y, nullptr, nullptr, nullptr, nullptr}, s);
  LAUNCH_CHECK();
  h->last_replayed = false;
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  if (graphs && !P->gfailed && P->eager_runs > 0 && cudaStreamIsCapturing(s, &cst) == cudaSuccess &&
      cst == cudaStreamCaptureStatusNone) {
    if (!P->gexec) {
      if (!h->capture_stream && cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
        h->capture_stream = nullptr;
      cudaGraph_t graph = nullptr;
      int64_t nl = 0;
      if (h->capture_stream &&
          cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        const int brc = run_poly_body(h, *P, h->capture_stream, nl);
        const cudaError_t e = cudaStreamEndCapture(h->capture_stream, &graph);
        if (brc == SCS_PSD_OK && e == cudaSuccess && graph &&
            cudaGraphInstantiate(&P->gexec, graph, 0) == cudaSuccess)
          P->glaunches = nl;
        else
          P->gexec = nullptr;
        if (graph) cudaGraphDestroy(graph);
      }
      if (!P->gexec) P->gfailed = true;
      cudaGetLastError();
    }
    if (P->gexec) {
      CUDA_TRY(cudaGraphLaunch(P->gexec, s));
      h->last_launches = n_launch + P->glaunches;
      h->last_replayed = true;
      return SCS_PSD_OK;
    }
  }
  cudaGetLastError();
  if ((rc = run_poly_body(h, *P, s, n_launch))) return rc;
  ++P->eager_runs;
  h->last_launches = n_launch;
  return SCS_PSD_OK;
}

// ---- positivity post-processing (App. C instrument step, App. D process step) ----
int lambda_min(scs_psd_handle h, const double* x, double* lam, const int64_t* offsets, const int32_t* sides,
               int32_t count, const scs_psd_opts* opts, void* stream) {
  if (!h || !lam) return SCS_PSD_EINVAL;
  for (int i = 0; i < count && sides; ++i)
    if (sides[i] < 1) return SCS_PSD_EINVAL;  // a block without eigenvalues
  const IoSlot io{x, nullptr, nullptr, nullptr, nullptr, lam};
  return do_call(h, io, MODE_LMIN, offsets, sides, count, opts, stream);
}

int mix_identity(scs_psd_handle h, const double* x, double* y, const int64_t* offsets, const int32_t* sides,
                 int32_t count, const int32_t* groups, int32_t ngroups, const double* nu, double eps, double* p_out,
                 const scs_psd_opts* opts, void* stream) {
  if (!h || !x || !y || !groups || !nu || ngroups < 0 || count < 0) return SCS_PSD_EINVAL;
  int rc = check_shapes(offsets, sides, count);
  if (rc) return rc;
  if (groups[0] != 0 || groups[ngroups] != count) return SCS_PSD_EINVAL;
  for (int g = 0; g < ngroups; ++g)
    if (groups[g + 1] < groups[g]) return SCS_PSD_EINVAL;
  for (int i = 0; i < count; ++i)
    if (sides[i] < 1) return SCS_PSD_EINVAL;
  if (count == 0) return SCS_PSD_OK;
  MixPlan* mp = nullptr;
  {
    std::lock_guard<std::mutex> lock(h->mu);
    if (cudaSetDevice(h->device) != cudaSuccess) return SCS_PSD_ECUDA;
    std::string key = plan_key(sides, count, 0, 0, 0, 0);
    key.append(reinterpret_cast<const char*>(groups), sizeof(int32_t) * (size_t)(ngroups + 1));
    auto it = h->mix.find(key);
    if (it != h->mix.end()) {
      mp = it->second.get();
    } else {
      if (h->mix.size() >= 8) {
        cudaDeviceSynchronize();
        h->mix.clear();
      }
      auto np = std::make_unique<MixPlan>();
      np->count = count;
      np->ngroups = ngroups;
      std::vector<int64_t> meta(3 * (size_t)count);
      for (int g = 0; g < ngroups; ++g)
        for (int i = groups[g]; i < groups[g + 1]; ++i) {
          meta[3 * (size_t)i] = offsets[i];
          meta[3 * (size_t)i + 1] = sides[i];
          meta[3 * (size_t)i + 2] = g;
          np->maxn = std::max<int64_t>(np->maxn, sides[i]);
        }
      const size_t gb = align_up(sizeof(int) * (ngroups + 1)), mb2 = align_up(sizeof(int64_t) * meta.size());
      const size_t lb = align_up(sizeof(double) * count), vb = align_up(sizeof(double) * std::max(1, ngroups));
      if (cudaMalloc(&np->mem, gb + mb2 + lb + 2 * vb) != cudaSuccess) return SCS_PSD_ENOMEM;
      char* m = (char*)np->mem;
      np->groups_d = (int*)m;
      np->meta_d = (int64_t*)(m + gb);
      np->lam_d = (double*)(m + gb + mb2);
      np->nu_d = (double*)(m + gb + mb2 + lb);
      np->p_d = (double*)(m + gb + mb2 + lb + vb);
      if (cudaMemcpy(np->groups_d, groups, sizeof(int) * (ngroups + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(np->meta_d, meta.data(), sizeof(int64_t) * meta.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return SCS_PSD_ECUDA;
      mp = np.get();
      h->mix[key] = std::move(np);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (ngroups > 0) CUDA_TRY(cudaMemcpyAsync(mp->nu_d, nu, sizeof(double) * ngroups, cudaMemcpyHostToDevice, s));
  if ((rc = lambda_min(h, x, mp->lam_d, offsets, sides, count, opts, stream))) return rc;
  double* p = p_out ? p_out : mp->p_d;
  launch_mix_weight(mp->groups_d, mp->nu_d, mp->lam_d, eps, ngroups, p, s);
  launch_mix_apply(mp->meta_d, count, mp->maxn, x, y, p, mp->nu_d, s);
  if (cudaGetLastError() != cudaSuccess) return SCS_PSD_ECUDA;
  h->last_launches += 2;
  return SCS_PSD_OK;
}

// ---- the SCS iteration around the projection (App. D.1) ----
// The iterations for either operator (op.A dense, or op.kron structured with
// kron_n2 = N^2 doubles per work tensor).
int scs_run(scs_psd_handle h, ScsOp op, int64_t kron_n2, const double* b, const double* c, int64_t m, int64_t k,
            const int64_t* offsets, const int32_t* sides, int32_t count, double* u, double* v, int32_t iters,
            const scs_psd_opts* opts, void* stream) {
  if (!h || !b || !u || !v || m < 1 || k < 0 || iters < 0 || (k > 0 && !c)) return SCS_PSD_EINVAL;
  int rc = check_shapes(offsets, sides, count);
  if (rc) return rc;
  if (count < 1 || offsets[count] != m) return SCS_PSD_EINVAL;
  ScsPlan* sp = nullptr;
  {
    std::lock_guard<std::mutex> lock(h->mu);
    if (cudaSetDevice(h->device) != cudaSuccess) return SCS_PSD_ECUDA;
    auto it = h->scs.find({m, k});
    if (it != h->scs.end()) {
      sp = it->second.get();
    } else {
      if (h->scs.size() >= 8) {
        cudaDeviceSynchronize();
        h->scs.clear();
      }
      auto np = std::make_unique<ScsPlan>();
      np->m = m;
      np->k = k;
      const int nparts = scs_dot_parts(k + m);
      const int tchunks = scs_gemv_t_chunks(m, k);
      const size_t nd = (size_t)(k + m) * 2 + (size_t)std::max<int64_t>(k, 1) + (size_t)nparts + 2 + 2 * (size_t)m +
                        (size_t)tchunks * (size_t)std::max<int64_t>(k, 1);
      if (cudaMalloc(&np->mem, sizeof(double) * (nd + 64)) != cudaSuccess) return SCS_PSD_ENOMEM;
      double* q = (double*)np->mem;
      np->p = q; q += k + m;
      np->z = q; q += k + m;
      np->tk = q; q += std::max<int64_t>(k, 1);
      np->part = q; q += nparts;
      np->hp = q++;
      np->tau = q++;
      np->tin = q; q += m;
      np->uty = q; q += m;
      np->tpart = q;
      np->tchunks = tchunks;
      sp = np.get();
      h->scs[{m, k}] = std::move(np);
    }
    if (!op.A && kron_n2 > sp->kdoubles) {
      if (sp->kmem) cudaFree(sp->kmem);
      sp->kmem = nullptr;
      sp->kdoubles = 0;
      if (cudaMalloc(&sp->kmem, sizeof(double) * 2 * (size_t)kron_n2 + 256) != cudaSuccess) return SCS_PSD_ENOMEM;
      sp->kdoubles = kron_n2;
      sp->t0 = (double*)sp->kmem;
      sp->t1 = sp->t0 + kron_n2;
      sp->kstatus = (int*)(sp->t1 + kron_n2);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  int64_t launches = 6;  // dense: A^T in two launches
  op.tpart = sp->tpart;
  op.tchunks = sp->tchunks;
  if (!op.A) {
    op.t0 = sp->t0;
    op.t1 = sp->t1;
    op.status = h->status_word;
    kron_prepare();
    launches += 2 * (int64_t)kron_launches(op.kron) - 4;
  }
  launch_scs_setup(op, b, c, m, k, sp->p, sp->hp, sp->tk, sp->part, s);
  if (cudaGetLastError() != cudaSuccess) return SCS_PSD_ECUDA;
  const int64_t per_affine = op.A ? 7 : 3 + 2 * (int64_t)kron_launches(op.kron);
  for (int it = 0; it < iters; ++it) {
    launch_scs_affine(op, b, c, m, k, sp->p, sp->hp, u, v, sp->z, sp->tk, sp->part, sp->tau, sp->tin, sp->uty, s);
    if (cudaGetLastError() != cudaSuccess) return SCS_PSD_ECUDA;
    const IoSlot io{sp->tin, u + k, nullptr, nullptr, nullptr, nullptr};
    if ((rc = do_call(h, io, MODE_Y, offsets, sides, count, opts, stream))) return rc;
    launches += per_affine + h->last_launches;
    launch_scs_vy(v + k, sp->uty, u + k, m, s);
    if (cudaGetLastError() != cudaSuccess) return SCS_PSD_ECUDA;
    ++launches;
  }
  h->last_launches = launches;
  return SCS_PSD_OK;
}

int scs_iterate(scs_psd_handle h, const double* A, const double* b, const double* c, int64_t m, int64_t k,
                const int64_t* offsets, const int32_t* sides, int32_t count, double* u, double* v, int32_t iters,
                const scs_psd_opts* opts, void* stream) {
  if (k > 0 && !A) return SCS_PSD_EINVAL;
  ScsOp op;
  op.A = A;
  return scs_run(h, op, 0, b, c, m, k, offsets, sides, count, u, v, iters, opts, stream);
}

int scs_iterate_kron(scs_psd_handle h, const scs_psd_kron_op* K, const double* b, const double* c, double* u,
                     double* v, int32_t iters, const scs_psd_opts* opts, void* stream) {
  if (!h || !K || K->nmodes < 1 || K->nmodes > kKronMaxModes || K->nparams < 0) return SCS_PSD_EINVAL;
  ScsOp op;
  KronDev& kd = op.kron;
  kd.S = K->nmodes;
  int64_t N = 1, Kt = 1;
  for (int q = 0; q < kd.S; ++q) {
    const int d = K->dims[q], kb = K->nbasis[q];
    if (d < 1 || d > kKronMaxDim || kb < 1 || kb > d * d || !K->basis[q]) return SCS_PSD_EINVAL;
    kd.d[q] = d;
    kd.kb[q] = kb;
    kd.basis[q] = K->basis[q];
    N *= d;
    Kt *= kb;
  }
  if (N > kMaxSide || K->nparams > Kt || (K->nparams > 0 && !K->index)) return SCS_PSD_EINVAL;
  kd.index = K->index;
  kd.k = K->nparams;
  kd.N = N;
  kd.Kt = Kt;
  const int64_t offsets[2] = {0, svec_len(N)};
  const int32_t sides[1] = {(int32_t)N};
  return scs_run(h, op, N * N, b, c, svec_len(N), K->nparams, offsets, sides, 1, u, v, iters, opts, stream);
}

// ---- static-scratch entry point: no device allocation at all ----
// Callers that cannot allocate device memory (inside a memory pool that owns
// the GPU, in an embedding that forbids cudaMalloc after start-up) get the
// FP64 projection of one cone of side <= kStaticMaxSide with every buffer --
// the plan's metadata, the workspace and the status word -- carved from this
// file-scope array.  Every GPU that loads the library holds it until exit.
constexpr int64_t kStaticMaxSide = 256;
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticDeviceState {
  bool ready = false;
  char* base = nullptr;        // device address of g_static_scratch on this device
  scs_psd_handle_s hview;      // host-side view; its status word lives in the scratch
  std::unique_ptr<Plan> plan;  // layout the scratch currently holds
  int64_t plan_n = -1;
};
std::mutex g_static_mu;
StaticDeviceState g_static_state[64];

int proj_static(const double* x, double* y, int64_t n, void* stream) {
  if (n < 0 || n > kStaticMaxSide) return SCS_PSD_EINVAL;
  if (n == 0) return SCS_PSD_OK;
  if (!x || !y) return SCS_PSD_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SCS_PSD_ECUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticDeviceState& st = g_static_state[dev];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!st.ready || st.plan_n != n) {
    // set-up (the array's address, the plan copied in from host memory) is
    // not a stream operation that a capture could record
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cst) != cudaSuccess) return SCS_PSD_ECUDA;
    if (cst != cudaStreamCaptureStatusNone) return SCS_PSD_EINVAL;
  }
  if (!st.ready) {
    // once per device, with that device current: the array's device address
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return SCS_PSD_ECUDA;
    st.base = static_cast<char*>(p);
    st.hview.device = dev;
    cudaDeviceGetAttribute(&st.hview.sms, cudaDevAttrMultiProcessorCount, dev);
    st.hview.status_word = reinterpret_cast<int*>(st.base);  // first 256 bytes
    st.ready = true;
  }
  if (st.plan_n != n) {
    st.plan.reset();
    st.plan_n = -1;
    auto np = std::make_unique<Plan>();
    Arena ar;
    ar.base = st.base + 256;
    ar.size = kStaticScratchBytes - 256;
    ar.stream = s;
    const int32_t sides[1] = {(int32_t)n};
    const int rc = build_plan(&st.hview, *np, sides, 1, kDefaultBand, 0, 0, SCS_PSD_FP64, -1, Tuning(), &ar);
    if (rc) return rc;
    st.plan = std::move(np);
    st.plan_n = n;
  }
  if (cudaMemsetAsync(st.hview.status_word, 0, sizeof(int), s) != cudaSuccess) return SCS_PSD_ECUDA;
  const IoSlot io{x, y, nullptr, nullptr, nullptr, nullptr};
  return run_plan(&st.hview, *st.plan, io, MODE_Y, kDefaultWaitCycles, s, false);
}

}  // namespace

extern "C" {

int scs_psd_proj_static(const double* x, double* y, int64_t n, void* stream) { return proj_static(x, y, n, stream); }

int scs_psd_create(scs_psd_handle* h, int device) {
  if (!h) return SCS_PSD_EINVAL;
  *h = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return SCS_PSD_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return SCS_PSD_ECUDA;
  auto* H = new (std::nothrow) scs_psd_handle_s();
  if (!H) return SCS_PSD_ENOMEM;
  H->device = device;
  cudaDeviceGetAttribute(&H->sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&H->status_word, sizeof(int)) != cudaSuccess) {
    delete H;
    return SCS_PSD_ENOMEM;
  }
  cudaMemset(H->status_word, 0, sizeof(int));
  // the second stream and its fork/join events (without them everything runs on the caller's stream)
  if (cudaStreamCreateWithFlags(&H->aux_stream, cudaStreamNonBlocking) == cudaSuccess &&
      cudaEventCreateWithFlags(&H->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
      cudaEventCreateWithFlags(&H->ev_join, cudaEventDisableTiming) == cudaSuccess)
    H->use_aux = true;
  cudaGetLastError();
  *h = H;
  return SCS_PSD_OK;
}

int scs_psd_destroy(scs_psd_handle h) {
  if (!h) return SCS_PSD_EINVAL;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  h->plans.clear();
  h->herm.clear();
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  if (h->aux_stream) cudaStreamDestroy(h->aux_stream);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  cudaFree(h->status_word);
  delete h;
  return SCS_PSD_OK;
}

int scs_psd_proj(scs_psd_handle h, const double* x, double* y, int64_t n, const scs_psd_opts* opts, void* stream) {
  if (n < 0 || n > kMaxSide) return SCS_PSD_EINVAL;
  if (n == 0) return h ? SCS_PSD_OK : SCS_PSD_EINVAL;
  const int64_t offs[2] = {0, svec_len(n)};
  const int32_t sides[1] = {(int32_t)n};
  if (!y) return SCS_PSD_EINVAL;
  const IoSlot io{x, y, nullptr, nullptr, nullptr, nullptr};
  return do_call(h, io, MODE_Y, offs, sides, 1, opts, stream);
}

int scs_psd_proj_batched(scs_psd_handle h, const double* x, double* y, const int64_t* offsets, const int32_t* sides,
                         int32_t count, const scs_psd_opts* opts, void* stream) {
  const IoSlot io{x, y, nullptr, nullptr, nullptr, nullptr};
  return do_call(h, io, MODE_Y, offsets, sides, count, opts, stream);
}

int scs_psd_proj_vjp(scs_psd_handle h, const double* x, const double* g, double* xbar, double* y,
                     const int64_t* offsets, const int32_t* sides, int32_t count, const scs_psd_opts* opts,
                     void* stream) {
  const IoSlot io{x, y, g, xbar, nullptr, nullptr};
  return do_call(h, io, MODE_VJP | (y ? MODE_Y : 0), offsets, sides, count, opts, stream);
}

int scs_psd_proj_store(scs_psd_handle h, const double* x, double* y, double* V, double* lam, const int64_t* offsets,
                       const int32_t* sides, int32_t count, const scs_psd_opts* opts, void* stream) {
  const IoSlot io{x, y, nullptr, nullptr, V, lam};
  return do_call(h, io, MODE_EXPORT | (y ? MODE_Y : 0), offsets, sides, count, opts, stream);
}

int scs_psd_vjp_stored(scs_psd_handle h, const double* V, const double* lam, const double* g, double* xbar,
                       const int64_t* offsets, const int32_t* sides, int32_t count, const scs_psd_opts* opts,
                       void* stream) {
  const IoSlot io{nullptr, nullptr, g, xbar, const_cast<double*>(V), const_cast<double*>(lam)};
  return do_call(h, io, MODE_IMPORT | MODE_VJP, offsets, sides, count, opts, stream);
}

int scs_psd_reserve(scs_psd_handle h, int64_t max_n, int32_t max_count, const scs_psd_opts* opts) {
  if (!h || max_n < 0 || max_n > kMaxSide || max_count < 0) return SCS_PSD_EINVAL;
  if (max_n == 0 || max_count == 0) return SCS_PSD_OK;
  int side = 0, precision = SCS_PSD_FP64;
  Tuning tune;
  if (opts) {
    if (opts->precision != SCS_PSD_FP64 && opts->precision != SCS_PSD_SPLIT_TF32) return SCS_PSD_EINVAL;
    if (opts->band < 0 || opts->band > kMaxBand || opts->side < 0 || opts->side > 2) return SCS_PSD_EINVAL;
    precision = opts->precision;
    side = opts->side;
    tune.band = opts->band;
  }
  const std::vector<int32_t> sides((size_t)max_count, (int32_t)max_n);
  std::lock_guard<std::mutex> lock(h->mu);
  if (cudaSetDevice(h->device) != cudaSuccess) return SCS_PSD_ECUDA;
  if (!(opts && opts->band)) {
    auto t = h->tuned.find(tune_key(sides.data(), max_count, precision));
    if (t != h->tuned.end()) tune = t->second;
  }
  // the projection's plan (the derivative's is built on its first call)
  Plan* P = nullptr;
  return get_plan(h, sides.data(), max_count, 0, side, precision, tune, &P);
}

int scs_psd_proj_hermitian(scs_psd_handle h, const double* x, double* y, const int64_t* offsets,
                           const int32_t* sides, int32_t count, const scs_psd_opts* opts, void* stream) {
  return proj_hermitian(h, x, y, offsets, sides, count, opts, stream);
}

int scs_psd_proj_poly(scs_psd_handle h, const double* x, double* y, const int64_t* offsets, const int32_t* sides,
                      int32_t count, double lo, int32_t steps, const scs_psd_opts* opts, void* stream) {
  return proj_poly(h, x, y, offsets, sides, count, lo, steps, opts, stream);
}

int scs_psd_lambda_min(scs_psd_handle h, const double* x, double* lam_min, const int64_t* offsets,
                       const int32_t* sides, int32_t count, const scs_psd_opts* opts, void* stream) {
  return lambda_min(h, x, lam_min, offsets, sides, count, opts, stream);
}

int scs_psd_mix_identity(scs_psd_handle h, const double* x, double* y, const int64_t* offsets, const int32_t* sides,
                         int32_t count, const int32_t* groups, int32_t ngroups, const double* nu, double eps,
                         double* p_out, const scs_psd_opts* opts, void* stream) {
  return mix_identity(h, x, y, offsets, sides, count, groups, ngroups, nu, eps, p_out, opts, stream);
}

int scs_psd_scs_iterate_kron(scs_psd_handle h, const scs_psd_kron_op* op, const double* b, const double* c, double* u,
                             double* v, int32_t iters, const scs_psd_opts* opts, void* stream) {
  return scs_iterate_kron(h, op, b, c, u, v, iters, opts, stream);
}

int scs_psd_scs_iterate(scs_psd_handle h, const double* A, const double* b, const double* c, int64_t m, int64_t k,
                        const int64_t* offsets, const int32_t* sides, int32_t count, double* u, double* v,
                        int32_t iters, const scs_psd_opts* opts, void* stream) {
  return scs_iterate(h, A, b, c, m, k, offsets, sides, count, u, v, iters, opts, stream);
}

int scs_psd_proj_poly_hermitian(scs_psd_handle h, const double* x, double* y, const int64_t* offsets,
                                const int32_t* sides, int32_t count, double lo, int32_t steps,
                                const scs_psd_opts* opts, void* stream) {
  if (poly_schedule(lo, steps, nullptr, nullptr, nullptr) < 0) return SCS_PSD_EINVAL;
  return proj_hermitian(h, x, y, offsets, sides, count, opts, stream, lo, steps);
}

int32_t scs_psd_poly_schedule(double lo, int32_t steps, double* a, double* b, double* l_final) {
  std::vector<double> ca, cb;
  const int k = poly_schedule(lo, steps, &ca, &cb, l_final);
  if (k < 0) return -SCS_PSD_EINVAL;
  if (a) std::copy(ca.begin(), ca.end(), a);
  if (b) std::copy(cb.begin(), cb.end(), b);
  return k;
}

int scs_psd_autotune(scs_psd_handle h, const double* x, const int64_t* offsets, const int32_t* sides, int32_t count,
                     const scs_psd_opts* opts, void* stream, int32_t* chosen, double* best_ms) {
  return autotune(h, x, offsets, sides, count, opts, stream, chosen, best_ms);
}

int scs_psd_last_tuning(scs_psd_handle h, int32_t* out) {
  if (!h || !out) return SCS_PSD_EINVAL;
  out[0] = h->last_tune.band;
  out[1] = h->last_tune.gemm_ctas;
  out[2] = h->last_tune.bt1_cols;
  out[3] = h->last_tune.sy_share;
  return SCS_PSD_OK;
}

int scs_psd_status(scs_psd_handle h, int32_t* device_status) {
  if (!h || !device_status) return SCS_PSD_EINVAL;
  cudaSetDevice(h->device);
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return SCS_PSD_ECUDA;
  int v = 0;
  if (cudaMemcpy(&v, h->status_word, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SCS_PSD_ECUDA;
  cudaMemset(h->status_word, 0, sizeof(int));
  int code = SCS_PSD_OK;
  if (v & ST_BADARG) code = SCS_PSD_EINVAL;
  else if (v & ST_TIMEOUT) code = SCS_PSD_ETIMEOUT;
  else if (v & ST_NOCONV) code = SCS_PSD_ENOCONV;
  else if (v & ST_NONFINITE) code = SCS_PSD_ENONFINITE;
  *device_status = code;
  return SCS_PSD_OK;
}

int scs_psd_last_stats(scs_psd_handle h, scs_psd_cone_stats* out, int32_t count) {
  if (!h || !out || count < 0) return SCS_PSD_EINVAL;
  std::lock_guard<std::mutex> lock(h->mu);
  if (h->last_stats_key.empty() || count != h->last_stats_count) return SCS_PSD_EINVAL;
  auto it = h->plans.find(h->last_stats_key);
  if (it == h->plans.end() || !it->second->stats_out_d) return SCS_PSD_EINVAL;
  if (count == 0) return SCS_PSD_OK;
  static_assert(sizeof(ConeStats) == sizeof(scs_psd_cone_stats), "statistics record layout");
  if (cudaSetDevice(h->device) != cudaSuccess || cudaStreamSynchronize(h->last_stream) != cudaSuccess ||
      cudaMemcpy(out, it->second->stats_out_d, sizeof(ConeStats) * count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SCS_PSD_ECUDA;
  return SCS_PSD_OK;
}

int64_t scs_psd_last_launch_count(scs_psd_handle h) { return h ? h->last_launches : -1; }

int scs_psd_last_replayed(scs_psd_handle h) { return h ? (h->last_replayed ? 1 : 0) : -1; }

int scs_psd_trace(scs_psd_handle h, int enable) {
  if (!h) return SCS_PSD_EINVAL;
  h->trace = enable != 0;
  return SCS_PSD_OK;
}

int scs_psd_trace_read(scs_psd_handle h, double* ms, int64_t* intervals) {
  if (!h || !ms || !intervals) return SCS_PSD_EINVAL;
  cudaSetDevice(h->device);
  for (int p = 0; p < SCS_PSD_NPHASES; ++p) { ms[p] = 0.0; intervals[p] = 0; }
  int rc = SCS_PSD_OK;
  for (auto& e : h->trace_ev) {
    float t = 0.f;
    if (cudaEventSynchronize(e.second.second) != cudaSuccess ||
        cudaEventElapsedTime(&t, e.second.first, e.second.second) != cudaSuccess)
      rc = SCS_PSD_ECUDA;
    if (e.first >= 0 && e.first < SCS_PSD_NPHASES) { ms[e.first] += t; intervals[e.first] += 1; }
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
  h->trace_ev.clear();
  return rc;
}

const char* scs_psd_strerror(int code) {
  switch (code) {
    case SCS_PSD_OK: return "ok";
    case SCS_PSD_EINVAL: return "invalid argument";
    case SCS_PSD_ENOMEM: return "out of memory";
    case SCS_PSD_ECUDA: return "CUDA runtime error";
    case SCS_PSD_ETIMEOUT: return "bounded device wait ran out";
    case SCS_PSD_ENOCONV: return "iteration did not converge";
    case SCS_PSD_ENONFINITE: return "non-finite input";
    default: return "unknown error";
  }
}

}  // extern "C"
