// Internal declarations of the scs_psd CUDA library (not part of the ABI).
//
// Pipeline for one cone of side n >= 2 (every step is a kernel here):
//   svec unpack            -> dense symmetric A (column-major, ld = n)
//   dense -> band          blocked Householder, panels of width b factored by
//                          a thread-block cluster, trailing two-sided update by
//                          grouped GEMMs (sy2sb form W = X - 1/2 V T^T V^T X)
//   band -> tridiagonal    pipelined bulge chasing, one sweep per CTA at a time
//   tridiagonal eigensolve divide and conquer (Cuppen tearing, deflation,
//                          secular equation, Loewner/Gu-Eisenstat vectors)
//   back-transformation    stage-2 reflectors, then stage-1 WY blocks
//   clipped reconstruction lower triangle of V_k diag(l_k) V_k^T written
//                          straight into svec (positive part, or X minus the
//                          negative part by the Moreau decomposition)
#pragma once
#include <atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"

namespace scs {

// True on the first call for the current device with this flag word.  The
// launchers set their kernels' function attributes (dynamic shared memory
// beyond 48 KB, non-portable cluster sizes) once per device: each device's
// context keeps its own.
inline bool first_on_device(std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  return (done.fetch_or(bit) & bit) == 0;
}


// Per-cone device status bits (OR-ed together).
enum : int { ST_NONFINITE = 1, ST_NOCONV = 2, ST_TIMEOUT = 4, ST_BADARG = 8 };

constexpr int kMaxBand = 32;  // largest supported bandwidth b
constexpr int kSy1Block = 32; // reflectors per block of the one-stage back-transformation

// ------------------------------------------------------------------ GEMM
// C = alpha * op(A) op(B) + beta * C on column-major FP64 operands.
enum : int {
  GF_TRANS_A = 1,   // op(A) = A^T
  GF_TRANS_B = 2,   // op(B) = B^T
  GF_SYM_A = 4,     // A is square symmetric, only its lower triangle is read
  GF_LOWER_C = 8,   // only the lower triangle (i >= j) of C is computed
  GF_SCALE_B = 16,  // op(B)(k, j) is multiplied by bscale[k]
  GF_TRANS_C = 32,  // result element (i, j) is stored at C[j + i * ldc]
  GF_BETA_B = 64,   // the beta term reads B(i, j) = B[i + j * ldb] instead of C(i, j) (B not transposed, M = K)
};

struct GemmDesc {
  const double* A;
  const double* B;
  double* C;
  const double* bscale;  // GF_SCALE_B
  const int* dynM;       // if set: M = min(M, *dynM) (bounds only; layouts use the static M)
  const int* dynN;       // if set: N = min(N, *dynN)
  const int* dynK;       // if set: K = min(K, *dynK)
  const int* colmap;     // if set: column j of the result goes to column colmap[j] of C
  const int* skip;       // if set and *skip != 0 the problem is skipped (cone status)
  int M, N, K;
  int lda, ldb, ldc;
  double alpha, beta;
  int flags;
  int splitk;            // number of K slices (1: no split)
  double* partial;       // splitk > 1: scratch of splitk * M * N doubles
  const float* As;       // long-contraction tensor-core kernel: op(A) sliced by launch_tc2_slice
  const float* Bs;       //   and op(B) (as its N x K transpose)
};

// One operand of a long-contraction split-TF32 product, sliced once: the
// element (row, k) of a rows x K matrix is p[row + k ld] (mode 0),
// p[k + row ld] (mode 1) or the lower triangle of a symmetric p (mode 2),
// times scale[k] if scale is set; out receives ceil(rows/128) x ceil(K/16)
// blocks of 3 x 2048 floats.
struct SliceJob {
  const double* p;
  const double* scale;
  float* out;
  int64_t ld;
  int rows, K, mode;
  const int* dynRows;  // if set: rows at or past *dynRows are zero
  const int* dynK;     // if set: columns k at or past *dynK are zero
};
void launch_tc2_slice(const SliceJob* jobs, const int* prefix, int njobs, int total, cudaStream_t s);
void launch_tc2_gemm(const GemmDesc* descs, const int* tile_prefix, int count, int total_tiles, cudaStream_t s);
int64_t tc2_slice_floats(int rows, int K);
int tc2_slice_ctas(int rows, int K);

constexpr int kGemmBK = 16;
// 64x64, 128x16, 16x128, 16x16; GEMM_SQUARE_DF: 64x64 in double-float arithmetic (operands of magnitude
// at most about 1e30, as the eigenvector blocks of the divide and conquer)
enum : int { GEMM_SQUARE = 0, GEMM_TALL = 1, GEMM_SHORT = 2, GEMM_SMALL = 3, GEMM_SQUARE_DF = 4 };

void gemm_tile_shape(int variant, int* bm, int* bn);

// Split-TF32 tensor-core GEMM (tcgen05), same descriptors; tile 128 x 16 or 128 x 64.
enum : int { TC_N16 = 16, TC_N64 = 64 };
void tc_tile_shape(int variant, int* bm, int* bn);
void launch_tc_gemm(const GemmDesc* descs, const int* tile_prefix, int count, int total_tiles, int variant,
                    cudaStream_t s);
void launch_gemm_reduce(const GemmDesc* descs, int count, int64_t max_mn, cudaStream_t s);

// Launch one grouped GEMM over `count` problems whose descriptors are in
// device memory (`descs`); tile_prefix[p] = first tile of problem p,
// tile_prefix[count] = total tiles.  Problems with splitk > 1 are summed by a
// second kernel (needs_reduce), max_mn = largest M*N of the launch.
void launch_gemm(const GemmDesc* descs, const int* tile_prefix, int count, int total_tiles, int variant,
                 int needs_reduce, int64_t max_mn, cudaStream_t s);

// ------------------------------------------------------------------ cones
// Device view of one cone of the "large" path (n >= 2).
struct ConeDev {
  int64_t n;
  int64_t xoff;     // offset of the cone in the svec buffers
  int64_t voff;     // offset of the cone's n x n eigenvector block in IoSlot::V
  int64_t loff;     // offset of the cone's n eigenvalues in IoSlot::lam
  int path;         // 0: two-stage (dense -> band -> tridiagonal), 1: one-stage tridiagonalisation
  int b;            // bandwidth of stage 1 / 2
  int npanels;
  int nsweeps;      // number of bulge-chasing sweeps (n - 2, at least 0)
  int kmax;         // reflector slots per sweep
  double* A;        // n*n dense matrix (column-major)
  double* band;     // n * (2b) lower band with room for the bulge fill
  double* refl;     // nsweeps * kmax * (b + 1): c, u_0 .. u_{L-1} of H = I - c u u^T
  int* prog;        // nsweeps progress counters of the bulge chasing
  double* d;        // n diagonal of the tridiagonal matrix
  double* e;        // n off-diagonal (e[i] couples i and i+1)
  double* V1;       // stage-1 reflectors: npanels blocks of n*b (rows m_p); one-stage cones: FP32 pairs
                    // once larft1 has run (8 bytes per element either way)
  double* T1;       // npanels blocks of b*b (one-stage cones: FP32 pairs)
  double* Y;        // n*b   A22 V
  double* X;        // n*b   Y T
  double* U3;       // n*3b  [V | W | V] for the rank-2b update
  double* Mb;       // b*b
  double* Nb;       // b*b
  double* QA;       // n*n   D&C eigenvector blocks (ping)
  double* QB;       // n*n   (pong)
  double* lamA;     // n
  double* lamB;     // n
  double* Qin;      // n*n   permuted/deflated eigenvector block of a merge
  double* Ucm;      // n*n   secular eigenvectors, row i = eigenvector i
  double* Z;        // n*n   kept eigenvectors (columns), then back-transformed
  double* lamk;     // n     kept eigenvalues
  double* dsrt;     // n     sorted, deflated poles of each merge node
  double* zk;       // n     normalised rank-one vector on the kept poles
  double* dval;     // n     deflated eigenvalues
  double* tau;      // n     secular root offsets
  double* zhat;     // n     Loewner-corrected z
  double* rot;      // 2n    Givens rotations (c, s) of the deflation
  double* rho;      // n     rank-one weight per merge node (indexed by start)
  int* iperm;       // n     sorted position -> column of the child blocks
  int* ifp;         // n     sorted position -> column of the merged block (kept first)
  int* irot;        // 2n    rotation column pairs
  int* iorg;        // n     origin pole of each secular root
  int* imap;        // n     output column of each kept eigenvector of a merge
  int* icnt;        // 4n    per merge node: kept, deflated, rotations, kept-of-root (indexed by start)
  int* kinfo;       // [0] k kept, [1] route (0: positive part, 1: X - negative part), [2] kept secular
                    // roots, [3] keep all eigenpairs (derivative), [4] side option, [5] first kept root,
                    // [6] all-pairs mode: |S|, the pairs of the route's side, which come first,
                    // [7] the one-stage reduction wrote V1 as FP32 pairs (else FP64, converted by larft1),
                    // [8] eigenvalues > 0, [9] eigenvalues < 0, [10] largest biased exponent of the
                    // derivative's input g (16 ints)
  int* status;      // per-cone status bits
  double* tau1;     // n     tau of the one-stage reflectors (read by larft1 while the divide and conquer runs)
  int cidx;         // position of the cone in the call's shape list
};

// One merge node of the divide and conquer tree.
// Merges of at most this many rows build their permuted eigenvector block and
// apply their deflation rotations inside dc_prepare_kernel.
constexpr int kDcFuseK = 64;

struct MergeNode {
  int cone;
  int s;       // first row of the merged block
  int n1, n2;  // child sizes (n2 may be 0: plain copy)
  int root;    // 1 if this merge produces the cone's final decomposition
  int level;   // tree level (selects the ping-pong buffers)
};

// The caller's buffers of one call.  Kernels read them from this device slot
// (written by launch_set_io at the start of every call), so the rest of a
// call's launch sequence does not depend on them and can be replayed as a
// recorded graph.
struct IoSlot {
  const double* x;
  double* y;
  const double* g;
  double* xbar;
  double* V;    // all eigenvectors, cone i at voff (n x n column-major): written or read
  double* lam;  // all eigenvalues, cone i at loff
};

// Output modes of one call (bits).
enum : int {
  MODE_Y = 1,       // y = Pi(x)
  MODE_VJP = 2,     // xbar = DPi(X)[smat(g)]
  MODE_EXPORT = 4,  // write the eigendecomposition to io->V, io->lam
  MODE_IMPORT = 8,  // take the eigendecomposition from io->V, io->lam instead of computing it
  MODE_LMIN = 16,   // io->lam[i] = smallest eigenvalue of cone i (stops at the tridiagonal form)
  MODE_STATS = 32,  // per-cone statistics of the result (with MODE_Y)
};
constexpr int kModes = 64;

// ------------------------------------------------------------------ statistics
// Per-cone statistics of a call (layout of scs_psd_cone_stats in the ABI).
struct ConeStats {
  int k_pos, k_neg, route, status;
  double complementarity, norm_y, norm_x, reserved;
};
constexpr int kStatsChunk = 32768;  // svec entries per partial sum
// One cone of the call's shape list: its svec range, its device cone (-1 for
// sides 0 and 1) and its partial sums [part0, part0 + nparts).
struct StatsCone {
  int64_t off, len;
  int cone, side, part0, nparts;
};
void launch_stats_save_x(const IoSlot* io, double* xs, int64_t total, cudaStream_t s);
void launch_stats(const StatsCone* sc, int count, const int* part_cone, int nparts, const ConeDev* cones,
                  const int* triv_status, const double* xs, const IoSlot* io, double* part, ConeStats* out,
                  cudaStream_t s);

// ------------------------------------------------------------------ kernels
void launch_set_io(IoSlot* slot, const IoSlot& v, cudaStream_t s);
// which = 0: unpack io->x, 1: unpack io->g
void launch_unpack(const ConeDev* cones, int ncones, int64_t maxn2, const IoSlot* io, int which, cudaStream_t s);
// Cones of side 1: y, xbar, (V, lam) by `mode`; offs holds count svec, V and lam offsets each
// offs: 4 * count (svec, V, lam offsets and the cone's position in the call)
void launch_trivial(const int64_t* offs, int count, const IoSlot* io, int mode, int* status, cudaStream_t s);
void launch_panel(const ConeDev* cones, const int* cone_ids, int njobs, int panel, int b,
                  int cluster, int rows_per_cta, cudaStream_t s);
void launch_band_extract(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s);
int launch_bulge(const ConeDev* cones, int ncones, const int* cta_cone, const int* cta_rank,
                 const int* cta_count, int nctas, int b, long long wait_limit, cudaStream_t s);
int bulge_max_ctas(int b);
void launch_tridiag_extract(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s);
void launch_dc_leaves(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s);
void launch_dc_prepare(const ConeDev* cones, const MergeNode* nodes, int nnodes, int maxK, cudaStream_t s);
void launch_dc_secular(const ConeDev* cones, const MergeNode* nodes, const int* pos_node, int64_t total_pos,
                       int maxK, cudaStream_t s);
void launch_dc_loewner(const ConeDev* cones, const MergeNode* nodes, const int* pos_node, int64_t total_pos,
                       cudaStream_t s);
void launch_dc_select(const ConeDev* cones, const MergeNode* nodes, int nnodes, int maxK, cudaStream_t s);
void launch_dc_vectors(const ConeDev* cones, const MergeNode* nodes, const int* pos_node, int64_t total_pos,
                       int maxK, cudaStream_t s);
void launch_dc_copy_deflated(const ConeDev* cones, const MergeNode* nodes, int nnodes, int maxK, cudaStream_t s);
void launch_dc_build_qin(const ConeDev* cones, const MergeNode* nodes, int nnodes, int maxK, cudaStream_t s);
void launch_dc_apply_rot(const ConeDev* cones, const MergeNode* nodes, const int* pos_node, int64_t total_pos,
                         cudaStream_t s);
void launch_backtr2(const ConeDev* cones, int ncones, int maxn, int maxk, int kexp, int band, cudaStream_t s);
size_t panel_smem_bytes(int b, int R);
// Z, lamk (all n eigenpairs) <-> io->V, io->lam
void launch_export_eig(const ConeDev* cones, int ncones, int64_t maxn, const IoSlot* io, cudaStream_t s);
void launch_import_eig(const ConeDev* cones, int ncones, int64_t maxn, const IoSlot* io, cudaStream_t s);
// derivative: eigenpairs into S-first order (3 launches), then the k_S x n scaling
void launch_vjp_reorder(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s);
void launch_vjp_scale(const ConeDev* cones, int ncones, int64_t maxn, cudaStream_t s);
void launch_vjp_gexp(const ConeDev* cones, int ncones, const IoSlot* io, cudaStream_t s);
// The derivative's input scale: G enters the contractions as G / up, up = 2^(e - 1023)
// for e the largest biased exponent of g (kinfo[10]), clamped to [1, 2045].
__device__ __forceinline__ double vjp_gscale_up(int e) {
  e = e < 1 ? 1 : (e > 2045 ? 2045 : e);
  return __longlong_as_double((long long)e << 52);
}
__device__ __forceinline__ double vjp_gscale_down(int e) {
  e = e < 1 ? 1 : (e > 2045 ? 2045 : e);
  return __longlong_as_double((long long)(2046 - e) << 52);
}
void launch_pack_lower(const ConeDev* cones, int ncones, int64_t maxn, const IoSlot* io, cudaStream_t s);
void launch_recon(const ConeDev* cones, int ncones, int maxn, const IoSlot* io, cudaStream_t s);
int sytrd1_max_ctas(int maxn);
int sytrd1_max_ctas_for(size_t smem_bytes);
// dynamic shared memory of one CTA for side n in a group of G (resident: its columns in shared memory)
size_t sytrd1_smem_bytes(int n, int G, bool resident);
// the double-float route with the columns in global memory (glb launches)
size_t sytrd1_glb_smem_bytes(int n);
int launch_sytrd1(const ConeDev* cones, const int* cta_cone, const int* cta_rank, const int* cta_count, int nctas,
                  int maxn, size_t smem_bytes, int glb, long long wait_limit, cudaStream_t s);
void launch_larft1(const ConeDev* cones, const int* blk_cone, const int* blk_index, int nblocks, cudaStream_t s);
// Z <- Q1 Z for the stage-1 blocks in one launch (CTA tables as launch_sytrd1); cones of side <= bt1_max_side()
void launch_bt1(const ConeDev* cones, const int* cta_cone, const int* cta_rank, const int* cta_count, int nctas,
                int maxn, cudaStream_t s);
int bt1_max_side();
// whether a launch whose largest side is maxn can stage the reflector blocks in
// shared memory (it then does when it has at most one CTA per SM)
bool bt1_stages(int maxn);
// y = svec(S) or x - svec(S) from the lower triangle of S = Z diag(l) Z^T held in QA (split mode)
void launch_pack_recon(const ConeDev* cones, int ncones, int64_t maxn, const IoSlot* io, cudaStream_t s);
// complex Hermitian cones <-> real symmetric embeddings of side 2n (meta: n, Hermitian offset, real offset)
void launch_herm_embed(const int64_t* meta, int count, int64_t maxn, const double* hs, double* ms, cudaStream_t s);
void launch_herm_extract(const int64_t* meta, int count, int64_t maxn, const double* ms, double* hs, cudaStream_t s);
void launch_status_reduce(const int* status, int count, int* out, cudaStream_t s);
void launch_lmin(const ConeDev* cones, int ncones, const IoSlot* io, cudaStream_t s);
// Structured affine operator (App. D.2): column j of A is svec of the
// Kronecker product of local basis matrices F_s[mu_s], mu the multi-index of
// index[j] (C order over kb); local matrix b of mode s is column-major at
// basis[s] + b d_s^2.
constexpr int kKronMaxModes = 6;
constexpr int kKronMaxDim = 8;
struct KronDev {
  int S;
  int d[kKronMaxModes], kb[kKronMaxModes];
  const double* basis[kKronMaxModes];
  const int64_t* index;
  int64_t k, N, Kt;  // parameters, matrix side (prod d), prod kb
};
void kron_prepare();
int kron_launches(const KronDev& op);
// out = a1 (+ a2) + A x; t0, t1: work tensors of N^2 doubles each; bad indices set ST_BADARG in *status
void launch_kron_apply(const KronDev& op, const double* x, const double* a1, const double* a2, double* out,
                       double* t0, double* t1, int* status, cudaStream_t s);
// out = A^T (a1 (+ a2))
void launch_kron_apply_t(const KronDev& op, const double* a1, const double* a2, double* out, double* t0, double* t1,
                         int* status, cudaStream_t s);

// SCS iteration (App. D.1) around the projection; A with orthonormal columns,
// dense (m x k, column-major) or structured
struct ScsOp {
  const double* A = nullptr;  // dense, or null for the structured operator
  KronDev kron{};
  double* t0 = nullptr;
  double* t1 = nullptr;
  int* status = nullptr;
  double* tpart = nullptr;  // dense A^T: tchunks x k partial dot products
  int tchunks = 1;
};
int scs_dot_parts(int64_t len);
int scs_gemv_t_chunks(int64_t m, int64_t k);
void launch_scs_setup(const ScsOp& op, const double* b, const double* c, int64_t m, int64_t k, double* p,
                      double* hp, double* tk, double* part, cudaStream_t s);
void launch_scs_affine(const ScsOp& op, const double* b, const double* c, int64_t m, int64_t k, const double* p,
                       const double* hp, double* u, double* v, double* z, double* tk, double* part, double* tau,
                       double* tin, double* uty, cudaStream_t s);
void launch_scs_vy(double* vy, const double* uty, const double* uy, int64_t m, cudaStream_t s);
void launch_mix_weight(const int* groups, const double* nu, const double* lam, double eps, int ngroups, double* p,
                       cudaStream_t s);
void launch_mix_apply(const int64_t* meta, int count, int64_t maxn, const double* x, double* y, const double* p,
                      const double* nu, cudaStream_t s);

// ------------------------------------------------------------------ complex Hermitian cones (native)
// One complex Hermitian cone of side n: the real plan's cone (same index)
// holds its tridiagonal form (d, e), status, counters and the divide and
// conquer's output (Z, lamk, kinfo); the complex workspace holds the
// publication slabs of the reduction, the reflectors in blocks of 32 (V:
// rows 32 q + 1 .. n-1 of block q, unit diagonal, zeros above), their T
// factors, tau, and W = Q Z.
struct HConeDev {
  int64_t n, xoff;  // side, offset of the cone in the Hermitian svec buffers (n^2 reals each)
  double* d;
  double* e;
  int* status;
  int* prog;
  const double* Z;
  const double* lamk;
  const int* kinfo;
  dfl* pub;   // 2 n (n - 1) words
  cdf* V;     // hcone_v_elems(n)
  cdf* T;     // hcone_t_elems(n)
  cdf* tau;   // n
  cdf* W;     // n x n
};
constexpr int kHermNativeMax = 1100;  // largest side reduced natively (the columns must fit in shared memory)
constexpr size_t kHetrdSmemMax = 220 * 1024;  // dynamic shared memory of one reduction CTA
size_t hetrd1_smem_bytes(int n, int G);
int hetrd1_max_ctas_for(size_t smem);
size_t hcone_pub_doubles(int64_t n);
size_t hcone_v_elems(int64_t n);
size_t hcone_t_elems(int64_t n);
int hcone_blocks(int64_t n);
int launch_hetrd1(const HConeDev* cones, const int* cta_cone, const int* cta_rank, const int* cta_count, int nctas,
                  size_t smem, const IoSlot* io, long long wait_limit, cudaStream_t s);
void launch_hlarft(const HConeDev* cones, const int* blk_cone, const int* blk_index, int nblocks, cudaStream_t s);
void launch_hbt(const HConeDev* cones, const int* cta_cone, const int* cta_rank, const int* cta_count, int nctas,
                int maxn, cudaStream_t s);
void launch_hrecon(const HConeDev* cones, int ncones, int maxn, const IoSlot* io, cudaStream_t s);

// ------------------------------------------------------------------ polynomial projection
// One cone of the factorization-free approximate projection (S_0 = X / ||X||_F,
// S_{k+1} = a_k S_k + b_k S_k^3, Y = (X + S_K X) / 2; the products are grouped GEMMs).
constexpr int kPolyChunk = 16384;  // svec entries per partial sum of squares
struct PolyConeDev {
  int64_t n;
  int64_t xoff;     // offset of the cone in the svec buffers
  int part0;        // first partial sum of squares of this cone
  int nparts;       // ceil(n (n + 1) / 2 / kPolyChunk)
  double* X;        // n*n dense X (both triangles)
  double* S0;       // n*n S_0, then the even iterates
  double* S1;       // n*n the odd iterates
  int mirror;       // 1: the iterates are mirrored into their upper triangles (FP64 products)
  double* Y;        // n*n lower triangle of Y (the GEMMs' S^2 scratch before that)
  int* status;      // per-cone status bits
};
void launch_poly_prepare(const PolyConeDev* cones, int ncones, const int* part_cone, int nparts, int64_t maxn,
                         const IoSlot* io, double* part, double* inv, double nsq, cudaStream_t s);
void launch_poly_pack(const PolyConeDev* cones, int ncones, int64_t maxn, const IoSlot* io, cudaStream_t s);
// Upper triangle of the new iterate from its lower triangle (which = 0: S1, 1: S0).
void launch_poly_mirror(const PolyConeDev* cones, int ncones, int64_t maxn, int which, cudaStream_t s);

}  // namespace scs
