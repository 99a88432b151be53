/*
 * scs_psd -- projection onto the cone of positive-semidefinite matrices for
 * SCS-style conic solvers, on one NVIDIA GB300 (sm_103a).
 *
 * The operation is the cone step u = Pi_C(u~ - v) of the SCS iteration as the
 * paper describes it (App. D.1, "Operator splitting" and "Eliminating the dual
 * variables"), for the PSD cone: with X the symmetric matrix whose svec
 * (the vec_R map of App. D.1) is x,
 *
 *     Pi(X) = argmin_{Y >= 0} ||Y - X||_F = V diag(max(lambda, 0)) V^T,
 *
 * computed "by an eigendecomposition with the negative eigenvalues set to
 * zero" (App. D.2).  When fewer eigenvalues are negative than positive the
 * library forms X - V_- diag(lambda_-) V_-^T instead, which is the same matrix
 * by the Moreau decomposition Pi_{C*}(x) = x + Pi_C(-x) of App. D.1.
 *
 * svec layout (real symmetric case of vec_R, in the order SCS uses): the
 * lower triangle column by column, diagonal entries as they are and
 * off-diagonal entries multiplied by sqrt(2); a side-n cone holds
 * n(n+1)/2 doubles.  The map is an isometry: <svec A, svec B> = tr(AB).
 *
 * Conventions for every entry point:
 *  - Data buffers (x, y, g, xbar) are FP64, contiguous, in the device memory
 *    of the handle's GPU, and owned by the caller.
 *  - Shape arrays (offsets, sides) are HOST arrays owned by the caller; they
 *    are read during the call only (the library plans launches from them).
 *  - The library owns its workspace (device memory allocated per shape list
 *    on first use, or ahead of it by scs_psd_reserve) and keeps it until
 *    scs_psd_destroy (or until more than 16 shape lists are in use).
 *  - Work is enqueued on `stream` and is asynchronous; host-detectable errors
 *    (bad sizes, null pointers) are returned at once and nothing is enqueued.
 *    Errors found on the device (non-finite input, non-convergence, a bounded
 *    wait that ran out) are recorded in a device status word that
 *    scs_psd_status reads; the affected cone's output is filled with NaN.
 *  - y may alias x (in-place, as SCS updates its iterate).
 *  - No CPU fallback exists: every arithmetic step runs in this library's
 *    CUDA kernels.  No exception crosses the ABI.
 */
#ifndef SCS_PSD_H
#define SCS_PSD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scs_psd_handle_s* scs_psd_handle;

/* Return codes. */
enum {
  SCS_PSD_OK = 0,
  SCS_PSD_EINVAL = 1,     /* bad argument (null pointer, size mismatch, n < 0) */
  SCS_PSD_ENOMEM = 2,     /* device or host allocation failed */
  SCS_PSD_ECUDA = 3,      /* a CUDA runtime call failed */
  SCS_PSD_ETIMEOUT = 4,   /* a bounded device-side wait ran out */
  SCS_PSD_ENOCONV = 5,    /* an iteration did not converge */
  SCS_PSD_ENONFINITE = 6  /* the input held a NaN or an infinity */
};

/* Arithmetic used for the dense contractions. */
typedef enum {
  SCS_PSD_FP64 = 0,       /* FP64 throughout */
  SCS_PSD_SPLIT_TF32 = 1  /* dense contractions as split-TF32 tensor-core products: FP64 operands
                             sliced on a grid shared by each 16-wide K chunk into three TF32 parts
                             (10 + 11 + 11 bits), six part products, the leading ones summed exactly
                             in FP32, compensated FP32 sums across chunks; contractions with K >= 256
                             slice each operand once, on 64-wide K groups (9 + 11 + 11 bits, eight
                             part products).  Relative error of the projection about 2e-8 to 7e-8;
                             operands must lie within FP32's exponent range (magnitudes between about
                             1e-35 and 1e38).  Householder panels, bulge chasing, secular equations
                             and sign decisions stay FP64 */
} scs_psd_precision;

/* Options; a NULL pointer means all defaults (zero-initialised struct). */
typedef struct {
  int32_t precision;        /* scs_psd_precision */
  int32_t side;             /* 0 auto (fewer eigenpairs), 1 positive part, 2 X - negative part */
  int32_t recompute;        /* VJP: 0 auto, 1 always recompute V, 2 never (store) */
  int32_t band;             /* 0 = automatic (one-stage tridiagonalisation up to side 6144, two-stage
                               with band width 16 above; or the autotuner's choice), 1 = one-stage
                               for every cone up to side 7600 (two-stage above), 2..32 = two-stage
                               with this band width for every cone */
  int64_t mem_budget_bytes; /* VJP: workspace budget that triggers recompute; 0 = no limit */
  int64_t wait_limit_cycles;/* bound on device spin-waits; 0 = default */
  int32_t graphs;           /* 0 = replay a recorded CUDA graph from the second call with the same
                               shapes and options on, 1 = always launch kernel by kernel */
  int32_t stats;            /* 1 = record per-cone statistics of the result (scs_psd_last_stats);
                               only for calls that write y (scs_psd_proj, scs_psd_proj_batched,
                               scs_psd_proj_vjp and scs_psd_proj_store with y, scs_psd_scs_iterate:
                               its last projection); 0 = none */
} scs_psd_opts;

/* Per-cone statistics of a projection (opts->stats = 1), the error statement
 * that comes with every result.  With Y the returned projection of X:
 *   k_pos, k_neg     eigenvalues of X found > 0 and < 0 (FP64 sign decisions);
 *   route            0: Y formed from the positive eigenpairs, 1: as X minus the
 *                    negative part (Moreau decomposition, App. D.1);
 *   status           the cone's device status (an SCS_PSD_* code);
 *   complementarity  <Y, Y - X> / (||Y||_F ||X||_F) in FP64 from the svec
 *                    buffers (the vec_R map is an isometry, App. D.1): the
 *                    complementarity residual of the optimality conditions
 *                    Y >= 0, Y - X >= 0, <Y, Y - X> = 0, which the exact
 *                    projection satisfies (the PSD cone is self-dual).  With
 *                    Y = Pi(X) + E it equals (<E, |X|> + ||E||^2) / (||Y|| ||X||),
 *                    |X| = 2 Pi(X) - X: to first order the relative error's
 *                    component along |X|.  0 when Y = 0 or X = 0;
 *   norm_y, norm_x   ||Y||_F and ||X||_F.
 * Side-0 cones report zeros; side-1 cones their sign. */
typedef struct {
  int32_t k_pos, k_neg, route, status;
  double complementarity, norm_y, norm_x;
  double reserved;
} scs_psd_cone_stats;

/* Create a handle on CUDA device `device`.  Allocates no device memory yet. */
int scs_psd_create(scs_psd_handle* h, int device);

/* Release the handle and its workspace.  Synchronises the device first. */
int scs_psd_destroy(scs_psd_handle h);

/* Single cone: y = svec(Pi(smat(x))) for a side-n cone; x and y hold
 * n(n+1)/2 doubles.  n = 0 is a no-op; n = 1 gives y = max(x, 0).
 * `stream` is a cudaStream_t (NULL = legacy default stream).
 * Operation: App. D.2 (projection by eigendecomposition). */
int scs_psd_proj(scs_psd_handle h, const double* x, double* y, int64_t n,
                 const scs_psd_opts* opts, void* stream);

/* Many cones of uneven sides in one call: cone i occupies
 * x[offsets[i] .. offsets[i+1]) and has side sides[i], with
 * offsets[i+1] - offsets[i] == sides[i](sides[i]+1)/2 and offsets[0] == 0.
 * offsets (count+1 entries) and sides (count entries) are HOST arrays.
 * The first call for a shape list (with given options) launches kernel by
 * kernel; the second records that launch sequence once as a CUDA graph and
 * every later call replays it, after one small launch that hands the graph
 * this call's x and y.  A call issued while `stream` is itself being
 * captured is launched kernel by kernel into the caller's capture.
 * Operation: App. D.2, applied block by block (the PSD constraint split into
 * smaller blocks, as the paper's outlook on symmetry reduction proposes). */
int scs_psd_proj_batched(scs_psd_handle h, const double* x, double* y, const int64_t* offsets,
                         const int32_t* sides, int32_t count, const scs_psd_opts* opts, void* stream);

/* Vector-Jacobian product of the projection (App. E back-propagates through
 * the eigendecomposition): xbar = J^T g with J = DPi(X), by the
 * Daleckii-Krein formula
 *     DPi(X)[H] = V (L o (V^T H V)) V^T,  L_ij = (max(l_i,0) - max(l_j,0)) / (l_i - l_j),
 * L_ij = 1 if both are positive, 0 if neither is.  In svec coordinates J is
 * symmetric, so this is also the JVP.  Layout as scs_psd_proj_batched; the
 * eigenvectors are recomputed from x (opts->recompute).  y is optional: if
 * not NULL it receives Pi(x) from the same eigendecomposition. */
int scs_psd_proj_vjp(scs_psd_handle h, const double* x, const double* g, double* xbar, double* y,
                     const int64_t* offsets, const int32_t* sides, int32_t count,
                     const scs_psd_opts* opts, void* stream);

/* Complex Hermitian cones, the paper's own cone type (App. D.1's vec map
 * carries sqrt(2) Re X_ij and sqrt(2) Im X_ij): y = hsvec(Pi(hsmat(x))),
 * Pi(X) = V diag(max(lambda, 0)) V^H.  Hermitian svec order: column by
 * column the (real) diagonal entry, then for every row i > j the pair
 * sqrt(2) Re X_ij, sqrt(2) Im X_ij -- n^2 reals per cone.  Cone i occupies
 * x[offsets[i] .. offsets[i+1]) with offsets[i+1] - offsets[i] == sides[i]^2
 * (host arrays, offsets[0] == 0); y may alias x.  When every side is at most
 * 1100 and opts->band is 0, the cones are reduced natively: complex
 * Householder reflectors (real off-diagonals) to a real symmetric
 * tridiagonal form, the real divide and conquer, the complex
 * back-transformation of the kept eigenvectors and the reconstruction
 * straight into the Hermitian svec (complex double-float arithmetic in the
 * reduction, the back-transformation and the reconstruction).  Otherwise
 * through the real symmetric embedding [[Re X, -Im X], [Im X, Re X]] of
 * side 2n, whose projection is the embedding of Pi(X); sides up to 4096.
 * Options (opts->stats excepted) and errors as scs_psd_proj_batched. */
int scs_psd_proj_hermitian(scs_psd_handle h, const double* x, double* y, const int64_t* offsets,
                           const int32_t* sides, int32_t count, const scs_psd_opts* opts, void* stream);

/* Factorization-free APPROXIMATE projection (Conclusions, "Approximate
 * semidefinite-cone projections": a composite matrix polynomial built from
 * matrix-matrix products alone whose scalar map reproduces the thresholding
 * of the eigenvalues).  The paper names the approach but prints no
 * polynomial; this one is max(t, 0) = t (1 + sign t) / 2 with sign replaced
 * by a scaled Newton-Schulz composite:
 *     S_0 = X / ||X||_F,  S_{k+1} = a_k S_k + b_k S_k^3,  y = svec((X + S_K X) / 2),
 * a_k = 3 alpha_k / 2, b_k = -alpha_k^3 / 2,
 * alpha_k = min(sqrt(3 / (1 + l_k + l_k^2)), 2 cos(2 pi / 9)),
 * l_0 = lo, l_{k+1} = (alpha_k l_k / 2)(3 - alpha_k^2 l_k^2): the minimax
 * scaling of Chen & Chow (2014), capped where the cubic's value at 1 falls
 * to 1/2 (the uncapped cubic maps the top of the interval onto its bottom,
 * where the rounding of split-precision products is amplified).
 * Per eigenvalue l of X (sigma = ||X||_F) the result carries
 * l (1 + f(l / sigma)) / 2, f the composite, with |f(t) - sign t| <= 1 - l_K
 * for |t| >= lo and 0 <= f(t) sign t <= 1 otherwise; so eigenvalues above
 * lo * sigma in magnitude are thresholded to within a factor 1 - l_K, and
 * each smaller one contributes an error of at most |l| / 2.
 * lo in (0, 1); steps in [1, 200], or 0 for the smallest K with
 * 1 - l_K <= 1e-15 (for example 24 steps at lo = 1e-7, 29 at 1e-9).
 * Layout, host shape arrays, aliasing of y and x, graph replay and status
 * as scs_psd_proj_batched.  opts->precision: SCS_PSD_FP64, or
 * SCS_PSD_SPLIT_TF32 for the products of cones of side >= 64 on the
 * split-TF32 tensor-core kernel (smaller cones stay FP64); opts->graphs as
 * for the other calls; the remaining options are ignored.  ||x||_2^2 must
 * be finite (else the cone is marked SCS_PSD_ENONFINITE and its output is
 * NaN); x = 0 gives 0.  Per cone of side n the handle holds 4 n^2 doubles
 * for the shape list, and in split mode three sliced copies (9 n^2 floats)
 * for a cone of side >= 64.  Returns SCS_PSD_EINVAL for lo or steps out of
 * range. */
int scs_psd_proj_poly(scs_psd_handle h, const double* x, double* y, const int64_t* offsets,
                      const int32_t* sides, int32_t count, double lo, int32_t steps,
                      const scs_psd_opts* opts, void* stream);

/* The same composite for complex Hermitian cones (the construction acts on
 * the spectrum only, so it carries over): S_0 = X / ||X||_F with the complex
 * Frobenius norm, S_{k+1} = a_k S_k + b_k S_k^3, y = hsvec((X + S_K X) / 2),
 * on the Hermitian svec layout of scs_psd_proj_hermitian, computed through
 * the real embedding [[Re X, -Im X], [Im X, Re X]] (its norm halved, so
 * lo is relative to ||X||_F).  Arguments and errors as scs_psd_proj_poly;
 * sides up to 4096. */
int scs_psd_proj_poly_hermitian(scs_psd_handle h, const double* x, double* y, const int64_t* offsets,
                                const int32_t* sides, int32_t count, double lo, int32_t steps,
                                const scs_psd_opts* opts, void* stream);

/* Smallest eigenvalue of every cone: lam_min[i] = lambda_min(smat(x_i)), a
 * DEVICE array of count doubles; layout and host shape arrays as
 * scs_psd_proj_batched, every side >= 1 (else SCS_PSD_EINVAL).  The cones
 * are reduced to tridiagonal form as for the projection, then lambda_min is
 * found by multisection on Sturm counts (32 points per round, absolute
 * resolution eps ||T||).  Non-finite cones give NaN and SCS_PSD_ENONFINITE.
 * It serves the positivity post-processing of the paper's instrument and
 * process steps (App. C, App. D). */
int scs_psd_lambda_min(scs_psd_handle h, const double* x, double* lam_min, const int64_t* offsets,
                       const int32_t* sides, int32_t count, const scs_psd_opts* opts, void* stream);

/* Positivity post-processing by mixing with a multiple of the identity
 * (App. C: the outcome blocks C_a of one instrument input mixed with white
 * noise, nu = 1/(n_a d_Ao); App. D: a process matrix mixed with the trivial
 * process, nu = gamma).  Cones groups[g] .. groups[g+1]-1 form group g (host
 * array of ngroups + 1 entries, groups[0] = 0, groups[ngroups] = count,
 * non-decreasing); nu is a host array of ngroups values.  Per group, with
 * lambda_a = lambda_min of its blocks:
 *     p = 1 if min_a lambda_a >= 0, else p = min over lambda_a < eps of
 *     (nu - eps) / (nu - lambda_a),
 * and every block becomes y_a = svec(p C_a + (1 - p) nu 1), so that the
 * smallest eigenvalue of every mixed block is at least eps (up to rounding),
 * with equality for the worst block.  y may alias x; p_out (DEVICE, ngroups
 * doubles) receives the weights if not NULL.  Shapes as
 * scs_psd_proj_batched, every side >= 1; non-finite blocks make their
 * group's p and output NaN (status SCS_PSD_ENONFINITE). */
int scs_psd_mix_identity(scs_psd_handle h, const double* x, double* y, const int64_t* offsets,
                         const int32_t* sides, int32_t count, const int32_t* groups, int32_t ngroups,
                         const double* nu, double eps, double* p_out, const scs_psd_opts* opts, void* stream);

/* `iters` iterations of SCS around the projection (App. D.1, final iterates),
 * for  min c^T x  s.t.  A x + s = b,  s in K  (K the PSD cones of the shape
 * list, svec layout), in the homogeneous self-dual embedding:
 *     u~ = (I + Q)^{-1}(u + v),  u = Pi_C(u~ - v),  v = v - u~ + u,
 * u = (x [k], y [m], tau), v = (r [k], s [m], kappa), Q = [[0, A^T, c],
 * [-A, 0, b], [-c^T, -b^T, 0]], C = R^k x K x R_+.  A (DEVICE, m x k,
 * column-major) must have orthonormal columns (A^T A = I, as the paper's
 * parametrization has, App. D.3; not checked): the affine step is then
 * z_x = (a_x - A^T a_y)/2, z_y = a_y + A z_x, one product with A^T and one
 * with A.  b (m) and c (k) are DEVICE arrays (A and c may be NULL when
 * k = 0); u and v (k + m + 1 each, DEVICE) are updated in place.
 * offsets/sides (host) describe the cones of the y block, offsets[count] ==
 * m.  p = M^{-1}(c, b) is recomputed on every call (two more products).  The
 * projection runs with opts as in scs_psd_proj_batched; its device status is
 * read with scs_psd_status.  No acceleration, over-relaxation or rescaling. */
int scs_psd_scs_iterate(scs_psd_handle h, const double* A, const double* b, const double* c, int64_t m, int64_t k,
                        const int64_t* offsets, const int32_t* sides, int32_t count, double* u, double* v,
                        int32_t iters, const scs_psd_opts* opts, void* stream);

/* Structured affine operator for scs_psd_scs_iterate_kron, as the paper
 * applies A and A^T (App. D.2: tensor contractions over the local bases of
 * the subsystems, the Kronecker products never formed).  Column j of A is
 * svec(F_mu), mu = (mu_1 .. mu_S) the multi-index of index[j] in C order
 * over (nbasis[0] .. nbasis[S-1]) (mu_S varies fastest), and
 *     F_mu = B_1[mu_1] (x) B_2[mu_2] (x) ... (x) B_S[mu_S],
 * a matrix of side N = dims[0] * ... * dims[S-1] (row index (i_1 .. i_S) in
 * C order: the convention of numpy.kron).  B_s[b] is the d x d matrix
 * (d = dims[s]) at basis[s] + b d^2, COLUMN-major.  Every F_mu listed must be
 * symmetric, and the columns orthonormal (A^T A = I): orthonormal local bases
 * and distinct indices give that; neither is checked.  App. B's process
 * matrices, for example, take four subsystems (A_I, A_O, B_I, B_O) of side
 * d, a generalized Gell-Mann basis per subsystem, and the coefficients the
 * process constraints allow (2 d^6 - 3 d^4 + 2 d^2 of them). */
#define SCS_PSD_KRON_MAX_MODES 6
typedef struct {
  int32_t nmodes;                               /* S, 1 .. 6 */
  int32_t dims[SCS_PSD_KRON_MAX_MODES];         /* d_s, 1 .. 8; N = prod d_s <= 8192 */
  int32_t nbasis[SCS_PSD_KRON_MAX_MODES];       /* k_s, 1 .. d_s^2 */
  const double* basis[SCS_PSD_KRON_MAX_MODES];  /* DEVICE: k_s d_s^2 doubles each */
  int64_t nparams;                              /* k, 0 .. prod k_s */
  const int64_t* index;                         /* DEVICE: k flat indices in [0, prod k_s) */
} scs_psd_kron_op;

/* scs_psd_scs_iterate for one PSD cone of side N (m = N(N+1)/2) with the
 * structured operator `op` instead of a dense A: each product with A or A^T
 * costs S contractions of the coefficient tensor (at most N^2 doubles) with
 * the local bases, where a dense A would stream m k doubles.  b (m), c (k),
 * u and v (k + m + 1) as there; the handle keeps two work tensors of N^2
 * doubles for (m, k).  SCS_PSD_EINVAL for sizes out of range; an index
 * outside [0, prod k_s) is skipped on the device and makes scs_psd_status
 * report SCS_PSD_EINVAL. */
int scs_psd_scs_iterate_kron(scs_psd_handle h, const scs_psd_kron_op* op, const double* b, const double* c,
                             double* u, double* v, int32_t iters, const scs_psd_opts* opts, void* stream);

/* The composite's coefficients for (lo, steps) as scs_psd_proj_poly uses
 * them: returns K (the number of steps) and, where the pointers are not
 * NULL, writes a[0..K), b[0..K) and l_final = l_K; -SCS_PSD_EINVAL for lo or
 * steps out of range.  Host only (no handle, no GPU). */
int32_t scs_psd_poly_schedule(double lo, int32_t steps, double* a, double* b, double* l_final);

/* Forward pass that keeps the eigendecomposition for a later VJP (the
 * "store" side of the store-or-recompute choice for the derivative of App. E):
 * y = Pi(x) as scs_psd_proj_batched (y may be NULL), and every eigenpair of
 * every cone, X_i = V_i diag(lam_i) V_i^T.  V and lam are caller-owned device
 * buffers of sum_i sides[i]^2 and sum_i sides[i] doubles; cone i's V_i is
 * the column-major sides[i] x sides[i] block at sum_{j<i} sides[j]^2 and its
 * lam_i starts at sum_{j<i} sides[j].  The columns come in no particular
 * order.  A bad cone's V_i and lam_i are NaN. */
int scs_psd_proj_store(scs_psd_handle h, const double* x, double* y, double* V, double* lam,
                       const int64_t* offsets, const int32_t* sides, int32_t count,
                       const scs_psd_opts* opts, void* stream);

/* xbar = DPi(X)[smat(g)] (as scs_psd_proj_vjp) from an eigendecomposition
 * stored by scs_psd_proj_store instead of recomputing it; V, lam as there.
 * With the same shapes and options the result is bit-identical to
 * scs_psd_proj_vjp's, since the same kernels produce V and lam. */
int scs_psd_vjp_stored(scs_psd_handle h, const double* V, const double* lam, const double* g, double* xbar,
                       const int64_t* offsets, const int32_t* sides, int32_t count,
                       const scs_psd_opts* opts, void* stream);

/* Projection of one cone WITHOUT ANY DEVICE ALLOCATION, for callers that
 * cannot call cudaMalloc (a process whose GPU memory is owned by a pool or a
 * framework allocator, code that runs where allocation is forbidden after
 * start-up).  It has no counterpart in the paper.  y = svec(Pi(smat(x))) in
 * FP64 for a side-n cone, 0 <= n <= 256 (larger n returns SCS_PSD_EINVAL);
 * x and y are caller-owned device buffers of n(n+1)/2 doubles on the current
 * device, y may alias x.  All workspace -- the plan's metadata, the
 * eigensolver's buffers and a status word -- lives in a file-scope
 * __device__ array of 16 MiB that every GPU loading the library holds until
 * exit (side 256 takes about 8 MiB of it).  Set-up happens on the first call
 * on a device, which takes the array's address with cudaGetSymbolAddress,
 * and on every call whose side differs from the previous call's on that
 * device, which writes that side's plan into the array with cudaMemcpyAsync
 * on `stream`: such calls must not be issued while `stream` is being
 * captured (they return SCS_PSD_EINVAL then, having enqueued nothing).  A
 * plan that does not fit the array returns SCS_PSD_ENOMEM.  Every call
 * shares the array and leaves the last call's contents in it (the status
 * word is cleared at the start of each call), so calls that overlap on the
 * GPU race: issue them on one stream, or synchronise between them.
 * Device-side errors fill y with NaN; no handle is needed. */
int scs_psd_proj_static(const double* x, double* y, int64_t n, void* stream);

/* Autotuner (launch shapes are the project's own choice; the paper fixes
 * none).  Times candidate launch shapes of the projection for this shape
 * list and precision on the caller's input x (device, layout as
 * scs_psd_proj_batched; not modified): the route and band width (automatic,
 * one-stage, two-stage with 8, 16, 32), the GEMM split-K target (1, 2, 4
 * CTAs per SM), and for one-stage cones the back-transformation slab width
 * (1, 2, 4, 8 columns at most) and the one-stage group size (all, a half or
 * a quarter of the SMs),
 * by coordinate search, three timed runs each (CUDA events on `stream`).
 * The winner is kept in the handle and used by every later call with these
 * shapes and precision whose opts->band is 0.  chosen (may be NULL)
 * receives {band, gemm CTAs per SM, slab columns, group share}, best_ms (may
 * be NULL) its time per call.  Allocates a scratch output for the duration;
 * synchronises `stream`; drops the handle's cached plans. */
int scs_psd_autotune(scs_psd_handle h, const double* x, const int64_t* offsets, const int32_t* sides,
                     int32_t count, const scs_psd_opts* opts, void* stream, int32_t* chosen,
                     double* best_ms);

/* The launch shapes of the last call, as scs_psd_autotune's `chosen`. */
int scs_psd_last_tuning(scs_psd_handle h, int32_t* out);

/* Optional set-up ahead of the first call: builds and caches the plan (the
 * workspace and launch metadata) of the projection of max_count cones of
 * side max_n with these options, so that a later scs_psd_proj_batched (or,
 * for max_count 1, scs_psd_proj) with exactly these shapes and options
 * allocates nothing.  Other shape lists are planned on their first call. */
int scs_psd_reserve(scs_psd_handle h, int64_t max_n, int32_t max_count, const scs_psd_opts* opts);

/* Statistics of the last call made on this handle with opts->stats = 1:
 * synchronises its stream and copies `count` records (the call's number of
 * cones, in its order) into the caller's HOST array `out`.  SCS_PSD_EINVAL
 * if no such call was made, if count differs from its cone count, or if the
 * handle's cached plans were dropped since (more than 16 shape lists, or
 * scs_psd_autotune).  A call with opts->stats costs one copy of the input and
 * one read of the input and the output (3 x 8 bytes per svec entry) more. */
int scs_psd_last_stats(scs_psd_handle h, scs_psd_cone_stats* out, int32_t count);

/* Synchronise the handle's last stream and return the device status of the
 * work enqueued since the previous call (an SCS_PSD_* code, OK if none). */
int scs_psd_status(scs_psd_handle h, int32_t* device_status);

/* Number of kernels the last call enqueued (for launch accounting), counting
 * each kernel of a replayed graph. */
int64_t scs_psd_last_launch_count(scs_psd_handle h);

/* 1 if the last call replayed a recorded graph, 0 if it launched kernel by
 * kernel, -1 for a NULL handle. */
int scs_psd_last_replayed(scs_psd_handle h);

/* Phase timing for profiling.  While enabled, every call records CUDA events
 * on its stream around each phase of the pipeline; scs_psd_trace_read
 * synchronises, returns the summed device time in milliseconds and the
 * number of recorded intervals of each phase (arrays of SCS_PSD_NPHASES
 * entries, caller-owned), and clears the record.  Phases: 0 svec unpack,
 * 1 dense->band (panels + trailing GEMMs), 2 band->tridiagonal, 3 tridiagonal
 * divide and conquer, 4 stage-2 back-transformation, 5 stage-1
 * back-transformation, 6 reconstruction + svec repack, 7 derivative. */
#define SCS_PSD_NPHASES 8
int scs_psd_trace(scs_psd_handle h, int enable);
int scs_psd_trace_read(scs_psd_handle h, double* ms, int64_t* intervals);

/* Human-readable text for a return code. */
const char* scs_psd_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* SCS_PSD_H */
