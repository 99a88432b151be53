/*
 * FP64 CPU oracle for the PSD-cone projection.  TEST INFRASTRUCTURE ONLY:
 * this file is compiled into liboracle.so, which only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark load.  The product
 * path never calls it and shares no code with it.
 *
 * What it computes (App. D of the paper, "Details on the SCS algorithm"):
 *   - the vec_R / mat_R maps of App. D.1 for real symmetric matrices
 *     (diagonal entries as they are, off-diagonal entries times sqrt(2)),
 *     in SCS order: lower triangle, column by column;
 *   - the Euclidean projection onto the PSD cone, which App. D.2 computes by
 *     "an eigendecomposition, negative eigenvalues set to zero":
 *         Pi(X) = V diag(max(lambda, 0)) V^T;
 *   - the same result through the Moreau decomposition of App. D.1,
 *         Pi(X) = X - Pi_-(X),  Pi_-(X) = V diag(min(lambda, 0)) V^T;
 *   - the directional derivative of Pi (needed because App. E back-propagates
 *     through the eigendecomposition), by the Daleckii-Krein formula
 *         DPi(X)[H] = V (L o (V^T H V)) V^T,
 *     L_ij the divided difference of max(.,0) at (lambda_i, lambda_j);
 *   - the same projection for complex Hermitian cones (the paper's own cone
 *     type), Pi(X) = V diag(max(lambda, 0)) V^H, by a complex Jacobi method.
 *
 * The eigendecomposition is a cyclic two-sided Jacobi method (rotation of
 * Golub & Van Loan, "Matrix Computations", Alg. 8.5.1 sym.schur2), with a
 * round-robin (circle-method) ordering so that the n/2 rotations of one round
 * touch disjoint index pairs; their angles are all computed from the same
 * matrix and the round is applied rows-then-columns, so the result does not
 * depend on the number of OpenMP threads.  No BLAS or LAPACK is used.
 * Compile with -O2 -ffp-contract=off (no fused multiply-add).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENOCONV 5
#define ORC_ENONFINITE 6

/* Mutation switch used only by the test suite to plant a mistake in the
 * oracle and show that the pins catch it.  0 = the correct oracle. */
static int g_mutation = 0;
void orc_set_mutation(int m) { g_mutation = m; }
int orc_get_mutation(void) { return g_mutation; }

static int g_threads = 0;
void orc_set_threads(int t) { g_threads = t; }
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
static int nthreads(void) {
#ifdef _OPENMP
  return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
  return 1;
#endif
}

int64_t orc_svec_len(int64_t n) { return n * (n + 1) / 2; }

/* mat_R of App. D.1: svec -> full symmetric n x n (row-major). */
void orc_smat(int64_t n, const double* s, double* A) {
  const double r2 = (g_mutation == 1) ? 1.0 : sqrt(2.0);
  int64_t k = 0;
  for (int64_t j = 0; j < n; ++j) {
    A[j * n + j] = s[k++];
    for (int64_t i = j + 1; i < n; ++i) {
      double v = s[k++] / r2;
      A[i * n + j] = v;
      A[j * n + i] = v;
    }
  }
}

/* vec_R of App. D.1: lower triangle of a symmetric matrix -> svec. */
void orc_svec(int64_t n, const double* A, double* s) {
  const double r2 = (g_mutation == 1) ? 1.0 : sqrt(2.0);
  int64_t k = 0;
  for (int64_t j = 0; j < n; ++j) {
    s[k++] = A[j * n + j];
    for (int64_t i = j + 1; i < n; ++i) s[k++] = r2 * A[i * n + j];
  }
}

/* One pair (p, q) of a round of the circle method over m (even) players:
 * round r pairs (r, m-1) and ((r+k) mod (m-1), (r-k) mod (m-1)), k >= 1. */
static void round_pair(int64_t m, int64_t r, int64_t k, int64_t* p, int64_t* q) {
  if (k == 0) {
    *p = r;
    *q = m - 1;
  } else {
    *p = (r + k) % (m - 1);
    *q = (r - k + (m - 1)) % (m - 1);
  }
  if (*p > *q) {
    int64_t t = *p;
    *p = *q;
    *q = t;
  }
}

/*
 * Jacobi eigendecomposition of the symmetric n x n matrix A (row-major, it is
 * overwritten).  On return lam[i] holds the i-th diagonal entry of the
 * converged matrix and column i of V (row-major n x n) its eigenvector.
 * Eigenvalues are not sorted.  Returns ORC_OK or ORC_ENOCONV.
 */
int orc_jacobi_eig(int64_t n, double* A, double* lam, double* V, int max_sweeps, int* sweeps_out) {
  for (int64_t i = 0; i < n * n; ++i) V[i] = 0.0;
  for (int64_t i = 0; i < n; ++i) V[i * n + i] = 1.0;
  if (sweeps_out) *sweeps_out = 0;
  if (n <= 1) {
    if (n == 1) lam[0] = A[0];
    return ORC_OK;
  }
  const int64_t m = (n % 2 == 0) ? n : n + 1; /* pad odd n with a dummy index */
  const int64_t half = m / 2;
  int64_t* P = (int64_t*)malloc(sizeof(int64_t) * half);
  int64_t* Q = (int64_t*)malloc(sizeof(int64_t) * half);
  double* C = (double*)malloc(sizeof(double) * half);
  double* S = (double*)malloc(sizeof(double) * half);
  double* T = (double*)malloc(sizeof(double) * half);
  if (!P || !Q || !C || !S || !T) {
    free(P); free(Q); free(C); free(S); free(T);
    return ORC_ENOMEM;
  }
  const double eps = 0x1p-53;
  const int nt = nthreads();
  int status = ORC_ENOCONV;
  int sweep;
  for (sweep = 0; sweep < max_sweeps; ++sweep) {
    int64_t rotated = 0;
    for (int64_t r = 0; r < m - 1; ++r) {
      /* angles of this round, all from the same A (pairs are disjoint) */
      int64_t np = 0;
      for (int64_t k = 0; k < half; ++k) {
        int64_t p, q;
        round_pair(m, r, k, &p, &q);
        if (q >= n) continue; /* dummy index */
        const double apq = A[p * n + q];
        const double app = A[p * n + p], aqq = A[q * n + q];
        if (fabs(apq) <= 1e-300 || fabs(apq) <= eps * sqrt(fabs(app)) * sqrt(fabs(aqq))) continue;
        /* Golub & Van Loan sym.schur2 */
        const double tau = (aqq - app) / (2.0 * apq);
        double t;
        if (fabs(tau) > 1e150) {
          t = 0.5 / tau;
        } else if (tau >= 0.0) {
          t = 1.0 / (tau + sqrt(1.0 + tau * tau));
        } else {
          t = -1.0 / (-tau + sqrt(1.0 + tau * tau));
        }
        if (g_mutation == 3) t = -t; /* planted sign error */
        const double c = 1.0 / sqrt(1.0 + t * t);
        P[np] = p; Q[np] = q; C[np] = c; S[np] = t * c; T[np] = t;
        ++np;
      }
      if (np == 0) continue;
      rotated += np;
      /* rows: A <- J^T A for every pair */
#pragma omp parallel for num_threads(nt) schedule(static)
      for (int64_t k = 0; k < np; ++k) {
        double* ap = A + P[k] * n;
        double* aq = A + Q[k] * n;
        const double c = C[k], s = S[k];
        for (int64_t j = 0; j < n; ++j) {
          const double x = ap[j], y = aq[j];
          ap[j] = c * x - s * y;
          aq[j] = s * x + c * y;
        }
      }
      /* columns: A <- A J and V <- V J, one matrix row at a time */
#pragma omp parallel for num_threads(nt) schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        double* ai = A + i * n;
        double* vi = V + i * n;
        for (int64_t k = 0; k < np; ++k) {
          const int64_t p = P[k], q = Q[k];
          const double c = C[k], s = S[k];
          double x = ai[p], y = ai[q];
          ai[p] = c * x - s * y;
          ai[q] = s * x + c * y;
          x = vi[p];
          y = vi[q];
          vi[p] = c * x - s * y;
          vi[q] = s * x + c * y;
        }
      }
      /* the rotated 2x2 blocks are diagonal by construction */
      for (int64_t k = 0; k < np; ++k) {
        A[P[k] * n + Q[k]] = 0.0;
        A[Q[k] * n + P[k]] = 0.0;
      }
    }
    if (rotated == 0) {
      status = ORC_OK;
      break;
    }
  }
  if (sweeps_out) *sweeps_out = sweep;
  for (int64_t i = 0; i < n; ++i) lam[i] = A[i * n + i];
  free(P); free(Q); free(C); free(S); free(T);
  return status;
}

static int all_finite(int64_t len, const double* x) {
  for (int64_t i = 0; i < len; ++i)
    if (!isfinite(x[i])) return 0;
  return 1;
}

/* Y = sum_i f_i v_i v_i^T over the i with keep[i], lower triangle only
 * (then mirrored).  V row-major, column i is eigenvector i. */
static void spectral_sum(int64_t n, const double* V, const double* f, double* Y) {
  const int nt = nthreads();
  const int transposed = (g_mutation == 4);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 8)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      double acc = 0.0;
      for (int64_t k = 0; k < n; ++k) {
        if (f[k] == 0.0) continue;
        const double vik = transposed ? V[k * n + i] : V[i * n + k];
        const double vjk = transposed ? V[k * n + j] : V[j * n + k];
        acc += f[k] * vik * vjk;
      }
      Y[i * n + j] = acc;
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) Y[i * n + j] = Y[j * n + i];
}

/*
 * Eigendecomposition of smat(x): lam (n) and V (n x n row-major, columns are
 * eigenvectors).  Used by the projection, the derivative and the tests.
 */
int orc_eig_svec(int64_t n, const double* x, double* lam, double* V, int* sweeps) {
  if (n < 0 || (n > 0 && (!x || !lam || !V))) return ORC_EINVAL;
  if (n == 0) return ORC_OK;
  if (!all_finite(orc_svec_len(n), x)) return ORC_ENONFINITE;
  double* A = (double*)malloc(sizeof(double) * n * n);
  if (!A) return ORC_ENOMEM;
  orc_smat(n, x, A);
  int st = orc_jacobi_eig(n, A, lam, V, 60, sweeps);
  free(A);
  return st;
}

/*
 * Pi(X) on svec buffers (App. D.2): y = svec(V diag(max(lam,0)) V^T).
 * If lam_out is not NULL it receives the eigenvalues (unsorted).
 * route: 0 = positive part sum_{lam>0} lam v v^T,
 *        1 = Moreau form X - sum_{lam<0} lam v v^T (App. D.1).
 */
int orc_psd_proj_route(int64_t n, const double* x, double* y, double* lam_out, int route) {
  if (n < 0 || (n > 0 && (!x || !y))) return ORC_EINVAL;
  if (n == 0) return ORC_OK;
  const int64_t len = orc_svec_len(n);
  if (!all_finite(len, x)) {
    for (int64_t i = 0; i < len; ++i) y[i] = NAN;
    return ORC_ENONFINITE;
  }
  double* A = (double*)malloc(sizeof(double) * n * n);
  double* V = (double*)malloc(sizeof(double) * n * n);
  double* Y = (double*)malloc(sizeof(double) * n * n);
  double* lam = (double*)malloc(sizeof(double) * n);
  double* f = (double*)malloc(sizeof(double) * n);
  if (!A || !V || !Y || !lam || !f) {
    free(A); free(V); free(Y); free(lam); free(f);
    return ORC_ENOMEM;
  }
  orc_smat(n, x, A);
  int st = orc_jacobi_eig(n, A, lam, V, 60, NULL);
  if (st == ORC_OK) {
    for (int64_t i = 0; i < n; ++i) {
      if (route == 0)
        f[i] = (lam[i] > 0.0 || g_mutation == 2) ? lam[i] : 0.0;
      else
        f[i] = (lam[i] < 0.0) ? lam[i] : 0.0;
    }
    spectral_sum(n, V, f, Y);
    if (route == 1) {
      orc_smat(n, x, A);
      for (int64_t i = 0; i < n * n; ++i) Y[i] = A[i] - Y[i];
    }
    orc_svec(n, Y, y);
    if (lam_out) memcpy(lam_out, lam, sizeof(double) * n);
  }
  free(A); free(V); free(Y); free(lam); free(f);
  return st;
}

int orc_psd_proj(int64_t n, const double* x, double* y) { return orc_psd_proj_route(n, x, y, NULL, 0); }

/* Divided difference of max(., 0) at (a, b); f'(0) is taken as 0. */
static double loewner(double a, double b) {
  const int pa = a > 0.0, pb = b > 0.0;
  if (pa && pb) return 1.0;
  if (!pa && !pb) return 0.0;
  /* opposite signs: (max(a,0) - max(b,0)) / (a - b) = positive one / |a - b| */
  const double pos = pa ? a : b;
  return pos / fabs(a - b);
}

/*
 * Daleckii-Krein derivative on svec buffers:
 *   out = svec(V (L o (V^T smat(h) V)) V^T),  L_ij = loewner(lam_i, lam_j).
 * In svec coordinates this map is symmetric, so it is both the JVP and VJP.
 */
int orc_psd_jvp(int64_t n, const double* x, const double* h, double* out) {
  if (n < 0 || (n > 0 && (!x || !h || !out))) return ORC_EINVAL;
  if (n == 0) return ORC_OK;
  const int64_t len = orc_svec_len(n);
  if (!all_finite(len, x) || !all_finite(len, h)) {
    for (int64_t i = 0; i < len; ++i) out[i] = NAN;
    return ORC_ENONFINITE;
  }
  double* V = (double*)malloc(sizeof(double) * n * n);
  double* H = (double*)malloc(sizeof(double) * n * n);
  double* W = (double*)malloc(sizeof(double) * n * n);
  double* lam = (double*)malloc(sizeof(double) * n);
  if (!V || !H || !W || !lam) {
    free(V); free(H); free(W); free(lam);
    return ORC_ENOMEM;
  }
  int st = orc_eig_svec(n, x, lam, V, NULL);
  if (st == ORC_OK) {
    const int nt = nthreads();
    orc_smat(n, h, H);
    /* W = H V */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t k = 0; k < n; ++k) acc += H[i * n + k] * V[k * n + j];
        W[i * n + j] = acc;
      }
    /* H <- L o (V^T W) */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t k = 0; k < n; ++k) acc += V[k * n + i] * W[k * n + j];
        H[i * n + j] = loewner(lam[i], lam[j]) * acc;
      }
    /* W = V H */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t k = 0; k < n; ++k) acc += V[i * n + k] * H[k * n + j];
        W[i * n + j] = acc;
      }
    /* H = W V^T, then symmetrise the rounding and pack */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t k = 0; k < n; ++k) acc += W[i * n + k] * V[j * n + k];
        H[i * n + j] = acc;
      }
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < i; ++j) {
        const double v = 0.5 * (H[i * n + j] + H[j * n + i]);
        H[i * n + j] = v;
        H[j * n + i] = v;
      }
    orc_svec(n, H, out);
  }
  free(V); free(H); free(W); free(lam);
  return st;
}

/* ------------------------------------------------------------------------
 * Complex Hermitian cones (the paper's cones are complex Hermitian: the
 * vec map of App. D.1 lists X_ii, sqrt(2) Re X_ij, sqrt(2) Im X_ij).  Taken
 * order (SCS's complex PSD cone): column by column, the diagonal entry, then
 * for every row i > j the pair sqrt(2) Re X_ij, sqrt(2) Im X_ij; n^2 reals.
 * Matrices are held as separate real and imaginary row-major arrays.
 */
int64_t orc_hsvec_len(int64_t n) { return n * n; }

void orc_hsmat(int64_t n, const double* s, double* Ar, double* Ai) {
  const double r = 0.70710678118654752440;  /* 1 / sqrt(2) */
  int64_t k = 0;
  for (int64_t j = 0; j < n; ++j) {
    Ar[j * n + j] = s[k++];
    Ai[j * n + j] = 0.0;
    for (int64_t i = j + 1; i < n; ++i) {
      const double re = s[k++] * r, im = s[k++] * r;
      Ar[i * n + j] = re; Ai[i * n + j] = im;    /* X_ij */
      Ar[j * n + i] = re; Ai[j * n + i] = -im;   /* X_ji = conj(X_ij) */
    }
  }
}

void orc_hsvec(int64_t n, const double* Ar, const double* Ai, double* s) {
  const double r2 = 1.41421356237309504880;
  int64_t k = 0;
  for (int64_t j = 0; j < n; ++j) {
    s[k++] = Ar[j * n + j];
    for (int64_t i = j + 1; i < n; ++i) {
      s[k++] = r2 * Ar[i * n + j];
      s[k++] = r2 * Ai[i * n + j];
    }
  }
}

/*
 * Jacobi for Hermitian matrices.  For a pair (p, q) with A_pq = |b| e^{i phi},
 * the unitary U = D J, D = diag(1, e^{-i phi}) (which makes the pair's
 * off-diagonal entry real, |b|) and J the real rotation of sym.schur2 for
 * [[A_pp, |b|], [|b|, A_qq]], zeroes A_pq:
 *   columns: col_p <- c col_p - s e^{-i phi} col_q,  col_q <- s col_p + c e^{-i phi} col_q;
 *   rows   : row_p <- c row_p - s e^{i phi} row_q,   row_q <- s row_p + c e^{i phi} row_q.
 * Same round-robin order and thread-count independence as the real method.
 */
int orc_herm_jacobi_eig(int64_t n, double* Ar, double* Ai, double* lam, double* Vr, double* Vi, int max_sweeps) {
  for (int64_t i = 0; i < n * n; ++i) { Vr[i] = 0.0; Vi[i] = 0.0; }
  for (int64_t i = 0; i < n; ++i) Vr[i * n + i] = 1.0;
  if (n <= 1) {
    if (n == 1) lam[0] = Ar[0];
    return ORC_OK;
  }
  const int64_t m = (n % 2 == 0) ? n : n + 1;
  const int64_t half = m / 2;
  int64_t* P = (int64_t*)malloc(sizeof(int64_t) * half);
  int64_t* Q = (int64_t*)malloc(sizeof(int64_t) * half);
  double* C = (double*)malloc(sizeof(double) * half);
  double* S = (double*)malloc(sizeof(double) * half);
  double* ER = (double*)malloc(sizeof(double) * half);  /* cos(phi) */
  double* EI = (double*)malloc(sizeof(double) * half);  /* sin(phi) */
  if (!P || !Q || !C || !S || !ER || !EI) {
    free(P); free(Q); free(C); free(S); free(ER); free(EI);
    return ORC_ENOMEM;
  }
  const double eps = 0x1p-53;
  const int nt = nthreads();
  int status = ORC_ENOCONV;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int64_t rotated = 0;
    for (int64_t r = 0; r < m - 1; ++r) {
      int64_t np = 0;
      for (int64_t k = 0; k < half; ++k) {
        int64_t p, q;
        round_pair(m, r, k, &p, &q);
        if (q >= n) continue;
        const double br = Ar[p * n + q], bi = Ai[p * n + q];
        const double ab = hypot(br, bi);
        const double app = Ar[p * n + p], aqq = Ar[q * n + q];
        if (ab <= 1e-300 || ab <= eps * sqrt(fabs(app)) * sqrt(fabs(aqq))) continue;
        const double tau = (aqq - app) / (2.0 * ab);
        double t;
        if (fabs(tau) > 1e150) t = 0.5 / tau;
        else if (tau >= 0.0) t = 1.0 / (tau + sqrt(1.0 + tau * tau));
        else t = -1.0 / (-tau + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t);
        P[np] = p; Q[np] = q; C[np] = c; S[np] = t * c; ER[np] = br / ab; EI[np] = bi / ab;
        ++np;
      }
      if (np == 0) continue;
      rotated += np;
      /* rows: row_p <- c row_p - s e^{i phi} row_q, row_q <- s row_p + c e^{i phi} row_q */
#pragma omp parallel for num_threads(nt) schedule(static)
      for (int64_t k = 0; k < np; ++k) {
        double* pr = Ar + P[k] * n; double* pi = Ai + P[k] * n;
        double* qr = Ar + Q[k] * n; double* qi = Ai + Q[k] * n;
        const double c = C[k], s = S[k], er = ER[k], ei = EI[k];
        for (int64_t j = 0; j < n; ++j) {
          const double xr = pr[j], xi = pi[j], yr = qr[j], yi = qi[j];
          const double zr = er * yr - ei * yi, zi = er * yi + ei * yr;  /* e^{i phi} y */
          pr[j] = c * xr - s * zr; pi[j] = c * xi - s * zi;
          qr[j] = s * xr + c * zr; qi[j] = s * xi + c * zi;
        }
      }
      /* columns of A and V: col_p <- c col_p - s e^{-i phi} col_q, col_q <- s col_p + c e^{-i phi} col_q */
#pragma omp parallel for num_threads(nt) schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = 0; k < np; ++k) {
          const int64_t p = P[k], q = Q[k];
          const double c = C[k], s = S[k], er = ER[k], ei = EI[k];
          for (int w = 0; w < 2; ++w) {
            double* mr = (w == 0 ? Ar : Vr) + i * n;
            double* mi = (w == 0 ? Ai : Vi) + i * n;
            const double xr = mr[p], xi = mi[p], yr = mr[q], yi = mi[q];
            const double zr = er * yr + ei * yi, zi = er * yi - ei * yr;  /* e^{-i phi} y */
            mr[p] = c * xr - s * zr; mi[p] = c * xi - s * zi;
            mr[q] = s * xr + c * zr; mi[q] = s * xi + c * zi;
          }
        }
      }
      for (int64_t k = 0; k < np; ++k) {
        Ar[P[k] * n + Q[k]] = 0.0; Ai[P[k] * n + Q[k]] = 0.0;
        Ar[Q[k] * n + P[k]] = 0.0; Ai[Q[k] * n + P[k]] = 0.0;
        Ai[P[k] * n + P[k]] = 0.0; Ai[Q[k] * n + Q[k]] = 0.0;
      }
    }
    if (rotated == 0) { status = ORC_OK; break; }
  }
  for (int64_t i = 0; i < n; ++i) lam[i] = Ar[i * n + i];
  free(P); free(Q); free(C); free(S); free(ER); free(EI);
  return status;
}

/*
 * Pi(X) for a complex Hermitian cone on its svec (n^2 reals):
 * y = svec(sum_{lam > 0} lam v v^H) (route 0) or svec(X - sum_{lam < 0} lam v v^H) (route 1).
 */
int orc_herm_proj_route(int64_t n, const double* x, double* y, double* lam_out, int route) {
  if (n < 0 || (n > 0 && (!x || !y))) return ORC_EINVAL;
  if (n == 0) return ORC_OK;
  const int64_t len = n * n;
  if (!all_finite(len, x)) {
    for (int64_t i = 0; i < len; ++i) y[i] = NAN;
    return ORC_ENONFINITE;
  }
  double* Ar = (double*)malloc(sizeof(double) * n * n);
  double* Ai = (double*)malloc(sizeof(double) * n * n);
  double* Vr = (double*)malloc(sizeof(double) * n * n);
  double* Vi = (double*)malloc(sizeof(double) * n * n);
  double* Yr = (double*)malloc(sizeof(double) * n * n);
  double* Yi = (double*)malloc(sizeof(double) * n * n);
  double* lam = (double*)malloc(sizeof(double) * n);
  if (!Ar || !Ai || !Vr || !Vi || !Yr || !Yi || !lam) {
    free(Ar); free(Ai); free(Vr); free(Vi); free(Yr); free(Yi); free(lam);
    return ORC_ENOMEM;
  }
  orc_hsmat(n, x, Ar, Ai);
  int st = orc_herm_jacobi_eig(n, Ar, Ai, lam, Vr, Vi, 60);
  if (st == ORC_OK) {
    const int nt = nthreads();
    /* Y_ij = sum_k f_k V_ik conj(V_jk), lower triangle then mirrored */
#pragma omp parallel for num_threads(nt) schedule(dynamic, 8)
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t j = 0; j <= i; ++j) {
        double sr = 0.0, si = 0.0;
        for (int64_t k = 0; k < n; ++k) {
          const double f = route == 0 ? (lam[k] > 0.0 ? lam[k] : 0.0) : (lam[k] < 0.0 ? lam[k] : 0.0);
          if (f == 0.0) continue;
          const double ar = Vr[i * n + k], ai = Vi[i * n + k], br = Vr[j * n + k], bi = Vi[j * n + k];
          sr += f * (ar * br + ai * bi);
          si += f * (ai * br - ar * bi);
        }
        Yr[i * n + j] = sr; Yi[i * n + j] = si;
      }
    }
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = i + 1; j < n; ++j) { Yr[i * n + j] = Yr[j * n + i]; Yi[i * n + j] = -Yi[j * n + i]; }
    if (route == 1) {
      orc_hsmat(n, x, Ar, Ai);
      for (int64_t i = 0; i < n * n; ++i) { Yr[i] = Ar[i] - Yr[i]; Yi[i] = Ai[i] - Yi[i]; }
    }
    orc_hsvec(n, Yr, Yi, y);
    if (lam_out) memcpy(lam_out, lam, sizeof(double) * n);
  }
  free(Ar); free(Ai); free(Vr); free(Vi); free(Yr); free(Yi); free(lam);
  return st;
}
