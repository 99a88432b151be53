"""Seeded synthetic inputs for the PSD-cone projection, shared by the tests,
the benchmark and the smoke check.

This module only *makes inputs*: random orthogonal factors, spectra and the
svec storage layout the projection reads (the vec_R map of App. D.1 of the
paper, real symmetric case: lower triangle column by column, off-diagonal
entries times sqrt(2)).  It holds none of the projection's arithmetic; the
expected projection of a constructed matrix Q diag(lam) Q^T is formed by the
tests themselves.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.  The
workloads mirror the process-matrix step (n = d^4) and the instrument step
(n = d^2) of the paper's see-saw (Sec. III, App. B.4, App. A.3).  The paper
solves SDPs from GYNI games whose iterates are not available here, so every
matrix is synthetic: a spectrum of the stated shape under a Haar-random
orthogonal basis, or a symmetrised Gaussian matrix.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SQRT2 = np.sqrt(2.0)
SEED_BASE = 20519


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def svec_len(n: int) -> int:
    return n * (n + 1) // 2


def to_svec(X: np.ndarray) -> np.ndarray:
    """Storage layout of a symmetric matrix: lower triangle, column-major,
    off-diagonals scaled by sqrt(2).  For a symmetric matrix this equals the
    upper triangle read row by row."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    r, c = np.triu_indices(n)
    s = X[r, c].copy()
    s[r != c] *= SQRT2
    return s


def haar_orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the
    signs of R's diagonal moved into Q (Mezzadri 2007)."""
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def from_spectrum(rng: np.random.Generator, lam: np.ndarray):
    """X = Q diag(lam) Q^T with Haar Q.  Returns (X, Q, lam)."""
    lam = np.asarray(lam, dtype=np.float64)
    Q = haar_orthogonal(rng, lam.size)
    X = (Q * lam[None, :]) @ Q.T
    X = 0.5 * (X + X.T)
    return X, Q, lam


def sym_gaussian(rng: np.random.Generator, n: int) -> np.ndarray:
    """Sym(G) = (G + G^T) / 2 with G iid N(0, 1)."""
    G = rng.standard_normal((n, n))
    return 0.5 * (G + G.T)


# ---------------------------------------------------------------- spectra

def spectrum_plain(rng, n: int) -> np.ndarray:
    """Single-projection spectrum: about half U[0.1, 2], half U[-2, -0.1],
    one exact zero when n is odd (n = 81: 40 / 40 / 1)."""
    npos = (n - 1) // 2 if n % 2 else n // 2
    nneg = n - npos - (1 if n % 2 else 0)
    parts = [rng.uniform(0.1, 2.0, npos), rng.uniform(-2.0, -0.1, nneg)]
    if n % 2:
        parts.append(np.zeros(1))
    return np.concatenate(parts)


def spectrum_admm(rng, n: int) -> np.ndarray:
    """ADMM-like start spectrum: 48 % N(0, std 1e-6) clustered at zero, 32 %
    U[0.01, 1], the rest U[-1, -0.01] (n = 625: 300 / 200 / 125)."""
    n0 = int(round(n * 300 / 625))
    npos = int(round(n * 200 / 625))
    nneg = n - n0 - npos
    return np.concatenate([rng.normal(0.0, 1e-6, n0), rng.uniform(0.01, 1.0, npos),
                           rng.uniform(-1.0, -0.01, nneg)])


def spectrum_precision(rng, n: int) -> np.ndarray:
    """Precision stress spectrum: half U[-1, 1], a quarter N(0, std 1e-8),
    a quarter of magnitude 10^U[-4, 2] with a random sign."""
    h = n // 2
    q = (n - h) // 2
    r = n - h - q
    mags = 10.0 ** rng.uniform(-4.0, 2.0, r)
    signs = np.where(rng.uniform(size=r) < 0.5, -1.0, 1.0)
    return np.concatenate([rng.uniform(-1.0, 1.0, h), rng.normal(0.0, 1e-8, q), signs * mags])


def spectrum_vjp(rng, n: int, cluster: float = 1e-9) -> np.ndarray:
    """Derivative stress spectrum: U[-1, 1] with 10 % of the eigenvalues at
    +cluster and -cluster, half each (n = 1296: 65 + 65)."""
    nc = int(round(0.1 * n))
    nc -= nc % 2
    base = rng.uniform(-1.0, 1.0, n - nc)
    return np.concatenate([base, np.full(nc // 2, cluster), np.full(nc // 2, -cluster)])


# ---------------------------------------------------------------- workloads

@dataclass
class Batch:
    """Packed svec cones: x[offsets[i]:offsets[i+1]] is cone i of side sides[i]."""
    x: np.ndarray
    offsets: np.ndarray
    sides: np.ndarray
    extra: dict = field(default_factory=dict)

    @property
    def count(self) -> int:
        return int(self.sides.size)


def pack(svecs, sides) -> Batch:
    sides = np.asarray(sides, dtype=np.int32)
    lens = np.array([svec_len(int(n)) for n in sides], dtype=np.int64)
    offsets = np.zeros(sides.size + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    x = np.concatenate(svecs) if len(svecs) else np.zeros(0)
    return Batch(x=x, offsets=offsets, sides=sides)


def single_projection(seed: int = SEED_BASE + 1, n: int = 81):
    """One n x n matrix Q diag(lam) Q^T with the plain spectrum
    (n = 81 = d^4 at d = 3).  Returns (svec, Q, lam)."""
    rng = rng_for(seed)
    lam = spectrum_plain(rng, n)
    X, Q, lam = from_spectrum(rng, lam)
    return to_svec(X), Q, lam


def admm_sequence(seed: int = SEED_BASE + 2, n: int = 625, steps: int = 200, step_scale: float = 1e-3):
    """ADMM-like sequence X_{k+1} = X_k + 1e-3 Sym(G_k) starting from
    Q diag(lam0) Q^T with the clustered spectrum (n = 625 = d^4 at d = 5).
    Returns (list of svecs, Q, lam0)."""
    rng = rng_for(seed)
    lam = spectrum_admm(rng, n)
    X, Q, lam = from_spectrum(rng, lam)
    out = [to_svec(X)]
    for _ in range(steps - 1):
        X = X + step_scale * sym_gaussian(rng, n)
        out.append(to_svec(X))
    return out, Q, lam


def precision_batch(seed: int = SEED_BASE + 3, n: int = 4096, batch: int = 4) -> Batch:
    """``batch`` matrices with the precision stress spectrum
    (n = 4096 = d^4 at d = 8).  extra['Q'], extra['lam'] hold the factors."""
    rng = rng_for(seed)
    svecs, Qs, lams = [], [], []
    for _ in range(batch):
        lam = spectrum_precision(rng, n)
        X, Q, lam = from_spectrum(rng, lam)
        svecs.append(to_svec(X))
        Qs.append(Q)
        lams.append(lam)
    b = pack(svecs, [n] * batch)
    b.extra.update(Q=Qs, lam=lams)
    return b


INSTRUMENT_SIDES = (4, 9, 16, 25, 36, 49, 64)


def uneven_batch(seed: int = SEED_BASE + 4, restarts: int = 64, small_sides=INSTRUMENT_SIDES,
                 copies: int = 2, big_sides=(625, 1296)) -> Batch:
    """Many uneven cones: each see-saw restart contributes ``copies`` blocks
    of every instrument side d^2 plus one process block whose side alternates
    through ``big_sides``.  Entries are Sym(G) + u I with u ~ U[-0.5, 0.5] per
    block.  Default: 64 x (14 + 1) = 960 cones."""
    rng = rng_for(seed)
    svecs, sides = [], []
    for r in range(restarts):
        blocks = [s for s in small_sides for _ in range(copies)]
        if big_sides:
            blocks.append(big_sides[r % len(big_sides)])
        for n in blocks:
            X = sym_gaussian(rng, n) + rng.uniform(-0.5, 0.5) * np.eye(n)
            svecs.append(to_svec(X))
            sides.append(n)
    return pack(svecs, sides)


def vjp_batch(seed: int = SEED_BASE + 5, n: int = 1296, batch: int = 8, cluster: float = 1e-9) -> Batch:
    """``batch`` matrices with the derivative stress spectrum (n = 1296 = d^4
    at d = 6) plus Gaussian cotangents in extra['g'] (same layout as x)."""
    rng = rng_for(seed)
    svecs, Qs, lams = [], [], []
    for _ in range(batch):
        lam = spectrum_vjp(rng, n, cluster)
        X, Q, lam = from_spectrum(rng, lam)
        svecs.append(to_svec(X))
        Qs.append(Q)
        lams.append(lam)
    b = pack(svecs, [n] * batch)
    b.extra.update(Q=Qs, lam=lams, g=rng.standard_normal(b.x.size))
    return b


# ---- complex Hermitian cones (the paper's cones are complex Hermitian)
def haar_unitary(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-random unitary: QR of a complex Gaussian with the phases of R's
    diagonal moved into Q (Mezzadri 2007)."""
    G = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(G)
    d = np.diag(R)
    return Q * (d / np.abs(d))[None, :]


def herm_from_spectrum(rng: np.random.Generator, lam: np.ndarray):
    """X = U diag(lam) U^H with Haar U.  Returns (X, U, lam)."""
    lam = np.asarray(lam, dtype=np.float64)
    U = haar_unitary(rng, lam.size)
    X = (U * lam[None, :]) @ U.conj().T
    X = 0.5 * (X + X.conj().T)
    return X, U, lam


def herm_gaussian(rng: np.random.Generator, n: int) -> np.ndarray:
    """(G + G^H) / 2 with G iid complex Gaussian (unit variance per entry)."""
    G = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    return 0.5 * (G + G.conj().T)


def to_hsvec(X: np.ndarray) -> np.ndarray:
    """Hermitian svec: per column the (real) diagonal entry, then for every
    row below it sqrt(2) Re X_ij, sqrt(2) Im X_ij (n^2 reals)."""
    X = np.asarray(X, dtype=np.complex128)
    n = X.shape[0]
    out = np.empty(n * n)
    k = 0
    r2 = np.sqrt(2.0)
    for j in range(n):
        out[k] = X[j, j].real
        k += 1
        col = X[j + 1:, j]
        m = col.size
        out[k:k + 2 * m:2] = r2 * col.real
        out[k + 1:k + 2 * m:2] = r2 * col.imag
        k += 2 * m
    return out


def herm_admm_sequence(seed: int = SEED_BASE + 6, n: int = 625, steps: int = 50, step_scale: float = 1e-3):
    """The ADMM-like sequence for a complex Hermitian cone (the paper's cones
    are complex): X_0 = U diag(lam0) U^H with the clustered spectrum of the
    real sequence and Haar U, X_{k+1} = X_k + 1e-3 (G + G^H)/2.
    Returns (list of Hermitian svecs, U, lam0)."""
    rng = rng_for(seed)
    lam = spectrum_admm(rng, n)
    X, U, lam = herm_from_spectrum(rng, lam)
    out = [to_hsvec(X)]
    for _ in range(steps - 1):
        X = X + step_scale * herm_gaussian(rng, n)
        out.append(to_hsvec(X))
    return out, U, lam


def orthonormal_columns(rng: np.random.Generator, m: int, k: int) -> np.ndarray:
    """First k columns of H1 H2 (two Householder reflectors of random
    direction): an m x k matrix with orthonormal columns in O(m k) work.
    Returned as a C-contiguous k x m array (the m x k matrix column-major)."""
    w1, w2 = rng.standard_normal(m), rng.standard_normal(m)
    B = np.zeros((k, m))
    B[np.arange(k), np.arange(k)] = 1.0                      # rows of B = columns of E = I[:, :k]
    B -= (2.0 / (w2 @ w2)) * np.outer(w2[:k], w2)            # H2 E
    B -= (2.0 / (w1 @ w1)) * np.outer(B @ w1, w1)            # H1 H2 E
    return B


def scs_problem(seed: int = SEED_BASE + 7, n: int = 625, k: int = 1000):
    """One PSD cone of side n (d = 5) in SCS form: A (m x k, orthonormal
    columns, as a k x m array), b ~ N(0, 1/m) (svec), c ~ N(0, 1/k), and the
    SCS initial iterates u = v = (0, 0, 1)."""
    rng = rng_for(seed)
    m = n * (n + 1) // 2
    At = orthonormal_columns(rng, m, k)
    b = rng.standard_normal(m) / np.sqrt(m)
    c = rng.standard_normal(k) / np.sqrt(k)
    u = np.zeros(k + m + 1)
    u[-1] = 1.0
    return At, b, c, u, u.copy()



# ---- structured operator of the process-matrix step (App. B, App. D.2)
def real_local_basis(d: int):
    """Orthonormal basis of the real d x d matrices in the real form of the
    generalized Gell-Mann basis: element 0 the identity / sqrt(d), then the
    d - 1 traceless diagonal matrices diag(1, .., 1, -l, 0, ..) / sqrt(l (l + 1)),
    then (E_ij + E_ji) / sqrt(2) and (E_ij - E_ji) / sqrt(2) for i < j.
    Returns (B of shape (d^2, d, d), antisym flags of length d^2).  The
    antisymmetric elements are the imaginary Gell-Mann matrices divided by i."""
    B, anti = [np.eye(d) / np.sqrt(d)], [False]
    for l in range(1, d):
        D = np.zeros((d, d))
        D[np.arange(l), np.arange(l)] = 1.0
        D[l, l] = -float(l)
        B.append(D / np.sqrt(l * (l + 1.0)))
        anti.append(False)
    for i in range(d):
        for j in range(i + 1, d):
            S = np.zeros((d, d))
            S[i, j] = S[j, i] = 1.0 / np.sqrt(2.0)
            A = np.zeros((d, d))
            A[i, j], A[j, i] = 1.0 / np.sqrt(2.0), -1.0 / np.sqrt(2.0)
            B += [S, A]
            anti += [False, True]
    return np.stack(B), np.array(anti)


def process_allowed(d: int, real: bool = True) -> np.ndarray:
    """Flat indices (C order over (A_I, A_O, B_I, B_O) basis indices, 0 the
    identity) of the coefficients a bipartite process matrix may carry
    (App. B): w_{a0,c0} for all a, c; w_{a j,c 0} with j, c traceless; w_{a 0,c l}
    with a, l traceless -- 2 d^6 - 3 d^4 + 2 d^2 of them.  real=True keeps the
    ones whose Kronecker product is real symmetric: an even number of
    antisymmetric local factors."""
    k = d * d
    _, anti = real_local_basis(d)
    a, j, c, l = np.meshgrid(np.arange(k), np.arange(k), np.arange(k), np.arange(k), indexing="ij")
    ok = ((j == 0) & (l == 0)) | ((j > 0) & (l == 0) & (c > 0)) | ((j == 0) & (l > 0) & (a > 0))
    if real:
        na = anti[a].astype(int) + anti[j] + anti[c] + anti[l]
        ok &= (na % 2) == 0
    return np.flatnonzero(ok.reshape(-1)).astype(np.int64)


def scs_kron_problem(seed: int = SEED_BASE + 8, d: int = 5):
    """The process-matrix SDP step of App. D at local dimension d: one PSD
    cone of side n = d^4 (four subsystems), A x = svec(sum_mu x_mu F_mu) over
    the real process subspace (``process_allowed``), F_mu Kronecker products
    of ``real_local_basis(d)``; b ~ N(0, 1/m), c ~ N(0, 1/k), and SCS's
    initial iterates u = v = (0, 0, 1).  Returns (bases, index, b, c, u, v)."""
    rng = rng_for(seed)
    B, _ = real_local_basis(d)
    index = process_allowed(d)
    n = d ** 4
    m, k = n * (n + 1) // 2, index.size
    b = rng.standard_normal(m) / np.sqrt(m)
    c = rng.standard_normal(k) / np.sqrt(k)
    u = np.zeros(k + m + 1)
    u[-1] = 1.0
    return [B] * 4, index, b, c, u, u.copy()
