"""Plain FP64 CPU oracle for the sparse Fast Chebyshev Transform (Jones et al.,
"A Sparse Fast Chebyshev Transform for High-Dimensional Approximation").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import or run this module.
It shares no code with the CUDA path; the only thing both read is the seeded
input generator package ``workloads`` (random draws, no arithmetic of the
method).

What it computes (Algorithm 3, Sec. 3.4): for an L-grid of K tensor grids,
    b = F f   (per grid, the multi-dimensional DCT-I interpolation coefficients
               of the samples; Eq. (main_linear_system), rows of empty bins
               dropped)
    A         (stacked per-grid alias matrices, Eq. (L-grid_A_mat), entries
               from the fold relation, the extrema-grid analogue of
               Lemma (lem:aliasing) / Eq. (aliasing_matrix_nd_diff))
    c* = argmin_c || b - A c ||_2      (the least-squares problem of Sec. 3.4)
and the grid-count selection of Algorithm 2 (Sec. 3.3): grids are appended
in a given candidate order until kappa(A) <= kappa0.

Readings of the paper this oracle follows:
  * grid: Chebyshev extrema x_j = cos(pi j / (n-1)), j = 0..n-1, with a DCT-I
    per axis and an unsigned fold; the paper's own form (first-kind points,
    1/M DCT-II quadrature, signed half-weight alias entries, Eq.
    (aliasing_matrix_1d)) is the ``kind="first"`` variant;
  * normalisation: b holds the exact Chebyshev coefficients of the grid
    interpolant, so A has unit entries times single-point weights;
  * an axis with one point samples at a given node xi and contributes the
    weight T_{m_i}(xi) to every entry of that column;
  * solver: the least-squares minimiser itself (dense Householder QR, normal
    equations with refinement, or CGLS to a tight tolerance, by size).

Parity pins: every function here is checked by ``tests/test_oracle_pins.py``
against closed forms, library routines, brute force or invariants.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

import workloads as W


# ==========================================================================
# Sec. 2: Chebyshev polynomials, index sets
# ==========================================================================
def chebyshev_T(n, x):
    """T_n(x) = cos(n arccos x)  (definition, Sec. 2)."""
    x = np.clip(np.asarray(x, dtype=np.float64), -1.0, 1.0)
    return np.cos(np.asarray(n, dtype=np.float64) * np.arccos(x))


def chebyshev_T_table(nmax: int, x) -> np.ndarray:
    """[len(x), nmax+1] table of T_0..T_nmax by the three-term recurrence
    T_{n+1} = 2 x T_n - T_{n-1} (Sec. 2)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    t = np.empty((x.size, nmax + 1), dtype=np.float64)
    t[:, 0] = 1.0
    if nmax >= 1:
        t[:, 1] = x
    for n in range(1, nmax):
        t[:, n + 1] = 2.0 * x * t[:, n] - t[:, n - 1]
    return t


def support_size_total_degree(d: int, D: int) -> int:
    """|S^1_{d,D}| = C(d + D, d), Eq. (N_1norm)."""
    return math.comb(d + D, d)


def support_total_degree_bruteforce(d: int, D: int) -> np.ndarray:
    """S^1_{d,D} by filtering the full box {0..d}^D (tiny D only)."""
    grids = np.meshgrid(*[np.arange(d + 1)] * D, indexing="ij")
    allm = np.stack([g.reshape(-1) for g in grids], axis=1)
    return allm[allm.sum(axis=1) <= d]


# ==========================================================================
# Grids and samples
# ==========================================================================
def extrema_nodes(n: int, xi: float = 1.0) -> np.ndarray:
    """Chebyshev extrema x_j = cos(pi j/(n-1)), j = 0..n-1 (reading O-1).

    The angle is reduced exactly: x_{n-1-j} = -x_j is enforced by computing
    the first half and mirroring, so the endpoints are exactly +-1 and the
    middle point of an odd grid is exactly 0.  n == 1 is the single node xi.
    """
    if n == 1:
        return np.array([xi], dtype=np.float64)
    j = np.arange(n)
    x = np.cos(np.pi * j / (n - 1))
    half = n // 2
    x[n - half:] = -x[:half][::-1]
    if n % 2 == 1:
        x[half] = 0.0
    x[0], x[-1] = 1.0, -1.0
    return x


def grid_axes(sizes_l, nodes_l, kind: str = "extrema") -> list[np.ndarray]:
    nodes_fn = extrema_nodes if kind == "extrema" else first_kind_nodes
    return [nodes_fn(int(n), float(xi)) for n, xi in zip(sizes_l, nodes_l)]


def _broadcast_axis(v: np.ndarray, i: int, D: int) -> np.ndarray:
    shape = [1] * D
    shape[i] = v.size
    return v.reshape(shape)


def sample_grid(family: int, params: np.ndarray, support: np.ndarray, axes) -> np.ndarray:
    """f on the tensor grid spanned by ``axes`` (row-major tensor)."""
    D = len(axes)
    shape = tuple(a.size for a in axes)
    if family in (W.FAMILY_GAUSSCOS, W.FAMILY_POLY_GAUSSCOS):
        a, b = params[:D], params[D:2 * D]
        quad = sum(a[i] * _broadcast_axis(axes[i] ** 2, i, D) for i in range(D))
        lin = sum(b[i] * _broadcast_axis(axes[i], i, D) for i in range(D))
        f = np.exp(-quad) * np.cos(lin)
        if family == W.FAMILY_POLY_GAUSSCOS:
            f = f + sample_poly_bruteforce(params[2 * D:], support, axes)
        return np.broadcast_to(f, shape).copy()
    if family == W.FAMILY_RATIONAL:
        c = params[:D]
        quad = sum(c[i] * _broadcast_axis(axes[i] ** 2, i, D) for i in range(D))
        return np.broadcast_to(1.0 / (1.0 + quad), shape).copy()
    if family == W.FAMILY_POLY:
        return sample_poly_bruteforce(params, support, axes)
    raise ValueError(family)


def sample_poly_bruteforce(coeffs: np.ndarray, support: np.ndarray, axes) -> np.ndarray:
    """p(x) = sum_m c_m prod_i T_{m_i}(x_i) at every grid point, term by term
    (Eq. (chebyshev_expansion)); T from the recurrence."""
    D = len(axes)
    shape = tuple(a.size for a in axes)
    dmax = int(support.max()) if support.size else 0
    tabs = [chebyshev_T_table(dmax, ax) for ax in axes]           # [n_i, dmax+1]
    pts = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), -1).reshape(-1, D)
    out = np.zeros(pts.shape[0])
    sup = support.astype(np.int64)
    step = max(1, 2_000_000 // max(1, sup.shape[0]))
    for s0 in range(0, pts.shape[0], step):
        p = pts[s0:s0 + step]
        prod = np.ones((p.shape[0], sup.shape[0]))
        for i in range(D):
            prod *= tabs[i][p[:, i]][:, sup[:, i]]
        out[s0:s0 + step] = prod @ coeffs
    return out.reshape(shape)


def sample_lgrid(family, params, support, sizes, nodes, kind: str = "extrema") -> np.ndarray:
    """Concatenated samples of all K grids (row-major per grid)."""
    return np.concatenate([sample_grid(family, params, support, grid_axes(sizes[l], nodes[l], kind)).ravel()
                           for l in range(sizes.shape[0])])


# ==========================================================================
# DCT-I (per axis) -- the F^(l) blocks of Eq. (main_linear_system)
# ==========================================================================
def dct1_matrix(n: int) -> np.ndarray:
    """Interpolation DCT-I on n >= 2 extrema points:
        y_k = (2 e_k/(n-1)) sum_j e_j cos(pi j k/(n-1)) x_j,  e_0 = e_{n-1} = 1/2, else 1,
    so that samples of sum_k a_k T_k (k < n) map to a.  The cosine argument
    j k is reduced modulo 2(n-1) in integers first."""
    j = np.arange(n)
    jk = np.outer(j, j) % (2 * (n - 1))
    e = np.ones(n)
    e[0] = e[-1] = 0.5
    return (2.0 * e[:, None] / (n - 1)) * e[None, :] * np.cos(np.pi * jk / (n - 1))


def dct1_grid(f: np.ndarray) -> np.ndarray:
    """Apply the DCT-I along every axis with n >= 2 (axes of size 1 are the
    identity).  Direct O(n^2) per fibre; no fast transform."""
    y = np.asarray(f, dtype=np.float64)
    for axis, n in enumerate(y.shape):
        if n >= 2:
            y = np.moveaxis(np.tensordot(dct1_matrix(n), y, axes=([1], [axis])), 0, axis)
    return y


# ==========================================================================
# Aliasing: fold, per-grid alias matrix, stacked system
# ==========================================================================
def fold(m, n: int):
    """Alias of degree m on an n-point extrema grid (n >= 2): T_m and
    T_fold(m) agree on every node.  r = m mod 2(n-1); fold = r if r <= n-1
    else 2(n-1) - r."""
    m = np.asarray(m, dtype=np.int64)
    period = 2 * (n - 1)
    r = m % period
    return np.where(r <= n - 1, r, period - r)


def grid_bins(support: np.ndarray, sizes_l) -> np.ndarray:
    """Row-major linear bin index of every support element on grid l:
    sum over axes with n_i >= 2 of fold(m_i) * stride_i (Eq.
    (aliasing_matrix_nd_diff): the column of m has its one nonzero there)."""
    D = len(sizes_l)
    strides = np.ones(D, dtype=np.int64)
    for i in range(D - 2, -1, -1):
        strides[i] = strides[i + 1] * int(sizes_l[i + 1])
    sup = support.astype(np.int64)
    bins = np.zeros(sup.shape[0], dtype=np.int64)
    for i in range(D):
        n = int(sizes_l[i])
        if n >= 2:
            bins += fold(sup[:, i], n) * strides[i]
    return bins


def grid_weights(support: np.ndarray, sizes_l, nodes_l) -> np.ndarray:
    """Entry of the column of m: prod over single-point axes of T_{m_i}(xi_i)."""
    w = np.ones(support.shape[0])
    for i, n in enumerate(sizes_l):
        if int(n) == 1:
            w *= chebyshev_T(support[:, i].astype(np.int64), nodes_l[i])
    return w


def alias_matrix_grid(support, sizes_l, nodes_l) -> sp.csr_matrix:
    """A^(l) over all T_l bins (T_l x N), one nonzero per column."""
    T = int(np.prod(np.asarray(sizes_l, dtype=np.int64)))
    N = support.shape[0]
    return sp.csr_matrix((grid_weights(support, sizes_l, nodes_l),
                          (grid_bins(support, sizes_l), np.arange(N))), shape=(T, N))


def alias_matrix_grid_bruteforce(support, sizes_l, nodes_l) -> np.ndarray:
    """A^(l) with no fold formula: column m = DCT-I of T_m sampled on grid l
    (Eq. (multi_dim_dct) read column by column).  Tiny grids only."""
    axes = grid_axes(sizes_l, nodes_l)
    D = len(axes)
    cols = []
    for m in support.astype(np.int64):
        f = np.ones(tuple(a.size for a in axes))
        for i in range(D):
            f = f * _broadcast_axis(chebyshev_T(m[i], axes[i]), i, D)
        cols.append(dct1_grid(f).ravel())
    return np.stack(cols, axis=1)


# ==========================================================================
# The paper's own grid: first-kind Chebyshev points, DCT-II with the 1/M
# quadrature normalisation and the signed alias relation of Lemma
# (lem:aliasing) / Eq. (aliasing_matrix_1d).  An axis with M points here is the
# paper's "N + 1 points" (Eq. (chebyshev_grid)).
# ==========================================================================
def first_kind_nodes(M: int, xi: float = 1.0) -> np.ndarray:
    """x_k = cos(theta_k), theta_k = (k + 1/2) pi / M, k = 0..M-1 (Eq.
    (chebyshev_grid)); the mirror symmetry x_{M-1-k} = -x_k is enforced and the
    middle point of an odd grid is exactly 0.  M == 1 is the single node xi
    (the same reading of single-point axes as on the extrema grid)."""
    if M == 1:
        return np.array([xi], dtype=np.float64)
    k = np.arange(M)
    x = np.cos(np.pi * (2 * k + 1) / (2 * M))
    half = M // 2
    x[M - half:] = -x[:half][::-1]
    if M % 2 == 1:
        x[half] = 0.0
    return x


def dct2_matrix(M: int) -> np.ndarray:
    """The quadrature of Eq. (quad_1D): b_n = (1/M) sum_k cos(n theta_k) f_k,
    n, k = 0..M-1, with the cosine argument n (2k + 1) reduced modulo 4M in
    integers before the call to cos."""
    n = np.arange(M)
    a = np.outer(n, 2 * n + 1) % (4 * M)
    return np.cos(np.pi * a / (2 * M)) / M


def dct2_grid(f: np.ndarray) -> np.ndarray:
    """Apply dct2_matrix along every axis with M >= 2 (direct O(M^2))."""
    y = np.asarray(f, dtype=np.float64)
    for axis, M in enumerate(y.shape):
        if M >= 2:
            y = np.moveaxis(np.tensordot(dct2_matrix(M), y, axes=([1], [axis])), 0, axis)
    return y


def aliasing_delta(ell, M: int):
    """Delta_N of Eq. (aliasing_delta) for an M = N + 1 point grid."""
    r = np.asarray(ell, dtype=np.int64) % (4 * M)
    return np.where(r == 0, 1.0, np.where(r == 2 * M, -1.0, 0.0))


def aliasing_entry(n, m, M: int):
    """A_{n,m} = Delta(m + n)/2 + Delta(m - n)/2, Eq. (aliasing_matrix_1d)."""
    n = np.asarray(n, dtype=np.int64)
    m = np.asarray(m, dtype=np.int64)
    return 0.5 * aliasing_delta(m + n, M) + 0.5 * aliasing_delta(m - n, M)


def fold_first_kind(m, M: int):
    """Row and value of the one entry of column m in the M x inf matrix of Eq.
    (aliasing_matrix_1d), M >= 2.  With q = m div 2M and r = m mod 2M:
      r < M : row r,      value (-1)^q (1 if r == 0 else 1/2)
      r > M : row 2M - r, value -(-1)^q / 2
      r = M : no entry (T_m vanishes on every node); given row 0, value 0."""
    m = np.asarray(m, dtype=np.int64)
    q, r = np.divmod(m, 2 * M)
    sgn = np.where(q % 2 == 0, 1.0, -1.0)
    row = np.where(r < M, r, np.where(r > M, 2 * M - r, 0))
    val = np.where(r < M, sgn * np.where(r == 0, 1.0, 0.5), np.where(r > M, -0.5 * sgn, 0.0))
    return row, val


def grid_bins_first_kind(support: np.ndarray, sizes_l) -> np.ndarray:
    D = len(sizes_l)
    strides = np.ones(D, dtype=np.int64)
    for i in range(D - 2, -1, -1):
        strides[i] = strides[i + 1] * int(sizes_l[i + 1])
    sup = support.astype(np.int64)
    bins = np.zeros(sup.shape[0], dtype=np.int64)
    for i in range(D):
        M = int(sizes_l[i])
        if M >= 2:
            bins += fold_first_kind(sup[:, i], M)[0] * strides[i]
    return bins


def grid_weights_first_kind(support: np.ndarray, sizes_l, nodes_l) -> np.ndarray:
    """Entry of column m: product over axes of the 1D entries (Eq.
    (aliasing_matrix_nd_diff) on a tensor grid) times T_{m_i}(xi_i) on
    single-point axes."""
    w = np.ones(support.shape[0])
    for i, M in enumerate(sizes_l):
        mi = support[:, i].astype(np.int64)
        if int(M) == 1:
            w *= chebyshev_T(mi, nodes_l[i])
        else:
            w *= fold_first_kind(mi, int(M))[1]
    return w


def alias_matrix_grid_first_kind_bruteforce(support, sizes_l, nodes_l) -> np.ndarray:
    """Column m = the quadrature (dct2_grid) of T_m sampled on the grid; no
    fold formula.  Tiny grids only."""
    axes = grid_axes(sizes_l, nodes_l, "first")
    D = len(axes)
    cols = []
    for m in support.astype(np.int64):
        f = np.ones(tuple(a.size for a in axes))
        for i in range(D):
            f = f * _broadcast_axis(chebyshev_T(m[i], axes[i]), i, D)
        cols.append(dct2_grid(f).ravel())
    return np.stack(cols, axis=1)


class AliasSystem:
    """The stacked least-squares system of Eq. (main_linear_system), rows of
    empty bins dropped (they do not involve c).  kind = "extrema" (DCT-I on
    extrema points, interpolation normalisation) or "first" (the paper's
    first-kind points, 1/M quadrature and signed half-weight entries)."""

    def __init__(self, support, sizes, nodes, kind: str = "extrema"):
        if kind not in ("extrema", "first"):
            raise ValueError(kind)
        self.kind = kind
        self.support = np.asarray(support)
        self.sizes = np.asarray(sizes)
        self.nodes = np.asarray(nodes)
        K = self.sizes.shape[0]
        N = self.support.shape[0]
        self.T = np.prod(self.sizes.astype(np.int64), axis=1)
        self.offsets = np.concatenate([[0], np.cumsum(self.T)])
        blocks, self.rows = [], []
        for l in range(K):
            if kind == "extrema":
                bins = grid_bins(self.support, self.sizes[l])
                Al = alias_matrix_grid(self.support, self.sizes[l], self.nodes[l])
            else:
                bins = grid_bins_first_kind(self.support, self.sizes[l])
                Al = sp.csr_matrix((grid_weights_first_kind(self.support, self.sizes[l], self.nodes[l]),
                                    (bins, np.arange(N))), shape=(int(self.T[l]), N))
            nonempty = np.unique(bins)
            self.rows.append(nonempty)
            blocks.append(Al[nonempty])
        self.A = sp.vstack(blocks).tocsr()
        self.R = self.A.shape[0]

    def rhs(self, samples: np.ndarray) -> np.ndarray:
        """b: per grid DCT of its samples, restricted to nonempty bins."""
        transform = dct1_grid if self.kind == "extrema" else dct2_grid
        out = []
        for l in range(self.sizes.shape[0]):
            f = samples[self.offsets[l]:self.offsets[l + 1]].reshape(tuple(int(n) for n in self.sizes[l]))
            out.append(transform(f).ravel()[self.rows[l]])
        return np.concatenate(out)


# ==========================================================================
# Least-squares solvers (Sec. 3.4: "solve ... using CG"; direct forms for pins)
# ==========================================================================
class RankDeficient(RuntimeError):
    pass


def householder_lstsq(A: np.ndarray, b: np.ndarray, rank_tol: float = 1e-12) -> np.ndarray:
    """min ||A c - b|| by Householder QR and back substitution (own code)."""
    A = np.array(A, dtype=np.float64, copy=True)
    b = np.array(b, dtype=np.float64, copy=True)
    m, n = A.shape
    if m < n:
        raise RankDeficient("fewer rows than columns")
    for k in range(n):
        x = A[k:, k]
        nx = np.linalg.norm(x)
        if nx == 0.0:
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv == 0.0:
            continue
        v /= nv
        A[k:, k:] -= 2.0 * np.outer(v, v @ A[k:, k:])
        b[k:] -= 2.0 * v * (v @ b[k:])
    Rm = np.triu(A[:n, :n])
    diag = np.abs(np.diag(Rm))
    if diag.min() <= rank_tol * diag.max():
        raise RankDeficient(f"min |R_kk| / max |R_kk| = {diag.min() / diag.max():.3e}")
    c = np.zeros(n)
    for k in range(n - 1, -1, -1):
        c[k] = (b[k] - Rm[k, k + 1:] @ c[k + 1:]) / Rm[k, k]
    return c


def csne_lstsq(A: sp.spmatrix, b: np.ndarray, refine: int = 4) -> np.ndarray:
    """Corrected semi-normal equations: Cholesky of A^T A, then corrections
    c += (A^T A)^{-1} A^T (b - A c).  Medium sizes (N up to ~2e4)."""
    import scipy.linalg as sla
    AtA = (A.T @ A).toarray()
    try:
        cf = sla.cho_factor(AtA, lower=False, check_finite=False)
    except np.linalg.LinAlgError as e:
        raise RankDeficient(str(e))
    c = sla.cho_solve(cf, A.T @ b, check_finite=False)
    for _ in range(refine):
        c = c + sla.cho_solve(cf, A.T @ (b - A @ c), check_finite=False)
    return c


def cgls(A, b: np.ndarray, tol: float = 1e-15, maxit: int = 100000):
    """Conjugate gradients on the normal equations of min ||A c - b|| (the
    "CG method" of Sec. 3.4), from c = 0.  Stops when
    ||A^T r|| <= tol ||A^T b|| or when ||A^T r|| has not improved for 200
    iterations.  Returns (c, iterations, ||A^T r|| / ||A^T b||)."""
    x = np.zeros(A.shape[1])
    r = np.array(b, dtype=np.float64, copy=True)
    s = A.T @ r
    p = s.copy()
    gamma = float(s @ s)
    gamma0 = gamma
    if gamma0 == 0.0:
        return x, 0, 0.0
    best, best_it, it = math.inf, 0, 0
    for it in range(1, maxit + 1):
        q = A @ p
        delta = float(q @ q)
        if delta == 0.0:
            break
        alpha = gamma / delta
        x += alpha * p
        r -= alpha * q
        s = A.T @ r
        gnew = float(s @ s)
        rel = math.sqrt(gnew / gamma0)
        if rel <= tol:
            gamma = gnew
            break
        if rel < best:
            best, best_it = rel, it
        elif it - best_it > 200:
            gamma = gnew
            break
        beta = gnew / gamma
        p = s + beta * p
        gamma = gnew
    return x, it, math.sqrt(gamma / gamma0)


def solve(system: AliasSystem, b: np.ndarray, method: str = "auto", tol: float = 1e-15):
    """The least-squares minimiser c* of Algorithm 3, by the tier that fits."""
    N = system.A.shape[1]
    if method == "auto":
        method = "qr" if N <= 600 else ("csne" if N <= 12000 else "cgls")
    if method == "qr":
        return householder_lstsq(system.A.toarray(), b)
    if method == "lstsq":
        return np.linalg.lstsq(system.A.toarray(), b, rcond=None)[0]
    if method == "csne":
        return csne_lstsq(system.A, b)
    if method == "cgls":
        return cgls(system.A, b, tol=tol)[0]
    raise ValueError(method)


def fct(support, sizes, nodes, samples, method: str = "auto", tol: float = 1e-15, kind: str = "extrema"):
    """Algorithm 3 end to end on given samples: build A, DCT, solve."""
    system = AliasSystem(support, sizes, nodes, kind)
    b = system.rhs(samples)
    return solve(system, b, method=method, tol=tol)


def condition_number(A) -> float:
    """kappa(A) = sigma_max / sigma_min, the singular values of the dense A
    (N up to a few thousand).  Returns inf when A has fewer rows than columns
    or sigma_min is below rounding level (R * eps * sigma_max)."""
    A = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    if A.shape[0] < A.shape[1]:
        return math.inf
    sv = np.linalg.svd(A, compute_uv=False)
    if sv[-1] <= sv[0] * A.shape[0] * np.finfo(np.float64).eps:
        return math.inf
    return float(sv[0] / sv[-1])


def evaluate_expansion(coeffs, support, points) -> np.ndarray:
    """p(x) = sum_m c_m prod_i T_{m_i}(x_i) (Eq. (chebyshev_expansion)) at each
    row of points [P, D], term by term with T from its definition
    cos(m arccos x).  The paper measures approximation error this way, at
    random points (Sec. 4)."""
    pts = np.atleast_2d(np.asarray(points, dtype=np.float64))
    sup = np.asarray(support).astype(np.int64)
    c = np.asarray(coeffs, dtype=np.float64)
    out = np.empty(pts.shape[0])
    for p in range(pts.shape[0]):
        terms = np.ones(sup.shape[0])
        for i in range(sup.shape[1]):
            terms *= chebyshev_T(sup[:, i], pts[p, i])
        out[p] = terms @ c
    return out


def construct_alias_system(support, cand_sizes, cand_nodes, kappa0: float = 1e4):
    """Algorithm 2 (Sec. 3.3): starting from no grids, append the next grid of
    the candidate sequence (each one an Algorithm 1 draw, passed in) until the
    stacked alias matrix has kappa(A) <= kappa0; a rank-deficient A has
    kappa = inf.  Returns ``(L, kappa(A))`` for the first L grids, or
    ``(None, kappa)`` when every candidate has been used."""
    cand_sizes = np.asarray(cand_sizes)
    kappa = math.inf
    for L in range(1, cand_sizes.shape[0] + 1):
        kappa = condition_number(AliasSystem(support, cand_sizes[:L], np.asarray(cand_nodes)[:L]).A)
        if kappa <= kappa0:
            return L, kappa
    return None, kappa


def numerical_rank(A, rtol: float = 1e-10) -> int:
    """Number of singular values of A above rtol * sigma_max (the definition
    of numerical rank; the singular values come from the dense SVD of A
    itself, since the eigenvalues of A^T A cannot resolve sigma below about
    1e-8 sigma_max)."""
    A = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
    if A.size == 0:
        return 0
    sv = np.linalg.svd(A, compute_uv=False)
    if sv[0] == 0.0:
        return 0
    return int((sv > sv[0] * rtol).sum())
