"""Seeded workload generators for the sparse FCT (random draws only).

Every random number the transform's inputs need is drawn here, from one
PCG64 stream per (seed, purpose), and handed to both the CUDA path and the
CPU oracle as data.  Nothing in this module evaluates a Chebyshev polynomial,
a DCT, a fold or a solve.

Conventions shared by both sides
--------------------------------
* ``support``: ``uint16[N, D]`` multi-indices; coefficient order = row order.
* ``sizes``: ``int32[K, D]``, points per axis of each grid (n >= 1).
* ``nodes``: ``float64[K, D]``, the single sample position used on an axis
  whose size is 1 (ignored elsewhere).
* samples of grid l form a row-major tensor of shape ``sizes[l]`` (last axis
  fastest); the K tensors are concatenated in grid order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Function families understood by the samplers (the values are part of the
# C interface, see include/fct.h: FCT_FAMILY_*).
FAMILY_POLY = 0            # f = sum_m c_m T_m(x); params = c[N] over the support
FAMILY_GAUSSCOS = 1        # f = exp(-sum a_i x_i^2) cos(sum b_i x_i); params = [a(D), b(D)]
FAMILY_RATIONAL = 2        # f = 1 / (1 + sum c_i x_i^2); params = [c(D)]
FAMILY_POLY_GAUSSCOS = 3   # poly + gausscos; params = [a(D), b(D), c(N)]

# Sub-stream ids: one independent stream per purpose of a seed.
_PURPOSE = {
    "coeffs": 1,     # sparse-polynomial coefficients
    "function": 2,   # a_i, b_i, c_i of the analytic families
    "sizes": 3,      # Algorithm 1 draws (permutation + per-axis sizes)
    "nodes": 4,      # single-point node positions
    "batch": 5,      # per-transform shapes inside a batch
    "arrivals": 6,   # serving arrival process
    "probe": 7,      # start vectors of condition probes and test matrices
    "support": 8,    # random sparse supports
    "support_vec": 9,  # random sparse supports drawn in vectorised batches
}


def stream(seed: int, purpose: str) -> np.random.Generator:
    """Independent PCG64 generator for ``(seed, purpose)``."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), _PURPOSE[purpose]])))


# --------------------------------------------------------------------------
# Supports
# --------------------------------------------------------------------------
def total_degree_support(D: int, d: int) -> np.ndarray:
    """All n in N^D with |n|_1 <= d, lexicographic (axis 0 slowest), uint16[N, D].

    This is the total-degree index set S^1_{d,D} of Sec. 2.
    """
    rows = np.zeros((1, 0), dtype=np.int64)
    rem = np.array([d], dtype=np.int64)
    for _ in range(D):
        counts = rem + 1
        total = int(counts.sum())
        starts = np.cumsum(counts) - counts
        vals = np.arange(total, dtype=np.int64) - np.repeat(starts, counts)
        rows = np.concatenate([np.repeat(rows, counts, axis=0), vals[:, None]], axis=1)
        rem = np.repeat(rem, counts) - vals
    return rows.astype(np.uint16)


def euclidean_support(D: int, d: int) -> np.ndarray:
    """All n in N^D with |n|_2 <= d (the Euclidean index set S^2_{d,D} of
    Sec. 2), lexicographic, uint16[N, D]: the total-degree set filtered by the
    integer test sum n_i^2 <= d^2 (|n|_2 <= d implies |n|_1 <= d sqrt(D))."""
    cap = int(np.floor(d * np.sqrt(D))) + 1
    rows = np.zeros((1, 0), dtype=np.int64)
    sq = np.zeros(1, dtype=np.int64)
    for _ in range(D):
        vals = np.arange(min(d, cap) + 1, dtype=np.int64)
        ok = sq[:, None] + vals[None, :] ** 2 <= d * d
        r_idx, v_idx = np.nonzero(ok)
        rows = np.concatenate([rows[r_idx], vals[v_idx][:, None]], axis=1)
        sq = sq[r_idx] + vals[v_idx] ** 2
    return rows.astype(np.uint16)


def sparse_infinity_support(seed: int, D: int, d: int, N: int, nonzeros: int) -> np.ndarray:
    """N distinct multi-indices of S^inf_{d,D} (max degree d), each with
    exactly `nonzeros` nonzero components at uniformly drawn axes with values
    uniform in {1..d}, plus the zero index; sorted lexicographically.  (The
    paper's sparse-support family draws N multi-indices of S^inf_{d,D} at
    random; `nonzeros` fixes how many components of each are nonzero.)"""
    g = stream(seed, "support")
    seen = {tuple([0] * D)}
    out = [np.zeros(D, dtype=np.int64)]
    while len(out) < N:
        m = np.zeros(D, dtype=np.int64)
        axes = g.choice(D, size=nonzeros, replace=False)
        m[axes] = g.integers(1, d + 1, size=nonzeros)
        t = tuple(m.tolist())
        if t not in seen:
            seen.add(t)
            out.append(m)
    arr = np.stack(out)
    order = np.lexsort(arr.T[::-1])
    return arr[order].astype(np.uint16)


def sparse_support_vectorised(seed: int, D: int, d: int, N: int, nonzeros: int) -> np.ndarray:
    """N distinct multi-indices of S^inf_{d,D}: the zero index, then indices with
    exactly `nonzeros` nonzero components at uniformly drawn axes with values
    uniform in {1..d}, in the order they were drawn (duplicates dropped).  The
    same family as sparse_infinity_support, drawn in vectorised batches for
    supports of 1e5..1e7 indices (a different random sequence)."""
    g = stream(seed, "support_vec")
    rows = [np.zeros((1, 2 * nonzeros), dtype=np.uint8)]
    have = 1
    while have < N:
        n = int((N - have) * 1.2) + 1024
        keys = g.random((n, D), dtype=np.float32)
        axes = np.sort(np.argpartition(keys, nonzeros, axis=1)[:, :nonzeros], axis=1)
        vals = g.integers(1, d + 1, size=(n, nonzeros))
        rows.append(np.hstack([axes, vals]).astype(np.uint8))
        allr = np.ascontiguousarray(np.vstack(rows))
        view = allr.view(np.dtype((np.void, allr.shape[1]))).ravel()
        _, first = np.unique(view, return_index=True)
        keep = np.sort(first)
        rows = [allr[keep]]
        have = len(keep)
    sel = rows[0][:N]
    out = np.zeros((N, D), dtype=np.uint16)
    r = np.arange(1, N)
    for j in range(nonzeros):
        out[r, sel[1:, j].astype(np.int64)] = sel[1:, nonzeros + j]
    return out


# --------------------------------------------------------------------------
# L-grids
# --------------------------------------------------------------------------
def alg1_sampling_rates(g: np.random.Generator, N: int, D: int, lo: int, hi: int) -> np.ndarray:
    """One draw of Algorithm 1 (sampling rate selection), Sec. 3.3.

    Visit the axes in a random order, give each a size drawn uniformly from
    {lo..hi}; once the running product exceeds N the draw that crossed is
    kept and every remaining axis gets one point.
    """
    perm = g.permutation(D)
    sizes = np.ones(D, dtype=np.int32)
    prod = 1
    for j in range(D):
        n = int(g.integers(lo, hi + 1))
        sizes[perm[j]] = n
        prod *= n
        if prod > N:
            break
    return sizes


def l_grid(seed: int, N: int, D: int, K: int, lo: int, hi: int):
    """K grids by repeated Algorithm 1 draws, plus single-point node positions.

    Returns ``(sizes int32[K, D], nodes float64[K, D])``.  A node is
    ``cos(pi u)`` with u ~ U(0, 1): an arcsine-distributed point in [-1, 1],
    used only on axes of size 1.
    """
    g = stream(seed, "sizes")
    sizes = np.stack([alg1_sampling_rates(g, N, D, lo, hi) for _ in range(K)]).astype(np.int32)
    u = stream(seed, "nodes").random((K, D))
    nodes = np.cos(np.pi * u)
    return sizes, nodes


# --------------------------------------------------------------------------
# Function parameters
# --------------------------------------------------------------------------
def poly_coefficients(seed: int, support: np.ndarray, decay: float = 0.8) -> np.ndarray:
    """c_m = z_m * decay^{|m|_1}, z_m ~ N(0, 1) i.i.d. over the support."""
    z = stream(seed, "coeffs").standard_normal(support.shape[0])
    deg = support.astype(np.int64).sum(axis=1)
    return z * decay ** deg


def gausscos_params(seed: int, D: int) -> np.ndarray:
    """[a(D), b(D)] with a_i ~ U[0.2, 1], b_i ~ U[0, 2]."""
    g = stream(seed, "function")
    a = g.uniform(0.2, 1.0, D)
    b = g.uniform(0.0, 2.0, D)
    return np.concatenate([a, b])


def rational_params(seed: int, D: int) -> np.ndarray:
    """[c(D)] with c_i ~ U[0.1, 1]."""
    return stream(seed, "function").uniform(0.1, 1.0, D)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    D: int
    d: int
    support: np.ndarray          # uint16[N, D]
    sizes: np.ndarray            # int32[K, D]
    nodes: np.ndarray            # float64[K, D]
    family: int
    params: np.ndarray           # float64, layout per family
    coeffs_true: np.ndarray | None  # float64[N] when f lies in the span of the support
    tol: float                   # solver stopping tolerance (relative |A^T r|)
    precision: str               # "fp64" or "mixed"

    @property
    def N(self) -> int:
        return int(self.support.shape[0])

    @property
    def K(self) -> int:
        return int(self.sizes.shape[0])

    @property
    def M(self) -> int:
        return int(np.prod(self.sizes.astype(np.int64), axis=1).sum())

    def grid_offsets(self) -> np.ndarray:
        t = np.prod(self.sizes.astype(np.int64), axis=1)
        return np.concatenate([[0], np.cumsum(t)]).astype(np.int64)


def make_workload(name: str, seed: int, D: int, d: int, K: int, lo: int, hi: int,
                  family: int, tol: float = 1e-13, precision: str = "fp64") -> Workload:
    support = total_degree_support(D, d)
    N = support.shape[0]
    sizes, nodes = l_grid(seed, N, D, K, lo, hi)
    coeffs = None
    if family == FAMILY_POLY:
        coeffs = poly_coefficients(seed, support)
        params = coeffs.copy()
    elif family == FAMILY_GAUSSCOS:
        params = gausscos_params(seed, D)
    elif family == FAMILY_RATIONAL:
        params = rational_params(seed, D)
    elif family == FAMILY_POLY_GAUSSCOS:
        params = np.concatenate([gausscos_params(seed, D), poly_coefficients(seed, support)])
    else:
        raise ValueError(f"unknown family {family}")
    return Workload(name, D, d, support, sizes, nodes, family, params, coeffs, tol, precision)


def config_small_poly(seed: int = 1) -> Workload:
    """D=2, total degree 16 (N=153), K=4 grids with 9..33 points per axis,
    seeded sparse polynomial; the case the oracle solves in seconds."""
    return make_workload("D2_d16_poly_K4", seed, 2, 16, 4, 9, 33, FAMILY_POLY, tol=1e-13)


def config_d6_gausscos(seed: int = 2, family: int = FAMILY_GAUSSCOS) -> Workload:
    """D=6, total degree 10 (N=8008), Gaussian-cosine target.  L = 3D = 18 grids
    drawn by Algorithm 1 with sizes in {1..d+1}."""
    tag = "gausscos" if family == FAMILY_GAUSSCOS else "poly"
    return make_workload(f"D6_d10_{tag}_K18", seed, 6, 10, 18, 1, 11, family, tol=1e-13)


def config_d10_rational(seed: int = 3, precision: str = "mixed") -> Workload:
    """D=10, total degree 8 (N=43758), rational target.  L = 3D = 30 grids,
    sizes in {1..d+1}."""
    return make_workload("D10_d8_rational_K30", seed, 10, 8, 30, 1, 9, FAMILY_RATIONAL,
                         tol=1e-12, precision=precision)


def binom(n: int, k: int) -> int:
    return math.comb(n, k)


def config_batch(seed: int = 4, B: int = 512, grids_per_dim: int = 3) -> list:
    """B independent transforms: D ~ U{3..8}, total degree d ~ U{6..14}, each
    target a seeded sparse polynomial on P^D_d plus the Gaussian-cosine
    function.  The nominal per-transform grid count is drawn from {4..10} and
    recorded in the name; the L-grid uses L = 3D grids with sizes {1..d+1}
    (Algorithm 1), the paper's default, because nominal counts that small
    leave total-degree supports rank-deficient.  A larger grids_per_dim
    extends each transform's grid sequence (the candidates of Algorithm 2)."""
    g = stream(seed, "batch")
    out = []
    for t in range(B):
        D = int(g.integers(3, 9))
        d = int(g.integers(6, 15))
        k_nominal = int(g.integers(4, 11))
        out.append(make_workload(f"b{t}_D{D}_d{d}_Knom{k_nominal}", seed * 1_000_003 + t, D, d, grids_per_dim * D,
                                 1, d + 1, FAMILY_POLY_GAUSSCOS, tol=1e-12, precision="mixed"))
    return out


def serving_shapes(seed: int = 5, dims=range(2, 21), nmin: int = 1000, nmax: int = 100000,
                   grids_per_dim: int = 3) -> list:
    """One plan shape per dimension D: total degree d drawn uniformly from the
    degrees whose support size C(D+d, d) lies in [nmin, nmax]; L = 3D grids
    (grids_per_dim * D) with sizes {1..d+1} (Algorithm 1).  Grid draws are
    sequential, so a larger grids_per_dim extends the same sequence: it is the
    candidate list for Algorithm 2.  Targets are filled in per request."""
    g = stream(seed, "batch")
    out = []
    for D in dims:
        valid = [d for d in range(1, 2000) if nmin <= math.comb(D + d, d) <= nmax]
        d = int(valid[int(g.integers(0, len(valid)))])
        out.append(make_workload(f"serve_D{D}_d{d}", seed * 1_000_003 + D, D, d, grids_per_dim * D, 1, d + 1,
                                 FAMILY_GAUSSCOS, tol=1e-12, precision="mixed"))
    return out


def first_grids(w: Workload, L: int) -> Workload:
    """The same workload on the first L grids of its L-grid."""
    return dataclasses.replace(w, name=f"{w.name}_L{L}", sizes=w.sizes[:L].copy(), nodes=w.nodes[:L].copy())


def serving_requests(seed: int, n: int, rate: float, n_shapes: int, poly_fraction: float = 0.05):
    """Poisson arrivals at `rate` req/s: list of (arrival_s, shape index,
    is_polynomial, parameter seed)."""
    g = stream(seed, "arrivals")
    t = np.cumsum(g.exponential(1.0 / rate, n))
    shape = g.integers(0, n_shapes, n)
    poly = g.random(n) < poly_fraction
    pseed = g.integers(0, 2**31 - 1, n)
    return [(float(t[i]), int(shape[i]), bool(poly[i]), int(pseed[i])) for i in range(n)]
