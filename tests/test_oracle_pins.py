"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: a closed
form derived by hand, a library routine, brute force, an invariant of the
alias structure, or exact recovery of a polynomial inside the support (the
consistent system of Eq. (main_linear_system)).  ``test_oracle_mutations.py``
plants plausible mistakes in the oracle and checks that these pins catch them.
"""
import itertools
import math
import os

import numpy as np
import numpy.polynomial.chebyshev as npcheb
import pytest
import scipy.fft

import workloads as W
from oracle import fct_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Sec. 2
def test_chebyshev_definition_recurrence_and_library_agree():
    """T_n(x) = cos(n arccos x) and the three-term recurrence (Sec. 2) agree
    with numpy's Chebyshev series evaluation."""
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-1, 1, 200), [-1.0, 0.0, 1.0]])
    tab = O.chebyshev_T_table(40, x)
    for n in range(41):
        e = np.zeros(n + 1)
        e[n] = 1.0
        ref = npcheb.chebval(x, e)
        assert np.max(np.abs(tab[:, n] - ref)) < 1e-12
        assert np.max(np.abs(O.chebyshev_T(n, x) - ref)) < 1e-12


def _golden_counts():
    rows = []
    with open(os.path.join(GOLDEN, "support_counts.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                D, d, N = (int(v) for v in line.split())
                rows.append((D, d, N))
    return rows


@pytest.mark.parametrize("D,d,N", _golden_counts())
def test_support_size_eq_N_1norm(D, d, N):
    """|S^1_{d,D}| = C(d+D, d) (Eq. (N_1norm)) for the oracle's count and the
    shared enumerator; brute force over the box where it is small."""
    assert O.support_size_total_degree(d, D) == N
    if N <= 50000:
        sup = W.total_degree_support(D, d)
        assert sup.shape == (N, D)
        assert len({tuple(r) for r in sup.tolist()}) == N
        assert int(sup.astype(np.int64).sum(axis=1).max(initial=0)) <= d
    if (d + 1) ** D <= 200000:
        bf = {tuple(r) for r in O.support_total_degree_bruteforce(d, D).tolist()}
        assert bf == {tuple(r) for r in W.total_degree_support(D, d).tolist()}


# ---------------------------------------------------------------- grids
@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 9, 33, 64])
def test_extrema_nodes(n):
    x = O.extrema_nodes(n)
    assert x[0] == 1.0 and x[-1] == -1.0
    assert np.all(np.diff(x) < 0)
    assert np.array_equal(x, -x[::-1])
    if n % 2:
        assert x[n // 2] == 0.0
    assert np.max(np.abs(x - np.cos(np.pi * np.arange(n) / (n - 1)))) < 1e-15


# ---------------------------------------------------------------- DCT-I
def _golden_dct():
    rows = []
    with open(os.path.join(GOLDEN, "dct1_closed_forms.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                n, f, a = line.split("|")
                rows.append((int(n), [float(v) for v in f.split()], [float(v) for v in a.split()]))
    return rows


@pytest.mark.parametrize("n,f,a", _golden_dct())
def test_dct1_closed_forms(n, f, a):
    assert np.allclose(O.dct1_matrix(n) @ np.array(f), np.array(a), atol=1e-15, rtol=0)


@pytest.mark.parametrize("n", [2, 3, 5, 9, 17, 33, 100, 446])
def test_dct1_maps_sampled_Tk_to_unit_vector(n):
    """DCT-I of T_k sampled on the n extrema is e_k for k < n (interpolation is
    exact for degree < n)."""
    x = O.extrema_nodes(n)
    C = O.dct1_matrix(n)
    V = np.stack([O.chebyshev_T(k, x) for k in range(n)], axis=1)   # V[j, k] = T_k(x_j)
    assert np.max(np.abs(C @ V - np.eye(n))) < 1e-12 * max(1, n / 10)


@pytest.mark.parametrize("n", [2, 3, 7, 16, 33])
def test_dct1_matches_scipy_type1(n):
    """scipy's unnormalised DCT-I y_k = x_0 + (-1)^k x_{n-1} + 2 sum_{j=1}^{n-2}
    x_j cos(pi j k/(n-1)) relates to ours by a_k = e_k y_k / (n-1)."""
    rng = np.random.default_rng(n)
    f = rng.standard_normal(n)
    y = scipy.fft.dct(f, type=1)
    e = np.ones(n)
    e[0] = e[-1] = 0.5
    assert np.max(np.abs(O.dct1_matrix(n) @ f - e * y / (n - 1))) < 1e-13


@pytest.mark.parametrize("shape", [(3, 4), (2, 5, 3), (1, 6, 4), (5, 1, 1, 3)])
def test_dct1_grid_equals_square_vandermonde_solve(shape):
    """On one tensor grid the multi-dimensional DCT-I is interpolation: it
    solves V a = f with V[pt, k] = prod_i T_{k_i}(x_{i,pt_i}) over all k in the
    grid's index box (brute-force linear solve, D <= 4)."""
    rng = np.random.default_rng(sum(shape))
    nodes = rng.uniform(-1, 1, len(shape))
    axes = O.grid_axes(np.array(shape), nodes)
    f = rng.standard_normal(shape)
    D = len(shape)
    idx = list(itertools.product(*[range(s) for s in shape]))
    V = np.array([[np.prod([O.chebyshev_T(k[i], axes[i][p[i]]) for i in range(D)]) for k in idx] for p in idx])
    a = np.linalg.solve(V, f.ravel())
    assert np.max(np.abs(O.dct1_grid(f).ravel() - a)) < 1e-12


# ---------------------------------------------------------------- fold
def test_fold_identity_exhaustive():
    """T_m(x_j) = T_fold(m)(x_j) on every extrema node (n <= 64, m <= 20 n),
    in FP64 and in the exact integer form m j = +-fold(m) j (mod 2(n-1))."""
    for n in range(2, 65):
        x = O.extrema_nodes(n)
        m = np.arange(0, 20 * n + 1)
        fm = O.fold(m, n)
        assert fm.min() >= 0 and fm.max() <= n - 1
        assert np.array_equal(fm[:n], np.arange(n))          # no alias below n
        j = np.arange(n)
        P = 2 * (n - 1)
        lhs = np.outer(m, j) % P
        rhs = np.outer(fm, j) % P
        assert np.all((lhs == rhs) | (lhs == (P - rhs) % P))
        err = np.abs(O.chebyshev_T(m[:, None], x[None, :]) - O.chebyshev_T(fm[:, None], x[None, :]))
        assert err.max() < 1e-9    # cos(n arccos x) at large n loses ~n*eps


# ---------------------------------------------------------------- alias matrix
TINY = [
    # (D, d, sizes, nodes)
    (1, 9, [[4]], [[1.0]]),
    (2, 6, [[3, 4], [5, 1], [1, 2]], [[0.3, 0.1], [0.2, -0.7], [0.45, 0.9]]),
    (3, 4, [[2, 3, 1], [1, 1, 4], [3, 2, 2]], [[0.1, 0.2, 0.6], [-0.3, 0.8, 0.0], [0.5, 0.5, 0.5]]),
]


@pytest.mark.parametrize("D,d,sizes,nodes", TINY)
def test_alias_matrix_fold_equals_bruteforce(D, d, sizes, nodes):
    """A^(l) from the fold formula equals, column by column, the DCT-I of T_m
    sampled on the grid (no fold formula involved)."""
    sup = W.total_degree_support(D, d)
    for sz, nd in zip(np.array(sizes), np.array(nodes)):
        Af = O.alias_matrix_grid(sup, sz, nd).toarray()
        Ab = O.alias_matrix_grid_bruteforce(sup, sz, nd)
        assert np.array_equal(Af != 0, np.abs(Ab) > 1e-12)
        assert np.max(np.abs(Af - Ab)) < 1e-12


def test_alias_invariants():
    """One nonzero per column per grid (Sec. 3.5); with xi = 1 every entry is 1,
    so ||A||_F^2 = K N and each grid's rows sum to N."""
    w = W.config_small_poly()
    ones = np.ones_like(w.nodes)
    s = O.AliasSystem(w.support, w.sizes, ones)
    assert s.A.nnz == w.K * w.N
    assert np.allclose(s.A.data, 1.0)
    assert abs(s.A.multiply(s.A).sum() - w.K * w.N) < 1e-9
    start = 0
    for l in range(w.K):
        Rl = len(s.rows[l])
        blk = s.A[start:start + Rl]
        assert np.all(np.diff(blk.tocsc().indptr) == 1)
        assert abs(blk.sum() - w.N) < 1e-9
        start += Rl
    # with generic nodes the entry magnitudes are |prod T(xi)| <= 1
    s2 = O.AliasSystem(w.support, w.sizes, w.nodes)
    assert np.all(np.abs(s2.A.data) <= 1.0 + 1e-15)


def test_adjoint_identity():
    rng = np.random.default_rng(5)
    w = W.make_workload("t", 11, 3, 6, 6, 1, 7, W.FAMILY_GAUSSCOS)
    s = O.AliasSystem(w.support, w.sizes, w.nodes)
    p = rng.standard_normal(s.A.shape[1])
    r = rng.standard_normal(s.A.shape[0])
    lhs, rhs = (s.A @ p) @ r, p @ (s.A.T @ r)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs) + 1e-13


# ---------------------------------------------------------------- recovery
RECOVERY = [
    ("D1", 21, 1, 12, 5, 2, 9),
    ("D2", 22, 2, 8, 4, 3, 9),
    ("D3", 23, 3, 5, 9, 1, 6),
    ("D4", 24, 4, 4, 12, 1, 5),
]


@pytest.mark.parametrize("name,seed,D,d,K,lo,hi", RECOVERY)
def test_exact_recovery_of_polynomials_in_support(name, seed, D, d, K, lo, hi):
    """A polynomial whose coefficients live on the support makes the system
    consistent (Eq. (main_linear_system)); the least-squares solution is the
    true coefficient vector.  Samples by brute-force evaluation."""
    w = W.make_workload(name, seed, D, d, K, lo, hi, W.FAMILY_POLY)
    s = O.AliasSystem(w.support, w.sizes, w.nodes)
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    b = s.rhs(f)
    for method in ("qr", "lstsq", "csne"):
        c = O.solve(s, b, method)
        assert np.linalg.norm(c - w.coeffs_true) <= 1e-11 * np.linalg.norm(w.coeffs_true), method
    c, it, rel = O.cgls(s.A, b, tol=1e-15)
    assert np.linalg.norm(c - w.coeffs_true) <= 1e-11 * np.linalg.norm(w.coeffs_true)


def test_config_small_recovers_exactly():
    w = W.config_small_poly()
    c = O.fct(w.support, w.sizes, w.nodes, O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes), "qr")
    assert np.linalg.norm(c - w.coeffs_true) <= 1e-13 * np.linalg.norm(w.coeffs_true)


def test_full_grid_is_selection_and_returns_dct_output():
    """One grid resolving every degree of the support (n_i >= d+1) has no
    collision: A selects rows, and c* is the DCT output at the support's bins
    (the classical tensor DCT approach of Sec. 4.2)."""
    D, d = 3, 4
    sup = W.total_degree_support(D, d)
    sizes = np.array([[d + 1, d + 2, d + 1]], dtype=np.int32)
    nodes = np.ones((1, D))
    s = O.AliasSystem(sup, sizes, nodes)
    assert s.R == sup.shape[0]
    f = O.sample_lgrid(W.FAMILY_RATIONAL, W.rational_params(3, D), sup, sizes, nodes)
    y = O.dct1_grid(f.reshape(tuple(sizes[0])))
    c = O.solve(s, s.rhs(f), "qr")
    assert np.max(np.abs(c - y[tuple(sup.T.astype(np.int64))])) < 1e-14


# ---------------------------------------------------------------- solvers
def test_solver_tiers_agree_and_are_optimal():
    """Householder QR, LAPACK lstsq, corrected semi-normal equations and CGLS
    agree on a non-polynomial target, and the answer satisfies the normal
    equations A^T (b - A c) = 0."""
    w = W.make_workload("tiers", 31, 4, 5, 12, 1, 6, W.FAMILY_GAUSSCOS)
    s = O.AliasSystem(w.support, w.sizes, w.nodes)
    b = s.rhs(O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes))
    cq = O.solve(s, b, "qr")
    cl = O.solve(s, b, "lstsq")
    cn = O.solve(s, b, "csne")
    cg, it, rel = O.cgls(s.A, b, tol=1e-15)
    nq = np.linalg.norm(cq)
    for c in (cl, cn, cg):
        assert np.linalg.norm(c - cq) <= 1e-12 * nq
    g = s.A.T @ (b - s.A @ cq)
    assert np.linalg.norm(g) <= 1e-13 * np.linalg.norm(s.A.T @ b)


# ---------------------------------------------------------------- samplers
def _golden_samples():
    rows = {}
    for line in open(os.path.join(GOLDEN, "sampler_values.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        fam, idx, val, _ = [t.strip() for t in line.split("|")]
        i0, i1 = (int(t) for t in idx.split())
        rows.setdefault(fam, {})[(i0, i1)] = float(val)
    return rows


# the hand-picked grid of the golden file: n = 4, n = 3, one point at xi = 1/2
_GOLDEN_SIZES = np.array([4, 3, 1], dtype=np.int32)
_GOLDEN_NODES = np.array([0.0, 0.0, 0.5])
_GOLDEN_PARAMS = {
    "gausscos": (W.FAMILY_GAUSSCOS, np.array([0.5, 0.25, 1.0, 1.0, 2.0, 0.5])),
    "rational": (W.FAMILY_RATIONAL, np.array([0.5, 0.25, 1.0])),
    "runge": (W.FAMILY_RATIONAL, np.array([10.0, 10.0, 10.0])),
}


@pytest.mark.parametrize("family", ["gausscos", "rational", "runge"])
def test_sampler_families_match_hand_values(family):
    """The analytic targets on a small grid equal values worked out by hand
    (tests/golden/sampler_values.txt); the Runge case is the paper's f_1
    (Sec. 4, Function Class #1) on that grid."""
    fam, params = _GOLDEN_PARAMS[family]
    want = _golden_samples()[family]
    sup = np.zeros((1, 3), dtype=np.uint16)
    got = O.sample_grid(fam, params, sup, O.grid_axes(_GOLDEN_SIZES, _GOLDEN_NODES))
    assert got.shape == (4, 3, 1)
    assert len(want) == 12
    for (i0, i1), v in want.items():
        assert abs(got[i0, i1, 0] - v) <= 2e-16 * max(1.0, abs(v)), (family, i0, i1, got[i0, i1, 0], v)


@pytest.mark.parametrize("D", [1, 4, 9])
def test_sampler_families_at_the_origin_and_on_an_axis(D):
    """Special cases: both families are 1 at x = 0; with x = t e_k the
    Gaussian-cosine reduces to exp(-a_k t^2) cos(b_k t) and the rational form
    to 1 / (1 + c_k t^2), independent of the other parameters."""
    g = W.stream(31, "probe")
    sizes = np.ones(D, dtype=np.int32)
    gp = W.gausscos_params(7, D)
    rp = W.rational_params(7, D)
    sup = np.zeros((1, D), dtype=np.uint16)
    zero = O.grid_axes(sizes, np.zeros(D))
    assert O.sample_grid(W.FAMILY_GAUSSCOS, gp, sup, zero).item() == 1.0
    assert O.sample_grid(W.FAMILY_RATIONAL, rp, sup, zero).item() == 1.0
    for k in range(D):
        t = float(g.uniform(-1.0, 1.0))
        nodes = np.zeros(D)
        nodes[k] = t
        axes = O.grid_axes(sizes, nodes)
        want_g = math.exp(-gp[k] * t * t) * math.cos(gp[D + k] * t)
        want_r = 1.0 / (1.0 + rp[k] * t * t)
        assert abs(O.sample_grid(W.FAMILY_GAUSSCOS, gp, sup, axes).item() - want_g) <= 1e-15
        assert abs(O.sample_grid(W.FAMILY_RATIONAL, rp, sup, axes).item() - want_r) <= 1e-15


def test_sampler_poly_gausscos_is_the_sum_of_its_parts():
    """The combined family is the Gaussian-cosine plus the polynomial."""
    D, d = 3, 4
    sup = W.total_degree_support(D, d)
    axes = O.grid_axes(np.array([5, 1, 4]), np.array([0.0, 0.3, 0.0]))
    gp = W.gausscos_params(3, D)
    c = W.poly_coefficients(3, sup)
    both = O.sample_grid(W.FAMILY_POLY_GAUSSCOS, np.concatenate([gp, c]), sup, axes)
    parts = O.sample_grid(W.FAMILY_GAUSSCOS, gp, sup, axes) + O.sample_grid(W.FAMILY_POLY, c, sup, axes)
    assert np.array_equal(both, parts)


def _matrix_with_singular_values(sv, rows, seed):
    """U diag(sv) V^T with random orthogonal U (rows x n) and V (n x n)."""
    g = W.stream(seed, "probe")
    n = len(sv)
    U, _ = np.linalg.qr(g.standard_normal((rows, n)))
    V, _ = np.linalg.qr(g.standard_normal((n, n)))
    return (U * np.asarray(sv)) @ V.T


def test_numerical_rank_of_constructed_matrices():
    """rank = number of singular values above rtol * sigma_max: exact on
    matrices built with known singular values (including ones too small for
    the eigenvalues of A^T A to resolve)."""
    sv = [1.0, 1e-3, 1e-6, 1e-9, 1e-12, 0.0, 0.0]
    A = _matrix_with_singular_values(sv, 12, 5)
    assert O.numerical_rank(A, rtol=1e-10) == 4
    assert O.numerical_rank(A, rtol=1e-7) == 3
    assert O.numerical_rank(A, rtol=1e-4) == 2
    assert O.numerical_rank(A, rtol=1e-2) == 1
    assert O.numerical_rank(_matrix_with_singular_values([2.0] * 6, 9, 6)) == 6
    assert O.numerical_rank(np.zeros((5, 3))) == 0


def test_rank_deficient_plan_is_detected():
    """All grids sharing one single-point node at x = 1 on the same axis: the
    polynomial T_1(x_0) - 1 vanishes on every grid, so A loses rank and the
    QR tier refuses."""
    D, d = 2, 3
    sup = W.total_degree_support(D, d)
    sizes = np.array([[1, 5], [1, 4], [1, 6]], dtype=np.int32)
    s = O.AliasSystem(sup, sizes, np.ones((3, D)))
    with pytest.raises(O.RankDeficient):
        O.householder_lstsq(s.A.toarray(), np.ones(s.R))
    # T_{m_0}(1) = 1, so every column depends on m_1 alone; the four values
    # m_1 = 0..3 fold to distinct bins of the 5-point axis: rank exactly 4
    assert O.numerical_rank(s.A) == 4


# ---------------------------------------------------------------- workloads
def test_alg1_postconditions():
    """Algorithm 1: sizes in {lo..hi} on drawn axes, 1 elsewhere; the running
    product first exceeds N at the last drawn axis (or never)."""
    g = W.stream(7, "sizes")
    for _ in range(500):
        D = int(g.integers(1, 12))
        N = int(g.integers(1, 10000))
        sizes = W.alg1_sampling_rates(g, N, D, 2, 9)
        assert sizes.min() >= 1 and sizes.max() <= 9
        prod = int(np.prod(sizes.astype(np.int64)))
        drawn = sizes[sizes > 1]
        # at most one draw past N: dropping the smallest drawn factor leaves <= N
        assert prod <= N or prod // int(drawn.min()) <= N * 9
        if prod <= N:
            assert drawn.size == D       # never crossed: every axis was drawn


def test_workload_shapes():
    w = W.config_small_poly()
    assert (w.N, w.D, w.K) == (153, 2, 4)
    assert w.sizes.min() >= 9 and w.sizes.max() <= 33
    assert w.M == int(np.prod(w.sizes, axis=1).sum())
    w2 = W.config_d6_gausscos()
    assert (w2.N, w2.K) == (8008, 18)


# ---------------------------------------------------------------- Algorithm 2
def _stacked_bruteforce(support, sizes, nodes):
    """Alias matrices of the grids from the definition (every bin, empty rows
    included: zero rows change no singular value)."""
    return np.vstack([O.alias_matrix_grid_bruteforce(support, sizes[l], nodes[l]) for l in range(len(sizes))])


def _kappa_eig(A):
    ev = np.linalg.eigvalsh(A.T @ A)
    return math.sqrt(ev[-1] / ev[0]) if ev[0] > 0 else math.inf


def test_condition_number_closed_forms():
    """kappa of a diagonal matrix is max/min of |d|; of an orthogonal one, 1;
    a wide matrix is rank-deficient; for a moderately conditioned alias
    matrix it equals the eigenvalue route sqrt(lambda_max/lambda_min) of A^T A."""
    d = np.array([3.0, -0.5, 2.0, 0.25])
    assert O.condition_number(np.diag(d)) == pytest.approx(12.0, rel=1e-14)
    q, _ = np.linalg.qr(W.stream(11, "probe").standard_normal((7, 7)))
    assert O.condition_number(q) == pytest.approx(1.0, rel=1e-13)
    assert O.condition_number(np.ones((2, 3))) == math.inf
    assert O.condition_number(np.outer(np.arange(1.0, 6.0), np.arange(1.0, 4.0))) == math.inf
    sup = W.total_degree_support(3, 4)
    sizes, nodes = W.l_grid(12, sup.shape[0], 3, 9, 2, 5)
    A = _stacked_bruteforce(sup, sizes, nodes)
    k = _kappa_eig(A)
    assert 1.0 < k < 1e4
    assert O.condition_number(O.AliasSystem(sup, sizes, nodes).A) == pytest.approx(k, rel=1e-9)


def test_alg2_single_full_grid_stops_at_one():
    """One axis with n = d + 1 extrema points resolves every degree without
    collision: A is the identity, kappa = 1 and Algorithm 2 stops at L = 1."""
    d = 9
    sup = np.arange(d + 1, dtype=np.uint16).reshape(-1, 1)
    sizes = np.array([[d + 1], [3], [4]], dtype=np.int32)
    L, kappa = O.construct_alias_system(sup, sizes, np.ones((3, 1)), kappa0=1.0 + 1e-12)
    assert L == 1 and kappa == pytest.approx(1.0, abs=1e-12)


def test_alg2_single_point_grids_need_N_grids():
    """Grids of one point each contribute one row: below N grids A is
    rank-deficient (kappa = inf), and at generic points exactly N grids give a
    nonsingular square A, so Algorithm 2 with a loose bound returns L = N."""
    D, d = 2, 2
    sup = W.total_degree_support(D, d)
    N = sup.shape[0]
    K = N + 3
    sizes = np.ones((K, D), dtype=np.int32)
    nodes = np.cos(np.pi * W.stream(13, "nodes").random((K, D)))
    L, kappa = O.construct_alias_system(sup, sizes, nodes, kappa0=1e12)
    assert L == N
    # the same matrix from the definition: T_{m1}(x1) T_{m2}(x2) at the N points
    V = np.array([[O.chebyshev_T(int(m[0]), nodes[l, 0]) * O.chebyshev_T(int(m[1]), nodes[l, 1]) for m in sup]
                  for l in range(N)])
    sv = np.linalg.svd(V, compute_uv=False)
    assert kappa == pytest.approx(sv[0] / sv[-1], rel=1e-9)


@pytest.mark.parametrize("kappa0", [4.5, 6.0, 7.3, 1e3])
def test_alg2_returns_the_first_prefix_within_bound(kappa0):
    """Algorithm 2's stopping rule, checked on matrices built from the
    definition: kappa(first L grids) <= kappa0 < kappa(first L-1 grids)."""
    D, d = 3, 4
    sup = W.total_degree_support(D, d)
    sizes, nodes = W.l_grid(14, sup.shape[0], D, 24, 2, d + 1)
    L, kappa = O.construct_alias_system(sup, sizes, nodes, kappa0)
    assert L is not None
    assert _kappa_eig(_stacked_bruteforce(sup, sizes[:L], nodes[:L])) <= kappa0 * (1 + 1e-9)
    if L > 1:
        assert _kappa_eig(_stacked_bruteforce(sup, sizes[:L - 1], nodes[:L - 1])) > kappa0 * (1 - 1e-9)


# ---------------------------------------------------------------- first-kind grid (the paper's own form)
@pytest.mark.parametrize("M", [1, 2, 3, 4, 7, 16, 33])
def test_first_kind_nodes_are_roots_of_T_M(M):
    x = O.first_kind_nodes(M, xi=0.3)
    if M == 1:
        assert x.tolist() == [0.3]
        return
    assert np.allclose(x, np.cos((np.arange(M) + 0.5) * np.pi / M), atol=2e-16)
    assert np.all(x[::-1] == -x)
    assert np.all(np.diff(x) < 0)
    assert np.max(np.abs(npcheb.chebval(x, [0] * M + [1]))) < 1e-13


def test_dct2_closed_forms():
    """From the quadrature b_n = (1/M) sum_k cos(n theta_k) f_k, by hand:
    M=2 (x = +-1/sqrt2): b0 = (f0+f1)/2, b1 = (f0-f1)/(2 sqrt2);
    M=3 (x = sqrt3/2, 0, -sqrt3/2): b0 = (f0+f1+f2)/3, b1 = (f0-f2)/(2 sqrt3),
    b2 = (f0/2 - f1 + f2/2)/3."""
    f2 = np.array([0.7, -1.3])
    assert np.allclose(O.dct2_matrix(2) @ f2, [(f2[0] + f2[1]) / 2, (f2[0] - f2[1]) / (2 * math.sqrt(2))],
                       atol=1e-16)
    f3 = np.array([0.4, 2.0, -0.9])
    want = [f3.sum() / 3, (f3[0] - f3[2]) / (2 * math.sqrt(3)), (f3[0] / 2 - f3[1] + f3[2] / 2) / 3]
    assert np.allclose(O.dct2_matrix(3) @ f3, want, atol=1e-16)
    assert O.dct2_matrix(1).tolist() == [[1.0]]


@pytest.mark.parametrize("M", [2, 5, 8, 31, 100])
def test_dct2_matches_scipy_type2(M):
    f = W.stream(M, "probe").standard_normal(M)
    assert np.allclose(O.dct2_matrix(M) @ f, scipy.fft.dct(f, type=2) / (2 * M), atol=1e-14)


@pytest.mark.parametrize("M", [2, 3, 6, 13])
def test_dct2_of_sampled_T_is_half_unit_vector(M):
    """Below M the quadrature is exact: T_0 -> e_0, T_n -> e_n / 2 (orthogonality)."""
    x = O.first_kind_nodes(M)
    for n in range(M):
        b = O.dct2_matrix(M) @ O.chebyshev_T(n, x)
        e = np.zeros(M)
        e[n] = 1.0 if n == 0 else 0.5
        assert np.allclose(b, e, atol=1e-14)


def test_first_kind_fold_equals_lemma_and_quadrature_exhaustive():
    """Lemma (lem:aliasing): the quadrature of cos(n theta) cos(m theta) over
    the M first-kind points equals Delta(m+n)/2 + Delta(m-n)/2 (computed from
    Eq. (aliasing_delta)); the signed fold gives exactly those entries."""
    for M in range(2, 41):
        th = (np.arange(M) + 0.5) * np.pi / M
        n = np.arange(M)
        m = np.arange(20 * M)
        quad = np.cos(np.outer(n, th)) @ np.cos(np.outer(th, m)) / M          # [M, 20M]
        lem = O.aliasing_entry(n[:, None], m[None, :], M)
        assert np.max(np.abs(quad - lem)) < 1e-12
        row, val = O.fold_first_kind(m, M)
        dense = np.zeros((M, m.size))
        dense[row, m] = val
        assert np.array_equal(dense, lem)


TINY_FIRST = [
    (1, 9, [[4], [7]], [[0.0], [0.0]]),
    (2, 5, [[3, 4], [1, 6], [5, 1]], [[0.0, 0.0], [0.41, 0.0], [0.0, -0.77]]),
    (3, 3, [[2, 3, 2], [4, 1, 3]], [[0.0, 0.0, 0.0], [0.0, 0.25, 0.0]]),
]


@pytest.mark.parametrize("D,d,sizes,nodes", TINY_FIRST)
def test_first_kind_alias_matrix_equals_bruteforce(D, d, sizes, nodes):
    sup = W.total_degree_support(D, d)
    for l in range(len(sizes)):
        bins = O.grid_bins_first_kind(sup, sizes[l])
        w = O.grid_weights_first_kind(sup, sizes[l], nodes[l])
        T = int(np.prod(sizes[l]))
        dense = np.zeros((T, sup.shape[0]))
        dense[bins, np.arange(sup.shape[0])] = w
        brute = O.alias_matrix_grid_first_kind_bruteforce(sup, sizes[l], nodes[l])
        assert np.max(np.abs(dense - brute)) < 1e-13


@pytest.mark.parametrize("seed,D,d,K,lo,hi", [(61, 1, 14, 6, 4, 11), (62, 2, 9, 5, 2, 8), (63, 3, 5, 9, 1, 6),
                                              (64, 4, 4, 12, 1, 5)])
def test_first_kind_exact_recovery(seed, D, d, K, lo, hi):
    w = W.make_workload("fk", seed, D, d, K, lo, hi, W.FAMILY_POLY)
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes, kind="first")
    c = O.fct(w.support, w.sizes, w.nodes, f, "qr", kind="first")
    assert np.linalg.norm(c - w.coeffs_true) <= 1e-12 * np.linalg.norm(w.coeffs_true)


def test_first_kind_full_grid_is_scaled_selection():
    """One grid with M_i >= d + 1 points per axis: no collision; the entry of
    m is prod_i (1 if m_i = 0 else 1/2), and c* = b / entry."""
    D, d = 3, 4
    sup = W.total_degree_support(D, d)
    sizes = np.array([[d + 1, d + 2, d + 1]], dtype=np.int32)
    s = O.AliasSystem(sup, sizes, np.zeros((1, D)), kind="first")
    assert s.R == sup.shape[0]
    want = np.prod(np.where(sup == 0, 1.0, 0.5), axis=1)
    assert np.allclose(np.abs(s.A).sum(axis=0).A1, want, atol=0)
    f = O.sample_lgrid(W.FAMILY_RATIONAL, W.rational_params(3, D), sup, sizes, np.zeros((1, D)), kind="first")
    c = O.solve(s, s.rhs(f), "qr")
    y = O.dct2_grid(f.reshape(tuple(sizes[0])))[tuple(sup.T.astype(np.int64))]
    assert np.max(np.abs(c - y / want)) < 1e-14


# ---------------------------------------------------------------- evaluation of the expansion
def test_evaluate_matches_numpy_chebval_1d_and_2d():
    g = W.stream(71, "probe")
    c1 = g.standard_normal(13)
    x = g.uniform(-1, 1, 50)
    sup1 = np.arange(13, dtype=np.uint16).reshape(-1, 1)
    assert np.allclose(O.evaluate_expansion(c1, sup1, x[:, None]), npcheb.chebval(x, c1), atol=1e-13)
    sup2 = W.total_degree_support(2, 8)
    c2 = g.standard_normal(sup2.shape[0])
    dense = np.zeros((9, 9))
    dense[sup2[:, 0], sup2[:, 1]] = c2
    pts = g.uniform(-1, 1, (40, 2))
    want = npcheb.chebval2d(pts[:, 0], pts[:, 1], dense)
    assert np.allclose(O.evaluate_expansion(c2, sup2, pts), want, atol=1e-13)


def test_evaluate_at_grid_points_equals_recurrence_sampler():
    w = W.make_workload("ev", 72, 3, 5, 2, 2, 5, W.FAMILY_POLY)
    axes = O.grid_axes(w.sizes[0], w.nodes[0])
    pts = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    got = O.evaluate_expansion(w.coeffs_true, w.support, pts)
    want = O.sample_poly_bruteforce(w.coeffs_true, w.support, axes).ravel()
    assert np.allclose(got, want, atol=1e-13)


# ---------------------------------------------------------------- other supports (generators)
@pytest.mark.parametrize("D,d", [(1, 7), (2, 50), (3, 9), (5, 6)])
def test_euclidean_support_is_the_l2_ball(D, d):
    sup = W.euclidean_support(D, d)
    brute = np.array([m for m in itertools.product(range(d + 1), repeat=D) if sum(x * x for x in m) <= d * d],
                     dtype=np.uint16)
    assert np.array_equal(sup, brute)


def test_sparse_infinity_support_properties():
    sup = W.sparse_infinity_support(3, 40, 9, 3000, 3)
    assert sup.shape == (3000, 40) and sup.max() <= 9
    assert len({tuple(r) for r in sup.tolist()}) == 3000
    nz = (sup > 0).sum(axis=1)
    assert nz[0] == 0 and np.all(nz[1:] == 3)
    assert np.array_equal(sup, sup[np.lexsort(sup.T[::-1])])
