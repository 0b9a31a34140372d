"""Plant plausible mistakes in the oracle (CPU only) and check that at least
one pin in test_oracle_pins fails for each.  A pin set that let one of these
through would not pin the oracle."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import fct_oracle as O
from tests import test_oracle_pins as P


def _fold_off_by_one(m, n):
    m = np.asarray(m, dtype=np.int64)
    period = 2 * (n - 1)
    r = m % period
    return np.where(r <= n - 1, r, period - r - 1)


def _dct_no_output_weight(n):
    j = np.arange(n)
    jk = np.outer(j, j) % (2 * (n - 1))
    e = np.ones(n)
    e[0] = e[-1] = 0.5
    return (2.0 / (n - 1)) * e[None, :] * np.cos(np.pi * jk / (n - 1))


_orig_dct = O.dct1_matrix
_orig_T = O.chebyshev_T
_orig_nodes = O.extrema_nodes
_orig_weights = O.grid_weights
_orig_bins = O.grid_bins


def _dct_wrong_period(n):
    j = np.arange(n)
    e = np.ones(n)
    e[0] = e[-1] = 0.5
    return (2.0 * e[:, None] / (n - 1)) * e[None, :] * np.cos(np.pi * np.outer(j, j) / n)


def _weights_dropped(support, sizes_l, nodes_l):
    return np.ones(support.shape[0])


def _bins_colmajor(support, sizes_l):
    D = len(sizes_l)
    strides = np.ones(D, dtype=np.int64)
    for i in range(1, D):
        strides[i] = strides[i - 1] * int(sizes_l[i - 1])
    sup = support.astype(np.int64)
    bins = np.zeros(sup.shape[0], dtype=np.int64)
    for i in range(D):
        n = int(sizes_l[i])
        if n >= 2:
            bins += O.fold(sup[:, i], n) * strides[i]
    return bins


def _nodes_mirrored(n, xi=1.0):
    return -_orig_nodes(n, xi)


def _T_table_bad(nmax, x):
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    t = np.empty((x.size, nmax + 1))
    t[:, 0] = 1.0
    if nmax >= 1:
        t[:, 1] = x
    for n in range(1, nmax):
        t[:, n + 1] = x * t[:, n] - t[:, n - 1]
    return t


def _cgls_wrong_sign(A, b, tol=1e-15, maxit=100000):
    x = np.zeros(A.shape[1]); r = b.copy(); s = A.T @ r; p = s.copy()
    gamma = float(s @ s); g0 = gamma
    for it in range(1, 2000):
        q = A @ p; alpha = gamma / float(q @ q)
        x += alpha * p; r += alpha * q
        s = A.T @ r; gn = float(s @ s)
        if gn <= tol * tol * g0:
            break
        p = s + (gn / gamma) * p; gamma = gn
    return x, it, 0.0


_orig_cond = O.condition_number
_orig_construct = O.construct_alias_system


def _cond_squared(A):
    k = _orig_cond(A)
    return k * k


def _construct_one_late(support, cand_sizes, cand_nodes, kappa0=1e4):
    # tests the bound only after appending the next grid
    L, _ = _orig_construct(support, cand_sizes, cand_nodes, kappa0)
    if L is None or L >= len(cand_sizes):
        return L, math.inf
    return L + 1, _orig_cond(O.AliasSystem(support, cand_sizes[:L + 1], cand_nodes[:L + 1]).A)


_orig_fold1 = O.fold_first_kind


def _fold1_unsigned(m, M):
    row, val = _orig_fold1(m, M)
    return row, np.abs(val)


def _fold1_full_weight(m, M):
    row, val = _orig_fold1(m, M)
    return row, np.sign(val)


def _fold1_no_zero_column(m, M):
    row, val = _orig_fold1(m, M)
    r = np.asarray(m, dtype=np.int64) % (2 * M)
    return np.where(r == M, M - 1, row), np.where(r == M, 0.5, val)


_orig_eval = O.evaluate_expansion


def _eval_axes_swapped(coeffs, support, points):
    return _orig_eval(coeffs, support, np.atleast_2d(points)[:, ::-1])


_orig_sample_grid = O.sample_grid


def _sampler_variant(cos_arg_squared=False, drop_a=False, drop_c=False, rational_unsquared=False):
    def sample_grid(family, params, support, axes):
        D = len(axes)
        shape = tuple(a.size for a in axes)
        bc = O._broadcast_axis
        if family in (W.FAMILY_GAUSSCOS, W.FAMILY_POLY_GAUSSCOS):
            a, b = params[:D], params[D:2 * D]
            quad = sum((1.0 if drop_a else a[i]) * bc(axes[i] ** 2, i, D) for i in range(D))
            lin = sum(b[i] * bc(axes[i] ** 2 if cos_arg_squared else axes[i], i, D) for i in range(D))
            return np.broadcast_to(np.exp(-quad) * np.cos(lin), shape).copy()
        if family == W.FAMILY_RATIONAL:
            c = params[:D]
            quad = sum((1.0 if drop_c else c[i]) * bc(axes[i] if rational_unsquared else axes[i] ** 2, i, D)
                       for i in range(D))
            return np.broadcast_to(1.0 / (1.0 + quad), shape).copy()
        return _orig_sample_grid(family, params, support, axes)
    return sample_grid


def _rank_from_normal_eigenvalues(A, rtol=1e-10):
    A = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    ev = np.linalg.eigvalsh(A.T @ A)
    return int((ev > ev[-1] * rtol * rtol).sum())


def _rank_rtol_unsquared(A, rtol=1e-10):
    A = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    sv = np.linalg.svd(A, compute_uv=False)
    return int((sv * sv > sv[0] * sv[0] * rtol).sum()) if sv.size and sv[0] > 0 else 0


def _golden_sampler_pins():
    for fam in ("gausscos", "rational", "runge"):
        P.test_sampler_families_match_hand_values(fam)


MUTATIONS = [
    ("gausscos_cos_of_squares", "sample_grid", _sampler_variant(cos_arg_squared=True), _golden_sampler_pins),
    ("gausscos_a_dropped", "sample_grid", _sampler_variant(drop_a=True), _golden_sampler_pins),
    ("rational_c_dropped", "sample_grid", _sampler_variant(drop_c=True), _golden_sampler_pins),
    ("rational_unsquared", "sample_grid", _sampler_variant(rational_unsquared=True), _golden_sampler_pins),
    ("rank_from_normal_eigenvalues", "numerical_rank", _rank_from_normal_eigenvalues,
     lambda: P.test_numerical_rank_of_constructed_matrices()),
    ("rank_rtol_unsquared", "numerical_rank", _rank_rtol_unsquared,
     lambda: P.test_numerical_rank_of_constructed_matrices()),
    ("fold_off_by_one", "fold", _fold_off_by_one, lambda: P.test_fold_identity_exhaustive()),
    ("fold_off_by_one_recovery", "fold", _fold_off_by_one,
     lambda: P.test_exact_recovery_of_polynomials_in_support(*P.RECOVERY[1])),
    ("dct_no_output_weight", "dct1_matrix", _dct_no_output_weight,
     lambda: [P.test_dct1_closed_forms(*r) for r in P._golden_dct()]),
    ("dct_wrong_period", "dct1_matrix", _dct_wrong_period, lambda: P.test_dct1_maps_sampled_Tk_to_unit_vector(9)),
    ("weights_dropped", "grid_weights", _weights_dropped,
     lambda: P.test_exact_recovery_of_polynomials_in_support(*P.RECOVERY[2])),
    ("bins_colmajor", "grid_bins", _bins_colmajor, lambda: P.test_alias_matrix_fold_equals_bruteforce(*P.TINY[1])),
    ("nodes_mirrored", "extrema_nodes", _nodes_mirrored, lambda: P.test_extrema_nodes(5)),
    ("T_recurrence_bad", "chebyshev_T_table", _T_table_bad,
     lambda: P.test_chebyshev_definition_recurrence_and_library_agree()),
    ("cgls_wrong_sign", "cgls", _cgls_wrong_sign, lambda: P.test_solver_tiers_agree_and_are_optimal()),
    ("condition_squared", "condition_number", _cond_squared, lambda: P.test_condition_number_closed_forms()),
    ("alg2_one_late", "construct_alias_system", _construct_one_late,
     lambda: P.test_alg2_returns_the_first_prefix_within_bound(6.0)),
    ("fold1_unsigned", "fold_first_kind", _fold1_unsigned,
     lambda: P.test_first_kind_alias_matrix_equals_bruteforce(*P.TINY_FIRST[1])),
    ("fold1_full_weight", "fold_first_kind", _fold1_full_weight,
     lambda: P.test_first_kind_exact_recovery(62, 2, 9, 5, 2, 8)),
    ("fold1_no_zero_column", "fold_first_kind", _fold1_no_zero_column,
     lambda: P.test_first_kind_fold_equals_lemma_and_quadrature_exhaustive()),
    ("eval_axes_swapped", "evaluate_expansion", _eval_axes_swapped,
     lambda: P.test_evaluate_matches_numpy_chebval_1d_and_2d()),
]


@pytest.mark.parametrize("name,attr,bad,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, attr, bad, pin, monkeypatch):
    monkeypatch.setattr(O, attr, bad)
    with pytest.raises((AssertionError, O.RankDeficient, np.linalg.LinAlgError, ZeroDivisionError, ValueError)):
        pin()
