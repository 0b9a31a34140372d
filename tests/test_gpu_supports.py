"""Supports other than total degree on the device: the Euclidean set S^2
and random sparse subsets of S^inf (the paper's second and third function
classes), against the oracle and by exact recovery of polynomials."""
import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _solve(sup, sizes, nodes, f, **opts):
    plan = F.Plan(sup, sizes, nodes, **opts)
    c = torch.full((plan.N,), float("nan"), dtype=torch.float64, device="cuda")
    rep = plan.execute(torch.from_numpy(f).cuda(), c)
    plan.close()
    return c.cpu().numpy(), rep


# name, support, D, d, grids per dimension (the Euclidean sets need 6D grids
# for full rank at these seeds; 3D leaves them rank-deficient)
SUPPORTS = [
    ("S2_D3_d9", lambda: W.euclidean_support(3, 9), 3, 9, 6),
    ("S2_D5_d5", lambda: W.euclidean_support(5, 5), 5, 5, 6),
    ("Sinf_D10_d3", lambda: W.sparse_infinity_support(11, 10, 3, 1500, 3), 10, 3, 3),
    ("Sinf_D30_d9", lambda: W.sparse_infinity_support(12, 30, 9, 2000, 3), 30, 9, 3),
]


@pytest.mark.parametrize("name,mk,D,d,kpd", SUPPORTS, ids=[s[0] for s in SUPPORTS])
def test_other_supports_match_oracle(name, mk, D, d, kpd):
    sup = mk()
    N = sup.shape[0]
    sizes, nodes = W.l_grid(100 + D, N, D, kpd * D, 1, d + 1)
    params = W.gausscos_params(5, D)
    f = O.sample_lgrid(W.FAMILY_GAUSSCOS, params, sup, sizes, nodes)
    ref = O.fct(sup, sizes, nodes, f, "csne")
    for opts, tol in ((dict(precision=F.FCT_FP64, tol=1e-14), 1e-11),
                      (dict(precision=F.FCT_MIXED, tol=1e-13, inner_tol=1e-5), 1e-10)):
        got, rep = _solve(sup, sizes, nodes, f, **opts)
        assert rep["status"] == 0, rep
        assert rel(got, ref) <= tol, (rel(got, ref), rep)


@pytest.mark.parametrize("name,mk,D,d,kpd", SUPPORTS, ids=[s[0] for s in SUPPORTS])
def test_other_supports_exact_recovery(name, mk, D, d, kpd):
    sup = mk()
    sizes, nodes = W.l_grid(200 + D, sup.shape[0], D, kpd * D, 1, d + 1)
    c_true = W.poly_coefficients(9, sup)
    plan = F.Plan(sup, sizes, nodes, precision=F.FCT_MIXED, tol=1e-13, inner_tol=1e-5)
    x = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(W.FAMILY_POLY, c_true, x)
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    rep = plan.execute(x, c)
    plan.close()
    assert rep["status"] == 0
    assert rel(c.cpu().numpy(), c_true) <= 1e-10


@pytest.mark.slow
def test_sparse_support_D100_large_exact_recovery():
    """The paper's sparse-support setting at D = 100: 2 x 10^4 random multi-indices
    of degree <= 9 (3 nonzero components each), 1000 grids by Algorithm 1
    (10 D: with so few nonzero components most columns share bin 0 of a grid,
    and 3 D grids leave kappa(A) ~ 165, measured with fct_plan_condition);
    a polynomial on that support is recovered by the mixed path."""
    D, d, N = 100, 9, 20_000
    sup = W.sparse_infinity_support(13, D, d, N, 3)
    sizes, nodes = W.l_grid(300, N, D, 10 * D, 1, d + 1)
    c_true = W.poly_coefficients(10, sup)
    plan = F.Plan(sup, sizes, nodes, precision=F.FCT_MIXED, tol=1e-13, inner_tol=1e-5)
    x = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(W.FAMILY_POLY | F.fct.FCT_SAMPLE_FOLDED, c_true, x)
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    rep = plan.execute(x, c)
    plan.close()
    assert rep["status"] == 0, rep
    assert rel(c.cpu().numpy(), c_true) <= 1e-10


@pytest.mark.slow
def test_sparse_support_D100_N1e6_exact_recovery():
    """The paper's sparse-support scale: 10^6 random multi-indices at D = 100
    (10 nonzero components of degree <= 3 each), 600 grids by Algorithm 1
    (K N = 6e8 table entries, M = 1.2e9 samples); a polynomial on that support
    is recovered by the mixed path (the check that holds at any size)."""
    D, d, N, K = 100, 3, 1_000_000, 600
    sup = W.sparse_support_vectorised(3, D, d, N, 10)
    sizes, nodes = W.l_grid(500, N, D, K, 1, d + 1)
    c_true = W.poly_coefficients(10, sup)
    plan = F.Plan(sup, sizes, nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-4, block_threads=512)
    assert plan.info["nnz"] == K * N
    x = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(W.FAMILY_POLY | F.fct.FCT_SAMPLE_FOLDED, c_true, x)
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    rep = plan.execute(x, c)
    plan.close()
    assert rep["status"] == 0, rep
    assert rel(c.cpu().numpy(), c_true) <= 1e-10


@pytest.mark.parametrize("bt", [128, 256, 512])
def test_wide_rows_match_oracle_and_batch(bt):
    """Sparse supports put most columns in bin 0 of a grid: rows of more than
    16 x 32 x (entries per lane) entries are gathered by every warp of a block
    (the warps' partial sums added in a fixed order); 2 entries per lane put
    this plan's ~1.5k-entry rows above that.  The plan must hold such rows,
    the FP64 and mixed solves match the oracle, and a batch on small teams
    gives the coefficients of the transform alone bit for bit."""
    sup = W.sparse_infinity_support(12, 30, 9, 2000, 3)
    N, D = sup.shape
    sizes, nodes = W.l_grid(130, N, D, 3 * D, 1, 10)
    params = W.gausscos_params(5, D)
    f = O.sample_lgrid(W.FAMILY_GAUSSCOS, params, sup, sizes, nodes)
    ref = O.fct(sup, sizes, nodes, f, "csne")
    x = torch.from_numpy(f).cuda()
    for opts, tol in ((dict(precision=F.FCT_FP64, tol=1e-14), 1e-11),
                      (dict(precision=F.FCT_MIXED, tol=1e-13, inner_tol=1e-5), 1e-10)):
        plan = F.Plan(sup, sizes, nodes, block_threads=bt, entries_per_lane=2, **opts)
        lens = np.diff(F.fct_plan_tables(plan.handle)["rowptr"])
        assert lens.max() > 16 * 32 * 2 and plan.info["wide_rows"] > 0
        c = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        rep = plan.execute(x, c)
        assert rep["status"] == 0, rep
        got = c.cpu().numpy()
        assert rel(got, ref) <= tol, (rel(got, ref), rep)
        clones = [plan.clone() for _ in range(3)]   # own workspace each
        outs = [torch.full((N,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
        reps = F.fct_execute_batch([p.handle for p in clones], [x] * 3, outs, team_blocks=4)
        assert all(r["status"] == 0 for r in reps)
        for o in outs:
            assert torch.equal(o, c)
        for p in clones:
            p.close()
        plan.close()
