"""Mixed path with the stored normal matrix W = A^T A (pipelined CG inner
solve, one team barrier per iteration) against the FP64 oracle, against the
two-phase inner solve, and for determinism across team sizes."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-10

CASES = [
    # name, seed, D, d, K, lo, hi, family
    ("D1_poly", 21, 1, 12, 5, 2, 9, W.FAMILY_POLY),
    ("D2_gc", 41, 2, 9, 5, 3, 12, W.FAMILY_GAUSSCOS),
    ("D3_rat", 42, 3, 6, 9, 1, 7, W.FAMILY_RATIONAL),
    ("D4_gc", 43, 4, 5, 12, 1, 6, W.FAMILY_GAUSSCOS),
    ("D5_rat", 45, 5, 4, 15, 1, 5, W.FAMILY_RATIONAL),
]
MIXED = dict(precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5)


def _w(case):
    name, seed, D, d, K, lo, hi, fam = case
    return W.make_workload(name, seed, D, d, K, lo, hi, fam)


def _solve(w, f, **opts):
    plan = F.Plan(w.support, w.sizes, w.nodes, **opts)
    x = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    c = torch.full((plan.N,), float("nan"), dtype=torch.float64, device="cuda")
    rep = plan.execute(x, c)
    info = plan.info
    plan.close()
    return c.cpu().numpy(), rep, info


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_normal_matrix_pattern_is_that_of_AtA(case):
    w = _w(case)
    A = O.AliasSystem(w.support, w.sizes, w.nodes).A
    pat = (abs(A) > 0).astype(np.int64)
    nnz = (pat.T @ pat).nnz
    plan = F.Plan(w.support, w.sizes, w.nodes, normal_matrix=1, **MIXED)
    assert plan.info["normal_nnz"] == nnz
    plan.close()
    plan = F.Plan(w.support, w.sizes, w.nodes, normal_matrix=-1, **MIXED)
    assert plan.info["normal_nnz"] == 0
    plan.close()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_mixed_with_and_without_normal_matrix_match_oracle(case):
    w = _w(case)
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "qr")
    for nm in (1, -1):
        got, rep, info = _solve(w, f, normal_matrix=nm, **MIXED)
        assert rep["status"] == 0, (nm, rep)
        assert (info["normal_nnz"] > 0) == (nm == 1)
        assert rel(got, ref) <= TOL_MIXED, (nm, rel(got, ref), rep)
        if w.coeffs_true is not None:
            assert rel(got, w.coeffs_true) <= TOL_MIXED


def test_d6_mixed_normal_matrix_matches_oracle():
    w = W.config_d6_gausscos()
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "csne")
    got, rep, info = _solve(w, f, normal_matrix=1, **MIXED)
    assert info["normal_nnz"] > 0
    assert rep["status"] == 0, rep
    assert rel(got, ref) <= TOL_MIXED, (rel(got, ref), rep)


def test_d6_poly_exact_recovery_with_normal_matrix():
    w = W.config_d6_gausscos(family=W.FAMILY_POLY)
    plan = F.Plan(w.support, w.sizes, w.nodes, normal_matrix=1, **MIXED)
    x = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(w.family, w.params, x)
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    rep = plan.execute(x, c)
    plan.close()
    assert rep["status"] == 0
    assert rel(c.cpu().numpy(), w.coeffs_true) <= TOL_MIXED


def test_normal_matrix_batch_bitwise_equals_alone():
    """W's rows are split into units of fixed rows and every reduction has a
    fixed order, so a transform gives the same bits on any team size."""
    ws = [_w(c) for c in CASES[1:]] + [W.config_small_poly()]
    plans, samples, alone = [], [], []
    for w in ws:
        p = F.Plan(w.support, w.sizes, w.nodes, normal_matrix=1, **MIXED)
        s = torch.empty(p.M, dtype=torch.float64, device="cuda")
        p.sample(w.family, w.params, s)
        c = torch.empty(p.N, dtype=torch.float64, device="cuda")
        assert p.execute(s, c)["status"] == 0
        plans.append(p)
        samples.append(s)
        alone.append(c.clone())
    outs = [torch.full((p.N,), float("nan"), dtype=torch.float64, device="cuda") for p in plans]
    for team_blocks in (1, 3, 0):
        reps = F.fct_execute_batch([p.handle for p in plans], samples, outs, team_blocks=team_blocks)
        assert all(r["status"] == 0 for r in reps)
        for a, o in zip(alone, outs):
            assert torch.equal(a, o)
    for p in plans:
        p.close()


@pytest.mark.parametrize("bt", [128, 512])
def test_normal_matrix_block_sizes_agree(bt):
    w = _w(CASES[3])
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "qr")
    got, rep, info = _solve(w, f, normal_matrix=1, block_threads=bt, **MIXED)
    assert rep["status"] == 0 and info["normal_nnz"] > 0
    assert rel(got, ref) <= TOL_MIXED
