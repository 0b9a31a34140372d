"""DCT passes on the tensor cores (fct_options.tensor_dct) against the oracle.

Grids with a long axis run Algorithm 3's per-grid DCT as BF16 digit-slice
products on the tensor cores (tcgen05, FP32 accumulation kept exact, FP64
combination).  The right-hand side b = F f must match the oracle's direct
FP64 DCT row by row at the FP64 bar, and whole transforms must match the
oracle's least-squares solution at the parity tolerances.
"""
import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11
TOL_MIXED = 1e-10


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(name):
    """(support, sizes, nodes): explicit grids with long, ragged and
    single-point axes."""
    if name == "D1_n300":
        return W.total_degree_support(1, 280), np.array([[300], [131]], np.int32), np.zeros((2, 1))
    if name == "D2_long":
        sup = W.total_degree_support(2, 120)
        sizes = np.array([[130, 97], [70, 121], [1, 200], [45, 40]], np.int32)
        return sup, sizes, np.cos(np.pi * W.stream(3, "nodes").random((4, 2)))
    if name == "D3_mid":
        sup = W.total_degree_support(3, 30)
        sizes = np.array([[70, 1, 66], [33, 80, 9], [1, 64, 100], [12, 13, 14]], np.int32)
        return sup, sizes, np.cos(np.pi * W.stream(4, "nodes").random((4, 3)))
    if name == "D2_short_forced":
        w = W.config_small_poly()
        return w.support, w.sizes, w.nodes
    raise KeyError(name)


CASES = ["D1_n300", "D2_long", "D3_mid", "D2_short_forced"]


def _rhs(plan, f):
    b = torch.empty(plan.info["R"], dtype=torch.float64, device="cuda")
    bins = F.fct_plan_rhs(plan.handle, torch.from_numpy(f).cuda(), b)
    order = np.argsort(bins, kind="stable")
    return bins[order], b.cpu().numpy()[order]


@pytest.mark.parametrize("kind", ["extrema", "first"])
@pytest.mark.parametrize("name", CASES)
def test_tensor_core_rhs_matches_oracle(name, kind):
    """b from the tensor-core passes equals the oracle's direct DCT row by row
    (bins exactly, values within the FP64 bar), and equals the FP64-unit DCT of
    the same plan shape to a few units of FP64 rounding."""
    sup, sizes, nodes = _case(name)
    gk = F.FCT_GRID_EXTREMA if kind == "extrema" else F.FCT_GRID_FIRST_KIND
    mode = 1 if name.endswith("forced") else 0
    params = W.gausscos_params(11, sup.shape[1])
    f = O.sample_lgrid(W.FAMILY_GAUSSCOS, params, sup, sizes, nodes, kind=kind)
    s = O.AliasSystem(sup, sizes, nodes, kind=kind)
    ref = s.rhs(f)
    tc = F.Plan(sup, sizes, nodes, grid_kind=gk, tensor_dct=mode)
    plain = F.Plan(sup, sizes, nodes, grid_kind=gk, tensor_dct=-1)
    assert tc.info["tensor_dct_grids"] >= 1 and plain.info["tensor_dct_grids"] == 0
    bins, got = _rhs(tc, f)
    bins_p, got_p = _rhs(plain, f)
    tc.close()
    plain.close()
    want_bins = np.concatenate([s.offsets[l] + s.rows[l] for l in range(len(s.rows))])
    assert np.array_equal(bins, want_bins) and np.array_equal(bins_p, want_bins)
    scale = max(1.0, float(np.max(np.abs(f))))
    assert np.max(np.abs(got - ref)) <= 1e-13 * scale, np.max(np.abs(got - ref))
    assert np.max(np.abs(got - got_p)) <= 1e-14 * scale, np.max(np.abs(got - got_p))


def test_tensor_core_grid_selection():
    """Auto mode takes the grids whose longest active axis has 64..1024 points."""
    sup, sizes, nodes = _case("D3_mid")
    p = F.Plan(sup, sizes, nodes)
    assert p.info["tensor_dct_grids"] == 3   # 70, 80 and 100 points; the 14-point grid stays
    assert p.info["tensor_dct_flops"] > 0 and p.info["tensor_dct_flops"] % (36 * 2 * 128 * 64 * 16) == 0
    p.close()
    p = F.Plan(sup, sizes, nodes, tensor_dct=-1)
    assert p.info["tensor_dct_grids"] == 0 and p.info["tensor_dct_flops"] == 0
    p.close()
    p = F.Plan(sup, sizes, nodes, tensor_dct=1)
    assert p.info["tensor_dct_grids"] == 4
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tensor_core_transform_matches_oracle(prec):
    """A whole transform on a D=2 L-grid of Algorithm 1 (degree 90, axes up to
    91 points): Gaussian-cosine samples, both solver paths, against the
    oracle's least-squares solution (semi-normal equations)."""
    D, d = 2, 90
    sup = W.total_degree_support(D, d)
    sizes, nodes = W.l_grid(21, sup.shape[0], D, 6, 1, d + 1)
    params = W.gausscos_params(12, D)
    f = O.sample_lgrid(W.FAMILY_GAUSSCOS, params, sup, sizes, nodes)
    ref = O.fct(sup, sizes, nodes, f, "csne")
    opts = dict(precision=F.FCT_FP64, tol=1e-13) if prec == "fp64" else \
        dict(precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-4)
    plan = F.Plan(sup, sizes, nodes, **opts)
    assert plan.info["tensor_dct_grids"] >= 1
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    rep = plan.execute(torch.from_numpy(f).cuda(), c)
    plan.close()
    assert rep["status"] == 0
    assert _rel(c.cpu().numpy(), ref) <= (TOL_FP64 if prec == "fp64" else TOL_MIXED)


def test_tensor_core_exact_recovery_of_a_polynomial():
    """Samples of a polynomial on the support (device sampler): the transform
    recovers its coefficients; the same with the tensor cores off."""
    D, d = 2, 150
    sup = W.total_degree_support(D, d)
    sizes, nodes = W.l_grid(22, sup.shape[0], D, 6, 1, d + 1)
    c_true = W.poly_coefficients(23, sup)
    out = {}
    for mode in (0, -1):
        plan = F.Plan(sup, sizes, nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-4, tensor_dct=mode)
        x = torch.empty(plan.M, dtype=torch.float64, device="cuda")
        plan.sample(W.FAMILY_POLY | F.fct.FCT_SAMPLE_FOLDED, c_true, x)
        c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
        rep = plan.execute(x, c)
        assert rep["status"] == 0
        out[mode] = c.cpu().numpy()
        if mode == 0:
            assert plan.info["tensor_dct_grids"] >= 1
        plan.close()
    assert _rel(out[0], c_true) <= TOL_MIXED
    assert _rel(out[0], out[-1]) <= TOL_MIXED


def test_tensor_core_nonfinite_sample_is_reported():
    sup, sizes, nodes = _case("D2_long")
    plan = F.Plan(sup, sizes, nodes)
    x = torch.zeros(plan.M, dtype=torch.float64, device="cuda")
    x[int(plan.offsets[1]) + 17] = float("nan")   # a sample of a tensor-core grid
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FctError) as e:
        plan.execute(x, c)
    assert e.value.status == F.fct.FCT_ERR_NONFINITE
    plan.close()
