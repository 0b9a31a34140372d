"""Alias tables built on the device (fct_options.plan_build): bit-identical
to the host builder for every table, consistent with the oracle's bins and
entries (Sec. 3.3, Eq. (aliasing_matrix_nd_diff)), and the transform through
them bit-identical to the transform through host-built tables."""
import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O

pytestmark = pytest.mark.gpu

HOST, DEVICE = F.FCT_PLAN_BUILD_HOST, F.FCT_PLAN_BUILD_DEVICE


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def _wl(w):
    return w.support, w.sizes, w.nodes


def _sparse(seed, D, d, N, kpd):
    sup = W.sparse_infinity_support(seed, D, d, N, 3)
    sizes, nodes = W.l_grid(300 + D, N, D, kpd * D, 1, d + 1)
    return sup, sizes, nodes


def _sparse10(N, K):
    """D = 100, 10 nonzero components of degree <= 3: rows of every length from
    1 to thousands of entries (32-lane rows of several load rounds)."""
    sup = W.sparse_support_vectorised(3, 100, 3, N, 10)
    sizes, nodes = W.l_grid(500, N, 100, K, 1, 4)
    return sup, sizes, nodes


# name, (support, sizes, nodes) maker, plan options.  Sizes span one radix
# tile (K N < 4096) to K N = 6e6 (several hundred tiles, three 8-bit passes),
# single-point axes, both grid kinds, the three block sizes (different entries
# per lane) and a sparse support whose bin 0 rows hold thousands of entries.
CASES = [
    ("small", lambda: _wl(W.config_small_poly()), {}),
    ("d1", lambda: _wl(W.make_workload("t1", 21, 1, 12, 5, 2, 9, W.FAMILY_POLY)), {}),
    ("d4_single_point", lambda: _wl(W.make_workload("t4", 43, 4, 5, 12, 1, 6, W.FAMILY_GAUSSCOS)), {}),
    ("d6", lambda: _wl(W.config_d6_gausscos()), {}),
    ("d6_first_kind", lambda: _wl(W.config_d6_gausscos()), {"grid_kind": F.FCT_GRID_FIRST_KIND}),
    ("d6_bt128", lambda: _wl(W.config_d6_gausscos()), {"block_threads": 128}),
    ("d6_bt512_epl2", lambda: _wl(W.config_d6_gausscos()), {"block_threads": 512, "entries_per_lane": 2}),
    ("d10", lambda: _wl(W.config_d10_rational()), {}),
    ("sinf_d30", lambda: _sparse(12, 30, 9, 2000, 3), {}),
    ("sinf_d100", lambda: _sparse(13, 100, 6, 20000, 3), {}),
    ("sinf_d100_nz10", lambda: _sparse10(20000, 60), {}),
    ("sinf_d100_nz10_rounds", lambda: _sparse10(40000, 220), {}),
]


@pytest.mark.parametrize("name,mk,opts", CASES, ids=[c[0] for c in CASES])
def test_device_tables_equal_host_tables(name, mk, opts):
    sup, sizes, nodes = mk()
    ph = F.Plan(sup, sizes, nodes, plan_build=HOST, **opts)
    pd = F.Plan(sup, sizes, nodes, plan_build=DEVICE, **opts)
    try:
        th, td = F.fct_plan_tables(ph.handle), F.fct_plan_tables(pd.handle)
        for k in ("rowptr", "col", "crow", "bins"):
            assert np.array_equal(th[k], td[k]), k
        for k in ("wcsr", "wcm"):
            assert np.array_equal(_bits(th[k]), _bits(td[k])), k
        for k in ("R", "M", "grid_blocks", "coef_lanes", "device_bytes", "normal_nnz"):
            assert ph.info[k] == pd.info[k], k
    finally:
        ph.close()
        pd.close()


ORACLE_CASES = [
    ("small", lambda: _wl(W.config_small_poly()), F.FCT_GRID_EXTREMA),
    ("d4_single_point", lambda: _wl(W.make_workload("t4", 43, 4, 5, 12, 1, 6, W.FAMILY_GAUSSCOS)),
     F.FCT_GRID_EXTREMA),
    ("d6", lambda: _wl(W.config_d6_gausscos()), F.FCT_GRID_EXTREMA),
    ("d6_first_kind", lambda: _wl(W.config_d6_gausscos()), F.FCT_GRID_FIRST_KIND),
    ("sinf_d30", lambda: _sparse(12, 30, 9, 2000, 3), F.FCT_GRID_EXTREMA),
]


@pytest.mark.parametrize("name,mk,kind", ORACLE_CASES, ids=[c[0] for c in ORACLE_CASES])
def test_device_tables_match_oracle(name, mk, kind):
    """Every column's entry on every grid sits in the oracle's bin with the
    oracle's value, and the CSR is the transpose of the coefficient-major
    table with columns ascending in each row."""
    sup, sizes, nodes = mk()
    first = kind == F.FCT_GRID_FIRST_KIND
    p = F.Plan(sup, sizes, nodes, plan_build=DEVICE, grid_kind=kind)
    try:
        t = F.fct_plan_tables(p.handle)
        off = p.offsets
    finally:
        p.close()
    K, N = sizes.shape[0], sup.shape[0]
    rows_of_grid = np.searchsorted(off, t["bins"], side="right") - 1
    for l in range(K):
        ob = (O.grid_bins_first_kind if first else O.grid_bins)(sup, sizes[l])
        ow = (O.grid_weights_first_kind if first else O.grid_weights)(sup, sizes[l], nodes[l])
        r = t["crow"][l]
        assert np.all(rows_of_grid[r] == l)
        assert np.array_equal(t["bins"][r] - off[l], ob)
        if np.all(sizes[l] >= 2):
            assert np.array_equal(t["wcm"][l], ow)
        assert np.max(np.abs(t["wcm"][l] - ow)) <= 1e-13
    # CSR = transpose of the coefficient-major table, m ascending inside a row
    rp, col, wcsr = t["rowptr"], t["col"], t["wcsr"]
    assert rp[0] == 0 and rp[-1] == K * N and np.all(np.diff(rp) >= 1)
    row_of_entry = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    grid_of_entry = rows_of_grid[row_of_entry]
    assert np.array_equal(t["crow"][grid_of_entry, col], row_of_entry)
    assert np.array_equal(_bits(t["wcm"][grid_of_entry, col]), _bits(wcsr))
    inner = np.ones(len(col), dtype=bool)
    inner[rp[:-1]] = False
    assert np.all(np.diff(col)[inner[1:]] > 0)


def _solve(w, samples, **opts):
    plan = F.Plan(w.support, w.sizes, w.nodes, **opts)
    c = torch.full((plan.N,), float("nan"), dtype=torch.float64, device="cuda")
    rep = plan.execute(samples, c)
    torch.cuda.synchronize()
    plan.close()
    return c.cpu().numpy(), rep


@pytest.mark.parametrize("precision,tol", [(F.FCT_FP64, 1e-11), (F.FCT_MIXED, 1e-10)], ids=["fp64", "mixed"])
@pytest.mark.parametrize("mk", [W.config_small_poly, W.config_d6_gausscos], ids=["small", "d6"])
def test_transform_through_device_tables_is_bit_identical(mk, precision, tol):
    """Same samples, same launch: the coefficients are bit-identical whichever
    builder made the tables, and match the oracle.  The small plan also stores
    W = A^T A on the mixed path (built on the host from the downloaded
    device tables)."""
    w = mk()
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    x = torch.from_numpy(f).cuda()
    opts = dict(precision=precision, tol=1e-13 if precision == F.FCT_MIXED else 1e-14, inner_tol=1e-5)
    ch, rh = _solve(w, x, plan_build=HOST, **opts)
    cd, rd = _solve(w, x, plan_build=DEVICE, **opts)
    assert rh["status"] == 0 and rd["status"] == 0
    assert rh["iterations"] == rd["iterations"]
    assert np.array_equal(_bits(ch), _bits(cd))
    ref = O.fct(w.support, w.sizes, w.nodes, f, "csne")
    assert np.linalg.norm(cd - ref) / np.linalg.norm(ref) <= tol


def test_default_build_is_on_the_device_and_bad_value_is_rejected():
    assert F.fct_default_options().plan_build == F.FCT_PLAN_BUILD_AUTO
    w = W.config_small_poly()
    with pytest.raises(F.FctError):
        F.Plan(w.support, w.sizes, w.nodes, plan_build=3)


def _lanes_for(length, epl):
    lanes = 1
    while lanes < 32 and lanes * epl < length:
        lanes *= 2
    return 64 if length > 16 * 32 * epl else lanes


@pytest.mark.parametrize("epl", [2, 8])
def test_solver_row_order_of_a_large_plan(epl):
    """K N = 8.8e6 table entries (at least 2^23): rows in solver order have
    non-increasing gather lanes (wide rows first); inside the 32-lane class
    and among wide rows, non-increasing load rounds ceil(len / (32 epl)); rows
    with equal lanes and rounds keep ascending bin order."""
    sup, sizes, nodes = _sparse10(40000, 220)
    assert sizes.shape[0] * sup.shape[0] >= 1 << 23
    p = F.Plan(sup, sizes, nodes, entries_per_lane=epl)
    try:
        t = F.fct_plan_tables(p.handle)
        assert p.info["entries_per_lane"] == epl
    finally:
        p.close()
    lens = np.diff(t["rowptr"])
    lanes = np.array([_lanes_for(int(n), epl) for n in lens])
    rounds = -(-lens // (32 * epl))
    assert np.all(np.diff(lanes) <= 0)
    assert (lanes == 32).sum() > 1000 and len(np.unique(rounds[lanes == 32])) >= 5
    same = lanes[1:] == lanes[:-1]
    long_rows = same & (lanes[1:] >= 32)
    assert np.all(np.diff(rounds)[long_rows] <= 0)
    tie = same & ((lanes[1:] < 32) | (rounds[1:] == rounds[:-1]))
    assert np.all(np.diff(t["bins"])[tie] > 0)


def test_solver_row_order_of_a_small_plan():
    """Below 2^23 table entries the rows keep ascending bin order inside each
    lane class, whatever their load rounds."""
    sup, sizes, nodes = _sparse10(20000, 60)
    p = F.Plan(sup, sizes, nodes, entries_per_lane=2)
    try:
        t = F.fct_plan_tables(p.handle)
    finally:
        p.close()
    lens = np.diff(t["rowptr"])
    lanes = np.array([_lanes_for(int(n), 2) for n in lens])
    assert np.all(np.diff(lanes) <= 0)
    rounds = -(-lens // 64)
    assert len(np.unique(rounds[lanes == 32])) >= 5
    same = lanes[1:] == lanes[:-1]
    assert np.all(np.diff(t["bins"])[same] > 0)
