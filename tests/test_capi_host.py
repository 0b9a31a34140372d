"""CPU-side checks of the C ABI library: it loads, exports every entry point of
include/fct.h, and its host-built alias tables equal the oracle's bit for bit."""
import re
import os

import numpy as np
import pytest

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "fct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fct_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2309_14584_gb300 import build
    build.build()
    return F.lib()


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "fct_execute" in names and "fct_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in F.fct.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_default_options_and_status_strings(lib):
    o = F.fct_default_options()
    assert o.precision == F.FCT_FP64 and o.tol == 1e-13 and o.max_iter == 50000
    assert F.fct.status_string(0) == "FCT_OK"
    assert F.fct.status_string(4) == "FCT_ERR_TIMEOUT"


CASES = [
    ("small", lambda: W.config_small_poly()),
    ("d6", lambda: W.config_d6_gausscos()),
    ("d3", lambda: W.make_workload("t", 11, 3, 6, 6, 1, 7, W.FAMILY_GAUSSCOS)),
    ("d10", lambda: W.config_d10_rational()),
]


@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_alias_tables_bit_exact_vs_oracle(lib, name, mk):
    w = mk()
    b, c, wt, R = F.fct_alias_tables_host(w.support, w.sizes, w.nodes)
    s = O.AliasSystem(w.support, w.sizes, w.nodes)
    assert R == s.R
    off = 0
    for l in range(w.K):
        ob = O.grid_bins(w.support, w.sizes[l])
        assert np.array_equal(b[l], ob)
        assert np.array_equal(c[l], off + np.searchsorted(s.rows[l], ob))
        off += len(s.rows[l])
        ow = O.grid_weights(w.support, w.sizes[l], w.nodes[l])
        assert np.max(np.abs(wt[l] - ow)) <= 1e-13


FIRST_CASES = [
    ("small", lambda: W.config_small_poly()),
    ("d3", lambda: W.make_workload("t", 11, 3, 6, 6, 1, 7, W.FAMILY_GAUSSCOS)),
    ("d6", lambda: W.config_d6_gausscos()),
    ("d1", lambda: W.make_workload("t1", 61, 1, 14, 6, 4, 11, W.FAMILY_POLY)),
]


@pytest.mark.parametrize("name,mk", FIRST_CASES, ids=[c[0] for c in FIRST_CASES])
def test_first_kind_alias_tables_bit_exact_vs_oracle(lib, name, mk):
    """The paper's first-kind grid: signed 1, +-1/2, 0 entries (exact in
    FP64, so compared bitwise where no single-point weight enters)."""
    w = mk()
    b, c, wt, R = F.fct_alias_tables_host(w.support, w.sizes, w.nodes, grid_kind=F.FCT_GRID_FIRST_KIND)
    s = O.AliasSystem(w.support, w.sizes, w.nodes, kind="first")
    assert R == s.R
    off = 0
    for l in range(w.K):
        ob = O.grid_bins_first_kind(w.support, w.sizes[l])
        assert np.array_equal(b[l], ob)
        assert np.array_equal(c[l], off + np.searchsorted(s.rows[l], ob))
        off += len(s.rows[l])
        ow = O.grid_weights_first_kind(w.support, w.sizes[l], w.nodes[l])
        if np.all(w.sizes[l] >= 2):
            assert np.array_equal(wt[l], ow)
        assert np.max(np.abs(wt[l] - ow)) <= 1e-13


def test_unknown_grid_kind_rejected(lib):
    w = W.config_small_poly()
    with pytest.raises(F.FctError):
        F.fct_alias_tables_host(w.support, w.sizes, w.nodes, grid_kind=7)


def test_alias_tables_reject_bad_input(lib):
    sup = np.zeros((3, 2), dtype=np.uint16)
    with pytest.raises(F.FctError):
        F.fct_alias_tables_host(sup, np.array([[0, 2]], dtype=np.int32))
    with pytest.raises(F.FctError):
        F.fct_alias_tables_host(sup, np.array([[1, 2]], dtype=np.int32), np.array([[1.5, 0.0]]))
    with pytest.raises(F.FctError) as e:
        F.fct_alias_tables_host(sup, np.array([[2, 5000]], dtype=np.int32))
    assert "4096" in str(e.value)


def test_plan_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(F.FctError) as e:
        F.Plan(np.zeros((1, 1), dtype=np.uint16), np.array([[2]], dtype=np.int32))
    assert e.value.status in (F.fct.FCT_ERR_NO_DEVICE, F.fct.FCT_ERR_CUDA)
