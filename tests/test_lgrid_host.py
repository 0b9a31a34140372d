"""Host logic of the Algorithm 2 driver (which prefixes it probes and what it
returns), with the device probe replaced by a table of kappa values."""
import math

import numpy as np
import pytest

from paper_2309_14584_gb300 import lgrid


def _run(monkeypatch, kappas, kappa0, start=1, step=1):
    calls = []

    def fake_probe(support, sizes, nodes, iterations=200, seed=0, device="cuda", **kw):
        L = len(sizes)
        calls.append(L)
        return {"kappa": kappas[L - 1]}

    monkeypatch.setattr(lgrid, "probe_condition", fake_probe)
    K = len(kappas)
    r = lgrid.select_grids(np.zeros((1, 1), np.uint16), np.ones((K, 1), np.int32), np.ones((K, 1)), kappa0=kappa0,
                           start=start, step=step)
    return r, calls


def _first_within(kappas, kappa0, start=1):
    for L in range(start, len(kappas) + 1):
        if kappas[L - 1] <= kappa0:
            return L
    return None


SEQ = [math.inf] * 5 + [40.0, 31.0, 20.0, 12.5, 9.0, 8.8, 7.0, 6.5, 5.1, 5.0, 4.2]


@pytest.mark.parametrize("kappa0", [1e4, 30.0, 9.0, 8.9, 5.0, 4.2, 1.0])
@pytest.mark.parametrize("step", [1, 2, 3, 5, 16])
def test_monotone_sequence_gives_algorithm2_answer(monkeypatch, kappa0, step):
    r, calls = _run(monkeypatch, SEQ, kappa0, step=step)
    assert r["L"] == _first_within(SEQ, kappa0)
    assert len(calls) == len(set(calls))           # no prefix probed twice
    if r["L"] is not None:
        assert r["kappa"] == SEQ[r["L"] - 1]
        assert r["L"] in r["probes"]


def test_step_one_is_the_sequential_loop(monkeypatch):
    seq = [math.inf, 50.0, 3.0, 80.0, 2.0]           # not monotone
    r, calls = _run(monkeypatch, seq, 10.0, start=2, step=1)
    assert r["L"] == 3 and calls == [2, 3]


def test_start_beyond_candidates_is_rejected(monkeypatch):
    with pytest.raises(ValueError):
        _run(monkeypatch, SEQ, 10.0, start=len(SEQ) + 1)


def test_serving_candidates_extend_the_default_lgrid():
    import workloads as W
    a = W.serving_shapes(dims=range(2, 9))
    b = W.serving_shapes(dims=range(2, 9), grids_per_dim=10)
    for x, y in zip(a, b):
        assert y.K == 10 * y.D and x.K == 3 * x.D
        assert np.array_equal(x.sizes, y.sizes[:x.K]) and np.array_equal(x.nodes, y.nodes[:x.K])
        z = W.first_grids(y, x.K)
        assert np.array_equal(z.sizes, x.sizes) and z.M == x.M
