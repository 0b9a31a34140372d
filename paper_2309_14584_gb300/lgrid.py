"""Algorithm 2 (Sec. 3.3) on the device: how many grids of a candidate L-grid
to use.  Grids are appended in candidate order (each one an Algorithm 1 draw,
supplied by the caller) until the stacked alias matrix A has
kappa(A) <= kappa0.

kappa(A) comes from fct_plan_condition: a Lanczos estimate from the
coefficients of CG on A^T A started at a random vector, computed in
libfct_gb300.so.  This module only chooses which prefix to probe next.

With step = 1 the probes follow Algorithm 2 exactly (every prefix from
`start` on, the first one within the bound wins).  A larger step probes every
step-th prefix and then bisects between the last failing and the first
passing one, which returns the same L whenever kappa decreases with L (rows
appended to A can only raise sigma_min).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import fct as F


def probe_condition(support, sizes, nodes, iterations: int = 200, seed: int = 0, device="cuda",
                    **plan_options) -> dict:
    """kappa estimate of the alias matrix of one L-grid (sizes[K, D], nodes[K, D])."""
    p = F.Plan(support, sizes, nodes, **plan_options)
    try:
        N, R = p.N, p.info["R"]
        if R < N:
            return {"kappa": math.inf, "iterations": 0, "N": N, "R": R}
        g = torch.Generator(device=device)
        g.manual_seed(int(seed))
        start = torch.randn(N, dtype=torch.float64, device=device, generator=g)
        work = torch.empty_like(start)
        r = F.fct_plan_condition(p.handle, start, work, max(2, min(int(iterations), N + 1)))
        r.update(N=N, R=R)
        return r
    finally:
        p.close()


def select_grids(support, cand_sizes, cand_nodes, kappa0: float = 1e4, start: int = 1, step: int = 1,
                 probe_iterations: int = 200, seed: int = 0, device="cuda", **plan_options) -> dict:
    """Returns {"L": grids to use (None if no prefix meets the bound),
    "kappa": its estimate, "probes": {L: kappa} of every prefix probed}."""
    cand_sizes = np.asarray(cand_sizes, dtype=np.int32)
    cand_nodes = np.asarray(cand_nodes, dtype=np.float64)
    K_max = cand_sizes.shape[0]
    if not 1 <= start <= K_max or step < 1:
        raise ValueError("need 1 <= start <= number of candidates and step >= 1")
    probes: dict[int, float] = {}

    def kappa_of(L: int) -> float:
        if L not in probes:
            probes[L] = probe_condition(support, cand_sizes[:L], cand_nodes[:L], probe_iterations, seed, device,
                                        **plan_options)["kappa"]
        return probes[L]

    fail, L = start - 1, start
    while L <= K_max and kappa_of(L) > kappa0:
        fail, L = L, L + step
    if L > K_max:
        if fail < K_max and kappa_of(K_max) <= kappa0:
            L = K_max
        else:
            return {"L": None, "kappa": probes.get(K_max, probes[fail]), "probes": probes}
    while L - fail > 1:  # bisect (L passes, fail fails or is below start)
        mid = (fail + L) // 2
        if mid < start:
            break
        if kappa_of(mid) <= kappa0:
            L = mid
        else:
            fail = mid
    return {"L": L, "kappa": probes[L], "probes": probes}
