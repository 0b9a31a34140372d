"""Serving loop with continuous batching on top of the C ABI.

Requests name a plan shape and a device-resident input.  The engine keeps
device-resident plans (one per shape) and solver slots (clones of the plan,
each with its own workspace) within an HBM budget, and one persistent server
launch (fct_server_*) whose teams take jobs as they are submitted.  A request
is admitted as soon as a slot of its shape is free and its workspace fits the
budget; it then joins the work already on the device.  Latency = completion
time - arrival time on the host clock.

All numerical work happens in libfct_gb300.so; this module only schedules.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import fct as F


class ServingEngine:
    """Admission and scheduling of transform requests onto one serving launch.

    lazy_plans = False: every shape's plan is built up front and, while the
    HBM budget lasts, up to max_slots_per_shape - 1 clones per shape (round
    robin).  lazy_plans = True: a shape's plan is built when its first request
    is admitted (a plan-cache miss, reported as a cold request), while the
    serving launch keeps running; extra slots are cloned on demand.  Either
    way a request is admitted only when a free slot of its shape exists or
    can be cloned, and the device bytes of every plan and slot held stay
    within the budget (live accounting from each plan's fct_plan_info).
    Building plans while the launch runs needs free SMs: pass teams below
    the maximum (the launch then leaves the rest of the device to the plan
    builder's kernels)."""

    def __init__(self, shapes, hbm_budget_bytes: float = 8e9, max_slots_per_shape: int = 4,
                 block_threads: int = 256, team_blocks: int = 16, teams: int = 0, idle_timeout_s: float = 0.05,
                 lazy_plans: bool = False, **plan_options):
        self.shapes = list(shapes)
        self.budget = float(hbm_budget_bytes)
        self.max_slots = int(max_slots_per_shape)
        self.block_threads = block_threads
        self.plan_options = dict(plan_options)
        n = len(self.shapes)
        self.plans = [None] * n   # one base plan per shape (holds the tables)
        self.slots = [[] for _ in range(n)]   # per shape: plan handles (base + clones)
        self.free = [[] for _ in range(n)]    # per shape: free slot indices
        self.slot_bytes = [0.0] * n           # per shape: workspace bytes of one slot
        self.used_bytes = 0.0                 # device bytes of every plan and clone held
        self.in_flight_bytes = 0.0
        self.clones = []
        self.plan_build_s = {}                # shape -> seconds of its (cold) plan build
        if not lazy_plans:
            for s in range(n):
                self._build_plan(s)
            # clones up front, round-robin over shapes while the budget lasts
            grew = True
            while grew:
                grew = False
                for s in range(n):
                    if len(self.slots[s]) < self.max_slots and self.used_bytes + self.slot_bytes[s] <= self.budget:
                        self._clone(s)
                        grew = True
        self.server = F.fct_server_create(block_threads, team_blocks, teams, idle_timeout_s)

    # -- plans and slots ------------------------------------------------------------
    def _build_plan(self, s: int):
        w = self.shapes[s]
        t0 = time.perf_counter()
        p = F.Plan(w.support, w.sizes, w.nodes, block_threads=self.block_threads, **self.plan_options)
        self.plan_build_s[s] = time.perf_counter() - t0
        self.plans[s] = p
        self.slots[s].append(p.handle)
        self.free[s].append(0)
        N, M, R = p.info["N"], p.info["M"], p.info["R"]
        self.slot_bytes[s] = 8.0 * (2 * M + 3 * R + 2 * N) + 4.0 * (R + 3 * N)
        self.used_bytes += float(p.info["device_bytes"])

    def _clone(self, s: int):
        c = self.plans[s].clone()
        self.clones.append(c)
        self.slots[s].append(c.handle)
        self.free[s].append(len(self.slots[s]) - 1)
        self.used_bytes += self.slot_bytes[s]

    def _take_slot(self, s: int):
        if self.plans[s] is None:
            return None
        if not self.free[s] and len(self.slots[s]) < self.max_slots and \
                self.used_bytes + self.slot_bytes[s] <= self.budget:
            self._clone(s)
        if self.in_flight_bytes + self.slot_bytes[s] > self.budget:
            return None
        if not self.free[s]:
            return None
        k = self.free[s].pop()
        self.in_flight_bytes += self.slot_bytes[s]
        return k

    def _give_slot(self, s: int, k: int):
        self.free[s].append(k)
        self.in_flight_bytes -= self.slot_bytes[s]

    # -- serving ---------------------------------------------------------------------
    def run(self, requests, inputs, outputs, timeout_s: float = 600.0):
        """requests: list of (arrival_s, shape, input_key) sorted by arrival;
        inputs[input_key]: device samples; outputs[i]: device coefficient
        buffer of request i.  Returns per-request dicts (latency, report)."""
        n = len(requests)
        pending = collections.deque()
        in_flight = {}
        cold = set()   # requests whose plan was built on admission
        results = [None] * n
        nxt = 0
        done = 0
        t0 = time.perf_counter()
        while done < n:
            now = time.perf_counter() - t0
            if now > timeout_s:
                raise TimeoutError(f"serving run exceeded {timeout_s} s ({done}/{n} done)")
            while nxt < n and requests[nxt][0] <= now:
                pending.append(nxt)
                nxt += 1
            # admission, in arrival order per shape; a shape without a plan gets
            # one now (plan-cache miss) if its tables fit the budget
            blocked = set()
            for _ in range(len(pending)):
                i = pending.popleft()
                s = requests[i][1]
                if self.plans[s] is None and s not in blocked:
                    self._build_plan(s)
                    cold.add(i)
                k = None if s in blocked else self._take_slot(s)
                if k is None:
                    blocked.add(s)
                    pending.append(i)
                    continue
                t = F.fct_server_submit(self.server, self.slots[s][k], inputs[requests[i][2]], outputs[i])
                in_flight[t] = (i, s, k, time.perf_counter() - t0)
            for t in list(in_flight):
                # a device-side error of the serving launch (a bounded wait that
                # expired) comes back as an exception here and ends the run
                rep = F.fct_server_poll(self.server, t)
                if rep is not None:
                    i, s, k, t_sub = in_flight.pop(t)
                    t_done = time.perf_counter() - t0
                    results[i] = {"latency_s": t_done - requests[i][0], "queue_s": t_sub - requests[i][0],
                                  "arrival_s": requests[i][0], "done_s": t_done, "report": rep,
                                  "cold": i in cold}
                    self._give_slot(s, k)
                    done += 1
        return results

    def close(self):
        if getattr(self, "server", None):
            F.fct_server_destroy(self.server)
            self.server = None
        for c in getattr(self, "clones", []):
            c.close()
        for p in getattr(self, "plans", []):
            if p is not None:
                p.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def latency_summary(results, coeffs_per_request) -> dict:
    """p50 / p99 latency and whole-run throughput (coefficients over the span
    from the first arrival to the last completion)."""
    lat = np.array([r["latency_s"] for r in results])
    span = max(r["done_s"] for r in results) - min(r["arrival_s"] for r in results)
    coeffs = int(np.sum(coeffs_per_request))
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "requests": len(results), "coeffs": coeffs,
            "span_s": float(span), "coeffs_per_s": coeffs / span if span > 0 else None,
            "all_converged": all(r["report"]["status"] == 0 for r in results)}
