"""Continuous-batching OTOC server over the batched engine (syk_batch_*).

Requests (one disorder realisation each: N, couplings, beta, time grid,
seeds) arrive over time.  The loop compiles each arriving request's Hamiltonian
(syk_build_terms), admits it into the running batch as soon as a slot and
enough arena memory are free (admission by device footprint), advances all
admitted jobs a few ticks at a time, and retires finished ones — so requests
that arrive while others are on the GPU join them at the next tick instead of
waiting for a batch to drain.  Latency = completion time - arrival time.
All compute runs in libsyk; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from .api import Batch, Terms


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float  # seconds from the start of the run
    N: int
    quads: np.ndarray
    J: np.ndarray
    beta: float
    t_grid: np.ndarray
    seed: int
    state_id: int = 0
    a: int = -1  # Majoranas (default N-1, N-2)
    b: int = -2


@dataclasses.dataclass
class Result:
    rid: int
    N: int
    F: np.ndarray
    otoc: np.ndarray
    arrival: float
    admitted: float
    done: float
    matvecs: int
    status: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def poisson_arrivals(n: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times of n requests of a Poisson process of the given rate (1/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def percentile(values, q: float) -> float:
    v = np.sort(np.asarray(values, dtype=np.float64))
    if len(v) == 0:
        return float("nan")
    k = (len(v) - 1) * q / 100.0
    lo, hi = math.floor(k), math.ceil(k)
    return float(v[lo] + (v[hi] - v[lo]) * (k - lo))


class OtocServer:
    """batch / make_terms can be injected (tests drive the scheduling with fakes)."""

    def __init__(self, dtype: str = "c64", max_slots: int = 256, hbm_budget_bytes: int = 8 << 30, m: int = 30,
                 tol=None, ticks_per_step: int = 4, batch=None, make_terms=None, policy: str = "fifo"):
        self.batch = batch if batch is not None else Batch(dtype=dtype, max_slots=max_slots,
                                                           max_bytes=hbm_budget_bytes, m=m, tol=tol)
        self.make_terms = make_terms if make_terms is not None else (
            lambda r: Terms(r.N, r.quads, r.J, dtype=dtype))
        self.ticks = ticks_per_step
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be 'fifo' or 'sjf'")
        self.policy = policy
        self.live = {}  # rid -> (Request, Terms, admitted time)

    def close(self):
        for _, (_, h, _) in list(self.live.items()):
            h.close()
        self.live.clear()
        self.batch.close()

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep):
        """Serve the requests (arrival times in seconds from now); returns the
        Results in completion order."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue = []  # arrived and compiled, waiting for admission (FIFO without overtaking, or SJF)
        out = []
        t0 = clock()
        now = lambda: clock() - t0
        i = 0
        while i < len(pending) or queue or self.live:
            t = now()
            while i < len(pending) and pending[i].arrival <= t:
                queue.append((pending[i], self.make_terms(pending[i])))
                i += 1
            if self.policy == "sjf":  # shortest estimated work first (stable for equal work)
                queue.sort(key=lambda rh: work_estimate(rh[0], rh[1]))
            while queue:
                r, h = queue[0]
                a = r.a if r.a >= 0 else r.N + r.a
                b = r.b if r.b >= 0 else r.N + r.b
                if not self.batch.submit(h, a, b, r.beta, r.t_grid, r.seed, r.state_id, r.rid):
                    break
                self.live[r.rid] = (r, h, now())
                queue.pop(0)
            if self.live:
                for res in self.batch.run(max_ticks=self.ticks, ticks_per_sync=self.ticks):
                    r, h, adm = self.live.pop(res["tag"])
                    out.append(Result(r.rid, r.N, res["F"], res["otoc"], r.arrival, adm, now(), res["matvecs"],
                                      res["status"]))
                    h.close()
            elif i < len(pending):
                sleep(max(0.0, min(0.01, pending[i].arrival - now())))
        return out


def work_estimate(r: Request, h) -> float:
    """Term x amplitude updates of a request, up to a common factor: its
    matvecs grow like the sum over the grid of |t| (the ket chain evolves
    by t at every point), each costing terms x D."""
    nterms = getattr(h, "n_terms", len(r.J))
    D = getattr(h, "D", 1 << (r.N // 2 - 1))
    t = np.asarray(r.t_grid, dtype=np.float64)
    return float(nterms) * float(D) * float(len(t) + np.sum(np.abs(t)))


def calibrated_rate(capacity_requests, capacity_wall_s: float, served, load: float) -> tuple:
    """Poisson arrival rate that offers `load` (e.g. 0.75) of the server's
    capacity for the requests in `served`.

    The capacity is measured by a closed-loop pass over `capacity_requests`
    (all present at t = 0, finished in capacity_wall_s); it is taken in work
    units per second (work_estimate) and converted to requests per second of
    the served sample through the served sample's own mean work, so that a
    capacity sample lighter or heavier than the served one (a heavy-tailed
    size mix) does not over- or under-load the server.  Returns
    (rate, capacity in requests per second of the served sample)."""
    if capacity_wall_s <= 0 or not capacity_requests or not served:
        raise ValueError("need a positive wall time and non-empty samples")
    cap_work = sum(work_estimate(r, None) for r in capacity_requests) / capacity_wall_s
    mean_work = float(np.mean([work_estimate(r, None) for r in served]))
    cap = cap_work / mean_work
    return load * cap, cap


def summarize(results, wall: float, windows: int = 4, work=None, capacity_work_per_s=None) -> dict:
    """Latency percentiles over all results and, to show whether the load is
    sustained, over `windows` consecutive groups of requests in arrival order
    (a queue that keeps growing shows as latencies rising window by window).
    With work (rid -> work_estimate) and the closed-loop capacity in work units
    per second, each window also reports its offered load: the work that
    arrived in it over its arrival span, as a fraction of the capacity (a
    heavy-tailed mix offers some windows much more than the average)."""
    lat = [r.latency for r in results]
    by_arrival = sorted(results, key=lambda r: r.arrival)
    win = []
    if results and windows > 1:
        parts = np.array_split(np.arange(len(by_arrival)), windows)
        for k, part in enumerate(parts):
            lw = [by_arrival[i].latency for i in part]
            w = {"arrivals_s": [by_arrival[part[0]].arrival, by_arrival[part[-1]].arrival],
                 "p50_latency_s": percentile(lw, 50), "p99_latency_s": percentile(lw, 99)}
            if work is not None and capacity_work_per_s:
                # span from the window's first arrival to the next window's first
                end = by_arrival[parts[k + 1][0]].arrival if k + 1 < len(parts) else by_arrival[part[-1]].arrival
                span = end - by_arrival[part[0]].arrival
                if span > 0:
                    w["offered_load"] = sum(work[by_arrival[i].rid] for i in part) / span / capacity_work_per_s
            win.append(w)
    return {"requests": len(results), "wall_s": wall, "realizations_per_s": len(results) / wall if wall > 0 else None,
            "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
            "mean_latency_s": float(np.mean(lat)) if lat else None,
            "failed": sum(1 for r in results if r.status != 0), "windows": win}
