"""Continuous-batching serving loop over the pool API.

Simulation requests (a hierarchy shape and its physics) arrive over time.  The
server admits them first-come first-served while their device memory fits the
HBM budget, keeps every admitted hierarchy resident on the GPU, advances all of
them together (one pool step = one coarse step of every active run), and retires
a run when its force has converged: |F(t) - F(t - t_cross)| <= tol |F(t)| for the
force along the perturber's motion, checked every coarse step once t >= 2 t_cross,
where t_cross = 2 l_f / (c_s + V) is the crossing time of the finest level (l_f its
half-width); or when the step cap is reached.  Freed slots take the next queued
requests at once, so work that arrives while others run overlaps with them.

``solve_sequential`` is the baseline: the same requests, one at a time, each in its
own FP64 context, with the same stopping rule.
"""
from __future__ import annotations

import bisect
import time
from dataclasses import dataclass, field

import numpy as np

from . import binding


def crossing_time(spec) -> float:
    p = spec["params"]
    half = 0.5 * (spec["hi"][0] - spec["lo"][0]) / 2 ** (spec["n_levels"] - 1)
    return 2.0 * half / (p["cs"] + p["mach"] * p["cs"])


def along_motion(F, spec) -> float:
    d = np.asarray(spec["params"]["flow_dir"], dtype=float)
    return -float(np.dot(F, d / np.linalg.norm(d)))


@dataclass
class Track:
    rid: int
    spec: dict
    arrival: float
    admitted: float
    t_cross: float
    ts: list = field(default_factory=list)
    Fs: list = field(default_factory=list)
    steps: int = 0

    def converged(self, tol) -> bool:
        if not self.ts or self.ts[-1] < 2 * self.t_cross:
            return False
        t, F = self.ts[-1], self.Fs[-1]
        j = bisect.bisect_right(self.ts, t - self.t_cross) - 1
        if j < 0:
            return False
        return abs(F - self.Fs[j]) <= tol * abs(F)


@dataclass
class Result:
    rid: int
    arrival: float
    finish: float
    steps: int
    t: float
    F: np.ndarray
    F_along: float
    capped: bool

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def summarize(results, t_begin, t_end):
    lat = np.array([r.latency for r in results])
    return {
        "requests": len(results),
        "throughput_req_per_s": len(results) / max(t_end - t_begin, 1e-12),
        "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "capped_fraction": float(np.mean([r.capped for r in results])) if results else None,
        "makespan_s": t_end - t_begin,
    }


class Server:
    def __init__(self, budget_bytes, precision=binding.DF_FP32_STATE, tol=1e-3, step_cap=4000,
                 device=0, stream=None, tiles=None):
        self.pool = binding.Pool(budget_bytes, precision=precision, device=device, stream=stream)
        self.tol = tol
        self.step_cap = step_cap
        self.tiles = tiles
        self.max_active = 0

    def close(self):
        self.pool.close()

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep):
        """requests: list of (arrival time in s from the start, spec).  Returns the
        per-request results (in completion order) and the summary."""
        order = sorted(range(len(requests)), key=lambda i: requests[i][0])
        pending = [(requests[i][0], i, requests[i][1]) for i in order]
        queue, active, done = [], {}, []
        t0 = clock()
        nxt = 0
        if self.tiles is not None:
            self.pool.set_tiles(self.tiles)
        while nxt < len(pending) or queue or active:
            now = clock() - t0
            while nxt < len(pending) and pending[nxt][0] <= now:
                queue.append(pending[nxt])
                nxt += 1
            # admit FIFO while the budget allows
            while queue:
                arr, rid, spec = queue[0]
                slot = self.pool.admit(spec["n_levels"], spec["n"], spec["lo"], spec["hi"],
                                       spec["G"], spec["params"])
                if slot is None:
                    if not active:
                        raise RuntimeError(f"request {rid} does not fit the empty pool")
                    break
                queue.pop(0)
                active[slot] = Track(rid, spec, arr, clock() - t0, crossing_time(spec))
            self.max_active = max(self.max_active, len(active))
            if not active:
                if nxt < len(pending):
                    sleep(max(0.0, pending[nxt][0] - (clock() - t0)))
                continue
            self.pool.step(1)
            q = self.pool.query()
            finished = []
            for slot, tr in active.items():
                row = q[slot]
                tr.steps += 1
                tr.ts.append(float(row[3]))
                tr.Fs.append(along_motion(row[:3], tr.spec))
                if row[5] != 0:
                    raise RuntimeError(f"request {tr.rid}: unhealthy state")
                capped = tr.steps >= self.step_cap
                if tr.converged(self.tol) or capped:
                    finished.append((slot, tr, row, capped))
            for slot, tr, row, capped in finished:
                done.append(Result(tr.rid, tr.arrival, clock() - t0, tr.steps, float(row[3]),
                                   np.array(row[:3]), tr.Fs[-1], capped))
                self.pool.release(slot)
                del active[slot]
        t_end = clock() - t0
        return done, summarize(done, 0.0, t_end)


def solve_one(spec, precision, tol, step_cap, device=0, stream=None):
    """One request alone in its own context, with the serving stopping rule."""
    sim = binding.Sim(spec["n_levels"], spec["n"], spec["lo"], spec["hi"], spec["G"],
                      spec["params"], precision=precision, device=device, stream=stream)
    tr = Track(-1, spec, 0.0, 0.0, crossing_time(spec))
    capped = False
    while True:
        sim.step(1)
        F, _ = sim.force()
        t, _, _ = sim.status()
        tr.steps += 1
        tr.ts.append(t)
        tr.Fs.append(along_motion(F, spec))
        if tr.converged(tol):
            break
        if tr.steps >= step_cap:
            capped = True
            break
    sim.close()
    return tr, F, capped


def solve_sequential(requests, precision=binding.DF_FP64, tol=1e-3, step_cap=4000,
                     clock=time.perf_counter, sleep=time.sleep):
    """Single-server FIFO baseline: each request solved alone when it arrives and the
    previous one is done."""
    order = sorted(range(len(requests)), key=lambda i: requests[i][0])
    t0 = clock()
    done = []
    for i in order:
        arr, spec = requests[i]
        wait = arr - (clock() - t0)
        if wait > 0:
            sleep(wait)
        tr, F, capped = solve_one(spec, precision, tol, step_cap)
        done.append(Result(i, arr, clock() - t0, tr.steps, tr.ts[-1], F, tr.Fs[-1], capped))
    t_end = clock() - t0
    return done, summarize(done, 0.0, t_end)
