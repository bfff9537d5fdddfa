"""Continuous-batching serving loop over the pool API.

Simulation requests (a hierarchy shape and its physics) arrive over time.  The
server admits them first-come first-served while their device memory fits the
HBM budget, keeps every admitted hierarchy resident on the GPU, advances all of
them together (one pool step = one coarse step of every active run), and retires
a run when its force has converged: |F(t) - F(t - t_cross)| <= tol |F(t)| for the
force along the perturber's motion, checked at every coarse step once t >= 2 t_cross,
where t_cross = 2 l_f / (c_s + V) is the crossing time of the finest level (l_f its
half-width); or when the step cap is reached.  Freed slots take the next queued
requests at once, so work that arrives while others run overlaps with them.

The host does not wait on every coarse step: it issues a batch of steps, then reads
each run's force history (the device keeps F and t of every step) and applies the
rule step by step.  A batch ends early enough that no run can pass its earliest
possible convergence step by more than `check_every` steps, and that a request
arriving while there is room is admitted within about one batch.

Failures stay with their request: a run whose state goes bad (NaN, rho <= 0 or
e <= 0, found by the device's time-step reduction) is retired with an error result
and its slot freed, and a request that cannot fit even an empty pool is rejected
with an error result; the other requests are unaffected.

``serve_sequential`` is the baseline: the same requests, one at a time on the same
machinery (a server with one slot), in FP64 or FP32 state, with the same stepping and
stopping rule; ``solve_sequential`` does the same with a context per request that
reads the force after every coarse step.
"""
from __future__ import annotations

import bisect
import math
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
    F3: list = field(default_factory=list)
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
    error: str | None = None
    history: list | None = None  # F along the motion after each coarse step

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def summarize(results, t_begin, t_end):
    ok = [r for r in results if r.error is None]
    lat = np.array([r.latency for r in ok])
    return {
        "requests": len(results),
        "failed": len(results) - len(ok),
        "throughput_req_per_s": len(ok) / max(t_end - t_begin, 1e-12),
        "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "capped_fraction": float(np.mean([r.capped for r in ok])) if ok else None,
        "makespan_s": t_end - t_begin,
    }


class Server:
    def __init__(self, budget_bytes, precision=binding.DF_FP32_STATE, tol=1e-3, step_cap=4000,
                 device=0, stream=None, tiles=None, check_every=8, keep_history=False,
                 max_slots=None, transport=binding.TRANSPORT_AUTO):
        """max_slots: at most this many runs at once (1: one request at a time, the
        sequential baseline with the same stepping and stopping machinery);
        transport: the pool's transport kernels (binding.TRANSPORT_*)"""
        self.pool = binding.Pool(budget_bytes, precision=precision, device=device, stream=stream)
        if transport != binding.TRANSPORT_AUTO:
            self.pool.set_transport(transport)
        self.max_slots = max_slots
        self.budget = budget_bytes
        self.precision = precision
        self.tol = tol
        self.step_cap = step_cap
        self.tiles = tiles
        self.check_every = max(1, int(check_every))
        self.keep_history = keep_history
        self.max_active = 0
        self.batches = 0
        self.step_s = None  # running estimate of the wall time of one pool step

    def close(self):
        self.pool.close()

    def _batch(self, active, queue_waiting, next_arrival_in):
        """coarse steps to issue before the next look at the runs"""
        k = 4000  # the device keeps 4096 steps of history per run
        for tr in active.values():
            k = min(k, self.step_cap - tr.steps)
            if tr.ts and tr.ts[-1] < 2 * tr.t_cross and len(tr.ts) >= 2:
                dt = tr.ts[-1] - tr.ts[-2]
                k = min(k, max(self.check_every,
                               math.ceil((2 * tr.t_cross - tr.ts[-1]) / max(dt, 1e-300))))
            else:
                k = min(k, self.check_every)
        full = self.max_slots is not None and len(active) >= self.max_slots
        if queue_waiting and full:
            queue_waiting = False  # nothing can be admitted before a run finishes
            next_arrival_in = None
        elif full:
            next_arrival_in = None
        if queue_waiting or next_arrival_in is not None:
            # come back for requests waiting for room, or about to arrive
            horizon = 0.0 if queue_waiting else next_arrival_in
            if self.step_s:
                k = min(k, max(1, int(horizon / self.step_s) + 1))
            else:
                k = 1
        return max(1, k)

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep, on_admit=None):
        """requests: list of (arrival time in s from the start, spec).  Returns the
        per-request results (in completion order) and the summary.  on_admit(pool,
        slot, rid), if given, is called after each admission (tests use it to plant a
        fault in one run's state)."""
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
            # admit FIFO while the budget (and the slot limit) allows
            while queue and (self.max_slots is None or len(active) < self.max_slots):
                arr, rid, spec = queue[0]
                try:
                    slot = self.pool.admit(spec["n_levels"], spec["n"], spec["lo"], spec["hi"],
                                           spec["G"], spec["params"])
                except binding.DfError as exc:  # a malformed request fails alone
                    queue.pop(0)
                    done.append(self._failed(rid, arr, clock() - t0, str(exc)))
                    continue
                if slot is None:
                    need = binding.run_bytes(spec["n_levels"], spec["n"], spec["G"],
                                             self.precision)
                    if need > self.budget:  # it would never fit: reject it alone
                        queue.pop(0)
                        done.append(self._failed(
                            rid, arr, clock() - t0,
                            f"needs {need} bytes, more than the {self.budget}-byte budget"))
                        continue
                    break
                queue.pop(0)
                active[slot] = Track(rid, spec, arr, clock() - t0, crossing_time(spec))
                if on_admit is not None:
                    on_admit(self.pool, slot, rid)
            self.max_active = max(self.max_active, len(active))
            if not active:
                if nxt < len(pending):
                    sleep(max(0.0, pending[nxt][0] - (clock() - t0)))
                continue
            nai = pending[nxt][0] - (clock() - t0) if nxt < len(pending) else None
            k = self._batch(active, bool(queue), nai)
            tb = clock()
            self.pool.step(k)
            q = self.pool.query()  # waits for the batch; health and time of every slot
            self.batches += 1
            per = (clock() - tb) / k
            self.step_s = per if self.step_s is None else 0.7 * self.step_s + 0.3 * per
            finished = []
            for slot, tr in active.items():
                row = q[slot]
                if row[5] != 0:
                    finished.append((slot, tr, None, "unhealthy state: NaN, rho <= 0 or e <= 0"))
                    continue
                hist = self.pool.history(slot, k)
                for F3 in hist:
                    tr.steps += 1
                    tr.ts.append(float(F3[3]))
                    tr.F3.append(F3[:3].copy())
                    tr.Fs.append(along_motion(F3[:3], tr.spec))
                    if tr.converged(self.tol) or tr.steps >= self.step_cap:
                        finished.append((slot, tr, tr.steps >= self.step_cap
                                         and not tr.converged(self.tol), None))
                        break
            fin_t = clock() - t0
            for slot, tr, capped, err in finished:
                if err is not None:
                    done.append(self._failed(tr.rid, tr.arrival, fin_t, err))
                else:
                    done.append(Result(tr.rid, tr.arrival, fin_t, tr.steps, tr.ts[-1],
                                       np.array(tr.F3[-1]), tr.Fs[-1], bool(capped),
                                       history=list(tr.Fs) if self.keep_history else None))
                self.pool.release(slot)
                del active[slot]
        t_end = clock() - t0
        return done, summarize(done, 0.0, t_end)

    @staticmethod
    def _failed(rid, arrival, finish, msg):
        return Result(rid, arrival, finish, 0, float("nan"), np.full(3, np.nan), float("nan"),
                      False, error=msg)


def solve_one(spec, precision, tol, step_cap, device=0, stream=None):
    """One request alone in its own context, with the serving stopping rule."""
    sim = binding.Sim(spec["n_levels"], spec["n"], spec["lo"], spec["hi"], spec["G"],
                      spec["params"], precision=precision, device=device, stream=stream)
    tr = Track(-1, spec, 0.0, 0.0, crossing_time(spec))
    capped = False
    while True:
        t = sim.step(1, want_t=True)
        F, _ = sim.force()
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


def serve_sequential(requests, budget_bytes, precision=binding.DF_FP64, tol=1e-3,
                     step_cap=4000, keep_history=False, tiles=None,
                     transport=binding.TRANSPORT_AUTO):
    """Sequential baseline on the serving machinery: one request at a time, FIFO, each
    alone on the GPU with the same batched stepping and stopping rule."""
    srv = Server(budget_bytes, precision=precision, tol=tol, step_cap=step_cap,
                 keep_history=keep_history, max_slots=1, tiles=tiles, transport=transport)
    try:
        return srv.run(requests)
    finally:
        srv.close()


def solve_sequential(requests, precision=binding.DF_FP64, tol=1e-3, step_cap=4000,
                     clock=time.perf_counter, sleep=time.sleep, keep_history=False):
    """Single-server FIFO baseline in contexts: each request solved alone when it
    arrives and the previous one is done, reading the force every coarse step."""
    order = sorted(range(len(requests)), key=lambda i: requests[i][0])
    t0 = clock()
    done = []
    for i in order:
        arr, spec = requests[i]
        wait = arr - (clock() - t0)
        if wait > 0:
            sleep(wait)
        tr, F, capped = solve_one(spec, precision, tol, step_cap)
        done.append(Result(i, arr, clock() - t0, tr.steps, tr.ts[-1], F, tr.Fs[-1], capped,
                           history=list(tr.Fs) if keep_history else None))
    t_end = clock() - t0
    return done, summarize(done, 0.0, t_end)
