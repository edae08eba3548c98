"""Continuous-batching request loop over the C ABI.

A request is one rollout: a scenario, a horizon in steps, and a seed for the
signal actions it receives every ``action_every`` steps (the optimisation
loops of the paper's benchmarks, §4 / App. E: an agent sets signal phases,
steps the simulator and reads metrics).  The server

* admits waiting requests while the device-memory budget and the slot count
  allow (requests that arrive while others run are admitted as soon as
  memory and slots free up),
* keeps every admitted rollout's state resident on the device (one handle
  each, on its own CUDA stream, so the steps of different rollouts overlap
  on the GPU),
* applies each request's actions between its steps, and
* records every step's latency (CUDA events around the step on the request's
  stream) and the vehicle updates performed.

All simulation work runs in the CUDA library; this module only orders calls.
"""
from __future__ import annotations

import dataclasses
import heapq
import math
import time
from typing import Dict, List, Optional

import numpy as np

from . import binding
from .scenario import Scenario, Stream


# bytes of device memory a handle allocates (the layout of moss_create)
def estimate_device_bytes(scen: Scenario, precision: int = 32) -> int:
    n = int(scen.veh.n)
    r = 16 if precision == 32 else 32
    real = 4 if precision == 32 else 8
    # two snapshots, code, stayer (s, v), entrant records, entrant links,
    # candidate records and gap heads, per-vehicle tables
    cand = 96 if precision == 32 else 144
    per_vehicle = 2 * (r + 16) + 1 + 2 * real + r + 16 + 4 + cand + 8 + 4 * 7
    per_lane = 32 + 2 * 4 + 8 + 3 * 4 + 2 * 4 + 8
    lanes = int(scen.net.n_lanes)
    return (n * per_vehicle + int(scen.veh.routes.size) * 4 + lanes * per_lane +
            int(scen.net.n_junctions) * 48 + 64 * 1024)


@dataclasses.dataclass
class Request:
    rid: int
    scenario: Scenario
    horizon: int
    arrival: float = 0.0        # seconds after the start of run()
    action_seed: int = 0
    # filled by the server
    admitted_at: Optional[float] = None
    finished_at: Optional[float] = None
    metrics: Optional[Dict[str, float]] = None
    state: Optional[Dict[str, np.ndarray]] = None
    step_ms: List[float] = dataclasses.field(default_factory=list)


def actions_for(req: Request, step: int, n_junctions: int) -> np.ndarray:
    """The phase the request's agent sets on every junction at `step`
    (seeded, reproducible; one draw per junction)."""
    st = Stream(req.action_seed, 600 + step)
    return st.integers(0, 4, n_junctions).astype(np.int32)


class _Active:
    def __init__(self, req: Request, sim: binding.Simulation, stream, bytes_: int, actual: int):
        self.req = req
        self.sim = sim
        self.stream = stream
        self.bytes = bytes_      # admission accounting (the estimate, or more if larger)
        self.actual = actual     # bytes the handle holds
        self.step = 0
        self.pending: List = []  # (start event, end event, steps in between)


class Server:
    def __init__(self, hbm_budget_bytes: int, max_slots: int = 64, precision: int = 32,
                 action_every: int = 10, keep_state: bool = False):
        self.budget = int(hbm_budget_bytes)
        self.max_slots = int(max_slots)
        self.precision = precision
        self.action_every = int(action_every)
        self.keep_state = keep_state
        self.active: List[_Active] = []
        self.bytes_in_use = 0
        self.updates = 0
        self.peak_slots = 0
        self.peak_bytes = 0

    def _can_admit(self, req: Request) -> bool:
        need = estimate_device_bytes(req.scenario, self.precision)
        if need > self.budget:
            raise binding.MossError(binding.MOSS_EBUDGET,
                                    f"request {req.rid} needs {need} B, more than the whole budget")
        return len(self.active) < self.max_slots and self.bytes_in_use + need <= self.budget

    def _admit(self, req: Request, now: float) -> None:
        import torch
        stream = torch.cuda.Stream()
        sc = req.scenario
        sim = binding.Simulation(sc.net, sc.veh, sc.params, precision=self.precision,
                                 stream=stream.cuda_stream)
        actual = sim.device_bytes()
        b = max(actual, estimate_device_bytes(sc, self.precision))
        self.active.append(_Active(req, sim, stream, b, actual))
        self.bytes_in_use += b
        self.actual_in_use = getattr(self, "actual_in_use", 0) + actual
        req.admitted_at = now
        self.peak_slots = max(self.peak_slots, len(self.active))
        self.peak_bytes = max(self.peak_bytes, self.actual_in_use)

    def _launch_step(self, a: _Active) -> None:
        """The request's actions (at an action step) and then its steps up to
        the next action step or its horizon, as one launch on its stream."""
        import torch
        req = a.req
        if a.step % self.action_every == 0:
            nj = int(req.scenario.net.n_junctions)
            if nj:
                a.sim.set_signal_phase(np.arange(nj, dtype=np.int32), actions_for(req, a.step, nj))
        k = min(self.action_every - a.step % self.action_every, req.horizon - a.step)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(a.stream)
        a.sim.step(k)
        e1.record(a.stream)
        a.pending.append((e0, e1, k))
        a.step += k

    def _collect(self, a: _Active, block: bool) -> None:
        """Per-step latency of finished launches: the launch's GPU time over
        its steps (one entry per step)."""
        keep = []
        for e0, e1, k in a.pending:
            if block or e1.query():
                e1.synchronize()
                a.req.step_ms.extend([e0.elapsed_time(e1) / k] * k)
            else:
                keep.append((e0, e1, k))
        a.pending = keep

    def _retire(self, a: _Active, now: float) -> None:
        self._collect(a, block=True)
        m = a.sim.metrics()
        a.req.metrics = m
        if self.keep_state:
            a.req.state = a.sim.state()
        a.req.finished_at = now
        self.updates += int(m["vehicle_updates"])
        a.sim.close()
        self.bytes_in_use -= a.bytes
        self.actual_in_use -= a.actual
        self.active.remove(a)

    def run(self, requests: List[Request], realtime: bool = True) -> Dict[str, float]:
        """Serve the requests (arrival times relative to the start; with
        realtime=False every request is available at once).  Returns summary
        statistics."""
        waiting: List = []
        future = sorted(requests, key=lambda r: (r.arrival, r.rid))
        t0 = time.perf_counter()
        fi = 0
        while fi < len(future) or waiting or self.active:
            now = time.perf_counter() - t0
            while fi < len(future) and (not realtime or future[fi].arrival <= now):
                heapq.heappush(waiting, (future[fi].arrival, future[fi].rid, future[fi]))
                fi += 1
            while waiting and self._can_admit(waiting[0][2]):
                self._admit(heapq.heappop(waiting)[2], now)
            if not self.active:
                if fi < len(future):
                    time.sleep(max(0.0, min(0.01, future[fi].arrival - now)))
                continue
            for a in list(self.active):
                if a.step < a.req.horizon:
                    self._launch_step(a)
            for a in list(self.active):
                self._collect(a, block=False)
                if a.step >= a.req.horizon:
                    a.sim.synchronize()
                    self._retire(a, time.perf_counter() - t0)
        wall = time.perf_counter() - t0
        lat = np.concatenate([np.asarray(r.step_ms, dtype=np.float64) for r in requests]) \
            if requests else np.zeros(0)
        return {
            "requests": len(requests), "wall_s": wall, "vehicle_updates": self.updates,
            "vehicle_updates_per_s": self.updates / wall if wall > 0 else 0.0,
            "p50_step_ms": float(np.percentile(lat, 50)) if lat.size else 0.0,
            "p99_step_ms": float(np.percentile(lat, 99)) if lat.size else 0.0,
            "steps": int(lat.size), "peak_slots": self.peak_slots, "peak_bytes": self.peak_bytes,
        }


def shard(items, rank: int, world: int):
    """The share of `items` (scenarios of a batch, or requests) that process
    `rank` of `world` serves when each GPU has its own process and the items
    are independent (no exchange between the processes): every world-th item,
    starting at `rank`."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    return items[rank::world]


def poisson_requests(n: int, rate_hz: float = 20.0, seed: int = 0, n_lo: int = 5000,
                     n_hi: int = 500_000, h_lo: int = 300, h_hi: int = 3600,
                     make=None) -> List[Request]:
    """n rollout requests: Poisson arrivals at rate_hz, vehicles log-uniform in
    [n_lo, n_hi], grid side from the vehicle count (5..40), horizon uniform in
    [h_lo, h_hi], departures uniform over [0, min(horizon, 1800))."""
    from . import scenario as sc
    st = Stream(seed, 700)
    gaps = -np.log1p(-st.uniform(n)) / rate_hz
    arrivals = np.cumsum(gaps)
    u = st.uniform(n)
    ns = np.round(np.exp(np.log(n_lo) + u * (np.log(n_hi) - np.log(n_lo)))).astype(np.int64)
    horizons = st.integers(h_lo, h_hi + 1, n)
    out = []
    for i in range(n):
        G = int(np.clip(round(5 * 8 ** (math.log(ns[i] / 2000.0) / math.log(150.0))), 5, 40))
        s_i = seed * 100_000 + i + 1
        if make is not None:
            scen = make(i, G, int(ns[i]), int(horizons[i]), s_i)
        else:
            net = sc.grid_network(G, 300.0, 3, vmax_choices=(11.1, 13.89, 16.67), offsets=True, seed=s_i)
            veh = sc.random_demand(net, int(ns[i]), min(int(horizons[i]), 1800), seed=s_i,
                                   dest_pool=256)
            scen = sc.Scenario(net, veh, sc.Params(seed=s_i, scenario=i), f"req{i}_g{G}_{ns[i]}")
        out.append(Request(rid=i, scenario=scen, horizon=int(horizons[i]), arrival=float(arrivals[i]),
                           action_seed=s_i))
    return out
