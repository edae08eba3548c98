"""Continuous-batching request loop over the C ABI.

A request is one rollout: a scenario, a horizon in steps, and a seed for the
signal actions it receives every ``action_every`` steps (the optimisation
loops of the paper's benchmarks, §4 / App. E: an agent sets signal phases,
steps the simulator and reads metrics).  The server

* keeps one resident slot batch (moss_slots_create) whose slots are sized
  for the request set and the device-memory budget,
* admits waiting requests into free slots that fit them while others run
  (requests that arrive while others run are admitted as soon as a slot
  frees up), so one set of launches per step advances every request in
  flight,
* applies each request's actions between its steps, freezes a request at its
  horizon on the device, reads its metrics and retires its slot, and
* records every step's latency (CUDA events around each chunk of steps) and
  the vehicle updates performed.

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
    def __init__(self, req: Request, slot: int):
        self.req = req
        self.slot = slot
        self.step = 0


class Server:
    """Continuous batching over one resident slot batch (moss_slots_create):
    every in-flight request occupies a slot, and one set of launches per step
    (moss_step on the slot batch, replayed from a CUDA graph) advances all of
    them.  Requests are admitted into free slots that fit them while others
    run; a finished request is frozen at its horizon, its metrics are read,
    and its slot is retired and reused.  All slots share the same action
    points (requests are admitted at chunk boundaries, every chunk is
    ``action_every`` steps), so a chunk is one launch sequence; a request
    whose horizon falls inside a chunk is frozen there by the device.

    The pool of slots is sized from the requests: up to ``max_slots`` slots
    in three size classes (the sizes below the median, below the 85th
    percentile, and up to the largest request, a quarter, a quarter and half
    of the slots), shrunk to fit the device-memory budget."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 32, precision: int = 32,
                 action_every: int = 10, keep_state: bool = False):
        self.budget = int(hbm_budget_bytes)
        self.max_slots = int(max_slots)
        self.precision = precision
        self.action_every = int(action_every)
        self.keep_state = keep_state
        self.updates = 0
        self.peak_slots = 0
        self.peak_bytes = 0

    def pool(self, requests: List[Request]) -> List[Dict[str, int]]:
        """Slot capacities for the request set (see the class docstring)."""
        needs = [binding.slot_caps(r.scenario) for r in requests]
        order = sorted(range(len(needs)), key=lambda i: (needs[i]["n_vehicles"], needs[i]["n_lanes"]))
        n = len(order)
        S = max(1, min(self.max_slots, n))

        def cap_of(idx):
            return {k: max(needs[i][k] for i in idx) for k in needs[0]}

        if S < 3 or n < 3:
            caps = [cap_of(order)] * S
        else:
            b1, b2 = order[: max(1, n // 2)], order[: max(1, (85 * n) // 100)]
            n_small = S // 4
            n_mid = S // 4
            caps = [cap_of(b1)] * n_small + [cap_of(b2)] * n_mid + [cap_of(order)] * (S - n_small - n_mid)
        # fit the budget: drop slots, smallest first, while the pool is too large
        while len(caps) > 1 and sum(estimate_slot_bytes(c, self.precision) for c in caps) > self.budget:
            caps = caps[1:]
        if estimate_slot_bytes(caps[-1], self.precision) > self.budget:
            raise binding.MossError(binding.MOSS_EBUDGET, "the largest request does not fit the budget")
        return caps

    def run(self, requests: List[Request], realtime: bool = True) -> Dict[str, float]:
        """Serve the requests (arrival times relative to the start; with
        realtime=False every request is available at once).  Returns summary
        statistics."""
        import torch
        if not requests:
            return {"requests": 0, "wall_s": 0.0, "vehicle_updates": 0, "vehicle_updates_per_s": 0.0,
                    "p50_step_ms": 0.0, "p99_step_ms": 0.0, "steps": 0, "peak_slots": 0, "peak_bytes": 0}
        caps = self.pool(requests)
        stream = torch.cuda.Stream()
        slots = binding.Slots(caps, requests[0].scenario.params, precision=self.precision,
                              stream=stream.cuda_stream)
        self.peak_bytes = slots.device_bytes()
        free = list(range(len(caps)))
        retiring: Dict[int, int] = {}
        active: List[_Active] = []
        waiting: List = []
        future = sorted(requests, key=lambda r: (r.arrival, r.rid))
        steps_done = 0
        pending = []    # (event start, event end, [(request, steps)])
        finishing = []  # (active request, readback slot) frozen at its horizon
        rb_free = list(range(binding.METRIC_SLOTS))
        largest = caps[-1]
        t0 = time.perf_counter()
        fi = 0
        try:
            while fi < len(future) or waiting or active or finishing:
                now = time.perf_counter() - t0
                while fi < len(future) and (not realtime or future[fi].arrival <= now):
                    r = future[fi]
                    if not binding.fits(largest, binding.slot_caps(r.scenario)):
                        raise binding.MossError(binding.MOSS_EBUDGET, f"request {r.rid} fits no slot")
                    heapq.heappush(waiting, (r.arrival, r.rid, r))
                    fi += 1
                for sl, at in list(retiring.items()):
                    if steps_done > at:
                        free.append(sl)
                        del retiring[sl]
                # admission: the smallest free slot that fits, in arrival order
                while waiting and free:
                    r = waiting[0][2]
                    need = binding.slot_caps(r.scenario)
                    cand = [sl for sl in free if binding.fits(caps[sl], need)]
                    if not cand:
                        break
                    sl = min(cand, key=lambda x: (caps[x]["n_vehicles"], caps[x]["n_lanes"], x))
                    heapq.heappop(waiting)
                    free.remove(sl)
                    slots.load(sl, r.scenario)
                    slots.set_horizon(sl, r.horizon)
                    r.admitted_at = time.perf_counter() - t0
                    active.append(_Active(r, sl))
                self.peak_slots = max(self.peak_slots, len(active))
                # results of the requests frozen in the previous chunk: their
                # metric copies were queued behind it, so reading them waits
                # for that chunk only (the one launched since keeps running)
                for a, rb in finishing:
                    a.req.metrics = slots.metrics_read(rb) if rb is not None else slots.metrics(a.slot)
                    if rb is not None:
                        rb_free.append(rb)
                    if self.keep_state:
                        a.req.state = slots.state(a.slot)
                    a.req.finished_at = time.perf_counter() - t0
                    self.updates += int(a.req.metrics["vehicle_updates"])
                    slots.retire(a.slot)
                    retiring[a.slot] = steps_done
                finishing = []
                if not active:
                    if retiring and waiting:
                        # a step removes the retired slots' vehicles, so the
                        # waiting requests can be loaded
                        slots.step(1)
                        steps_done += 1
                    elif fi < len(future):
                        time.sleep(max(0.0, min(0.01, future[fi].arrival - now)))
                    continue
                # the requests' actions at their (shared) action points, in
                # one call for all of them
                acts = [(a, int(a.req.scenario.net.n_junctions)) for a in active
                        if a.step % self.action_every == 0 and a.req.scenario.net.n_junctions]
                if acts:
                    slots.set_signal_phases(
                        np.concatenate([np.full(nj, a.slot, dtype=np.int32) for a, nj in acts]),
                        np.concatenate([np.arange(nj, dtype=np.int32) for a, nj in acts]),
                        np.concatenate([actions_for(a.req, a.step, nj) for a, nj in acts]))
                k = self.action_every
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                slots.step(k)
                e1.record(stream)
                steps_done += k
                adv = []
                for a in active:
                    d = min(k, a.req.horizon - a.step)
                    adv.append((a.req, d))
                    a.step += d
                pending.append((e0, e1, k, adv))
                # finished requests: frozen at their horizon on the device; their
                # metrics are copied behind this chunk and read after the next
                # one is launched
                for a in [a for a in active if a.step >= a.req.horizon]:
                    rb = rb_free.pop() if rb_free else None
                    if rb is not None:
                        slots.metrics_enqueue(rb, scenario=a.slot)
                    finishing.append((a, rb))
                    active.remove(a)
                # per-step latency of finished chunks (chunk time over its steps)
                keep = []
                for e0_, e1_, k_, adv_ in pending:
                    if e1_.query():
                        ms = e0_.elapsed_time(e1_) / k_
                        for r, d in adv_:
                            r.step_ms.extend([ms] * d)
                    else:
                        keep.append((e0_, e1_, k_, adv_))
                pending = keep
            stream.synchronize()
            for e0_, e1_, k_, adv_ in pending:
                ms = e0_.elapsed_time(e1_) / k_
                for r, d in adv_:
                    r.step_ms.extend([ms] * d)
        finally:
            slots.close()
        wall = time.perf_counter() - t0
        lat = np.concatenate([np.asarray(r.step_ms, dtype=np.float64) for r in requests])
        return {
            "requests": len(requests), "wall_s": wall, "vehicle_updates": self.updates,
            "vehicle_updates_per_s": self.updates / wall if wall > 0 else 0.0,
            "p50_step_ms": float(np.percentile(lat, 50)) if lat.size else 0.0,
            "p99_step_ms": float(np.percentile(lat, 99)) if lat.size else 0.0,
            "steps": int(lat.size), "peak_slots": self.peak_slots, "peak_bytes": self.peak_bytes,
            "slots": len(caps), "slot_steps": steps_done,
        }


def estimate_slot_bytes(caps: Dict[str, int], precision: int = 32) -> int:
    """Device bytes a slot of the given capacities takes in a slot batch."""
    r = 16 if precision == 32 else 32
    real = 4 if precision == 32 else 8
    cand = 96 if precision == 32 else 144
    per_vehicle = 2 * (r + 16) + 1 + 2 * real + r + 16 + 4 + cand + 8 + 4 * 7
    per_lane = 32 + 2 * 4 + 8 + 3 * 4 + 2 * 4 + 8 + 4 + 8
    return (caps["n_vehicles"] * per_vehicle + caps["n_route_entries"] * 4 + (caps["n_lanes"] + 1) * per_lane +
            (caps["n_junctions"] + 1) * 48 + caps["n_phases"] * 8 + 4096)


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
