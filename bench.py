#!/usr/bin/env python
"""Benchmark of the per-timestep vehicle update on GB300.

Workload: the city-scale synthetic scenario (perturbed 100x100 grid, 39,600
roads, 2,464,950 trips departing uniformly over 3,600 s).  Set-up (untimed)
simulates the first 3,600 steps on the GPU, so the timed steps start from the
state the simulation itself reaches once every trip has departed (about two
million vehicles on the network); inputs are resident in HBM before timing.
A step is one pass of the whole hot path (signals, insertion, sensing, IDM,
MOBIL with conflict resolution, integration, transfer, arrival, snapshot
rebuild) over all active vehicles.

Metric: vehicle-updates/s = sum over timed steps of the active vehicles
updated / summed device time of those steps (CUDA events on the simulation
stream; L2 flushed by a 256 MiB write between timed steps, outside the
events).  ``--impl reference`` times the FP64 CPU oracle instead, on a
bounded slice of a synthetic state of the same workload at the same step.

Multi-GPU: replicas only (one independent city per rank, no collective on
the data path); value = all ranks' vehicle updates / max over ranks of the
timed duration.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

T_WARM = 3600   # the timed steps start at this step
SPEC_BYTES = {  # algorithmic bytes per unit with FP32 state (32 B snapshot record per vehicle)
    "decide": 41.0,    # per active vehicle: read its 32 B record, write code + s' + v' (9 B)
    "lanescan": 16.0,  # per lane: read its offset + leave + enter, write its next offset
    "place": 73.0,     # per active vehicle: read code, s', v' and the 32 B record, write 32 B
}
STEP_BYTES = 64.0      # whole step: read and write one 8x4 B state record per vehicle update


PROFILES = os.path.join(ROOT, "profiles")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2406_10661_gb300", "csrc", f)
                  for f in ("moss_device.cuh", "moss_kernels.cuh")]


def kernel_source_hash() -> str:
    """SHA-256 of the kernel sources without their comments and blank space
    (an edit of a comment does not invalidate a capture; any code change does)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def captured_traffic(kernel: str, workload: str = "city100x100_2464950"):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the
    committed ncu summary of that workload, if the capture was taken from the
    current kernel sources (the summary records their SHA-256); else None."""
    try:
        with open(os.path.join(PROFILES, f"step_kernels_{workload}.md")) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 4 and parts[0] == "traffic:" and parts[1] == kernel:
                    if parts[3] == "sha256:" + kernel_source_hash():
                        return float(parts[2])
    except OSError:
        pass
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.path = tempfile.mktemp(prefix="clk", suffix=".csv")
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0])); mx.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[3:7]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def city(args):
    from paper_2406_10661_gb300 import scenario as sc
    return sc.city_scenario(seed=args.seed, lane_groups=args.lane_groups)


def cpu_oracle_rate(scen, state, budget_s=15.0, max_road=4000, steps_cap=60, max_pressure=False,
                    t_state=T_WARM):
    """The FP64 oracle, as it stands, on the roads with id < max_road of the
    given state (a contiguous band of the grid at the same density) at step
    t_state."""
    import oracle
    from paper_2406_10661_gb300 import scenario as sc
    veh, sample = sc.region_band(state, scen.net, scen.veh, 0, max_road)
    o = oracle.Oracle(scen.net, veh, scen.params)
    o.set_state(sample["status"], sample["lane"], sample["s"], sample["v"], sample["rc"], t_state)
    if max_pressure:
        o.set_signal(list(range(scen.net.n_junctions)), oracle.POLICY_MAX_PRESSURE)
    o.step(1)  # untimed warm-up
    m0 = o.metrics()
    t0 = time.perf_counter()
    n = 0
    while n < steps_cap and (time.perf_counter() - t0) < budget_s:
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    m1 = o.metrics()
    upd = m1["vehicle_updates"] - m0["vehicle_updates"]
    return {"value": upd / dt, "unit": "vehicle-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle, {n} steps from the GPU's step-{t_state} state restricted to roads "
                      f"0..{max_road - 1} ({int((sample['status'] == 1).sum())} active vehicles), "
                      f"single thread, {dt:.1f} s"}


class OracleBands:
    """The FP64 oracle, as it stands, on n host cores at once: road ids
    [0, road_hi) are cut into n contiguous bands, each band's vehicles of the
    given state are stepped by their own oracle instance in their own thread
    (the oracle is C behind ctypes, which releases the GIL during a step),
    and the threads step in lockstep: one step() advances every band by one
    step and returns its wall time (the slowest band's)."""

    def __init__(self, scen, state, t_state, n=None, road_hi=None, max_pressure=False):
        import threading
        import oracle
        from paper_2406_10661_gb300 import scenario as sc
        self.n = n or os.cpu_count() or 1
        hi = scen.net.n_roads if road_hi is None else min(road_hi, scen.net.n_roads)
        bounds = np.linspace(0, hi, self.n + 1).astype(np.int64)
        self.orcs = []
        for k in range(self.n):
            veh, smp = sc.region_band(state, scen.net, scen.veh, int(bounds[k]), int(bounds[k + 1]))
            o = oracle.Oracle(scen.net, veh, scen.params)
            o.set_state(smp["status"], smp["lane"], smp["s"], smp["v"], smp["rc"], t_state)
            if max_pressure:
                o.set_signal(list(range(scen.net.n_junctions)), oracle.POLICY_MAX_PRESSURE)
            self.orcs.append(o)
        self._go = threading.Barrier(self.n + 1)
        self._done = threading.Barrier(self.n + 1)
        self._stop = False
        self._error = None
        self._threads = [threading.Thread(target=self._work, args=(k,), daemon=True) for k in range(self.n)]
        for t in self._threads:
            t.start()

    def _work(self, k):
        import threading
        try:
            while True:
                self._go.wait()
                if self._stop:
                    return
                self.orcs[k].step(1)
                self._done.wait()
        except threading.BrokenBarrierError:
            return
        except Exception as e:  # an oracle error ends the run instead of stalling it
            self._error = e
            self._go.abort()
            self._done.abort()

    def step(self) -> float:
        import threading
        t0 = time.perf_counter()
        try:
            self._go.wait()
            self._done.wait()
        except threading.BrokenBarrierError:
            raise RuntimeError(f"oracle band failed: {self._error!r}")
        return time.perf_counter() - t0

    def updates(self) -> float:
        return sum(o.metrics()["vehicle_updates"] for o in self.orcs)

    def active(self) -> int:
        return int(sum(o.metrics()["n_active"] for o in self.orcs))

    def close(self):
        import threading
        self._stop = True
        try:
            self._go.wait()
        except threading.BrokenBarrierError:
            pass
        for t in self._threads:
            t.join()


def cpu_oracle_all_cores(scen, state, budget_s=15.0, t_state=T_WARM, max_pressure=False, threads=None,
                         steps_cap=200):
    """The oracle on every host core (OracleBands over the whole state),
    stepped for max(2 s, budget_s / cores) of wall time: about budget_s of
    CPU work in all.  value = all updates / wall time."""
    pool = OracleBands(scen, state, t_state, n=threads, max_pressure=max_pressure)
    try:
        pool.step()  # untimed warm-up
        per_s = max(2.0, budget_s / pool.n)
        u0 = pool.updates()
        wall, steps = 0.0, 0
        while steps < steps_cap and wall < per_s:
            wall += pool.step()
            steps += 1
        upd = pool.updates() - u0
    finally:
        pool.close()
    n = pool.n
    return {"value": upd / wall, "unit": "vehicle-updates/s", "cores": n, "kind": "oracle",
            "sample": f"FP64 oracle on all {n} host cores: the GPU's step-{t_state} state cut into {n} "
                      f"bands of road ids, one oracle instance and thread per band, stepped together; "
                      f"{steps} steps of the whole network ({upd / max(steps, 1):.0f} vehicles per step) "
                      f"in {wall:.1f} s",
            "per_core": upd / wall / n}


def reduce_ranks(dist, dev_s: float, updates: float, device=None):
    """Replicas: the job's time is the slowest rank's, its work the sum of all
    ranks' vehicle updates.  Returns (max seconds, summed updates)."""
    import torch
    t = torch.tensor([dev_s], dtype=torch.float64, device=device)
    u = torch.tensor([updates], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    scen = city(args)
    from paper_2406_10661_gb300 import scenario as sc
    # a synthetic state of the same workload at the same step (built from the
    # inputs only; the reference arm runs none of the CUDA path), stepped by
    # the oracle on every host core (one band of road ids per core)
    warm = sc.warm_state(scen.net, scen.veh, T_WARM, spacing=9.0, seed=args.seed)
    pool = OracleBands(scen, warm, T_WARM, road_hi=args.ref_roads)
    try:
        for _ in range(args.warmup):
            pool.step()
        u0 = pool.updates()
        dt = sum(pool.step() for _ in range(args.steps))
        upd = pool.updates() - u0
        act = pool.active()
    finally:
        pool.close()
    value = upd / dt
    roads = scen.net.n_roads if args.ref_roads is None else min(args.ref_roads, scen.net.n_roads)
    line = {
        "impl": "reference", "metric": "vehicle-updates/s", "value": value, "unit": "vehicle-updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": scen.name, "roads": int(scen.net.n_roads), "vehicles": int(scen.veh.n),
                   "start": f"synthetic state at step {T_WARM} (9 m spacing)", "sample_roads": roads},
        "cpu_baseline": {"value": value, "unit": "vehicle-updates/s", "cores": pool.n, "kind": "oracle",
                         "sample": f"each step: the FP64 oracle over roads 0..{roads - 1} of a synthetic "
                                   f"step-{T_WARM} state on {pool.n} host cores (one band of road ids and "
                                   f"one oracle instance per core; {act} active vehicles after the run)"},
        "e2e": {"value": value, "unit": "vehicle-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_2406_10661_gb300 import binding

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    binding.load()
    saturated = None
    if args.workload == "saturated":
        # every trip on the road at once (the kernels at full occupancy)
        from paper_2406_10661_gb300 import scenario as sc
        scen, saturated = sc.saturated_city(seed=args.seed)
        t_start = 0
        start_desc = ("all trips on the road at step 0, evenly spaced in proportion to lane length "
                      "(set_state; set-up, untimed)")
    elif args.workload == "medium":
        # the 30x30 grid (100,000 trips) from its own step-1800 state: a small
        # case of the same kernels (for detailed profiles)
        from paper_2406_10661_gb300 import scenario as sc
        scen = sc.medium_scenario(seed=args.seed)
        t_start = 1800
        start_desc = "the simulation's own state at step 1800 (set-up, untimed)"
    else:
        scen = city(args)
        t_start = T_WARM
        start_desc = f"the simulation's own state at step {T_WARM} (set-up, untimed)"
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=32, stream=stream.cuda_stream)
        mp = args.policy == "max_pressure"
        if mp:  # every junction under the adaptive max-pressure policy from step 0
            sim.set_signal_policy(np.arange(scen.net.n_junctions, dtype=np.int32), binding.POLICY_MAX_PRESSURE)
        if saturated is not None:
            sim.set_state(*saturated, 0)
        else:
            sim.step(t_start)  # set-up: the simulation reaches its own state at the start step
        state0 = sim.state() if world == 1 else None
        for _ in range(args.warmup):
            sim.step(1)
        sim.synchronize()
        m0 = sim.metrics()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            w0 = time.perf_counter()
            for k in range(args.steps):
                flush.add_(1.0)           # > L2: evicts the previous step's lines
                evs[k][0].record(stream)
                sim.step(1)
                evs[k][1].record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - w0
        if dist:
            dist.barrier()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        m1 = sim.metrics()
        upd = m1["vehicle_updates"] - m0["vehicle_updates"]
        dev_s = sum(step_ms) / 1e3
        if dist:
            dev_s_all, upd_all = reduce_ranks(dist, dev_s, float(upd), device="cuda")
        else:
            dev_s_all, upd_all = dev_s, float(upd)
        value = upd_all / dev_s_all
        ms_per_step = 1e3 * dev_s_all / args.steps

        # per-kernel durations (events around each kernel, same L2 flushing)
        ksteps = max(3, min(args.steps, 20))
        m2 = sim.metrics()
        sim.set_kernel_timing(True)
        for _ in range(ksteps):
            flush.add_(1.0)
            sim.step(1)
        sim.synchronize()
        kt, kn = sim.kernel_times()
        m3 = sim.metrics()
        sim.set_kernel_timing(False)
        upd_k = (m3["vehicle_updates"] - m2["vehicle_updates"]) / max(kn, 1)
        mob_k = (m3["mobil_evals"] - m2["mobil_evals"]) / max(kn, 1)
        avg_ms = {k: v / max(kn, 1) for k, v in kt.items()}
        dom = max((k for k in avg_ms if k in SPEC_BYTES), key=avg_ms.get)
        n_lanes = int(scen.net.n_lanes)
        units = {"decide": upd_k, "lanescan": n_lanes, "place": upd_k}
        peak, peak_kind = _peaks()
        achieved = SPEC_BYTES[dom] * units[dom] / (avg_ms[dom] * 1e-3) / 1e9
        step_ms_k = sum(avg_ms.values())
        step_ach = STEP_BYTES * upd_k / (step_ms_k * 1e-3) / 1e9

        # end to end through the public API: every step the host writes the
        # signal actions of all junctions (pinned host arrays -> device), steps,
        # and reads the metrics back (device -> host); under max pressure the
        # junctions decide themselves and the host only steps and reads
        # (the fixed-time schedule of actions is laid out in pinned host
        # memory before the timed region; each step's row is copied inside it)
        J = int(scen.net.n_junctions)
        jids = torch.arange(J, dtype=torch.int32).pin_memory().numpy()
        offs = scen.net.junc_offset.astype(np.int64)
        e2e_steps = args.steps
        t_first = t_start + args.warmup + args.steps + ksteps
        phases = torch.empty((2 * e2e_steps, J), dtype=torch.int32).pin_memory().numpy()
        phases[:] = ((t_first + np.arange(2 * e2e_steps)[:, None] + offs[None, :]) % 132) // 33
        # pipelined loop (the headline): step k+1's actions and launch are
        # enqueued before step k's metrics are read (moss_metrics_enqueue /
        # moss_metrics_read), so the host work of a step overlaps the previous
        # step on the GPU; every step's actions go in and its metrics come out
        me0 = sim.metrics()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            if not mp:
                sim.set_signal_phase(jids, phases[k])
            sim.step(1)
            sim.metrics_enqueue(k % 2)
            if k > 0:
                mk = sim.metrics_read((k - 1) % 2)
        mk = sim.metrics_read((e2e_steps - 1) % 2)
        e2e_s = time.perf_counter() - t0
        e2e_upd = mk["vehicle_updates"] - me0["vehicle_updates"]
        # the same loop with a synchronous read after every step
        ms0 = sim.metrics()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            if not mp:
                sim.set_signal_phase(jids, phases[e2e_steps + k])
            sim.step(1)
            msk = sim.metrics()
        e2e_sync = (msk["vehicle_updates"] - ms0["vehicle_updates"]) / (time.perf_counter() - t0)
        # the lane / road metric calls of the public API on the same state
        # (kernel + device-to-host copy of the per-lane / per-road arrays)
        metric_ms = {}
        for name, call in (("lane_queue", sim.lane_queue), ("road_speed", sim.road_speed)):
            call()
            t1 = time.perf_counter()
            for _ in range(5):
                call()
            metric_ms[name] = (time.perf_counter() - t1) / 5 * 1e3
        e2e_val = e2e_upd / e2e_s
        if dist:
            e2e_s_all, e2e_upd_all = reduce_ranks(dist, e2e_s, float(e2e_upd), device="cuda")
            e2e_val = e2e_upd_all / e2e_s_all

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    wname = scen.name + ("_maxpressure" if args.policy == "max_pressure" else "")
    cpu = None
    if world == 1:
        # the oracle on all host cores (bands of the same state), and on one
        cpu = cpu_oracle_all_cores(scen, state0, budget_s=args.cpu_budget, t_state=t_start,
                                   max_pressure=args.policy == "max_pressure")
        cpu["single_thread"] = cpu_oracle_rate(scen, state0, budget_s=args.cpu_budget,
                                               max_pressure=args.policy == "max_pressure",
                                               t_state=t_start)
    n_total = int(scen.veh.n)
    line = {
        "metric": "vehicle-updates/s", "value": value, "unit": "vehicle-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wname, "roads": int(scen.net.n_roads), "lanes": n_lanes,
                   "vehicles": n_total, "dt_s": 1.0,
                   "start": start_desc,
                   "active_per_step": upd / args.steps,
                   "l2": "flushed between timed steps by a 256 MiB write (outside the events)",
                   "signal_policy": args.policy, "lane_groups": bool(args.lane_groups),
                   "parallelism": f"replicas x{world}"},
        "step_hz": 1e3 / ms_per_step,
        "nominal_vehicle_steps_per_s": n_total * 1e3 / ms_per_step,
        "paper_context": {"step_hz": 84.09, "vehicles": 2464950, "hardware": "RTX 4090 + Xeon 8462Y",
                          "note": "different network (CBLab Roadnet-L); context only"},
        "roofline": {"bound": "hbm", "kernel": f"k_{dom}", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": captured_traffic(f"k_{dom}", wname),
                     "peak_source": peak_kind,
                     "bytes_per_unit": SPEC_BYTES[dom], "units_per_launch": units[dom],
                     "avg_launch_ms": avg_ms[dom]},
        "kernel_ms": avg_ms,
        "step_roofline": {"achieved": step_ach, "frac": step_ach / peak, "bytes_per_update": STEP_BYTES},
        "clocks": clk.summary(),
        "e2e": {"value": e2e_val, "unit": "vehicle-updates/s", "h2d_bytes_per_step": 0 if mp else 8 * J,
                "d2h_bytes_per_step": 12 * 8 + 8 + 4,  # metric fields, step counter, error word
                "steps": e2e_steps,
                "api": ("" if mp else "moss_set_signal_phase + ") + "moss_step(1) + moss_metrics_enqueue per "
                       "step, step k's metrics read (moss_metrics_read) after step k+1 is enqueued",
                "sync_value": e2e_sync,
                "sync_api": ("" if mp else "moss_set_signal_phase + ") + "moss_step(1) + moss_get_metrics "
                            "(waits for the step) per step"},
        "gpu_launches": sim.step_launches() * args.steps,
        "metric_calls_ms": metric_ms,
        "wall_s_timed_region": wall,
        "cpu_baseline": cpu,
    }
    if world == 1 and args.workload == "city" and not args.city_only:
        # the batched (64 uneven scenarios) and served (Poisson rollout
        # requests) parts of the metric, each with its own clock record
        b = run_batched(args, emit=False)
        line["batched"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "step_hz", "p50_step_ms",
                                              "p99_step_ms", "batched_over_sequential", "clocks", "config",
                                              "sequential", "latency_how", "single_launch") if k in b}
        sv = run_serving(args, emit=False)
        line["served"] = {k: sv[k] for k in ("value", "unit", "p50_step_ms", "p99_step_ms", "wall_s", "config",
                                             "clocks", "all_at_once", "sequential", "all_at_once_over_sequential",
                                             "results_equal_alone_and_mixed", "peak_slots", "how")}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batched(args, emit=True):
    """64 uneven scenarios advanced together (one set of launches per step,
    replayed from a CUDA graph, autotuned schedule) against stepping the same
    scenarios one at a time; both from the step-900 state the simulation
    reaches, K timed steps each.  Under torchrun every rank takes every
    world-th scenario (no exchange between ranks); the job's rate is the
    summed updates over the slowest rank's time.  Returns the line (printed
    when emit)."""
    import torch
    from paper_2406_10661_gb300 import binding, scenario as sc, serving
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        if emit:
            dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    binding.load()
    t0 = time.perf_counter()
    mine = serving.shard(list(range(args.scenarios)), rank, world)
    scens = sc.batched_scenarios(args.scenarios, seed=args.seed, only=mine)
    gen_s = time.perf_counter() - t0
    pre = 900
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch = binding.Batch(scens, precision=32, stream=stream.cuda_stream)
        batch.step(pre)
        tuned = batch.autotune(1)
        batch.step(args.warmup)
        batch.synchronize()
        t_timed = int(batch.metrics(0)["step"])  # the step the timed steps start from
        u0 = sum(batch.metrics(i)["vehicle_updates"] for i in range(len(scens)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            e0.record(stream)
            batch.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
        b_ms = e0.elapsed_time(e1)
        u1 = sum(batch.metrics(i)["vehicle_updates"] for i in range(len(scens)))
        # per-step latency of the batch: K further steps, events around each
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for a, b in evs:
            a.record(stream)
            batch.step(1)
            b.record(stream)
        torch.cuda.synchronize()
        lat = np.array([a.elapsed_time(b) for a, b in evs])
        # the same steps as one cooperative launch each (moss_set_step_mode 1)
        batch.set_step_mode(1)
        batch.step(args.warmup)
        u2 = sum(batch.metrics(i)["vehicle_updates"] for i in range(len(scens)))
        e0.record(stream)
        batch.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        one_ms = e0.elapsed_time(e1)
        one_upd = sum(batch.metrics(i)["vehicle_updates"] for i in range(len(scens))) - u2
        batch.set_step_mode(0)
        batch.close()
        b_s, b_upd = b_ms / 1e3, float(u1 - u0)
        if dist:
            b_s, b_upd = reduce_ranks(dist, b_s, b_upd, device="cuda")
        seq_ms, seq_upd = 0.0, 0
        if world == 1:
            for s_ in scens:
                sim = binding.Simulation(s_.net, s_.veh, s_.params, precision=32, stream=stream.cuda_stream)
                sim.step(t_timed)  # the same state as the batch's timed steps start from
                sim.synchronize()
                m0 = sim.metrics()["vehicle_updates"]
                e0.record(stream)
                sim.step(args.steps)
                e1.record(stream)
                torch.cuda.synchronize()
                seq_ms += e0.elapsed_time(e1)
                seq_upd += sim.metrics()["vehicle_updates"] - m0
                sim.close()
    if dist and emit:
        dist.destroy_process_group()
    if rank != 0:
        return None
    b_val = b_upd / b_s
    line = {"metric": "vehicle-updates/s (batched)", "value": b_val, "unit": "vehicle-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * b_s / args.steps,
            "higher_is_better": True, "scaling": "strong", "dtype": "f32",
            "data": "synthetic",
            "step_hz": args.steps / b_s,
            "p50_step_ms": float(np.percentile(lat, 50)), "p99_step_ms": float(np.percentile(lat, 99)),
            "latency_how": f"{args.steps} further steps of the whole batch, CUDA events around each",
            "single_launch": {"value": one_upd / (one_ms / 1e3), "ms_per_step": one_ms / args.steps,
                              "how": "the same batch, each step one cooperative launch (grid-wide barriers "
                                     "between the phases), graph-replayed; further steps"},
            "clocks": clk.summary(),
            "config": {"workload": f"batched{args.scenarios}", "scenarios": args.scenarios,
                       "scenarios_rank0": len(scens),
                       "vehicles_rank0": int(sum(x.veh.n for x in scens)),
                       "vehicles_min_max_rank0": [int(min(x.veh.n for x in scens)), int(max(x.veh.n for x in scens))],
                       "start": f"each scenario's own step-{pre} state", "schedule": tuned,
                       "sharding": f"every {world}-th scenario per rank", "generation_s": gen_s}}
    if world == 1:
        s_val = seq_upd / (seq_ms / 1e3)
        line["sequential"] = {"value": s_val, "ms_per_step": seq_ms / args.steps,
                              "how": "the same scenarios, one handle each, stepped one scenario at a time"}
        line["batched_over_sequential"] = b_val / s_val
        line["same_updates"] = int(b_upd) == int(seq_upd)
    if emit:
        print(json.dumps(line), flush=True)
    return line


def _fresh(reqs):
    """the same requests with their results cleared (scenarios shared)"""
    from paper_2406_10661_gb300 import serving
    return [serving.Request(rid=r.rid, scenario=r.scenario, horizon=r.horizon, arrival=r.arrival,
                            action_seed=r.action_seed) for r in reqs]


def run_serving(args, emit=True):
    """A Poisson stream of rollout requests served by continuous batching: the
    requests share one resident slot batch (one set of launches per step for
    all in flight), admitted into free slots as they arrive; p50/p99 step
    latency and aggregate vehicle-updates/s, against serving the same
    requests one at a time, and with every request available at once (the
    capacity).  Returns the line (printed when emit)."""
    import torch
    from paper_2406_10661_gb300 import binding, serving
    binding.load()
    t0 = time.perf_counter()
    base = serving.poisson_requests(args.requests, rate_hz=20.0, seed=args.seed)
    gen_s = time.perf_counter() - t0
    free, total = torch.cuda.mem_get_info()
    budget = int(min(args.budget_gb * 2 ** 30, 0.8 * free))
    reqs = _fresh(base)
    with Clocks(torch.cuda.current_device()) as clk:
        stats = serving.Server(budget, max_slots=args.slots).run(reqs, realtime=True)
    sat_reqs = _fresh(base)
    sat = serving.Server(budget, max_slots=args.slots).run(sat_reqs, realtime=False)
    seq_reqs = _fresh(base[: args.seq_requests])
    seq = serving.Server(budget, max_slots=1).run(seq_reqs, realtime=False)
    same = all(a.metrics == b.metrics for a, b in zip(reqs, sat_reqs)) and \
        all(a.metrics == b.metrics for a, b in zip(reqs, seq_reqs))
    sat_head = sum(r.metrics["vehicle_updates"] for r in sat_reqs[: args.seq_requests])
    line = {"metric": "vehicle-updates/s (served)", "value": stats["vehicle_updates_per_s"],
            "unit": "vehicle-updates/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"serving{args.requests}", "arrivals": "Poisson 20/s",
                       "vehicles": "log-uniform 5k-500k", "horizon": "uniform 300-3600 steps",
                       "actions": "signal phases of every junction every 10 steps",
                       "budget_bytes": budget, "slots": stats["slots"], "generation_s": gen_s},
            "p50_step_ms": stats["p50_step_ms"], "p99_step_ms": stats["p99_step_ms"],
            "wall_s": stats["wall_s"], "peak_slots": stats["peak_slots"], "device_bytes": stats["peak_bytes"],
            "batch_steps": stats["slot_steps"], "request_steps": stats["steps"],
            "how": "one slot batch (moss_slots_create); requests loaded into free slots as they arrive, one "
                   "set of launches per step for all of them; latency = chunk time / steps",
            "clocks": clk.summary(),
            "all_at_once": {"value": sat["vehicle_updates_per_s"], "p50_step_ms": sat["p50_step_ms"],
                            "p99_step_ms": sat["p99_step_ms"], "wall_s": sat["wall_s"],
                            "how": "the same requests all available at once (capacity)"},
            "sequential": {"value": seq["vehicle_updates_per_s"], "requests": len(seq_reqs),
                           "p50_step_ms": seq["p50_step_ms"], "wall_s": seq["wall_s"],
                           "how": f"the first {len(seq_reqs)} requests one at a time (one slot)"},
            "all_at_once_over_sequential": sat["vehicle_updates_per_s"] / max(seq["vehicle_updates_per_s"], 1e-9),
            "results_equal_alone_and_mixed": same, "head_updates_all_at_once": sat_head}
    if emit:
        print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-roads", type=int, default=None,
                    help="reference arm: step only roads [0, REF_ROADS) (default: the whole network)")
    ap.add_argument("--workload", default="city", choices=["city", "saturated", "medium", "batched", "serving"],
                    help="city: the city from its own step-3600 state; saturated: the city network "
                         "with all 2,464,950 trips on the road at once")
    ap.add_argument("--policy", default="fixed", choices=["fixed", "max_pressure"],
                    help="signal policy of every junction on the city workload")
    ap.add_argument("--lane-groups", action="store_true",
                    help="city lanes serve turn groups (left+straight / straight / right+straight)")
    ap.add_argument("--scenarios", type=int, default=64)
    ap.add_argument("--requests", type=int, default=300)
    ap.add_argument("--seq-requests", type=int, default=40,
                    help="serving: requests served one at a time for the sequential comparison")
    ap.add_argument("--slots", type=int, default=32)
    ap.add_argument("--city-only", action="store_true",
                    help="city workload: leave out the batched and served sub-results")
    ap.add_argument("--budget-gb", type=float, default=64.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
