"""Thin ctypes binding of the C ABI in ``include/moss.h`` (argument
marshalling only: every step of the simulation runs in the CUDA library).

The functions carry the C names (``moss_create``, ``moss_step``, ...).  The
``Simulation`` and ``Batch`` classes wrap a handle for numpy inputs from
``paper_2406_10661_gb300.scenario``.  Loading fails loudly when the compiled
library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmoss.so")

MOSS_OK, MOSS_EINVAL, MOSS_ENOMEM, MOSS_ECUDA, MOSS_ETIMEOUT, MOSS_EBUDGET, MOSS_EDEVICE = range(7)
POLICY_FIXED_TIME, POLICY_MANUAL, POLICY_NONE, POLICY_MAX_PRESSURE = 0, 1, 2, 3
METRIC_SLOTS = 64  # readback slots of metrics_enqueue / metrics_read
F_FLAGGED, F_CHANGED, F_CANDIDATE, F_TRANSFER, F_ARRIVED, F_INSERTED, F_CONFLICT_LOST = (
    1, 2, 4, 8, 16, 32, 64)

_c_i32p = ctypes.POINTER(ctypes.c_int32)
_c_f32p = ctypes.POINTER(ctypes.c_float)
_c_f64p = ctypes.POINTER(ctypes.c_double)


class MossNetwork(ctypes.Structure):
    _fields_ = [("n_roads", ctypes.c_int32), ("n_road_lanes", ctypes.c_int32),
                ("n_lanes", ctypes.c_int32), ("n_junctions", ctypes.c_int32),
                ("road_lane_off", _c_i32p), ("lane_length", _c_f32p), ("lane_vmax", _c_f32p),
                ("jl_off", _c_i32p), ("jl_target", _c_i32p), ("jl_junction", _c_i32p),
                ("jl_mask", _c_i32p), ("junc_offset", _c_i32p), ("junc_phase_off", _c_i32p),
                ("phase_green", _c_i32p), ("phase_amber", _c_i32p), ("jl_plans", _c_i32p)]


class MossVehicles(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("route_off", _c_i32p), ("routes", _c_i32p),
                ("start_lane", _c_i32p), ("dep", _c_i32p), ("v0f", _c_f32p)]


class MossParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "dt", "a_max", "b_comf", "T", "s0", "delta", "veh_len", "politeness", "a_th", "b_safe",
        "p_attempt", "p_hi", "p_lo", "flag_band")] + [
        ("seed", ctypes.c_uint64), ("scenario", ctypes.c_uint32), ("precision", ctypes.c_int32)]


class MossMetrics(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("n_active", ctypes.c_int64),
                ("n_waiting", ctypes.c_int64), ("n_arrived", ctypes.c_int64),
                ("tt_sum", ctypes.c_double), ("speed_sum", ctypes.c_double),
                ("vehicle_updates", ctypes.c_int64), ("lane_changes", ctypes.c_int64),
                ("flagged", ctypes.c_int64), ("overlaps", ctypes.c_int64),
                ("inserted", ctypes.c_int64), ("errors", ctypes.c_int64),
                ("mobil_evals", ctypes.c_int64)]

    def as_dict(self) -> Dict[str, float]:
        return {k: getattr(self, k) for k, _ in self._fields_}


class MossState(ctypes.Structure):
    _fields_ = [("status", _c_i32p), ("lane", _c_i32p), ("s", _c_f64p), ("v", _c_f64p),
                ("rc", _c_i32p), ("flags", _c_i32p)]


class MossSlotCaps(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("n_lanes", "n_roads", "n_junctions", "n_phases", "n_vehicles",
                                              "n_route_entries")]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class MossAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", ctypes.c_void_p)]


def torch_allocator():
    """A MossAllocator backed by PyTorch's caching allocator (device memory
    of a handle comes from torch's pool, on the handle's stream).  Keep the
    returned object alive as long as the handle."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _release(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    return MossAllocator(ALLOC_FN(_alloc), RELEASE_FN(_release), None)


# every symbol include/moss.h declares, with its signature
_vp = ctypes.c_void_p
SIGNATURES = {
    "moss_create": (ctypes.c_int, [ctypes.POINTER(MossNetwork), ctypes.POINTER(MossVehicles),
                                   ctypes.POINTER(MossParams), _vp, ctypes.POINTER(_vp)]),
    "moss_step": (ctypes.c_int, [_vp, ctypes.c_int]),
    "moss_set_signal_phase": (ctypes.c_int, [_vp, ctypes.c_int, _c_i32p, _c_i32p]),
    "moss_set_signal_policy": (ctypes.c_int, [_vp, ctypes.c_int, _c_i32p, ctypes.c_int32]),
    "moss_get_signal_state": (ctypes.c_int, [_vp, ctypes.c_int, _c_i32p, _c_i32p, _c_i32p, _c_i32p]),
    "moss_set_vehicle_route": (ctypes.c_int, [_vp, ctypes.c_int, _c_i32p, _c_i32p, _c_i32p]),
    "moss_set_road_lane_plan": (ctypes.c_int, [_vp, ctypes.c_int, _c_i32p, _c_i32p]),
    "moss_set_lane_max_speed": (ctypes.c_int, [_vp, ctypes.c_int, _c_i32p, ctypes.POINTER(ctypes.c_float)]),
    "moss_set_lane_restriction": (ctypes.c_int, [_vp, ctypes.c_int, _c_i32p, _c_i32p]),
    "moss_get_lane_queue": (ctypes.c_int, [_vp, _c_i32p]),
    "moss_get_road_speed": (ctypes.c_int, [_vp, _c_f64p]),
    "moss_batch_get_lane_queue": (ctypes.c_int, [_vp, ctypes.c_int, _c_i32p]),
    "moss_batch_get_road_speed": (ctypes.c_int, [_vp, ctypes.c_int, _c_f64p]),
    "moss_get_metrics": (ctypes.c_int, [_vp, ctypes.POINTER(MossMetrics)]),
    "moss_get_state": (ctypes.c_int, [_vp, ctypes.POINTER(MossState)]),
    "moss_set_state": (ctypes.c_int, [_vp, ctypes.POINTER(MossState), ctypes.c_int64]),
    "moss_synchronize": (ctypes.c_int, [_vp]),
    "moss_device_bytes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "moss_destroy": (None, [_vp]),
    "moss_last_error": (ctypes.c_char_p, [_vp]),
    "moss_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(MossNetwork),
                                         ctypes.POINTER(MossVehicles), ctypes.POINTER(MossParams),
                                         _vp, ctypes.POINTER(_vp)]),
    "moss_batch_size": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "moss_slots_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(MossSlotCaps), ctypes.POINTER(MossParams),
                                         _vp, ctypes.POINTER(MossAllocator), ctypes.POINTER(_vp)]),
    "moss_slot_load": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(MossNetwork), ctypes.POINTER(MossVehicles),
                                      ctypes.POINTER(MossParams)]),
    "moss_slot_retire": (ctypes.c_int, [_vp, ctypes.c_int]),
    "moss_slot_set_horizon": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64]),
    "moss_batch_create_with_allocator": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(MossNetwork),
                                                        ctypes.POINTER(MossVehicles), ctypes.POINTER(MossParams),
                                                        _vp, ctypes.POINTER(MossAllocator), ctypes.POINTER(_vp)]),
    "moss_batch_get_metrics": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(MossMetrics)]),
    "moss_metrics_enqueue": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "moss_metrics_read": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(MossMetrics)]),
    "moss_batch_get_state": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(MossState)]),
    "moss_batch_set_signal_phase": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _c_i32p,
                                                   _c_i32p]),
    "moss_batch_set_signal_phases": (ctypes.c_int, [_vp, ctypes.c_int, _c_i32p, _c_i32p, _c_i32p]),
    "moss_set_kernel_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "moss_kernel_times": (ctypes.c_int, [_vp, _c_f64p, ctypes.POINTER(ctypes.c_int64)]),
    "moss_lane_offsets_noalloc": (ctypes.c_int, [ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "moss_autotune": (ctypes.c_int, [_vp, ctypes.c_int, _c_i32p]),
    "moss_get_schedule": (ctypes.c_int, [_vp, _c_i32p]),
    "moss_set_schedule": (ctypes.c_int, [_vp, _c_i32p]),
    "moss_set_step_mode": (ctypes.c_int, [_vp, ctypes.c_int]),
    "moss_step_launches": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "moss_selftest_bounded_wait": (ctypes.c_int, [_vp]),
}

NOALLOC_MAX_LANES = 1 << 22


def moss_lane_offsets_noalloc(n_lanes: int, d_off_cur: int, d_leave: int, d_enter: int,
                              d_off_next: int, d_lbefore: int, stream: int = 0) -> int:
    """Lane offsets of the next snapshot from per-lane leave/enter counts, for
    callers that cannot allocate device memory (device pointers in and out;
    see include/moss.h).  Returns the C status code."""
    return load().moss_lane_offsets_noalloc(int(n_lanes), _vp(d_off_cur), _vp(d_leave),
                                            _vp(d_enter), _vp(d_off_next), _vp(d_lbefore),
                                            _vp(stream) if stream else None)


def moss_selftest_bounded_wait(stream: int = 0) -> int:
    """Run the bounded-wait self-test (a look-back wait on a word nothing
    publishes); returns the C status, MOSS_ETIMEOUT when the wait gave up and
    reported it as designed."""
    return load().moss_selftest_bounded_wait(_vp(stream) if stream else None)


_LIB = None


def load(path: str = LIB_PATH):
    """Load the compiled library; raises if it is missing (no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA library {path} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


class MossError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"moss error {code}: {msg}")
        self.code = code


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc: int, h=None):
    if rc != MOSS_OK:
        msg = load().moss_last_error(h).decode() if h else ""
        raise MossError(rc, msg)


def _net_struct(net, keep: list) -> MossNetwork:
    def i32(a):
        x = np.ascontiguousarray(a, dtype=np.int32); keep.append(x); return _ptr(x, ctypes.c_int32)

    def f32(a):
        x = np.ascontiguousarray(a, dtype=np.float32); keep.append(x); return _ptr(x, ctypes.c_float)

    return MossNetwork(net.n_roads, net.n_road_lanes, net.n_lanes, net.n_junctions,
                       i32(net.road_lane_off), f32(net.lane_length), f32(net.lane_vmax),
                       i32(net.jl_off), i32(net.jl_target), i32(net.jl_junction), i32(net.jl_mask),
                       i32(net.junc_offset), i32(net.junc_phase_off), i32(net.phase_green),
                       i32(net.phase_amber),
                       i32(net.jl_plans) if getattr(net, "jl_plans", None) is not None else None)


def _veh_struct(veh, keep: list) -> MossVehicles:
    def i32(a):
        x = np.ascontiguousarray(a, dtype=np.int32); keep.append(x); return _ptr(x, ctypes.c_int32)

    v0 = np.ascontiguousarray(veh.v0f, dtype=np.float32)
    keep.append(v0)
    return MossVehicles(int(veh.n), i32(veh.route_off), i32(veh.routes), i32(veh.start_lane),
                        i32(veh.dep), _ptr(v0, ctypes.c_float))


def _prm_struct(p, precision: int) -> MossParams:
    return MossParams(p.dt, p.a_max, p.b_comf, p.T, p.s0, p.delta, p.veh_len, p.politeness,
                      p.a_th, p.b_safe, p.p_attempt, p.p_hi, p.p_lo, p.flag_band,
                      int(p.seed) & (2 ** 64 - 1), int(p.scenario) & 0xFFFFFFFF, precision)


class _Handle:
    def __init__(self):
        self.h = None
        self.lib = load()

    def close(self):
        if self.h:
            self.lib.moss_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1) -> None:
        _check(self.lib.moss_step(self.h, int(n)), self.h)

    def synchronize(self) -> None:
        _check(self.lib.moss_synchronize(self.h), self.h)

    def device_bytes(self) -> int:
        out = ctypes.c_size_t(0)
        _check(self.lib.moss_device_bytes(self.h, ctypes.byref(out)), self.h)
        return int(out.value)

    def step_launches(self) -> int:
        """Kernel launches of the library per step in the current mode."""
        out = ctypes.c_int(0)
        _check(self.lib.moss_step_launches(self.h, ctypes.byref(out)), self.h)
        return int(out.value)

    def set_step_mode(self, mode: int) -> None:
        """0: three kernels per step (graph); 1: one cooperative launch per step."""
        _check(self.lib.moss_set_step_mode(self.h, int(mode)), self.h)

    def set_kernel_timing(self, on: bool) -> None:
        _check(self.lib.moss_set_kernel_timing(self.h, int(bool(on))), self.h)

    SCHEDULE_KEYS = ("decide", "lanescan", "place", "road_weight", "lanes_per_thread", "step_mode",
                     "candidates_per_block")

    def autotune(self, trial_steps: int = 3):
        """Pick the fastest launch schedule on the next 16 * trial_steps steps;
        returns the whole schedule (``schedule()``)."""
        out = np.zeros(3, dtype=np.int32)
        _check(self.lib.moss_autotune(self.h, int(trial_steps), _ptr(out, ctypes.c_int32)), self.h)
        return self.schedule()

    def schedule(self) -> Dict[str, int]:
        out = np.zeros(7, dtype=np.int32)
        _check(self.lib.moss_get_schedule(self.h, _ptr(out, ctypes.c_int32)), self.h)
        return dict(zip(self.SCHEDULE_KEYS, out.tolist()))

    def set_schedule(self, **kw) -> None:
        cur = self.schedule()
        cur.update(kw)
        arr = np.array([cur[k] for k in self.SCHEDULE_KEYS], dtype=np.int32)
        _check(self.lib.moss_set_schedule(self.h, _ptr(arr, ctypes.c_int32)), self.h)

    def metrics_enqueue(self, slot: int, scenario: int = 0) -> None:
        """Queue a copy of the metrics (as after the work enqueued so far) into
        a readback slot without waiting."""
        _check(self.lib.moss_metrics_enqueue(self.h, int(scenario), int(slot)), self.h)

    def metrics_read(self, slot: int) -> Dict[str, float]:
        """Wait for the copy in a readback slot and return those metrics."""
        m = MossMetrics()
        _check(self.lib.moss_metrics_read(self.h, int(slot), ctypes.byref(m)), self.h)
        return m.as_dict()

    def kernel_times(self):
        ms = np.zeros(4, dtype=np.float64)
        n = ctypes.c_int64(0)
        _check(self.lib.moss_kernel_times(self.h, _ptr(ms, ctypes.c_double), ctypes.byref(n)), self.h)
        return dict(zip(("decide", "lanescan", "place", "resolve"), ms.tolist())), int(n.value)


def _state_arrays(n: int):
    st = {k: np.zeros(n, dtype=np.int32) for k in ("status", "lane", "rc", "flags")}
    st["s"] = np.zeros(n, dtype=np.float64)
    st["v"] = np.zeros(n, dtype=np.float64)
    ms = MossState(_ptr(st["status"], ctypes.c_int32), _ptr(st["lane"], ctypes.c_int32),
                   _ptr(st["s"], ctypes.c_double), _ptr(st["v"], ctypes.c_double),
                   _ptr(st["rc"], ctypes.c_int32), _ptr(st["flags"], ctypes.c_int32))
    return st, ms


class Simulation(_Handle):
    """One scenario on the GPU (``moss_create``)."""

    def __init__(self, net, veh, params, precision: int = 32, stream: Optional[int] = None,
                 allocator: Optional[MossAllocator] = None):
        super().__init__()
        keep: list = []
        n = _net_struct(net, keep)
        v = _veh_struct(veh, keep)
        p = _prm_struct(params, precision)
        h = _vp()
        if allocator is None:
            rc = self.lib.moss_create(ctypes.byref(n), ctypes.byref(v), ctypes.byref(p),
                                      _vp(stream) if stream else None, ctypes.byref(h))
        else:
            self._allocator = allocator  # the callbacks must outlive the handle
            rc = self.lib.moss_batch_create_with_allocator(1, ctypes.byref(n), ctypes.byref(v), ctypes.byref(p),
                                                           _vp(stream) if stream else None,
                                                           ctypes.byref(allocator), ctypes.byref(h))
        _check(rc)
        self.h = h
        self.n = int(veh.n)
        self.net = net
        self.precision = precision

    def metrics(self) -> Dict[str, float]:
        m = MossMetrics()
        _check(self.lib.moss_get_metrics(self.h, ctypes.byref(m)), self.h)
        return m.as_dict()

    def state(self) -> Dict[str, np.ndarray]:
        st, ms = _state_arrays(self.n)
        _check(self.lib.moss_get_state(self.h, ctypes.byref(ms)), self.h)
        return st

    def set_state(self, status, lane, s, v, rc, step: int) -> None:
        arr = [np.ascontiguousarray(status, dtype=np.int32), np.ascontiguousarray(lane, dtype=np.int32),
               np.ascontiguousarray(s, dtype=np.float64), np.ascontiguousarray(v, dtype=np.float64),
               np.ascontiguousarray(rc, dtype=np.int32), np.zeros(self.n, dtype=np.int32)]
        ms = MossState(_ptr(arr[0], ctypes.c_int32), _ptr(arr[1], ctypes.c_int32),
                       _ptr(arr[2], ctypes.c_double), _ptr(arr[3], ctypes.c_double),
                       _ptr(arr[4], ctypes.c_int32), _ptr(arr[5], ctypes.c_int32))
        _check(self.lib.moss_set_state(self.h, ctypes.byref(ms), ctypes.c_int64(int(step))), self.h)

    def set_signal_phase(self, junctions: Sequence[int], phases: Sequence[int]) -> None:
        j = np.ascontiguousarray(junctions, dtype=np.int32)
        p = np.ascontiguousarray(phases, dtype=np.int32)
        _check(self.lib.moss_set_signal_phase(self.h, len(j), _ptr(j, ctypes.c_int32),
                                              _ptr(p, ctypes.c_int32)), self.h)

    def set_signal_policy(self, junctions: Sequence[int], policy: int) -> None:
        j = np.ascontiguousarray(junctions, dtype=np.int32)
        _check(self.lib.moss_set_signal_policy(self.h, len(j), _ptr(j, ctypes.c_int32),
                                               int(policy)), self.h)

    def set_road_lane_plan(self, roads: Sequence[int], plans) -> None:
        r = np.ascontiguousarray(roads, dtype=np.int32)
        p = np.ascontiguousarray(plans, dtype=np.int32)
        _check(self.lib.moss_set_road_lane_plan(self.h, len(r), _ptr(r, ctypes.c_int32), _ptr(p, ctypes.c_int32)),
               self.h)

    def set_vehicle_route(self, vehicles: Sequence[int], routes) -> None:
        """New routes (lists of road ids) for the given vehicles (all or nothing)."""
        v = np.ascontiguousarray(vehicles, dtype=np.int32)
        off = np.zeros(len(v) + 1, dtype=np.int32)
        off[1:] = np.cumsum([len(r) for r in routes])
        flat = np.ascontiguousarray(np.concatenate([np.asarray(r, dtype=np.int32) for r in routes])
                                    if len(routes) else np.zeros(0, dtype=np.int32), dtype=np.int32)
        _check(self.lib.moss_set_vehicle_route(self.h, len(v), _ptr(v, ctypes.c_int32), _ptr(off, ctypes.c_int32),
                                               _ptr(flat, ctypes.c_int32)), self.h)

    def set_lane_max_speed(self, lanes: Sequence[int], vmax) -> None:
        l = np.ascontiguousarray(lanes, dtype=np.int32)
        v = np.ascontiguousarray(vmax, dtype=np.float32)
        _check(self.lib.moss_set_lane_max_speed(self.h, len(l), _ptr(l, ctypes.c_int32), _ptr(v, ctypes.c_float)),
               self.h)

    def set_lane_restriction(self, lanes: Sequence[int], flags) -> None:
        l = np.ascontiguousarray(lanes, dtype=np.int32)
        f = np.ascontiguousarray(flags, dtype=np.int32)
        _check(self.lib.moss_set_lane_restriction(self.h, len(l), _ptr(l, ctypes.c_int32), _ptr(f, ctypes.c_int32)),
               self.h)

    def lane_queue(self) -> np.ndarray:
        """Vehicles with v < 0.1 m/s within the last 50 m of every lane."""
        out = np.zeros(int(self.net.n_lanes), dtype=np.int32)
        _check(self.lib.moss_get_lane_queue(self.h, _ptr(out, ctypes.c_int32)), self.h)
        return out

    def road_speed(self) -> np.ndarray:
        """Mean vehicle speed of every road (its lanes' mean limit when empty)."""
        out = np.zeros(int(self.net.n_roads), dtype=np.float64)
        _check(self.lib.moss_get_road_speed(self.h, _ptr(out, ctypes.c_double)), self.h)
        return out

    def signal_state(self, junctions: Sequence[int]):
        """(phase shown or -1, steps in the current interval, phase after the
        amber or -1) per junction, at the current step."""
        j = np.ascontiguousarray(junctions, dtype=np.int32)
        ph, el, nx = (np.zeros(len(j), dtype=np.int32) for _ in range(3))
        _check(self.lib.moss_get_signal_state(self.h, len(j), _ptr(j, ctypes.c_int32), _ptr(ph, ctypes.c_int32),
                                              _ptr(el, ctypes.c_int32), _ptr(nx, ctypes.c_int32)), self.h)
        return ph, el, nx


class Batch(_Handle):
    """Several scenarios advanced together (``moss_batch_create``)."""

    def __init__(self, scenarios: List, precision: int = 32, stream: Optional[int] = None):
        super().__init__()
        keep: list = []
        k = len(scenarios)
        nets = (MossNetwork * k)(*[_net_struct(s.net, keep) for s in scenarios])
        vehs = (MossVehicles * k)(*[_veh_struct(s.veh, keep) for s in scenarios])
        prms = (MossParams * k)(*[_prm_struct(s.params, precision) for s in scenarios])
        h = _vp()
        _check(self.lib.moss_batch_create(k, nets, vehs, prms, _vp(stream) if stream else None,
                                          ctypes.byref(h)))
        self.h = h
        self.sizes = [int(s.veh.n) for s in scenarios]
        self.nets = [s.net for s in scenarios]
        self.k = k

    def metrics(self, i: int) -> Dict[str, float]:
        m = MossMetrics()
        _check(self.lib.moss_batch_get_metrics(self.h, int(i), ctypes.byref(m)), self.h)
        return m.as_dict()

    def state(self, i: int) -> Dict[str, np.ndarray]:
        st, ms = _state_arrays(self.sizes[i])
        _check(self.lib.moss_batch_get_state(self.h, int(i), ctypes.byref(ms)), self.h)
        return st

    def lane_queue(self, i: int) -> np.ndarray:
        out = np.zeros(int(self.nets[i].n_lanes), dtype=np.int32)
        _check(self.lib.moss_batch_get_lane_queue(self.h, int(i), _ptr(out, ctypes.c_int32)), self.h)
        return out

    def road_speed(self, i: int) -> np.ndarray:
        out = np.zeros(int(self.nets[i].n_roads), dtype=np.float64)
        _check(self.lib.moss_batch_get_road_speed(self.h, int(i), _ptr(out, ctypes.c_double)), self.h)
        return out

    def set_signal_phase(self, i: int, junctions, phases) -> None:
        j = np.ascontiguousarray(junctions, dtype=np.int32)
        p = np.ascontiguousarray(phases, dtype=np.int32)
        _check(self.lib.moss_batch_set_signal_phase(self.h, int(i), len(j), _ptr(j, ctypes.c_int32),
                                                    _ptr(p, ctypes.c_int32)), self.h)

    def set_signal_phases(self, scenarios, junctions, phases) -> None:
        """Phases of junctions of several scenarios in one call."""
        s = np.ascontiguousarray(scenarios, dtype=np.int32)
        j = np.ascontiguousarray(junctions, dtype=np.int32)
        p = np.ascontiguousarray(phases, dtype=np.int32)
        _check(self.lib.moss_batch_set_signal_phases(self.h, len(j), _ptr(s, ctypes.c_int32),
                                                     _ptr(j, ctypes.c_int32), _ptr(p, ctypes.c_int32)), self.h)


def slot_caps(scen) -> Dict[str, int]:
    """The capacities a slot needs to take scenario `scen` (moss_slot_load)."""
    net, veh = scen.net, scen.veh
    nph = int(net.junc_phase_off[net.n_junctions]) if net.n_junctions else 0
    return {"n_lanes": int(net.n_lanes), "n_roads": int(net.n_roads), "n_junctions": int(net.n_junctions),
            "n_phases": nph, "n_vehicles": int(veh.n),
            "n_route_entries": int(veh.route_off[veh.n]) if veh.n else 0}


def fits(caps: Dict[str, int], need: Dict[str, int]) -> bool:
    return all(need[k] <= caps[k] for k in need)


class Slots(Batch):
    """A slot batch (``moss_slots_create``): fixed-capacity slots into which
    scenarios are loaded while the others run; every ``step`` advances all
    loaded slots with one set of launches.  The per-slot getters and setters
    are those of ``Batch`` with the slot index."""

    def __init__(self, caps: List[Dict[str, int]], params, precision: int = 32, stream: Optional[int] = None,
                 allocator: Optional[MossAllocator] = None):
        _Handle.__init__(self)
        k = len(caps)
        arr = (MossSlotCaps * k)(*[MossSlotCaps(*[int(c[f]) for f, _ in MossSlotCaps._fields_]) for c in caps])
        p = _prm_struct(params, precision)
        h = _vp()
        if allocator is not None:
            self._allocator = allocator
        _check(self.lib.moss_slots_create(k, arr, ctypes.byref(p), _vp(stream) if stream else None,
                                          ctypes.byref(allocator) if allocator is not None else None,
                                          ctypes.byref(h)))
        self.h = h
        self.k = k
        self.precision = precision
        self.caps = [dict(c) for c in caps]
        self.sizes = [0] * k
        self.nets = [None] * k

    def load(self, slot: int, scen) -> None:
        keep: list = []
        n = _net_struct(scen.net, keep)
        v = _veh_struct(scen.veh, keep)
        p = _prm_struct(scen.params, self.precision)
        _check(self.lib.moss_slot_load(self.h, int(slot), ctypes.byref(n), ctypes.byref(v), ctypes.byref(p)), self.h)
        self.sizes[slot] = int(scen.veh.n)
        self.nets[slot] = scen.net

    def retire(self, slot: int) -> None:
        _check(self.lib.moss_slot_retire(self.h, int(slot)), self.h)
        self.sizes[slot] = 0
        self.nets[slot] = None

    def set_horizon(self, slot: int, stop_at: int) -> None:
        _check(self.lib.moss_slot_set_horizon(self.h, int(slot), int(stop_at)), self.h)
