"""ctypes front end of the FP64 CPU oracle (``moss_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it to check and time the CUDA path.  It
shares no code with the CUDA path; both consume the same plain input arrays
built by ``paper_2406_10661_gb300.scenario``.

Parity of everything here is pinned by ``tests/test_oracle_pins.py`` (IDM
closed forms, MOBIL hand cases, Philox known answers, invariants, textbook
special cases).  Full-rollout aggregates have no external reference: parity
unpinned for them beyond those invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "moss_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_moss_oracle.so")
_LIB = None

METRIC_NAMES = ("step", "n_active", "n_waiting", "n_arrived", "tt_sum", "speed_sum",
                "vehicle_updates", "lane_changes", "flagged", "overlaps", "inserted", "errors",
                "mobil_evals")

DECISION_NAMES = ("a_own", "eligible", "attempted", "cand", "dir", "u", "uL", "uR", "feasL",
                  "feasR", "uT", "pLC", "u_att", "u_lc", "u_dir", "at_ego_L", "at_ego_R",
                  "a_new_L", "a_new_R", "at_new_L", "at_new_R", "a_old", "at_old", "flag",
                  "TL", "TF", "own_has_leader", "own_gap", "own_stop", "tgt_a", "own_leader",
                  "TL_left", "TF_left", "TL_right", "TF_right", "OL", "OF")

F_FLAGGED, F_CHANGED, F_CANDIDATE, F_TRANSFER, F_ARRIVED, F_INSERTED, F_CONFLICT_LOST = (
    1, 2, 4, 8, 16, 32, 64)
POLICY_FIXED, POLICY_MANUAL, POLICY_NONE, POLICY_MAX_PRESSURE = 0, 1, 2, 3
LIGHT_GREEN, LIGHT_AMBER, LIGHT_RED = 0, 1, 2


def build(force: bool = False, cflags: Sequence[str] = ()) -> str:
    """Compile the oracle into ``oracle/_moss_oracle.so`` (plain C, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *cflags, "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_variant(out_path: str, defines: Sequence[str]) -> str:
    """Compile a variant of the oracle with extra -D defines (used by tests that
    plant a mistake in the oracle to show the pins catch it)."""
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           *[f"-D{d}" for d in defines], "-o", out_path, _SRC, "-lm"])
    return out_path


def _setup(lib):
    vp = ctypes.c_void_p
    lib.mo_create.restype = vp
    lib.mo_create.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                              ctypes.c_int, vp, vp, vp, vp, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                              ctypes.c_ulonglong, ctypes.c_uint]
    lib.mo_destroy.argtypes = [vp]
    lib.mo_step.argtypes = [vp, ctypes.c_int]
    lib.mo_get_metrics.argtypes = [vp, vp]
    lib.mo_get_state.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.mo_set_state.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_long]
    lib.mo_set_state.restype = ctypes.c_int
    lib.mo_set_signal.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp]
    lib.mo_light.argtypes = [vp, ctypes.c_int, ctypes.c_long]
    lib.mo_light.restype = ctypes.c_int
    lib.mo_signal_state.argtypes = [vp, ctypes.c_int, vp]
    lib.mo_set_lane_max_speed.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.mo_set_lane_restriction.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.mo_lane_queue.argtypes = [vp, vp]
    lib.mo_set_vehicle_route.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    lib.mo_set_lane_plans.argtypes = [vp, vp]
    lib.mo_set_road_plan.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.mo_set_vehicle_route.restype = ctypes.c_int
    lib.mo_road_speed.argtypes = [vp, vp]
    lib.mo_idm.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.mo_idm.restype = ctypes.c_double
    lib.mo_idm_free.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    lib.mo_idm_free.restype = ctypes.c_double
    lib.mo_p_lc.argtypes = [vp, ctypes.c_double]
    lib.mo_p_lc.restype = ctypes.c_double
    lib.mo_decision.argtypes = [vp, ctypes.c_int, vp]
    lib.mo_set_reverse_order.argtypes = [vp, ctypes.c_int]
    lib.mo_philox4x32_10.argtypes = [ctypes.c_uint32, ctypes.c_uint32, vp, vp]
    return lib


def lib(path: Optional[str] = None):
    global _LIB
    if path is not None:
        return _setup(ctypes.CDLL(path))
    if _LIB is None:
        _LIB = _setup(ctypes.CDLL(build()))
    return _LIB


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(k0: int, k1: int, ctr) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().mo_philox4x32_10(ctypes.c_uint32(k0), ctypes.c_uint32(k1), _p(c), _p(out))
    return out


class Oracle:
    """One scenario simulated by the FP64 oracle."""

    def __init__(self, net, veh, params, libpath: Optional[str] = None):
        self._lib = lib(libpath)
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)  # noqa: E731
        f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)  # noqa: E731
        self._keep = [i32(net.road_lane_off), f32(net.lane_length), f32(net.lane_vmax),
                      i32(net.jl_off), i32(net.jl_target), i32(net.jl_junction), i32(net.jl_mask),
                      i32(net.junc_offset), i32(net.junc_phase_off), i32(net.phase_green),
                      i32(net.phase_amber), i32(veh.route_off), i32(veh.routes),
                      i32(veh.start_lane), i32(veh.dep), f32(veh.v0f),
                      np.ascontiguousarray(params.as_array(), dtype=np.float64)]
        k = self._keep
        self.n = int(veh.n)
        self.net = net
        self.h = self._lib.mo_create(
            int(net.n_roads), _p(k[0]), int(net.n_lanes), int(net.n_road_lanes), _p(k[1]),
            _p(k[2]), _p(k[3]), _p(k[4]), _p(k[5]), _p(k[6]), int(net.n_junctions), _p(k[7]),
            _p(k[8]), _p(k[9]), _p(k[10]), self.n, _p(k[11]), _p(k[12]), _p(k[13]), _p(k[14]),
            _p(k[15]), _p(k[16]), ctypes.c_ulonglong(int(params.seed) & (2 ** 64 - 1)),
            ctypes.c_uint(int(params.scenario) & 0xFFFFFFFF))
        if not self.h:
            raise MemoryError("oracle creation failed")
        plans = getattr(net, "jl_plans", None)
        if plans is not None:
            pl = np.ascontiguousarray(plans, dtype=np.int32)
            self._lib.mo_set_lane_plans(self.h, _p(pl))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._lib.mo_destroy(h)
            self.h = None

    def step(self, n: int = 1) -> None:
        self._lib.mo_step(self.h, int(n))

    def metrics(self) -> Dict[str, float]:
        out = np.zeros(len(METRIC_NAMES), dtype=np.float64)
        self._lib.mo_get_metrics(self.h, _p(out))
        return dict(zip(METRIC_NAMES, out.tolist()))

    def state(self) -> Dict[str, np.ndarray]:
        n = self.n
        st = {k: np.zeros(n, dtype=np.int32) for k in ("status", "lane", "rc", "flags")}
        st["s"] = np.zeros(n, dtype=np.float64)
        st["v"] = np.zeros(n, dtype=np.float64)
        self._lib.mo_get_state(self.h, _p(st["status"]), _p(st["lane"]), _p(st["s"]),
                               _p(st["v"]), _p(st["rc"]), _p(st["flags"]))
        return st

    def set_state(self, status, lane, s, v, rc, step: int) -> None:
        a = [np.ascontiguousarray(status, dtype=np.int32), np.ascontiguousarray(lane, dtype=np.int32),
             np.ascontiguousarray(s, dtype=np.float64), np.ascontiguousarray(v, dtype=np.float64),
             np.ascontiguousarray(rc, dtype=np.int32)]
        rc_ = self._lib.mo_set_state(self.h, *[_p(x) for x in a], ctypes.c_long(int(step)))
        if rc_ != 0:
            raise ValueError("state violates the per-lane FIFO order of waiting vehicles")

    def set_signal(self, junctions, policy: int, phases=None) -> None:
        j = np.ascontiguousarray(junctions, dtype=np.int32)
        ph = np.ascontiguousarray(phases if phases is not None else np.zeros(len(j)), dtype=np.int32)
        self._lib.mo_set_signal(self.h, len(j), _p(j), int(policy), _p(ph))

    def signal_state(self, j: int):
        """Max-pressure state of junction j: (phase, steps in the current green
        or amber interval, phase after the amber or -1)."""
        out = np.zeros(3, dtype=np.int32)
        self._lib.mo_signal_state(self.h, int(j), _p(out))
        return int(out[0]), int(out[1]), int(out[2])

    def set_lane_max_speed(self, lanes, vmax) -> None:
        l = np.ascontiguousarray(lanes, dtype=np.int32)
        v = np.ascontiguousarray(vmax, dtype=np.float64)
        self._lib.mo_set_lane_max_speed(self.h, len(l), _p(l), _p(v))

    def set_lane_restriction(self, lanes, flags) -> None:
        l = np.ascontiguousarray(lanes, dtype=np.int32)
        f = np.ascontiguousarray(flags, dtype=np.int32)
        self._lib.mo_set_lane_restriction(self.h, len(l), _p(l), _p(f))

    def set_road_plan(self, roads, plans) -> None:
        r = np.ascontiguousarray(roads, dtype=np.int32)
        p = np.ascontiguousarray(plans, dtype=np.int32)
        self._lib.mo_set_road_plan(self.h, len(r), _p(r), _p(p))

    def set_vehicle_route(self, vid: int, roads) -> bool:
        """Replace the route of vehicle vid (reading R26); False if refused."""
        r = np.ascontiguousarray(roads, dtype=np.int32)
        return self._lib.mo_set_vehicle_route(self.h, int(vid), len(r), _p(r)) == 0

    def lane_queue(self) -> np.ndarray:
        out = np.zeros(int(self.net.n_lanes), dtype=np.int32)
        self._lib.mo_lane_queue(self.h, _p(out))
        return out

    def road_speed(self) -> np.ndarray:
        out = np.zeros(int(self.net.n_roads), dtype=np.float64)
        self._lib.mo_road_speed(self.h, _p(out))
        return out

    def light(self, jl: int, t: int) -> int:
        return int(self._lib.mo_light(self.h, int(jl), ctypes.c_long(int(t))))

    def idm(self, v, v0, gap, dv) -> float:
        return float(self._lib.mo_idm(self.h, v, v0, gap, dv))

    def idm_free(self, v, v0) -> float:
        return float(self._lib.mo_idm_free(self.h, v, v0))

    def p_lc(self, uT) -> float:
        return float(self._lib.mo_p_lc(self.h, uT))

    def decision(self, vid: int) -> Dict[str, float]:
        out = np.zeros(len(DECISION_NAMES), dtype=np.float64)
        self._lib.mo_decision(self.h, int(vid), _p(out))
        return dict(zip(DECISION_NAMES, out.tolist()))

    def set_reverse_order(self, rev: bool) -> None:
        self._lib.mo_set_reverse_order(self.h, int(bool(rev)))
