"""Seeded synthetic scenarios (road networks, travel demand, model parameters).

This module only builds INPUTS: grid and perturbed-grid road networks with
junction lanes and fixed-time signal programs, origin-destination demand with
shortest-path routes, and the model-parameter set.  It holds none of the
simulation arithmetic (no car-following, lane changing, signals evaluation or
integration), so both the FP64 oracle and the CUDA path consume its arrays as
plain data.

The paper's own inputs are protobuf maps and trips built from OpenStreetMap and
a diffusion OD model (§3.1 "Simulator Inputs and Toolchain", App. D); those are
not available, so the networks here are synthetic and shaped like the paper's
workloads (Table A2: up to 93,564 roads / 2,464,950 vehicles).

Randomness comes from splitmix64 (Steele, Lea & Flood, OOPSLA 2014), evaluated
with numpy uint64 arithmetic, so every platform builds bit-identical integer and
float32 arrays from the same seed.  Normal variates use the Irwin-Hall sum of
twelve uniforms (exact integer sums), not a transcendental transform.

Network layout conventions (shared by both consumers, documented in
``include/moss.h``):

* lanes ``[0, n_road_lanes)`` are road lanes, grouped by road; a road's lanes
  are contiguous and ordered from the leftmost (index 0) to the rightmost;
* lanes ``[n_road_lanes, n_lanes)`` are junction lanes, grouped by the road
  lane they leave from: the junction lanes leaving road lane ``l`` are
  ``[jl_off[l], jl_off[l+1])`` (absolute lane ids);
* ``jl_target[j - n_road_lanes]`` is the road lane junction lane ``j`` feeds;
* ``jl_mask`` bit ``p`` is set when the junction lane is green in phase ``p``;
* signal programs are in whole steps: per junction an offset and per phase a
  green and an amber duration.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)


# ----------------------------------------------------------------------------
# splitmix64 streams
# ----------------------------------------------------------------------------
def _shr(z: np.ndarray, k: int) -> np.ndarray:
    return np.right_shift(z, np.uint8(k))


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ _shr(z, 30)) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ _shr(z, 27)) * np.uint64(0x94D049BB133111EB)
        z = z ^ _shr(z, 31)
    return z


class Stream:
    """A splitmix64 stream: word k of stream (seed, tag) is mix64(base + (k+1)*gamma)."""

    def __init__(self, seed: int, tag: int):
        base = _mix64(np.array([(seed * 0x100000001B3 + tag) & 0xFFFFFFFFFFFFFFFF],
                               dtype=np.uint64))[0]
        self.base = np.uint64(base)
        self.pos = 0

    def words(self, n: int) -> np.ndarray:
        k = np.arange(self.pos + 1, self.pos + n + 1, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            return _mix64(self.base + k * _GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return _shr(self.words(n), 11).astype(np.float64) * (2.0 ** -53)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers uniform in [lo, hi) (multiply-shift on 32 high bits; hi-lo < 2^32)."""
        span = hi - lo
        assert 0 < span < 2 ** 32
        w = _shr(self.words(n), 32)
        with np.errstate(over="ignore"):
            r = _shr(w * np.uint64(span), 32)
        return (r.astype(np.int64) + lo)

    def normal(self, n: int) -> np.ndarray:
        """Approximate N(0,1): Irwin-Hall sum of 12 uniforms minus 6 (exact sums)."""
        w = _shr(self.words(12 * n), 40).astype(np.int64).reshape(n, 12)  # 24-bit ints
        tot = w.sum(axis=1)  # exact
        return tot.astype(np.float64) * (2.0 ** -24) - 6.0

    def choice(self, probs, n: int) -> np.ndarray:
        c = np.cumsum(np.asarray(probs, dtype=np.float64))
        c /= c[-1]
        return np.searchsorted(c, self.uniform(n), side="right")


# ----------------------------------------------------------------------------
# Parameters
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    """Model parameters (IDM of App. B.3, randomized MOBIL of App. B.3).

    Defaults are the workload's stated values: IDM T=1.5 s, a=2, b=4.5, s0=2,
    delta=4, length 5 m; MOBIL p=0.1, a_th=0.1, b_safe=4, attempt probability
    0.5; p_LC branch levels 0.9 and 2e-8 (App. B.3).
    """
    dt: float = 1.0
    a_max: float = 2.0
    b_comf: float = 4.5
    T: float = 1.5
    s0: float = 2.0
    delta: float = 4.0
    veh_len: float = 5.0
    politeness: float = 0.1
    a_th: float = 0.1
    b_safe: float = 4.0
    p_attempt: float = 0.5
    p_hi: float = 0.9
    p_lo: float = 2e-8
    flag_band: float = 1e-4
    seed: int = 0
    scenario: int = 0

    def as_array(self) -> np.ndarray:
        """The 14 floating parameters in the fixed order both consumers read."""
        return np.array([self.dt, self.a_max, self.b_comf, self.T, self.s0, self.delta,
                         self.veh_len, self.politeness, self.a_th, self.b_safe,
                         self.p_attempt, self.p_hi, self.p_lo, self.flag_band],
                        dtype=np.float64)


PARAM_ORDER = ("dt", "a_max", "b_comf", "T", "s0", "delta", "veh_len", "politeness",
               "a_th", "b_safe", "p_attempt", "p_hi", "p_lo", "flag_band")


# ----------------------------------------------------------------------------
# Network / vehicles containers
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Network:
    n_roads: int
    n_road_lanes: int
    n_lanes: int
    n_junctions: int
    road_lane_off: np.ndarray   # int32 [n_roads+1]
    lane_length: np.ndarray     # float32 [n_lanes]
    lane_vmax: np.ndarray       # float32 [n_lanes]
    jl_off: np.ndarray          # int32 [n_road_lanes+1], absolute lane ids
    jl_target: np.ndarray       # int32 [n_junction_lanes]
    jl_junction: np.ndarray     # int32 [n_junction_lanes]
    jl_mask: np.ndarray         # int32 [n_junction_lanes]
    junc_offset: np.ndarray     # int32 [n_junctions] (steps)
    junc_phase_off: np.ndarray  # int32 [n_junctions+1]
    phase_green: np.ndarray     # int32 [n_phases_total] (steps)
    phase_amber: np.ndarray     # int32 [n_phases_total] (steps)
    # descriptive extras (not consumed by the simulators)
    road_from: Optional[np.ndarray] = None
    road_to: Optional[np.ndarray] = None
    road_reverse: Optional[np.ndarray] = None
    jl_turn: Optional[np.ndarray] = None   # 0 straight, 1 left, 2 right
    # lane function plans: bit p of jl_plans[k] = junction lane k exists in plan p (None: all plans)
    jl_plans: Optional[np.ndarray] = None

    @property
    def n_junction_lanes(self) -> int:
        return self.n_lanes - self.n_road_lanes

    def lane_road(self) -> np.ndarray:
        r = np.full(self.n_lanes, -1, dtype=np.int32)
        r[: self.n_road_lanes] = np.repeat(np.arange(self.n_roads, dtype=np.int32),
                                           np.diff(self.road_lane_off))
        return r

    def validate(self) -> None:
        assert self.road_lane_off[0] == 0 and self.road_lane_off[-1] == self.n_road_lanes
        assert np.all(np.diff(self.road_lane_off) >= 1)
        assert self.jl_off[0] == self.n_road_lanes and self.jl_off[-1] == self.n_lanes
        assert np.all(np.diff(self.jl_off) >= 0)
        assert np.all(self.jl_target >= 0) and np.all(self.jl_target < self.n_road_lanes)
        assert np.all(self.lane_length > 0) and np.all(self.lane_vmax > 0)


@dataclasses.dataclass
class Vehicles:
    n: int
    route_off: np.ndarray   # int32 [n+1]
    routes: np.ndarray      # int32 [route_off[-1]] road ids
    start_lane: np.ndarray  # int32 [n] absolute lane id on road routes[route_off[i]]
    dep: np.ndarray         # int32 [n] departure step
    v0f: np.ndarray         # float32 [n] desired-speed factor

    def validate(self, net: Network) -> None:
        assert np.all(np.diff(self.route_off) >= 1)
        rl = net.lane_road()
        assert np.all(rl[self.start_lane] == self.routes[self.route_off[:-1]])


@dataclasses.dataclass
class Scenario:
    net: Network
    veh: Vehicles
    params: Params
    name: str = ""


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


# ----------------------------------------------------------------------------
# Generic builder from a junction graph with headings
# ----------------------------------------------------------------------------
def build_network(jxy: np.ndarray, links: np.ndarray, link_len: np.ndarray,
                  link_lanes: np.ndarray, link_vmax: np.ndarray,
                  junc_offset: np.ndarray, green: int = 30, amber: int = 3,
                  lane_width: float = 3.5, lane_groups: bool = False,
                  lane_plans: bool = False) -> Network:
    """Build a network from junction grid coordinates and undirected links.

    jxy: int [J,2] grid coordinates (headings are taken from them, so a
    perturbed geometry keeps grid topology); links: int [E,2] junction pairs.
    Each link gives two one-way roads with the link's length, lane count and
    speed limit.  Every road lane connects to every out-road of its end
    junction except the U-turn; in-lane i feeds out-lane min(i, n_out-1).
    With ``lane_groups`` the lanes of a road with two or more lanes serve
    turn groups instead: the leftmost lane left and straight, the rightmost
    lane right and straight, the lanes between straight only.  With
    ``lane_plans`` every lane keeps every turn but the junction lanes carry
    two lane plans: plan 0 all turns from every lane, plan 1 the turn groups.
    Junction lane lengths: box side W = 2 * lane_width * (max lanes of the
    junction's roads); straight W, right turn pi*W/8, left turn 3*pi*W/8.
    Signals: 4 phases (NS through+right, NS left, EW through+right, EW left),
    each ``green`` steps green then ``amber`` steps amber.
    """
    J = jxy.shape[0]
    E = links.shape[0]
    road_from = np.empty(2 * E, dtype=np.int64)
    road_to = np.empty(2 * E, dtype=np.int64)
    road_from[0::2], road_to[0::2] = links[:, 0], links[:, 1]
    road_from[1::2], road_to[1::2] = links[:, 1], links[:, 0]
    road_rev = np.arange(2 * E) ^ 1
    road_len = np.repeat(link_len, 2)
    road_lanes = np.repeat(link_lanes, 2).astype(np.int64)
    road_vmax = np.repeat(link_vmax, 2)
    R = 2 * E
    road_lane_off = np.zeros(R + 1, dtype=np.int64)
    road_lane_off[1:] = np.cumsum(road_lanes)
    n_road_lanes = int(road_lane_off[-1])

    heading = jxy[road_to] - jxy[road_from]  # grid heading of each road
    out_roads: List[List[int]] = [[] for _ in range(J)]
    for r in range(R):
        out_roads[road_from[r]].append(r)
    max_lanes_j = np.zeros(J, dtype=np.int64)
    np.maximum.at(max_lanes_j, road_from, road_lanes)
    np.maximum.at(max_lanes_j, road_to, road_lanes)

    jl_src, jl_tgt, jl_len, jl_vmax, jl_j, jl_mask, jl_turn, jl_plan = [], [], [], [], [], [], [], []
    jl_count = np.zeros(n_road_lanes, dtype=np.int64)
    for r in range(R):
        j = road_to[r]
        hin = heading[r]
        W = 2.0 * lane_width * max_lanes_j[j]
        ns = hin[1] != 0
        for i in range(road_lanes[r]):
            src = road_lane_off[r] + i
            for r2 in out_roads[j]:
                if r2 == road_rev[r]:
                    continue
                hout = heading[r2]
                cross = hin[0] * hout[1] - hin[1] * hout[0]
                if cross > 0:
                    turn, length = 1, 3.0 * math.pi * W / 8.0
                elif cross < 0:
                    turn, length = 2, math.pi * W / 8.0
                else:
                    turn, length = 0, W
                n_in = road_lanes[r]
                in_group = n_in == 1 or turn == 0 or (turn == 1 and i == 0) or (turn == 2 and i == n_in - 1)
                if lane_groups and not in_group:
                    continue
                phase = (0 if ns else 2) + (1 if turn == 1 else 0)
                tgt = road_lane_off[r2] + min(i, road_lanes[r2] - 1)
                jl_src.append(src); jl_tgt.append(tgt); jl_len.append(length)
                jl_vmax.append(min(road_vmax[r], road_vmax[r2])); jl_j.append(j)
                jl_mask.append(1 << phase); jl_turn.append(turn)
                jl_plan.append(1 | (2 if in_group else 0))
                jl_count[src] += 1
    # junction lanes are already grouped by source lane (loop order)
    jl_off = np.zeros(n_road_lanes + 1, dtype=np.int64)
    jl_off[1:] = np.cumsum(jl_count)
    jl_off += n_road_lanes
    lane_length = np.concatenate([np.repeat(road_len, road_lanes), np.array(jl_len)])
    lane_vmax = np.concatenate([np.repeat(road_vmax, road_lanes), np.array(jl_vmax)])
    junc_phase_off = np.arange(J + 1, dtype=np.int64) * 4
    net = Network(
        n_roads=R, n_road_lanes=n_road_lanes, n_lanes=n_road_lanes + len(jl_src),
        n_junctions=J, road_lane_off=_i32(road_lane_off), lane_length=_f32(lane_length),
        lane_vmax=_f32(lane_vmax), jl_off=_i32(jl_off), jl_target=_i32(jl_tgt),
        jl_junction=_i32(jl_j), jl_mask=_i32(jl_mask), junc_offset=_i32(junc_offset),
        junc_phase_off=_i32(junc_phase_off), phase_green=_i32(np.full(4 * J, green)),
        phase_amber=_i32(np.full(4 * J, amber)), road_from=_i32(road_from),
        road_to=_i32(road_to), road_reverse=_i32(road_rev), jl_turn=_i32(jl_turn),
        jl_plans=_i32(jl_plan) if lane_plans else None)
    net.validate()
    return net


def _grid_links(G: int) -> Tuple[np.ndarray, np.ndarray]:
    ii, jj = np.meshgrid(np.arange(G), np.arange(G), indexing="ij")
    jxy = np.stack([ii.ravel(), jj.ravel()], axis=1)
    idx = lambda a, b: a * G + b  # noqa: E731
    links = []
    for a in range(G):
        for b in range(G):
            if a + 1 < G:
                links.append((idx(a, b), idx(a + 1, b)))
            if b + 1 < G:
                links.append((idx(a, b), idx(a, b + 1)))
    return jxy, np.array(links, dtype=np.int64)


def grid_network(G: int, length: float = 200.0, lanes: int = 2, vmax: float = 13.89,
                 vmax_choices=None, offsets: bool = False, seed: int = 0,
                 green: int = 30, amber: int = 3, lane_groups: bool = False,
                 lane_plans: bool = False) -> Network:
    """Manhattan grid of G x G signalised junctions (configs "small"/"medium")."""
    jxy, links = _grid_links(G)
    E = len(links)
    st = Stream(seed, 101)
    if vmax_choices is None:
        lv = np.full(E, vmax)
    else:
        lv = np.asarray(vmax_choices, dtype=np.float64)[st.integers(0, len(vmax_choices), E)]
    cycle = 4 * (green + amber)
    off = st.integers(0, cycle, G * G) if offsets else np.zeros(G * G, dtype=np.int64)
    return build_network(jxy, links, np.full(E, length), np.full(E, lanes), lv, off,
                         green, amber, lane_groups=lane_groups, lane_plans=lane_plans)


def perturbed_grid_network(G: int = 100, seed: int = 0, median_len: float = 250.0,
                           sigma_ln: float = 0.4, len_clip=(50.0, 1500.0),
                           lane_probs=(0.2, 0.4, 0.3, 0.1),
                           vmax_choices=(11.1, 13.89, 16.67), green: int = 30,
                           amber: int = 3, lane_groups: bool = False) -> Network:
    """City-scale synthetic network: grid topology, log-normal link lengths
    (median 250 m, sigma_ln 0.4, clipped to [50, 1500] m), 1-4 lanes per link
    with the given probabilities, speed limits from the given set, random
    signal offsets.  G = 100 gives 39,600 one-way roads."""
    jxy, links = _grid_links(G)
    E = len(links)
    st = Stream(seed, 202)
    z = st.normal(E)
    lengths = np.clip(median_len * np.exp(sigma_ln * z), len_clip[0], len_clip[1])
    lanes = st.choice(lane_probs, E) + 1
    lv = np.asarray(vmax_choices, dtype=np.float64)[st.integers(0, len(vmax_choices), E)]
    off = st.integers(0, 4 * (green + amber), G * G)
    return build_network(jxy, links, lengths, lanes, lv, off, green, amber, lane_groups=lane_groups)


# ----------------------------------------------------------------------------
# Demand
# ----------------------------------------------------------------------------
def _line_graph(net: Network):
    import scipy.sparse as sp
    R = net.n_roads
    src, dst = [], []
    by_from = [[] for _ in range(net.n_junctions)]
    for r in range(R):
        by_from[int(net.road_from[r])].append(r)
    for r in range(R):
        for r2 in by_from[int(net.road_to[r])]:
            if r2 != net.road_reverse[r]:
                src.append(r); dst.append(r2)
    src = np.array(src); dst = np.array(dst)
    first_lane = net.road_lane_off[:-1]
    t_free = net.lane_length[first_lane].astype(np.float64) / net.lane_vmax[first_lane]
    # tiny deterministic perturbation so that shortest paths are unique
    h = _shr(_mix64(np.arange(R, dtype=np.uint64) + np.uint64(7)), 11).astype(
        np.float64) * (2.0 ** -53)
    w = t_free * (1.0 + 1e-6 * h)
    # reversed graph: edge r2 -> r with the cost of entering r2
    return sp.csr_matrix((w[dst], (dst, src)), shape=(R, R))


_WALK_LIB = None


def _walk_lib():
    """The optional compiled route walker (built by ``__graft_entry__.build``)."""
    global _WALK_LIB
    if _WALK_LIB is None:
        import ctypes
        import os
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_route_walk.so")
        _WALK_LIB = False
        if os.path.exists(path):
            try:
                lib = ctypes.CDLL(path)
                lib.moss_gen_walk.restype = ctypes.c_int
                lib.moss_gen_succ.restype = ctypes.c_int
                _WALK_LIB = lib
            except OSError:
                _WALK_LIB = False
    return _WALK_LIB


def _walk(pred, ds, sel, origins, row_all, lengths=None, routes=None, route_off=None):
    """Follow successor pointers from each origin to its destination; either
    count route lengths or write the road sequence."""
    lib = _walk_lib()
    if lib:
        import ctypes
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        sel64 = np.ascontiguousarray(sel, dtype=np.int64)
        org = np.ascontiguousarray(origins, dtype=np.int64)
        rows = np.ascontiguousarray(row_all, dtype=np.int64)
        dsa = np.ascontiguousarray(ds, dtype=np.int64)
        pr = np.ascontiguousarray(pred, dtype=np.int32)
        mode = 0 if routes is None else 1
        dummy64 = np.zeros(1, dtype=np.int64)
        dummy32 = np.zeros(1, dtype=np.int32)
        rc = lib.moss_gen_walk(
            ctypes.c_int(mode), ctypes.c_int64(len(sel64)), P(sel64), P(org), P(rows), P(dsa),
            P(pr), ctypes.c_int64(pr.shape[1]), ctypes.c_int64(pr.shape[1] + 1),
            P(lengths if lengths is not None else dummy64),
            P(route_off if route_off is not None else dummy64),
            P(routes if routes is not None else dummy32))
        assert rc == 0, "unreachable destination"
        return
    idx = sel
    cur = origins[sel].astype(np.int64)
    row = row_all[sel]
    pos = route_off[sel].copy() if routes is not None else None
    k = 1
    while idx.size:
        if routes is not None:
            routes[pos] = cur
        done = cur == ds[row]
        if lengths is not None and done.any():
            lengths[idx[done]] = k
        keep = ~done
        idx, cur, row = idx[keep], cur[keep], row[keep]
        if routes is not None:
            pos = pos[keep] + 1
        cur = pred[row, cur].astype(np.int64)
        assert np.all(cur >= 0), "unreachable destination"
        k += 1


def _successors(A, ds: np.ndarray) -> np.ndarray:
    """Rows of next-road pointers towards each destination in ds (reversed
    graph A): the compiled multithreaded Dijkstra when built, else scipy."""
    lib = _walk_lib()
    if lib:
        import ctypes
        import os
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        indices = np.ascontiguousarray(A.indices, dtype=np.int32)
        w = np.ascontiguousarray(A.data, dtype=np.float64)
        d = np.ascontiguousarray(ds, dtype=np.int64)
        succ = np.empty((len(d), A.shape[0]), dtype=np.int32)
        rc = lib.moss_gen_succ(ctypes.c_int(A.shape[0]), P(indptr), P(indices), P(w),
                               ctypes.c_int(len(d)), P(d), P(succ),
                               ctypes.c_int(max(1, min(32, os.cpu_count() or 1))))
        assert rc == 0, "route generation failed"
        return succ
    import scipy.sparse.csgraph as cg
    _, pred = cg.dijkstra(A, indices=ds, return_predecessors=True)
    return pred


def shortest_routes(net: Network, origins: np.ndarray, dests: np.ndarray,
                    chunk: int = 1024, keep_max: int = 4096) -> Tuple[np.ndarray, np.ndarray]:
    """Free-flow-time shortest routes (road sequences, origin..destination)
    on the road graph without U-turns.  Returns CSR (route_off, routes).
    Successor rows of up to ``keep_max`` destinations are kept between the
    length pass and the fill pass; beyond that they are recomputed."""
    A = _line_graph(net)
    n = len(origins)
    uniq, inv = np.unique(dests, return_inverse=True)
    order = np.argsort(inv, kind="stable")
    bounds = np.searchsorted(inv[order], np.arange(0, len(uniq) + chunk, chunk))
    keep = len(uniq) <= keep_max
    lengths = np.zeros(n, dtype=np.int64)
    chunks = []
    for ci, c0 in enumerate(range(0, len(uniq), chunk)):
        ds = uniq[c0:c0 + chunk].astype(np.int64)
        pred = _successors(A, ds)
        sel = order[bounds[ci]:bounds[ci + 1]]
        _walk(pred, ds, sel, origins, inv - c0, lengths=lengths)
        chunks.append((ds, pred if keep else None, sel, c0))
    route_off = np.zeros(n + 1, dtype=np.int64)
    route_off[1:] = np.cumsum(lengths)
    routes = np.empty(int(route_off[-1]), dtype=np.int32)
    for ds, pred, sel, c0 in chunks:
        if pred is None:
            pred = _successors(A, ds)
        _walk(pred, ds, sel, origins, inv - c0, routes=routes, route_off=route_off)
    return _i32(route_off), routes


def random_demand(net: Network, n: int, dep_horizon: int, seed: int = 0,
                  dest_pool: Optional[int] = None, v0_sigma: float = 0.1,
                  v0_clip=(0.7, 1.3)) -> Vehicles:
    """n trips: origin road uniform, destination road uniform (from a pool of
    ``dest_pool`` roads when given), distinct; shortest free-flow-time route;
    start lane uniform on the origin road; departure step uniform in
    [0, dep_horizon); desired-speed factor ~ N(1, v0_sigma) clipped."""
    st = Stream(seed, 303)
    R = net.n_roads
    if dest_pool is None or dest_pool >= R:
        dests = st.integers(0, R, n)
    else:
        pool = np.unique(st.integers(0, R, dest_pool))
        dests = pool[st.integers(0, len(pool), n)]
    origins = st.integers(0, R - 1, n)
    origins = origins + (origins >= dests)  # distinct from destination
    route_off, routes = shortest_routes(net, origins, dests)
    nl = np.diff(net.road_lane_off)[origins]
    start_lane = net.road_lane_off[origins] + (st.uniform(n) * nl).astype(np.int64)
    dep = st.integers(0, max(dep_horizon, 1), n)
    v0f = np.clip(1.0 + v0_sigma * st.normal(n), v0_clip[0], v0_clip[1])
    veh = Vehicles(n=n, route_off=route_off, routes=routes, start_lane=_i32(start_lane),
                   dep=_i32(dep), v0f=_f32(v0f))
    veh.validate(net)
    return veh


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------
def small_scenario(seed: int = 0) -> Scenario:
    """4x4 grid, 200 m two-lane roads at 13.89 m/s, 4-phase 30/3 s signals with
    offset 0, 1,000 trips departing uniformly over the first 300 s."""
    net = grid_network(4, 200.0, 2, 13.89, offsets=False, seed=seed)
    veh = random_demand(net, 1000, 300, seed=seed)
    return Scenario(net, veh, Params(seed=seed), "grid4x4_1k")


def small_groups_scenario(seed: int = 0) -> Scenario:
    """4x4 grid of 200 m three-lane roads whose lanes serve turn groups (left
    lane: left + straight, middle: straight, right lane: right + straight),
    1,500 trips departing over the first 300 s."""
    net = grid_network(4, 200.0, 3, 13.89, offsets=False, seed=seed, lane_groups=True)
    veh = random_demand(net, 1500, 300, seed=seed)
    return Scenario(net, veh, Params(seed=seed), "grid4x4_groups_1500")


def medium_scenario(seed: int = 0, n: int = 100_000) -> Scenario:
    """30x30 grid, 300 m three-lane roads, limits from {11.1, 13.89, 16.67} m/s,
    random signal offsets, 100,000 trips departing uniformly over 1,800 s."""
    net = grid_network(30, 300.0, 3, vmax_choices=(11.1, 13.89, 16.67), offsets=True,
                       seed=seed)
    veh = random_demand(net, n, 1800, seed=seed)
    return Scenario(net, veh, Params(seed=seed), "grid30x30_100k")


def city_scenario(seed: int = 0, n: int = 2_464_950, G: int = 100,
                  dest_pool: Optional[int] = 1024, dep_horizon: int = 3600,
                  lane_groups: bool = False) -> Scenario:
    """Perturbed 100x100 grid (39,600 roads, 1-4 lanes, log-normal lengths) with
    2,464,950 trips departing uniformly over 3,600 s; origins uniform over all
    roads, destinations uniform over a pool of 1,024 roads (trip attractors;
    it also bounds the shortest-path work to 1,024 Dijkstra runs)."""
    net = perturbed_grid_network(G, seed=seed, lane_groups=lane_groups)
    veh = random_demand(net, n, dep_horizon, seed=seed, dest_pool=dest_pool)
    return Scenario(net, veh, Params(seed=seed), f"city{G}x{G}_{n}" + ("_groups" if lane_groups else ""))


def saturated_city(seed: int = 0, n: int = 2_464_950, G: int = 100, hops: int = 24,
                   v0_sigma: float = 0.1, v0_clip=(0.7, 1.3)):
    """The city network with all n trips on the road at once (a measurement
    state, not a rollout): every road lane holds a share of the n vehicles in
    proportion to its length (largest remainders), evenly spaced; that is
    about 10 m per vehicle, the spacing at which n vehicles fit on the
    network.  Each vehicle drives at the speed whose IDM safe distance
    s0 + v T equals its gap (capped by its desired speed).  A trip's route
    starts on the road it stands on and continues for `hops` roads by a
    seeded random walk over the turns its junction lanes offer (ending early
    at a road without one).  Returns (scenario, state) where state is
    (status, lane, s, v, rc) for ``set_state`` at step 0."""
    net = perturbed_grid_network(G, seed=seed)
    prm = Params(seed=seed)
    st = Stream(seed, 606)
    NRL = net.n_road_lanes
    L = net.lane_length[:NRL].astype(np.float64)
    q = L / L.sum() * n
    cnt = np.floor(q).astype(np.int64)
    rest = n - int(cnt.sum())
    cnt[np.argsort(-(q - cnt), kind="stable")[:rest]] += 1
    lane = np.repeat(np.arange(NRL, dtype=np.int64), cnt)
    rank = np.arange(n) - np.repeat(np.cumsum(cnt) - cnt, cnt)  # 0 = front of the lane
    spacing = np.repeat(L / np.maximum(cnt, 1), cnt)
    s = np.repeat(L, cnt) - (rank + 0.5) * spacing
    v0f = np.clip(1.0 + v0_sigma * st.normal(n), v0_clip[0], v0_clip[1])
    vmax = net.lane_vmax[:NRL].astype(np.float64)[lane]
    v = np.clip((spacing - prm.veh_len - prm.s0) / prm.T, 0.0, v0f * vmax)
    # turns per road: the roads that the junction lanes of its lanes feed
    rl = net.lane_road()
    src = np.repeat(rl[:NRL], np.diff(net.jl_off))
    dst = rl[net.jl_target]
    pairs = np.unique(np.stack([src, dst], axis=1), axis=0)
    out_off = np.zeros(net.n_roads + 1, dtype=np.int64)
    np.add.at(out_off, pairs[:, 0] + 1, 1)
    out_off = np.cumsum(out_off)
    out_road = pairs[:, 1]
    road = rl[lane].astype(np.int64)
    routes = np.full((n, hops + 1), -1, dtype=np.int64)
    routes[:, 0] = road
    alive = np.ones(n, dtype=bool)
    cur = road.copy()
    for h in range(1, hops + 1):
        deg = out_off[cur + 1] - out_off[cur]
        alive &= deg > 0
        pick = (st.uniform(n) * np.maximum(deg, 1)).astype(np.int64)
        nxt = out_road[np.minimum(out_off[cur] + pick, len(out_road) - 1)]
        cur = np.where(alive, nxt, cur)
        routes[:, h] = np.where(alive, cur, -1)
    rlen = (routes >= 0).sum(axis=1)
    route_off = np.concatenate([[0], np.cumsum(rlen)])
    veh = Vehicles(n=n, route_off=_i32(route_off), routes=_i32(routes[routes >= 0]),
                   start_lane=_i32(lane), dep=_i32(np.zeros(n)), v0f=_f32(v0f))
    state = (np.ones(n, dtype=np.int32), _i32(lane), s, v, np.zeros(n, dtype=np.int32))
    return Scenario(net, veh, prm, f"city{G}x{G}_saturated_{n}"), state


def batched_scenarios(k: int = 64, seed: int = 0, n_lo: int = 2000, n_hi: int = 300_000,
                      dep_horizon: int = 1800, only=None) -> List[Scenario]:
    """k independent grid scenarios of uneven size: vehicles log-uniform in
    [n_lo, n_hi], grid side 5..40 grown with the vehicle count, medium-style
    roads, own seed and signal offsets.  `only` (indices) builds just those
    scenarios of the set, identical to the ones of the full set."""
    st = Stream(seed, 404)
    u = st.uniform(k)
    ns = np.round(np.exp(np.log(n_lo) + u * (np.log(n_hi) - np.log(n_lo)))).astype(np.int64)
    out = []
    keep = set(range(k)) if only is None else set(int(i) for i in only)
    for i, n in enumerate(ns):
        if i not in keep:
            continue
        G = int(np.clip(round(5 * 8 ** (math.log(n / 2000.0) / math.log(150.0))), 5, 40))
        s_i = seed * 1000 + i + 1
        net = grid_network(G, 300.0, 3, vmax_choices=(11.1, 13.89, 16.67), offsets=True,
                           seed=s_i)
        veh = random_demand(net, int(n), dep_horizon, seed=s_i)
        out.append(Scenario(net, veh, Params(seed=s_i, scenario=i), f"b{i}_g{G}_{n}"))
    return out


# ----------------------------------------------------------------------------
# Hand-built fixtures for tests
# ----------------------------------------------------------------------------
def corridor_network(n_lanes: int = 2, lengths=(1000.0, 1000.0), vmax: float = 13.89,
                     green: int = 30, amber: int = 3, offset: int = 0,
                     turn_len: float = 10.0) -> Network:
    """A straight corridor of len(lengths) roads joined by signalised junctions.
    Road k feeds road k+1 through one straight junction lane per lane (lane i
    -> lane i); junction k has a 2-phase program: phase 0 green for the
    corridor, phase 1 red for it (green/amber durations as given)."""
    R = len(lengths)
    road_lane_off = np.arange(R + 1) * n_lanes
    nrl = R * n_lanes
    jl_off = [nrl]
    jl_target, jl_junction, jl_mask, jl_len, jl_vmax = [], [], [], [], []
    for r in range(R):
        for i in range(n_lanes):
            if r + 1 < R:
                jl_target.append((r + 1) * n_lanes + i)
                jl_junction.append(r)
                jl_mask.append(1)
                jl_len.append(turn_len)
                jl_vmax.append(vmax)
            jl_off.append(nrl + len(jl_target))
    J = max(R - 1, 0)
    lane_length = np.concatenate([np.repeat(np.asarray(lengths, dtype=np.float64), n_lanes),
                                  np.asarray(jl_len, dtype=np.float64)])
    net = Network(
        n_roads=R, n_road_lanes=nrl, n_lanes=nrl + len(jl_target), n_junctions=J,
        road_lane_off=_i32(road_lane_off), lane_length=_f32(lane_length),
        lane_vmax=_f32(np.full(len(lane_length), vmax)), jl_off=_i32(jl_off),
        jl_target=_i32(jl_target), jl_junction=_i32(jl_junction), jl_mask=_i32(jl_mask),
        junc_offset=_i32(np.full(J, offset)), junc_phase_off=_i32(np.arange(J + 1) * 2),
        phase_green=_i32(np.full(2 * J, green)), phase_amber=_i32(np.full(2 * J, amber)))
    net.validate()
    return net


def corridor_vehicles(net: Network, start_lanes, deps, v0f=None, n_roads=None) -> Vehicles:
    """Vehicles driving the whole corridor from road 0 (or ``n_roads`` roads)."""
    n = len(start_lanes)
    R = net.n_roads if n_roads is None else n_roads
    route_off = np.arange(n + 1) * R
    routes = np.tile(np.arange(R), n)
    v0 = np.ones(n) if v0f is None else np.asarray(v0f)
    return Vehicles(n=n, route_off=_i32(route_off), routes=_i32(routes),
                    start_lane=_i32(start_lanes), dep=_i32(deps), v0f=_f32(v0))


# ----------------------------------------------------------------------------
# Warm-start states (inputs for measurement)
# ----------------------------------------------------------------------------
def warm_state(net: Network, veh: Vehicles, t_warm: int, spacing: float = 20.0,
               speed_frac: float = 0.8, seed: int = 0, rounds: int = 8):
    """A plausible mid-rollout state at step ``t_warm`` built directly from the
    inputs (no simulation): every trip with departure < t_warm is placed on a
    uniformly chosen road of its route and a uniform lane of that road; a lane
    holds at most floor(length / spacing) vehicles (20 m is about 35% of jam
    density for 5 m vehicles); a trip whose lane is full draws another road
    of its route, up to ``rounds`` times, and is marked finished if it never
    fits.  Vehicles of a lane are spaced evenly; speeds are speed_frac of the
    desired speed.  Trips with departure >= t_warm are waiting, so each start
    lane's queue keeps its (dep, id) order.  Returns per-vehicle arrays
    (status, lane, s, v, rc) for ``set_state``."""
    st = Stream(seed, 505)
    n = veh.n
    status = np.zeros(n, dtype=np.int32)
    lane = np.full(n, -1, dtype=np.int32)
    s = np.zeros(n, dtype=np.float64)
    v = np.zeros(n, dtype=np.float64)
    rc = np.zeros(n, dtype=np.int32)
    L = net.lane_length.astype(np.float64)
    cap = np.floor(L / spacing).astype(np.int64)
    cap[net.n_road_lanes:] = 0
    free = cap.copy()
    todo = np.nonzero(veh.dep < t_warm)[0]
    status[todo] = 2
    for _ in range(rounds):
        if todo.size == 0:
            break
        rlen = np.diff(veh.route_off)[todo]
        k = (st.uniform(len(todo)) * rlen).astype(np.int64)
        road = veh.routes[veh.route_off[todo] + k]
        nl = np.diff(net.road_lane_off)[road]
        ln = net.road_lane_off[road] + (st.uniform(len(todo)) * nl).astype(np.int64)
        order = np.lexsort((todo, ln))
        ids, ln, k = todo[order], ln[order], k[order]
        first = np.searchsorted(ln, ln, side="left")
        rank = np.arange(len(ids)) - first
        fits = rank < free[ln]
        a = ids[fits]
        status[a] = 1
        lane[a] = ln[fits]
        rc[a] = k[fits]
        np.subtract.at(free, ln[fits], 1)
        todo = np.sort(ids[~fits])
    act = np.nonzero(status == 1)[0]
    la = lane[act]
    order = np.lexsort((act, la))
    act, la = act[order], la[order]
    first = np.searchsorted(la, la, side="left")
    rank = np.arange(len(act)) - first
    m = (cap - free)[la]
    s[act] = L[la] * (m - rank) / (m + 1.0)
    v[act] = speed_frac * veh.v0f[act].astype(np.float64) * net.lane_vmax[la].astype(np.float64)
    s = s.astype(np.float32).astype(np.float64)
    v = v.astype(np.float32).astype(np.float64)
    return dict(status=status, lane=lane, s=s, v=v, rc=rc)


def vehicle_subset(veh: Vehicles, idx: np.ndarray) -> Vehicles:
    """The trips idx (sorted) of ``veh`` as a trip set of their own (new ids
    0..len(idx)-1 in the same order)."""
    idx = np.asarray(idx, dtype=np.int64)
    lens = np.diff(veh.route_off).astype(np.int64)[idx]
    off = np.concatenate([[0], np.cumsum(lens)])
    pos = np.repeat(veh.route_off[idx].astype(np.int64) - off[:-1], lens) + np.arange(off[-1])
    return Vehicles(n=len(idx), route_off=_i32(off), routes=_i32(veh.routes[pos]),
                    start_lane=_i32(veh.start_lane[idx]), dep=_i32(veh.dep[idx]), v0f=_f32(veh.v0f[idx]))


def region_band(state: dict, net: Network, veh: Vehicles, lo: int, hi: int):
    """The part of ``state`` that belongs to roads [lo, hi): the vehicles
    active on a lane of such a road (on a junction lane: of the road it
    leads to) and the waiting ones whose start lane is on one, as a trip set
    of their own with its state (so that a simulator holding only this band
    does work in proportion to it).  Bands that partition the road ids
    partition the active and waiting vehicles.  Returns (vehicles, state)."""
    lr = net.lane_road()
    lr[net.n_road_lanes:] = lr[net.jl_target]
    st, ln = state["status"], state["lane"]
    road = lr[np.maximum(ln, 0)]
    keep_a = (st == 1) & (road >= lo) & (road < hi)
    sroad = lr[veh.start_lane]
    keep_w = (st == 0) & (sroad >= lo) & (sroad < hi)
    idx = np.nonzero(keep_a | keep_w)[0]
    sub = {k: np.array(x)[idx].copy() for k, x in state.items()}
    return vehicle_subset(veh, idx), sub


