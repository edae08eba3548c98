"""Seeded input generators: the saturated city state (every trip on the road
at once) has the structure its docstring states, and the oracle steps from it
without overlaps or lost vehicles."""
import numpy as np

import oracle
from paper_2406_10661_gb300 import scenario as sc


def _small():
    return sc.saturated_city(seed=3, n=20_000, G=10, hops=6)


def test_saturated_state_structure():
    scen, (status, lane, s, v, rc) = _small()
    net, veh, prm = scen.net, scen.veh, scen.params
    net.validate()
    veh.validate(net)
    n = veh.n
    assert n == 20_000 and (status == 1).all() and (rc == 0).all()
    L = net.lane_length.astype(np.float64)
    # every vehicle on a road lane of its first route road, inside the lane
    rl = net.lane_road()
    assert (lane < net.n_road_lanes).all()
    assert (rl[lane] == veh.routes[veh.route_off[:-1]]).all()
    assert ((s > 0) & (s < L[lane])).all()
    # per-lane counts follow lane length (largest remainders) and sum to n
    cnt = np.bincount(lane, minlength=net.n_road_lanes)
    share = L[: net.n_road_lanes] / L[: net.n_road_lanes].sum() * n
    assert cnt.sum() == n and (np.abs(cnt - share) < 1.0).all()
    # evenly spaced, gaps > vehicle length + s0 is not required but gaps > 0 are
    order = np.lexsort((-s, lane))
    same = lane[order][1:] == lane[order][:-1]
    gaps = s[order][:-1] - s[order][1:] - prm.veh_len
    assert (gaps[same] > 0).all()
    # speeds: the IDM equilibrium for the gap, within [0, desired speed]
    v0 = veh.v0f.astype(np.float64) * net.lane_vmax[lane]
    assert ((v >= 0) & (v <= v0 + 1e-9)).all()
    # routes: consecutive roads joined by a junction lane of the earlier road
    src = np.repeat(rl[: net.n_road_lanes], np.diff(net.jl_off))
    turns = set(zip(src.tolist(), rl[net.jl_target].tolist()))
    for i in range(0, n, 997):
        r = veh.routes[veh.route_off[i]:veh.route_off[i + 1]]
        assert all((int(a), int(b)) in turns for a, b in zip(r[:-1], r[1:]))
    # reproducible
    _, (_, lane2, s2, v2, _) = _small()
    assert np.array_equal(lane, lane2) and np.array_equal(s, s2) and np.array_equal(v, v2)


def test_oracle_steps_from_saturated_state():
    scen, (status, lane, s, v, rc) = _small()
    o = oracle.Oracle(scen.net, scen.veh, scen.params)
    o.set_state(status, lane, s, v, rc, 0)
    o.step(3)
    st = o.state()
    m = o.metrics()
    assert m["n_active"] + m["n_arrived"] == scen.veh.n
    assert m["errors"] == 0 and m["vehicle_updates"] == 3 * scen.veh.n
    act = st["status"] == 1
    L = scen.net.lane_length.astype(np.float64)
    assert ((st["s"][act] >= 0) & (st["s"][act] <= L[st["lane"][act]])).all()
    # (vehicles that reach the same road lane from two junction lanes in one
    # step may overlap: the model has no merge rule, the overlap metric counts
    # them, so no gap bound is asserted here)


def test_region_bands_partition_the_state():
    """Bands of road ids partition the active and waiting vehicles; each band
    is a trip set of its own with the same routes, start lanes and state."""
    scen = sc.small_scenario()
    o = oracle.Oracle(scen.net, scen.veh, scen.params)
    o.step(150)
    st = o.state()
    st = {k: st[k] for k in ("status", "lane", "s", "v", "rc")}
    net, veh = scen.net, scen.veh
    bounds = [0, 10, 25, 48]
    seen = []
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        sub_veh, sub = sc.region_band(st, net, veh, lo, hi)
        sub_veh.validate(net)
        assert sub_veh.n == len(sub["status"])
        assert set(np.unique(sub["status"]).tolist()) <= {0, 1}
        # the band's trips, in id order, with their own routes
        keep = []
        lane_road = net.lane_road()
        for i in range(veh.n):
            ln = st["lane"][i]
            if st["status"][i] == 1 and ln < net.n_road_lanes:
                road = lane_road[ln]
            elif st["status"][i] == 1:  # junction lane: the road it leads to
                road = lane_road[net.jl_target[ln - net.n_road_lanes]]
            elif st["status"][i] == 0:
                road = net.lane_road()[veh.start_lane[i]]
            else:
                continue
            if lo <= road < hi:
                keep.append(i)
        assert len(keep) == sub_veh.n
        for j, i in enumerate(keep):
            assert np.array_equal(sub_veh.routes[sub_veh.route_off[j]:sub_veh.route_off[j + 1]],
                                  veh.routes[veh.route_off[i]:veh.route_off[i + 1]])
            assert sub_veh.start_lane[j] == veh.start_lane[i] and sub_veh.dep[j] == veh.dep[i]
            for k in st:
                assert sub[k][j] == st[k][i]
        seen += keep
    live = np.nonzero(st["status"] <= 1)[0]
    assert sorted(seen) == live.tolist()
    assert ((st["status"] == 1) & (st["lane"] >= net.n_road_lanes)).any()  # junction lanes covered


def test_oracle_bands_lockstep_equals_serial():
    """The all-cores CPU baseline: bands stepped together in threads give the
    same vehicle updates as the same band oracles stepped one after another;
    a band that fails ends the run with an error instead of stalling it."""
    import pytest
    bench = pytest.importorskip("bench")
    scen, (status, lane, s, v, rc) = _small()
    state = {"status": status, "lane": lane, "s": s, "v": v, "rc": rc}
    pool = bench.OracleBands(scen, state, 0, n=3)
    try:
        for _ in range(4):
            pool.step()
        par = [o.metrics() for o in pool.orcs]
    finally:
        pool.close()
    bounds = np.linspace(0, scen.net.n_roads, 4).astype(np.int64)
    for k in range(3):
        veh, smp = sc.region_band(state, scen.net, scen.veh, int(bounds[k]), int(bounds[k + 1]))
        o = oracle.Oracle(scen.net, veh, scen.params)
        o.set_state(smp["status"], smp["lane"], smp["s"], smp["v"], smp["rc"], 0)
        o.step(4)
        m = o.metrics()
        assert m["vehicle_updates"] == par[k]["vehicle_updates"] and m["n_active"] == par[k]["n_active"]
    assert sum(m["vehicle_updates"] for m in par) == 4 * scen.veh.n

    pool = bench.OracleBands(scen, state, 0, n=2)

    def planted(n):
        raise ValueError("planted")

    pool.orcs[1].step = planted
    with pytest.raises(RuntimeError, match="planted"):
        pool.step()
    pool.close()
