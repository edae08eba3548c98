"""Lane setters (reading R25) and lane/road metrics (reading R24) on the GPU
against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2406_10661_gb300 import binding, scenario as sc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    binding.load()


def test_metrics_match_oracle_medium():
    """Queue lengths (exact) and road speeds on a congested medium-grid state."""
    scen = sc.medium_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=32)
    sim.step(900)
    st = sim.state()
    ora = oracle.Oracle(scen.net, scen.veh, scen.params)
    ora.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], 900)
    gq, rq = sim.lane_queue(), ora.lane_queue()
    assert gq.sum() > 100  # the state has queues
    assert np.array_equal(gq, rq), np.nonzero(gq != rq)[0][:10]
    gs, rs = sim.road_speed(), ora.road_speed()
    assert np.allclose(gs, rs, rtol=1e-12, atol=1e-12), np.abs(gs - rs).max()


def test_batch_metrics_equal_alone():
    scens = [sc.small_scenario(seed=s) for s in (1, 2)]
    batch = binding.Batch(scens, precision=32)
    batch.step(200)
    for i, s_ in enumerate(scens):
        sim = binding.Simulation(s_.net, s_.veh, s_.params, precision=32)
        sim.step(200)
        assert np.array_equal(batch.lane_queue(i), sim.lane_queue())
        assert np.array_equal(batch.road_speed(i), sim.road_speed())
        sim.close()
    batch.close()


def test_fp64_rollout_with_lane_setters():
    """Restricted lanes (road and junction lanes) and changed speed limits
    during a rollout: vehicle states identical to the oracle's."""
    scen = sc.small_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=64)
    ora = oracle.Oracle(scen.net, scen.veh, scen.params)
    rng = np.random.default_rng(3)
    nrl, nl = scen.net.n_road_lanes, scen.net.n_lanes
    restricted = np.concatenate([rng.choice(nrl, 6, replace=False), nrl + rng.choice(nl - nrl, 8, replace=False)])
    limits = rng.choice(nrl, 10, replace=False)
    new_v = rng.uniform(5.0, 20.0, 10).astype(np.float32)
    for t0 in (0, 100, 250):
        if t0:
            sim.step(t0 - sim.metrics()["step"]); ora.step(t0 - int(ora.metrics()["step"]))
        if t0 == 0:
            sim.set_lane_restriction(restricted, np.ones(len(restricted)))
            ora.set_lane_restriction(restricted, np.ones(len(restricted)))
        elif t0 == 100:
            sim.set_lane_max_speed(limits, new_v)
            ora.set_lane_max_speed(limits, new_v.astype(np.float64))
        else:  # lift half of the restrictions
            half = restricted[::2]
            sim.set_lane_restriction(half, np.zeros(len(half)))
            ora.set_lane_restriction(half, np.zeros(len(half)))
    sim.step(150); ora.step(150)
    g, r = sim.state(), ora.state()
    assert np.array_equal(g["status"], r["status"])
    act = r["status"] == 1
    assert np.array_equal(g["lane"][act], r["lane"][act])
    assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6
    assert np.abs(g["v"][act] - r["v"][act]).max(initial=0) < 1e-6
    assert np.array_equal(g["flags"], r["flags"])
    gm, rm = sim.metrics(), ora.metrics()
    for k in ("n_arrived", "vehicle_updates", "lane_changes", "inserted"):
        assert gm[k] == rm[k], (k, gm[k], rm[k])
    # nobody entered a lane while it was restricted: the still-restricted
    # lanes hold no vehicle that was not already there (none at step 0)
    still = restricted[1::2]
    assert not np.isin(g["lane"][act], still).any()


def test_lane_setters_reject_bad_input():
    scen = sc.small_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=32)
    with pytest.raises(binding.MossError):
        sim.set_lane_max_speed([0], [0.0])
    with pytest.raises(binding.MossError):
        sim.set_lane_restriction([scen.net.n_lanes], [1])


def _cut_routes(scen, st, cur, rng, k):
    """Sub-paths of the vehicles' remaining routes (always valid re-routes):
    waiting -> a prefix of the route; on a road -> from the current road; on
    a junction lane -> from the road it enters.  cur[g] is vehicle g's stored
    route (the state's route cursor indexes it)."""
    nrl = scen.net.n_road_lanes
    cand = np.nonzero(st["status"] != 2)[0]
    vids = rng.choice(cand, min(k, len(cand)), replace=False)
    out = []
    for g in vids:
        r = cur[g]
        if st["status"][g] == 0:
            first = 0
        elif st["lane"][g] < nrl:
            first = st["rc"][g]
        else:
            first = st["rc"][g] + 1
        rest = r[first:]
        out.append(rest[:max(1, int(rng.integers(1, len(rest) + 1)))])
    return vids, out


def _stored(st, nrl, g, r, cur):
    """The route the simulators keep after re-routing g to r (reading R26):
    on a junction lane the road just left stays in front."""
    if st["status"][g] == 1 and st["lane"][g] >= nrl:
        return [cur[g][st["rc"][g]]] + list(r)
    return list(r)


def test_fp64_rollout_with_reroutes():
    """Reading R26: routes cut for waiting vehicles, vehicles on roads and on
    junction lanes, in several rounds (the route buffer grows and the step
    graphs are recaptured); states identical to the oracle's."""
    scen = sc.small_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=64)
    ora = oracle.Oracle(scen.net, scen.veh, scen.params)
    rng = np.random.default_rng(11)
    ro, roads = scen.veh.route_off, scen.veh.routes
    nrl = scen.net.n_road_lanes
    cur = {g: roads[ro[g]:ro[g + 1]].tolist() for g in range(scen.veh.n)}
    for rnd in range(14):
        sim.step(25); ora.step(25)
        st = ora.state()
        vids, routes = _cut_routes(scen, st, cur, rng, 400)
        sim.set_vehicle_route(vids, routes)
        for g, r in zip(vids, routes):
            assert ora.set_vehicle_route(int(g), r)
            cur[g] = _stored(st, nrl, g, r, cur)
        # the original routes again for everyone waiting, three times: every
        # call appends, so the device route buffer (64k spare entries here)
        # has to grow and the step graphs are captured again
        wait = np.nonzero(ora.state()["status"] == 0)[0]
        for _ in range(3 if len(wait) else 0):
            again = [roads[ro[g]:ro[g + 1]].tolist() for g in wait]
            sim.set_vehicle_route(wait, again)
            for g, r in zip(wait, again):
                assert ora.set_vehicle_route(int(g), r)
                cur[g] = list(r)
    sim.step(100); ora.step(100)
    g, r = sim.state(), ora.state()
    assert np.array_equal(g["status"], r["status"])
    act = r["status"] == 1
    assert np.array_equal(g["lane"][act], r["lane"][act])
    assert np.array_equal(g["rc"][act], r["rc"][act])
    assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6
    assert np.abs(g["v"][act] - r["v"][act]).max(initial=0) < 1e-6
    gm, rm = sim.metrics(), ora.metrics()
    for k in ("n_arrived", "vehicle_updates", "lane_changes", "inserted", "errors"):
        assert gm[k] == rm[k], (k, gm[k], rm[k])
    assert abs(gm["tt_sum"] - rm["tt_sum"]) < 1e-9


def test_reroute_refusals_change_nothing():
    scen = sc.small_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=32)
    sim.step(50)
    before = sim.state()
    ro, roads = scen.veh.route_off, scen.veh.routes
    g = int(np.nonzero(before["status"] == 1)[0][0])
    bad_first = [int(roads[ro[g + 1] - 1])] if ro[g + 1] - ro[g] > 1 else [int((roads[ro[g]] + 1) % scen.net.n_roads)]
    w = int(np.nonzero(before["status"] == 0)[0][0])
    for vids, routes in (([g], [bad_first]), ([w, w], [[int(roads[ro[w]])]] * 2), ([10 ** 7], [[0]])):
        with pytest.raises(binding.MossError):
            sim.set_vehicle_route(vids, routes)
    sim.step(10)
    sim2 = binding.Simulation(scen.net, scen.veh, scen.params, precision=32)
    sim2.step(60)
    a, b = sim.state(), sim2.state()
    assert np.array_equal(a["status"], b["status"]) and np.array_equal(a["lane"], b["lane"])
