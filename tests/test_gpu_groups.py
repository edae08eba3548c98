"""Lane groups (reading R27) on the GPU against the FP64 oracle: a grid of
three-lane roads whose lanes serve turn groups (left lane left + straight,
middle straight, right lane right + straight)."""
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


def test_fp64_rollout_lane_groups():
    scen = sc.small_groups_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=64)
    ora = oracle.Oracle(scen.net, scen.veh, scen.params)
    for chunk in range(8):
        sim.step(75); ora.step(75)
        g, r = sim.state(), ora.state()
        assert np.array_equal(g["status"], r["status"])
        act = r["status"] == 1
        assert np.array_equal(g["lane"][act], r["lane"][act])
        assert np.array_equal(g["rc"][act], r["rc"][act])
        assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6
        assert np.abs(g["v"][act] - r["v"][act]).max(initial=0) < 1e-6
        assert np.array_equal(g["flags"], r["flags"])
    gm, rm = sim.metrics(), ora.metrics()
    for k in ("n_arrived", "vehicle_updates", "lane_changes", "flagged", "overlaps", "inserted", "mobil_evals",
              "errors"):
        assert gm[k] == rm[k], (k, gm[k], rm[k])
    assert gm["lane_changes"] > 0 and gm["n_arrived"] > 0 and gm["errors"] == 0


def test_fp32_one_step_parity_lane_groups():
    scen = sc.small_groups_scenario()
    ora = oracle.Oracle(scen.net, scen.veh, scen.params)
    ora.step(240)
    st = ora.state()
    st["s"] = st["s"].astype(np.float32).astype(np.float64)
    st["v"] = st["v"].astype(np.float32).astype(np.float64)
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=32)
    ora2 = oracle.Oracle(scen.net, scen.veh, scen.params)
    for o in (sim, ora2):
        o.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], 240)
    sim.step(1); ora2.step(1)
    g, r = sim.state(), ora2.state()
    flagged = ((g["flags"] | r["flags"]) & binding.F_FLAGGED) != 0
    disc = (g["status"] != r["status"]) | ((r["status"] == 1) & (g["lane"] != r["lane"]))
    assert not (disc & ~flagged).any()
    ok = ~disc & (r["status"] == 1)
    for k in ("s", "v"):
        err = np.abs(g[k][ok] - r[k][ok]) / np.maximum(np.abs(r[k][ok]), 1.0)
        assert (err <= 1e-5).all(), (k, float(err.max()))


def test_fp64_rollout_lane_plan_switches():
    """Reading R28: roads switch between their two lane plans (all turns from
    every lane / turn groups) during the rollout; identical to the oracle."""
    net = sc.grid_network(4, 200.0, 3, 13.89, lane_plans=True)
    veh = sc.random_demand(net, 1500, 300, seed=3)
    scen = sc.Scenario(net, veh, sc.Params(seed=3), "plans")
    sim = binding.Simulation(net, veh, scen.params, precision=64)
    ora = oracle.Oracle(net, veh, scen.params)
    rng = np.random.default_rng(8)
    for chunk in range(8):
        roads = rng.choice(net.n_roads, net.n_roads // 2, replace=False)
        plans = rng.integers(0, 2, len(roads))
        sim.set_road_lane_plan(roads, plans)
        ora.set_road_plan(roads, plans)
        sim.step(60); ora.step(60)
        g, r = sim.state(), ora.state()
        assert np.array_equal(g["status"], r["status"]), chunk
        act = r["status"] == 1
        assert np.array_equal(g["lane"][act], r["lane"][act]), chunk
        assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6
        assert np.abs(g["v"][act] - r["v"][act]).max(initial=0) < 1e-6
        assert np.array_equal(g["flags"], r["flags"])
    gm, rm = sim.metrics(), ora.metrics()
    for k in ("n_arrived", "vehicle_updates", "lane_changes", "flagged", "inserted", "errors"):
        assert gm[k] == rm[k], (k, gm[k], rm[k])
    assert gm["errors"] == 0
