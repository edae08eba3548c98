"""CUDA path (through the C ABI) against the FP64 oracle.

Levels (tolerances from the method's specification):
  * FP64 kernels vs oracle over whole rollouts: identical discrete state,
    positions/speeds within 1e-6;
  * FP32 kernels vs oracle for one step from an identical state: identical
    discrete decisions except where either side flags the vehicle (a decision
    quantity within 1e-4 of its threshold), positions/speeds within
    1e-5 * max(|x|, 1);
  * FP32 rollouts: network speed and trip completions within 0.5%;
  * a batch equals its scenarios run alone.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from handmade import corridor, one_road
from paper_2406_10661_gb300 import binding, scenario as sc

pytestmark = pytest.mark.gpu

REL = 1e-5
DISCRETE_FLAGS = (binding.F_CHANGED | binding.F_TRANSFER | binding.F_ARRIVED | binding.F_INSERTED)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    binding.load()


def _sim(scen, precision=32):
    return binding.Simulation(scen.net, scen.veh, scen.params, precision=precision)


def _ora(scen):
    return oracle.Oracle(scen.net, scen.veh, scen.params)


def _set_both(sim, ora, st, step):
    sim.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], step)
    ora.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], step)


def _f32_state(st):
    out = {k: np.array(v, copy=True) for k, v in st.items()}
    out["s"] = out["s"].astype(np.float32).astype(np.float64)
    out["v"] = out["v"].astype(np.float32).astype(np.float64)
    return out


def compare_one_step(g, r, tol=REL):
    """Per-vehicle comparison after one step; returns (n_compared, n_excused)."""
    flagged = ((g["flags"] | r["flags"]) & binding.F_FLAGGED) != 0
    act = (g["status"] == 1) | (r["status"] == 1)
    disc = ((g["status"] != r["status"]) | (act & ((g["lane"] != r["lane"]) | (g["rc"] != r["rc"])))
            | ((g["flags"] & DISCRETE_FLAGS) != (r["flags"] & DISCRETE_FLAGS)))
    bad = disc & ~flagged
    assert not bad.any(), f"unflagged discrete mismatch at ids {np.nonzero(bad)[0][:10]}"
    ok = ~disc & (r["status"] == 1)
    for k in ("s", "v"):
        err = np.abs(g[k][ok] - r[k][ok]) / np.maximum(np.abs(r[k][ok]), 1.0)
        assert (err <= tol).all(), (k, float(err.max()), np.nonzero(ok)[0][np.argmax(err)])
    return int(ok.sum()), int((disc & flagged).sum())


# ---------------------------------------------------------------------------
def test_fp64_rollout_matches_oracle_small():
    scen = sc.small_scenario()
    sim, ora = _sim(scen, 64), _ora(scen)
    for chunk in range(6):
        sim.step(100); ora.step(100)
        g, r = sim.state(), ora.state()
        assert np.array_equal(g["status"], r["status"])
        act = r["status"] == 1
        assert np.array_equal(g["lane"][act], r["lane"][act])
        assert np.array_equal(g["rc"][act], r["rc"][act])
        assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6
        assert np.abs(g["v"][act] - r["v"][act]).max(initial=0) < 1e-6
        assert np.array_equal(g["flags"], r["flags"])
    gm, rm = sim.metrics(), ora.metrics()
    for k in ("step", "n_active", "n_waiting", "n_arrived", "vehicle_updates", "lane_changes",
              "flagged", "overlaps", "inserted", "mobil_evals"):
        assert gm[k] == rm[k], (k, gm[k], rm[k])
    assert abs(gm["tt_sum"] - rm["tt_sum"]) < 1e-9
    assert abs(gm["speed_sum"] - rm["speed_sum"]) <= 1e-6 * rm["speed_sum"]


def _with_attempt(scen, p_att):
    return dataclasses.replace(scen, params=dataclasses.replace(scen.params, p_attempt=p_att))


@pytest.mark.parametrize("p_att", [0.0, 1.0])
def test_fp64_rollout_attempt_extremes(p_att):
    """Attempt probability 0 (no vehicle evaluates MOBIL, the MOBIL queues stay
    empty) and 1 (every vehicle on a multi-lane road evaluates it, so the
    queues fill and drain in full rounds of 32): FP64 rollout identical to
    the oracle's."""
    scen = _with_attempt(sc.small_scenario(), p_att)
    sim, ora = _sim(scen, 64), _ora(scen)
    for chunk in range(3):
        sim.step(100); ora.step(100)
        g, r = sim.state(), ora.state()
        assert np.array_equal(g["status"], r["status"])
        act = r["status"] == 1
        assert np.array_equal(g["lane"][act], r["lane"][act])
        assert np.array_equal(g["rc"][act], r["rc"][act])
        assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6
        assert np.abs(g["v"][act] - r["v"][act]).max(initial=0) < 1e-6
        assert np.array_equal(g["flags"], r["flags"])
    gm, rm = sim.metrics(), ora.metrics()
    for k in ("n_active", "n_arrived", "vehicle_updates", "lane_changes", "flagged", "mobil_evals"):
        assert gm[k] == rm[k], (k, gm[k], rm[k])
    if p_att == 0.0:
        assert gm["mobil_evals"] == 0 and gm["lane_changes"] == 0
    else:
        assert gm["mobil_evals"] > 0.5 * gm["vehicle_updates"] and gm["lane_changes"] > 0


def test_medium_one_step_parity_every_vehicle_attempts_fp32():
    """30x30 grid of three-lane roads with attempt probability 1: one FP32 step
    from a step-600 state, every vehicle compared (MOBIL from full queues on
    tens of thousands of vehicles)."""
    scen = _with_attempt(sc.medium_scenario(), 1.0)
    sim = _sim(scen, 32)
    sim.step(600)
    st = sim.state()
    ora = _ora(scen)
    ora.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], 600)
    sim.step(1); ora.step(1)
    n, excused = compare_one_step(sim.state(), ora.state())
    assert n > 10_000 and excused <= n // 1000
    assert sim.metrics()["mobil_evals"] > 0


def test_fp64_rollout_matches_oracle_medium():
    """30x30 grid of three-lane roads, 100,000 trips: 600 FP64 steps on both
    sides (up to tens of thousands of vehicles, a third of them evaluating
    MOBIL each step); identical discrete state and flags every 100 steps,
    positions and speeds within 1e-6."""
    scen = sc.medium_scenario()
    sim, ora = _sim(scen, 64), _ora(scen)
    for chunk in range(6):
        sim.step(100); ora.step(100)
        g, r = sim.state(), ora.state()
        assert np.array_equal(g["status"], r["status"])
        act = r["status"] == 1
        assert np.array_equal(g["lane"][act], r["lane"][act])
        assert np.array_equal(g["rc"][act], r["rc"][act])
        assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6
        assert np.abs(g["v"][act] - r["v"][act]).max(initial=0) < 1e-6
        assert np.array_equal(g["flags"], r["flags"])
    assert act.sum() > 20_000
    gm, rm = sim.metrics(), ora.metrics()
    for k in ("n_active", "n_arrived", "vehicle_updates", "lane_changes", "flagged", "mobil_evals"):
        assert gm[k] == rm[k], (k, gm[k], rm[k])


@pytest.mark.parametrize("t0", [60, 150, 300, 450, 599])
def test_fp32_one_step_parity_small(t0):
    scen = sc.small_scenario()
    ora = _ora(scen)
    ora.step(t0)
    st = _f32_state(ora.state())
    sim, ora2 = _sim(scen, 32), _ora(scen)
    _set_both(sim, ora2, st, t0)
    sim.step(1); ora2.step(1)
    n, excused = compare_one_step(sim.state(), ora2.state())
    assert n > 0 and excused <= max(3, n // 100)


def test_fp32_rollout_aggregates_small():
    scen = sc.small_scenario()
    sim, ora = _sim(scen, 32), _ora(scen)
    sim.step(600); ora.step(600)
    gm, rm = sim.metrics(), ora.metrics()
    gs = gm["speed_sum"] / gm["vehicle_updates"]
    rs = rm["speed_sum"] / rm["vehicle_updates"]
    assert abs(gs - rs) <= 0.005 * rs, (gs, rs)
    assert abs(gm["n_arrived"] - rm["n_arrived"]) <= max(1, 0.005 * rm["n_arrived"]), (gm, rm)
    assert gm["errors"] == 0


@pytest.mark.slow
def test_fp32_rollout_aggregates_medium():
    """30x30 grid of three-lane roads, 100,000 trips: the full FP32 rollout of
    3,600 steps against the FP64 oracle's (about two minutes of oracle time);
    network speed and completions within 0.5%."""
    scen = sc.medium_scenario()
    sim, ora = _sim(scen, 32), _ora(scen)
    sim.step(3600); ora.step(3600)
    gm, rm = sim.metrics(), ora.metrics()
    gs = gm["speed_sum"] / gm["vehicle_updates"]
    rs = rm["speed_sum"] / rm["vehicle_updates"]
    assert abs(gs - rs) <= 0.005 * rs, (gs, rs)
    assert rm["n_arrived"] > 1000
    assert abs(gm["n_arrived"] - rm["n_arrived"]) <= 0.005 * rm["n_arrived"], (gm, rm)
    assert gm["errors"] == 0


def test_fp32_rollout_invariants_medium():
    """Invariants of the GPU state itself along an FP32 rollout of the 30x30
    grid (checked every 100 steps): conservation of trips, 0 <= s <= L and
    v >= 0 for active vehicles, a vehicle on a road lane sits on the road its
    route cursor names (on a junction lane: the junction lane leads to the
    next road of the route), no device error."""
    scen = sc.medium_scenario()
    net, veh = scen.net, scen.veh
    sim = _sim(scen, 32)
    L = net.lane_length.astype(np.float64)
    lane_road = net.lane_road()
    target_road = lane_road[net.jl_target]
    n_active_seen = 0
    for _ in range(9):
        sim.step(100)
        st, m = sim.state(), sim.metrics()
        assert m["errors"] == 0
        assert m["n_active"] + m["n_waiting"] + m["n_arrived"] == veh.n
        act = st["status"] == 1
        assert int(act.sum()) == m["n_active"] and int((st["status"] == 2).sum()) == m["n_arrived"]
        n_active_seen = max(n_active_seen, int(act.sum()))
        ln, s_, v_, rc = st["lane"][act], st["s"][act], st["v"][act], st["rc"][act]
        assert (s_ >= 0).all() and (s_ <= L[ln] + 1e-3).all() and (v_ >= 0).all()
        ids = np.nonzero(act)[0]
        cur_road = veh.routes[veh.route_off[ids] + rc]
        on_road = ln < net.n_road_lanes
        assert (lane_road[ln[on_road]] == cur_road[on_road]).all()
        jl = ~on_road
        nxt = veh.routes[np.minimum(veh.route_off[ids[jl]] + rc[jl] + 1, veh.route_off[ids[jl] + 1] - 1)]
        assert (target_road[ln[jl] - net.n_road_lanes] == nxt).all()
    assert n_active_seen > 20_000


# ---------------------------------------------------------------------------
# hand-built states
def _one_step_hand(scen, st, step, precision):
    sim, ora = _sim(scen, precision), _ora(scen)
    _set_both(sim, ora, st, step)
    sim.step(1); ora.step(1)
    return sim.state(), ora.state()


@pytest.mark.parametrize("precision", [32, 64])
def test_conflict_hand_case(precision):
    p = sc.Params(p_attempt=1.0)
    cars = [(0, 100.0, 10.0), (0, 115.0, 0.0), (2, 140.0, 10.0), (2, 165.0, 3.0)]
    scen, st = one_road(3, 1000.0, cars, params=p)
    ora = _ora(scen)
    t = next(t for t in range(400) if (ora.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], t)
                                       or (ora.decision(0)["cand"] and ora.decision(2)["cand"])))
    g, r = _one_step_hand(scen, st, t, precision)
    assert g["lane"].tolist() == r["lane"].tolist()
    assert (g["flags"] & ~binding.F_FLAGGED).tolist() == (r["flags"] & ~binding.F_FLAGGED).tolist()
    assert g["flags"][2] & binding.F_CONFLICT_LOST
    compare_one_step(g, r, 1e-5 if precision == 32 else 1e-12)


# the hand-worked lookahead states of the oracle pins (R11): the rearmost car
# of the next lane, of the lane after an empty junction lane, from a
# junction lane, and the two-lane bound
LOOKAHEAD_CASES = [
    [(0, 250.0, 10.0), (3, 8.0, 6.0), (3, 1.5, 4.0)],
    [(0, 250.0, 10.0), (1, 60.0, 9.0), (1, 20.0, 3.0)],
    [(3, 4.0, 8.0), (4, 3.0, 2.0)],
    [(0, 250.0, 10.0), (4, 5.0, 0.0)],
    [(0, 250.0, 10.0), (0, 290.0, 7.0), (3, 2.0, 0.0)],
]


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("case", range(len(LOOKAHEAD_CASES)))
def test_lookahead_hand_cases(case, precision):
    cars = LOOKAHEAD_CASES[case]
    scen = corridor((300.0, 300.0, 300.0), [(0, 0)] * len(cars), turn_len=10.0)
    rc_of = {0: 0, 1: 1, 2: 2, 3: 0, 4: 1}
    st = dict(status=np.ones(len(cars), dtype=np.int32), lane=np.array([c[0] for c in cars], dtype=np.int32),
              s=np.array([c[1] for c in cars]), v=np.array([c[2] for c in cars]),
              rc=np.array([rc_of[c[0]] for c in cars], dtype=np.int32))
    sim, ora = _sim(scen, precision), _ora(scen)
    _set_both(sim, ora, st, 0)
    sim.set_signal_policy([0, 1], binding.POLICY_NONE)
    ora.set_signal([0, 1], oracle.POLICY_NONE)
    for _ in range(3):
        sim.step(1); ora.step(1)
        g, r = sim.state(), ora.state()
        assert g["lane"].tolist() == r["lane"].tolist() and g["status"].tolist() == r["status"].tolist()
        tol = 1e-5 if precision == 32 else 1e-12
        assert np.all(np.abs(g["s"] - r["s"]) <= tol * np.maximum(np.abs(r["s"]), 1.0))
        assert np.all(np.abs(g["v"] - r["v"]) <= tol * np.maximum(np.abs(r["v"]), 1.0))


@pytest.mark.parametrize("precision", [32, 64])
def test_mobil_draw_gates_hand_states(precision):
    """The draw-gate pin states (R3-R6): both sides positive and equal (p_LC =
    p_hi), unequal with u_T in (0, 1), and u_T = 0 with p_lo raised: one step
    from each of 40 steps of draws; lane (change and side) and kinematics as
    the oracle's."""
    states = [([(1, 100.0, 10.0), (1, 120.0, 5.0)], sc.Params(seed=7)),
              ([(1, 100.0, 10.0), (1, 125.0, 8.0), (2, 150.0, 8.0)], sc.Params(seed=11, a_th=1.5)),
              ([(1, 100.0, 10.0)], sc.Params(seed=3, p_lo=0.3, p_attempt=1.0))]
    changed = 0
    for cars, prm in states:
        scen, st = one_road(3, 1000.0, cars, params=prm)
        for t in range(0, 40):
            g, r = _one_step_hand(scen, st, t, precision)
            assert g["lane"].tolist() == r["lane"].tolist(), (cars, t)
            assert (g["flags"] & ~binding.F_FLAGGED).tolist() == (r["flags"] & ~binding.F_FLAGGED).tolist()
            compare_one_step(g, r, 1e-5 if precision == 32 else 1e-12)
            changed += int(r["lane"][0] != st["lane"][0])
    assert changed > 20


@pytest.mark.parametrize("precision", [32, 64])
def test_red_light_and_transfer(precision):
    scen = corridor((300.0, 300.0), [(0, 0), (0, 3)])
    sim, ora = _sim(scen, precision), _ora(scen)
    for obj in (sim, ora):
        obj.set_signal_phase([0], [1]) if obj is sim else obj.set_signal([0], oracle.POLICY_MANUAL, [1])
    sim.step(100); ora.step(100)
    g, r = sim.state(), ora.state()
    assert g["lane"].tolist() == r["lane"].tolist() == [0, 0]
    assert np.allclose(g["s"], r["s"], atol=1e-4)
    sim.set_signal_phase([0], [0]); ora.set_signal([0], oracle.POLICY_MANUAL, [0])
    sim.step(150); ora.step(150)
    g, r = sim.state(), ora.state()
    assert g["status"].tolist() == r["status"].tolist() == [2, 2]
    assert sim.metrics()["tt_sum"] == pytest.approx(ora.metrics()["tt_sum"])


@pytest.mark.parametrize("precision", [32, 64])
def test_degenerate_scenarios(precision):
    # no vehicles at all
    net = sc.corridor_network(2, (500.0,))
    veh = sc.Vehicles(n=0, route_off=np.zeros(1, np.int32), routes=np.zeros(0, np.int32),
                      start_lane=np.zeros(0, np.int32), dep=np.zeros(0, np.int32),
                      v0f=np.zeros(0, np.float32))
    sim = binding.Simulation(net, veh, sc.Params(), precision=precision)
    sim.step(5)
    m = sim.metrics()
    assert m["step"] == 5 and m["vehicle_updates"] == 0
    # departures only after the horizon
    scen = corridor((300.0, 300.0), [(0, 1000), (0, 1000)])
    sim = _sim(scen, precision)
    sim.step(10)
    assert sim.metrics()["n_waiting"] == 2
    # single-road routes arrive at the end of their only road
    scen, st = one_road(1, 60.0, [(0, 50.0, 12.0), (0, 10.0, 5.0)])
    g, r = _one_step_hand(scen, st, 0, precision)
    assert g["status"].tolist() == r["status"].tolist() == [2, 1]


def test_signal_setter_parity_fp64():
    scen = sc.small_scenario()
    sim, ora = _sim(scen, 64), _ora(scen)
    rng = np.random.default_rng(1)
    J = scen.net.n_junctions
    for k in range(30):
        ph = rng.integers(0, 4, J)
        sim.set_signal_phase(np.arange(J), ph)
        ora.set_signal(np.arange(J), oracle.POLICY_MANUAL, ph)
        sim.step(10); ora.step(10)
    g, r = sim.state(), ora.state()
    assert np.array_equal(g["status"], r["status"])
    act = r["status"] == 1
    assert np.array_equal(g["lane"][act], r["lane"][act])
    assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6


def test_batch_equals_alone():
    scens = [sc.small_scenario(seed=s) for s in (0, 1, 2)]
    for i, s in enumerate(scens):
        s.params.scenario = i
    batch = binding.Batch(scens, precision=32)
    batch.step(300)
    for i, s in enumerate(scens):
        alone = _sim(s, 32)
        alone.step(300)
        a, b = alone.state(), batch.state(i)
        for k in ("status", "lane", "rc", "flags"):
            assert np.array_equal(a[k], b[k]), (i, k)
        for k in ("s", "v"):
            assert np.array_equal(a[k], b[k]), (i, k)
        ma, mb = alone.metrics(), batch.metrics(i)
        assert ma == mb, (i, ma, mb)


def test_medium_one_step_parity_fp32():
    """30x30 grid, 100,000 trips: one FP32 step from the oracle's state."""
    scen = sc.medium_scenario()
    sim = _sim(scen, 32)
    sim.step(900)  # let traffic build up on the GPU, then hand the state to the oracle
    st = sim.state()
    ora = _ora(scen)
    ora.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], 900)
    sim.step(1); ora.step(1)
    n, excused = compare_one_step(sim.state(), ora.state())
    assert n > 10_000 and excused <= n // 1000


def test_city_one_step_parity_fp32():
    """Full size, in the launch configuration the benchmark times: the city
    workload (39,600 roads, 2,464,950 trips) simulated on the GPU to step
    3600 (about two million vehicles on the network), then one step on both
    sides from that state; every vehicle compared."""
    scen = sc.city_scenario()
    sim = _sim(scen, 32)
    sim.step(3600)
    st = sim.state()
    assert (st["status"] == 1).sum() > 1_000_000
    ora = _ora(scen)
    ora.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], 3600)
    sim.step(1); ora.step(1)
    n, excused = compare_one_step(sim.state(), ora.state())
    assert n > 1_000_000 and excused <= n // 1000


def test_city_fp64_steps_identical_to_oracle():
    """Full size in FP64: the city simulated on the GPU to step 3600 (about two
    million vehicles), then three steps on both sides from that state; every
    vehicle's discrete state and flags identical, positions and speeds within
    1e-6."""
    scen = sc.city_scenario()
    sim = _sim(scen, 64)
    sim.step(3600)
    st = sim.state()
    assert (st["status"] == 1).sum() > 1_000_000
    ora = _ora(scen)
    ora.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], 3600)
    sim.step(3); ora.step(3)
    g, r = sim.state(), ora.state()
    assert np.array_equal(g["status"], r["status"])
    act = r["status"] == 1
    assert np.array_equal(g["lane"][act], r["lane"][act])
    assert np.array_equal(g["rc"][act], r["rc"][act])
    assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6
    assert np.abs(g["v"][act] - r["v"][act]).max(initial=0) < 1e-6
    assert np.array_equal(g["flags"], r["flags"])


def test_saturated_city_one_step_parity_fp32():
    """The state of the saturated measurement: all 2,464,950 trips of the
    city on the road at once, evenly spaced.  One FP32 step on both sides
    from the same (FP32-rounded) state, every vehicle compared."""
    scen, (status, lane, s, v, rc) = sc.saturated_city()
    st = _f32_state({"status": status, "lane": lane, "s": s, "v": v, "rc": rc})
    sim, ora = _sim(scen, 32), _ora(scen)
    _set_both(sim, ora, st, 0)
    sim.step(1); ora.step(1)
    n, excused = compare_one_step(sim.state(), ora.state())
    assert n > 2_000_000 and excused <= n // 1000


def test_ragged_batch_with_empty_member():
    """A batch of uneven members, one with no vehicles and no junctions, one
    with a single vehicle: every member equals its own run alone."""
    empty_net = sc.corridor_network(2, (500.0,))
    empty_veh = sc.Vehicles(n=0, route_off=np.zeros(1, np.int32), routes=np.zeros(0, np.int32),
                            start_lane=np.zeros(0, np.int32), dep=np.zeros(0, np.int32),
                            v0f=np.zeros(0, np.float32))
    empty = sc.Scenario(empty_net, empty_veh, sc.Params(), "empty")
    single = corridor((300.0, 300.0), [(1, 3)], n_lanes=2)
    scens = [sc.small_scenario(seed=4), empty, single, sc.small_scenario(seed=5)]
    for i, s in enumerate(scens):
        s.params.scenario = i
    batch = binding.Batch(scens, precision=32)
    batch.step(250)
    for i, s in enumerate(scens):
        alone = _sim(s, 32)
        alone.step(250)
        a, b = alone.state(), batch.state(i)
        for k in ("status", "lane", "rc", "flags", "s", "v"):
            assert np.array_equal(a[k], b[k]), (i, k)
        assert alone.metrics() == batch.metrics(i), i


def test_fp64_ragged_batch_matches_oracle_per_member():
    """A ragged FP64 batch against one oracle instance per member (not only
    against its members run alone): an empty member, a single-road member,
    grids of 3x3 to 8x8 with up to 6,000 trips, their own seeds and scenario
    ids (so their random streams differ), scenario-major lanes and vehicles
    at the batch boundaries.  After 300 steps every member's discrete state
    and flags equal its oracle's, positions and speeds within 1e-6, and its
    metrics match."""
    empty_net = sc.corridor_network(2, (500.0,))
    empty_veh = sc.Vehicles(n=0, route_off=np.zeros(1, np.int32), routes=np.zeros(0, np.int32),
                            start_lane=np.zeros(0, np.int32), dep=np.zeros(0, np.int32),
                            v0f=np.zeros(0, np.float32))
    empty = sc.Scenario(empty_net, empty_veh, sc.Params(), "empty")
    one_road_scen, _ = one_road(3, 800.0, [(0, 10.0, 5.0)])
    one_road_scen.veh.dep[:] = 0
    grids = []
    for k, (G, n, L) in enumerate([(3, 400, 150.0), (5, 2500, 200.0), (8, 6000, 250.0), (4, 1200, 300.0)]):
        net = sc.grid_network(G, L, 2 + (k % 2), 13.89, offsets=True, seed=10 + k)
        veh = sc.random_demand(net, n, 200, seed=10 + k)
        grids.append(sc.Scenario(net, veh, sc.Params(seed=100 + k), f"grid{G}"))
    scens = [grids[0], empty, grids[1], one_road_scen, grids[2], grids[3]]
    for i, s_ in enumerate(scens):
        s_.params.scenario = i
    batch = binding.Batch(scens, precision=64)
    batch.step(300)
    for i, s_ in enumerate(scens):
        ora = _ora(s_)
        ora.step(300)
        g, r = batch.state(i), ora.state()
        assert np.array_equal(g["status"], r["status"]), i
        act = r["status"] == 1
        for k in ("lane", "rc"):
            assert np.array_equal(g[k][act], r[k][act]), (i, k)
        assert np.array_equal(g["flags"], r["flags"]), i
        if act.any():
            assert np.abs(g["s"][act] - r["s"][act]).max() < 1e-6, i
            assert np.abs(g["v"][act] - r["v"][act]).max() < 1e-6, i
        gm, rm = batch.metrics(i), ora.metrics()
        for k in ("step", "n_active", "n_waiting", "n_arrived", "vehicle_updates", "lane_changes", "flagged",
                  "overlaps", "inserted", "mobil_evals"):
            assert gm[k] == rm[k], (i, k, gm[k], rm[k])
        assert abs(gm["tt_sum"] - rm["tt_sum"]) < 1e-9
        assert abs(gm["speed_sum"] - rm["speed_sum"]) <= 1e-6 * max(rm["speed_sum"], 1.0)


@pytest.mark.parametrize("precision", [32, 64])
def test_long_queue_lane_spans_many_tiles(precision):
    """One 8 km two-lane road holding a 1,500-car queue (the lane's segment
    spans several 256-slot tiles; adjacent-lane searches over long segments;
    entrants placed into long lanes) and exact position ties (order by id):
    50 steps against the oracle."""
    rng = np.random.default_rng(9)
    cars = []
    for k in range(1500):  # lane 0: a dense queue near the end, slowly moving
        cars.append((0, 7900.0 - 5.2 * k, float(rng.uniform(0.0, 2.0))))  # last one at 105 m
    for k in range(300):   # lane 1: sparser and faster, some cars side by side
        cars.append((1, 7950.0 - 24.0 * k, float(rng.uniform(5.0, 12.0))))
    for k in range(5):     # exact ties on lane 1 (ordered by id)
        cars.append((1, 3000.0 + 0.0 * k, 3.0))
    scen, st = one_road(2, 8000.0, cars, params=sc.Params(p_attempt=1.0))
    sim, ora = _sim(scen, precision), _ora(scen)
    _set_both(sim, ora, st if precision == 64 else _f32_state(st), 0)
    for _ in range(5):
        sim.step(10); ora.step(10)
        g, r = sim.state(), ora.state()
        if precision == 64:
            assert np.array_equal(g["status"], r["status"])
            act = r["status"] == 1
            assert np.array_equal(g["lane"][act], r["lane"][act])
            assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6
            assert np.abs(g["v"][act] - r["v"][act]).max(initial=0) < 1e-6
            assert np.array_equal(g["flags"], r["flags"])
    gm, rm = sim.metrics(), ora.metrics()
    assert gm["errors"] == 0
    if precision == 64:
        for k in ("lane_changes", "flagged", "overlaps", "n_arrived", "mobil_evals"):
            assert gm[k] == rm[k], (k, gm[k], rm[k])
    else:
        assert abs(gm["speed_sum"] - rm["speed_sum"]) <= 0.005 * rm["speed_sum"]


@pytest.mark.parametrize("precision", [32, 64])
def test_single_launch_step_equals_kernel_sequence(precision):
    """The step as one cooperative launch (moss_set_step_mode 1) gives the
    same state and metrics as the sequence of kernels, on a ragged batch;
    in FP64 both equal the oracle run per member."""
    scens = [sc.small_scenario(seed=4), sc.medium_scenario(n=15_000), sc.small_scenario(seed=5)]
    for i, s_ in enumerate(scens):
        s_.params.scenario = i
    a = binding.Batch(scens, precision=precision)
    b = binding.Batch(scens, precision=precision)
    b.set_step_mode(1)
    a.step(160); b.step(160)
    b.set_step_mode(0)
    a.step(7); b.step(7)
    b.set_step_mode(1)
    a.step(33); b.step(33)
    for i, s_ in enumerate(scens):
        x, y = a.state(i), b.state(i)
        for k in x:
            assert np.array_equal(x[k], y[k]), (i, k)
        assert a.metrics(i) == b.metrics(i), i
        if precision == 64:
            ora = _ora(s_)
            ora.step(200)
            r = ora.state()
            assert np.array_equal(y["status"], r["status"]), i
            act = r["status"] == 1
            assert np.array_equal(y["lane"][act], r["lane"][act]), i
            assert np.abs(y["s"][act] - r["s"][act]).max(initial=0) < 1e-6, i
