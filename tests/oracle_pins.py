"""Checks that pin the FP64 oracle to facts fixed by the paper and by
mathematics, independently of the oracle itself.

Each check takes an optional path to an oracle build so that
``test_oracle_planted.py`` can run the same battery against copies of the
oracle with a deliberately planted mistake and show that some check fails.
"""
import json
import math
import os

import numpy as np

import oracle
from handmade import corridor, one_road
from paper_2406_10661_gb300 import scenario as sc

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _oracle(scen, state=None, libpath=None, step=0):
    o = oracle.Oracle(scen.net, scen.veh, scen.params, libpath=libpath)
    if state is not None:
        o.set_state(state["status"], state["lane"], state["s"], state["v"], state["rc"], step)
    return o


def _probe(libpath=None):
    scen, st = one_road(1, 1000.0, [(0, 10.0, 0.0)])
    return _oracle(scen, st, libpath)


# --------------------------------------------------------------------------
# IDM (App. B.3, equations (1)-(2))
# --------------------------------------------------------------------------
def check_idm_free_road(libpath=None):
    g = _gold("idm_mobil_hand_cases.json")["idm_free_road"]
    o = _probe(libpath)
    a = o.idm_free(g["v"], 13.89)
    assert abs(a - g["expected"]) < 1e-12, a
    # interaction vanishes for a very distant leader at equal speed
    a_far = o.idm(g["v"], 13.89, 1e9, 0.0)
    assert abs(a_far - g["expected"]) < 1e-9, a_far


def check_idm_equilibrium(libpath=None):
    """a = 0 at the equilibrium gap s_e(v) of a uniform platoon (closed form)."""
    g = _gold("idm_mobil_hand_cases.json")["equilibrium_gap"]
    o = _probe(libpath)
    for v, se in zip(g["v"], g["s_e"]):
        a = o.idm(v, 13.89, se, 0.0)
        assert abs(a) < 1e-9, (v, a)
        # slightly closer -> braking, slightly farther -> accelerating
        assert o.idm(v, 13.89, se * 0.99, 0.0) < 0 < o.idm(v, 13.89, se * 1.01, 0.0)
    # standstill at the minimum gap s0: a = 0
    assert abs(o.idm(0.0, 13.89, 2.0, 0.0)) < 1e-12
    # approaching (dv > 0) brakes harder than following at equal speed
    assert o.idm(10.0, 13.89, 30.0, 3.0) < o.idm(10.0, 13.89, 30.0, 0.0) < o.idm(10.0, 13.89, 30.0, -3.0)


def check_p_lc(libpath=None):
    g = _gold("idm_mobil_hand_cases.json")["p_lc"]
    o = _probe(libpath)
    for u, e in zip(g["uT"], g["expected"]):
        assert abs(o.p_lc(u) - e) < 1e-15, (u, o.p_lc(u), e)


# --------------------------------------------------------------------------
# MOBIL hand cases (App. B.3, readings R1-R2)
# --------------------------------------------------------------------------
def _mobil_params():
    return sc.Params(p_attempt=1.0)


def check_mobil_case_A(libpath=None):
    g = _gold("idm_mobil_hand_cases.json")["case_A"]
    scen, st = one_road(2, 1000.0, [(1, 100.0, 10.0), (1, 120.0, 5.0)], params=_mobil_params())
    d = _oracle(scen, st, libpath).decision(0)
    assert d["attempted"] == 1
    assert abs(d["a_own"] - g["a_own"]) < 1e-9, d["a_own"]
    assert abs(d["at_ego_L"] - g["at_ego_L"]) < 1e-9, d["at_ego_L"]
    assert abs(d["uL"] - g["uL"]) < 1e-9, d["uL"]
    assert d["feasL"] == 1 and d["feasR"] == 0
    assert abs(d["pLC"] - 0.9) < 1e-15  # u_T >= 1


def check_mobil_case_B(libpath=None):
    g = _gold("idm_mobil_hand_cases.json")["case_B"]
    scen, st = one_road(2, 1000.0, [(1, 100.0, 10.0), (1, 120.0, 5.0), (0, 92.0, 15.0)],
                        params=_mobil_params())
    d = _oracle(scen, st, libpath).decision(0)
    assert abs(d["at_new_L"] - g["at_new_L"]) < 1e-6, d["at_new_L"]
    assert abs(d["a_new_L"] - g["a_new_L"]) < 1e-9, d["a_new_L"]
    assert d["feasL"] == g["feasL"]
    assert d["cand"] == 0 or d["dir"] != -1


def check_mobil_case_C(libpath=None):
    g = _gold("idm_mobil_hand_cases.json")["case_C"]
    scen, st = one_road(2, 1000.0, [(1, 100.0, 10.0), (1, 120.0, 5.0), (0, 65.0, 8.0)],
                        params=_mobil_params())
    d = _oracle(scen, st, libpath).decision(0)
    assert abs(d["a_new_L"] - g["a_new_L"]) < 1e-9, d["a_new_L"]
    assert abs(d["at_new_L"] - g["at_new_L"]) < 1e-9, d["at_new_L"]
    assert abs(d["uL"] - g["uL"]) < 1e-9, d["uL"]
    assert d["feasL"] == 1
    assert d["TF_left"] == 2 and d["TL_left"] == -1


def check_mobil_case_D(libpath=None):
    g = _gold("idm_mobil_hand_cases.json")["case_D"]
    scen, st = one_road(2, 1000.0, [(1, 100.0, 10.0), (1, 120.0, 5.0), (1, 80.0, 10.0)],
                        params=_mobil_params())
    d = _oracle(scen, st, libpath).decision(0)
    assert abs(d["a_old"] - g["a_old"]) < 1e-9, d["a_old"]
    assert abs(d["at_old"] - g["at_old"]) < 1e-9, d["at_old"]
    assert abs(d["uL"] - g["uL"]) < 1e-9, d["uL"]
    assert d["OF"] == 2 and d["OL"] == 1


def check_mobil_mirror(libpath=None):
    """Mirroring a 3-lane state left<->right swaps u_L and u_R."""
    rng = np.random.default_rng(5)
    cars = [(1, 200.0, 9.0)]
    for k in range(8):
        cars.append((int(rng.integers(0, 3)), float(rng.uniform(120, 280)), float(rng.uniform(0, 14))))
    # keep every car at least a length apart from the ego on other lanes to avoid overlaps
    cars = [c for i, c in enumerate(cars) if i == 0 or abs(c[1] - 200.0) > 6.0]
    mir = [(2 - c[0], c[1], c[2]) for c in cars]
    p = _mobil_params()
    s1, st1 = one_road(3, 1000.0, cars, params=p)
    s2, st2 = one_road(3, 1000.0, mir, params=p)
    d1 = _oracle(s1, st1, libpath).decision(0)
    d2 = _oracle(s2, st2, libpath).decision(0)
    assert abs(d1["uL"] - d2["uR"]) < 1e-12 and abs(d1["uR"] - d2["uL"]) < 1e-12, (d1, d2)
    assert d1["feasL"] == d2["feasR"] and d1["feasR"] == d2["feasL"]


# --------------------------------------------------------------------------
# Sensing: brute force over tiny lanes (§3.1 sensing index; reading R16)
# --------------------------------------------------------------------------
def _ahead(a, b):
    return a[0] > b[0] or (a[0] == b[0] and a[1] < b[1])


def check_neighbours_bruteforce(libpath=None, trials=40):
    rng = np.random.default_rng(11)
    p = _mobil_params()
    for _ in range(trials):
        n = int(rng.integers(2, 9))
        cars = []
        for k in range(n):
            s = float(rng.integers(0, 40)) * 2.5  # coarse grid -> exact ties happen
            cars.append((int(rng.integers(0, 3)), s, float(rng.uniform(0, 14))))
        scen, st = one_road(3, 500.0, cars, params=p)
        o = _oracle(scen, st, libpath)
        for ego in range(n):
            d = o.decision(ego)
            key = (st["s"][ego], ego)

            def lead(lane):
                c = [(st["s"][k], k) for k in range(n) if k != ego and st["lane"][k] == lane
                     and _ahead((st["s"][k], k), key)]
                return min(c, key=lambda x: (x[0], -x[1]))[1] if c else -1

            def foll(lane):
                c = [(st["s"][k], k) for k in range(n) if k != ego and st["lane"][k] == lane
                     and not _ahead((st["s"][k], k), key)]
                return max(c, key=lambda x: (x[0], -x[1]))[1] if c else -1

            el = st["lane"][ego]
            assert d["own_leader"] == lead(el), (cars, ego, d["own_leader"])
            assert d["OL"] == lead(el) and d["OF"] == foll(el)
            if el > 0:
                assert d["TL_left"] == lead(el - 1) and d["TF_left"] == foll(el - 1)
            if el < 2:
                assert d["TL_right"] == lead(el + 1) and d["TF_right"] == foll(el + 1)


# --------------------------------------------------------------------------
# Kinematics (reading R12): textbook reductions
# --------------------------------------------------------------------------
def check_free_road_vs_rk4(libpath=None):
    """A lone car on a free lane follows dv/dt = a(1-(v/v0)^4).  The ballistic
    update is first order in dt; its speed stays within 0.5 m/s (0.39 at worst for
    dt = 1 s) of a fine RK4
    solution and converges to v0; displacement per step is the trapezoid of
    the two speeds while no clamp binds."""
    scen, st = one_road(1, 5000.0, [(0, 0.0, 0.0)])
    o = _oracle(scen, st, libpath)
    v0, a = 13.89, 2.0
    f = lambda v: a * (1 - (v / v0) ** 4)  # noqa: E731
    vr, h = 0.0, 1e-3
    prev = o.state()
    for t in range(1, 60):
        o.step(1)
        cur = o.state()
        for _ in range(1000):
            k1 = f(vr); k2 = f(vr + h / 2 * k1); k3 = f(vr + h / 2 * k2); k4 = f(vr + h * k3)
            vr += h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        assert abs(cur["v"][0] - vr) < 0.5, (t, cur["v"][0], vr)
        ds = cur["s"][0] - prev["s"][0]
        assert abs(ds - 0.5 * (cur["v"][0] + prev["v"][0])) < 1e-9, (t, ds)
        prev = cur
    assert abs(prev["v"][0] - v0) < 1e-3


def check_platoon_equilibrium(libpath=None):
    """Followers of a uniform platoon at s_e(v) keep a = 0 (speed unchanged,
    displacement v dt) during the step."""
    v, v0 = 10.0, 14.0  # v0 exactly representable in the float32 lane table
    se = (2.0 + v * 1.5) / math.sqrt(1.0 - (v / v0) ** 4)  # closed form, a = 0
    n = 6
    cars = [(0, 100.0 + k * (se + 5.0), v) for k in range(n)]  # car n-1 is the head
    scen, st = one_road(1, 5000.0, cars, vmax=v0)
    o = _oracle(scen, st, libpath)
    o.step(1)
    cur = o.state()
    for k in range(n - 1):
        assert abs(cur["v"][k] - v) < 1e-9, (k, cur["v"][k])
        assert abs(cur["s"][k] - (st["s"][k] + v)) < 1e-9
    assert cur["v"][n - 1] > v  # the head is on free road below v0


def check_red_light(libpath=None):
    """Manual red: the car stops before the line (App. B.3 signal rule) and
    never enters the junction; after switching to green it crosses, transfers
    with exact kinematics and arrives."""
    scen = corridor((300.0, 300.0), [(0, 0)])
    o = _oracle(scen, None, libpath)
    o.set_signal([0], oracle.POLICY_MANUAL, [1])  # phase 1: corridor red
    L0 = float(scen.net.lane_length[0])
    for t in range(120):
        o.step(1)
        st = o.state()
        if st["status"][0] == 1:
            assert st["lane"][0] == 0, "entered a red junction lane"
            assert -1e-12 <= L0 - st["s"][0]
    st = o.state()
    assert st["v"][0] < 1e-6 and 0.0 <= L0 - st["s"][0] <= 2.0 + 1e-6, st
    o.set_signal([0], oracle.POLICY_MANUAL, [0])  # green
    crossed = False
    for t in range(200):
        before = o.state()
        o.step(1)
        after = o.state()
        if after["status"][0] == 1 and before["lane"][0] == 0 and after["lane"][0] != 0:
            crossed = True
            # exact transfer: s'' = s + d - L where d = trapezoid displacement
            d = 0.5 * (before["v"][0] + after["v"][0])
            if after["lane"][0] == 2:  # the junction lane
                assert abs(after["s"][0] - (before["s"][0] + d - L0)) < 1e-9
        if after["status"][0] == 2:
            break
    assert crossed and o.state()["status"][0] == 2
    m = o.metrics()
    assert m["n_arrived"] == 1 and m["errors"] == 0


def check_signal_program(libpath=None):
    """Fixed-time program (reading R19): phases 0,1 of 30 green + 3 amber;
    the corridor lane is green in phase 0 only."""
    scen = corridor((300.0, 300.0), [(0, 0)], green=30, amber=3)
    o = _oracle(scen, None, libpath)
    jl = scen.net.n_road_lanes  # the only junction lane
    exp = [oracle.LIGHT_GREEN] * 30 + [oracle.LIGHT_AMBER] * 3 + [oracle.LIGHT_RED] * 33
    got = [o.light(jl, t) for t in range(66)]
    assert got == exp
    assert [o.light(jl, t + 66) for t in range(66)] == exp  # periodic
    o.set_signal([0], oracle.POLICY_NONE)
    assert all(o.light(jl, t) == oracle.LIGHT_GREEN for t in range(66))


def check_arrival_and_travel_time(libpath=None):
    """A lone car departing at step 5 on an always-green corridor: it is
    inserted at step 5 (at t=6 it is at s=0), drives 600 m + junction and
    arrives; ATT = arrival time - departure time."""
    scen = corridor((300.0, 300.0), [(0, 5)], turn_len=10.0)
    o = _oracle(scen, None, libpath)
    o.set_signal([0], oracle.POLICY_NONE)
    total = 610.0
    pos = 0.0
    arrived_at = None
    for t in range(200):
        b = o.state()
        o.step(1)
        a = o.state()
        if b["status"][0] == 0 and a["status"][0] == 1:
            assert t == 5 and a["s"][0] == 0.0 and a["v"][0] == 0.0
        if b["status"][0] == 1:
            pos += 0.5 * (b["v"][0] + a["v"][0])
        if a["status"][0] == 2:
            arrived_at = t + 1
            break
    assert arrived_at is not None
    assert pos >= total - 1e-9 and pos - 0.5 * (b["v"][0] + a["v"][0]) < total
    m = o.metrics()
    assert m["n_arrived"] == 1 and abs(m["tt_sum"] - (arrived_at - 5)) < 1e-12


def check_insertion(libpath=None):
    """Two cars on one start lane, both due at step 0: FIFO by id, the second
    waits until the first has s - len >= s0 in the step's snapshot."""
    scen = corridor((1000.0, 300.0), [(0, 0), (0, 0)])
    o = _oracle(scen, None, libpath)
    o.set_signal([0], oracle.POLICY_NONE)
    o.step(1)
    st = o.state()
    assert st["status"].tolist() == [1, 0]
    t = 1
    while True:
        snap = o.state()
        o.step(1)
        st = o.state()
        if st["status"][1] == 1:
            assert snap["s"][0] - 5.0 >= 2.0
            break
        assert snap["s"][0] - 5.0 < 2.0
        t += 1
        assert t < 50
    assert o.metrics()["inserted"] == 2


def _find_step(scen, st, ids, libpath, want):
    o = _oracle(scen, st, libpath)
    for t in range(0, 400):
        o.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], t)
        ds = [o.decision(i) for i in ids]
        if all(want(d) for d in ds):
            return t, ds
    raise AssertionError("no step with the wanted draws")


def check_conflict(libpath=None):
    """Reading R9: candidates entering lane 1 from lanes 0 and 2 into the same
    gap: only the larger utility changes lanes; in different gaps both do."""
    p = _mobil_params()
    cars = [(0, 100.0, 10.0), (0, 115.0, 0.0),   # car 0 behind a stopped car
            (2, 140.0, 10.0), (2, 165.0, 3.0)]  # car 2 behind a slow car (smaller u)
    scen, st = one_road(3, 1000.0, cars, params=p)
    t, ds = _find_step(scen, st, [0, 2], libpath, lambda d: d["cand"] == 1)
    assert ds[0]["dir"] == 1 and ds[1]["dir"] == -1 and ds[0]["u"] > ds[1]["u"]
    assert (ds[0]["TL"], ds[0]["TF"]) == (ds[1]["TL"], ds[1]["TF"]) == (-1, -1)
    o = _oracle(scen, st, libpath, step=t)
    o.step(1)
    a = o.state()
    assert a["lane"][0] == 1 and a["flags"][0] & oracle.F_CHANGED
    assert a["lane"][2] == 2 and a["flags"][2] & oracle.F_CONFLICT_LOST
    assert o.metrics()["lane_changes"] == 1
    # a car in lane 1 between them separates the two gaps -> both change
    cars2 = cars + [(1, 120.0, 10.0)]
    scen2, st2 = one_road(3, 1000.0, cars2, params=p)
    t2, ds2 = _find_step(scen2, st2, [0, 2], libpath, lambda d: d["cand"] == 1)
    assert (ds2[0]["TL"], ds2[0]["TF"]) == (4, -1) and (ds2[1]["TL"], ds2[1]["TF"]) == (-1, 4)
    o2 = _oracle(scen2, st2, libpath, step=t2)
    o2.step(1)
    a2 = o2.state()
    assert a2["lane"][0] == 1 and a2["lane"][2] == 1


def check_permutation_invariance(libpath=None, steps=150):
    """Two-phase read/write separation (§3.1): processing vehicles in reverse
    order gives bit-identical states and metrics."""
    scen = sc.small_scenario()
    o1 = oracle.Oracle(scen.net, scen.veh, scen.params, libpath=libpath)
    o2 = oracle.Oracle(scen.net, scen.veh, scen.params, libpath=libpath)
    o2.set_reverse_order(True)
    o1.step(steps); o2.step(steps)
    a, b = o1.state(), o2.state()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert o1.metrics() == o2.metrics()


# ---------------------------------------------------------------------------
# Max pressure (reading R23), pinned to its definition written out here:
# movement pressure = vehicles on the road lane a junction lane leaves minus
# vehicles on the road lane it feeds (snapshot counts); phase pressure = sum
# over the junction lanes green in the phase; the current phase is kept when
# it is maximal, else the smallest index among the maxima.
def _mp_definition(net, counts, j, current):
    nrl = net.n_road_lanes
    frm = np.full(net.n_lanes, -1, dtype=np.int64)
    for l in range(nrl):
        frm[net.jl_off[l]:net.jl_off[l + 1]] = l
    P = int(net.junc_phase_off[j + 1] - net.junc_phase_off[j])
    press = [0] * P
    for jl in range(nrl, net.n_lanes):
        k = jl - nrl
        if net.jl_junction[k] != j:
            continue
        d = int(counts[frm[jl]]) - int(counts[net.jl_target[k]])
        for p in range(P):
            if (int(net.jl_mask[k]) >> p) & 1:
                press[p] += d
    m = max(press)
    if press[current] == m:
        return current
    return press.index(m)


def _parked(net, cars):
    """Vehicles standing still on road lanes: cars = list of (lane, s); each
    drives a one-road route on its lane's road.  Returns (vehicles, state)."""
    lr = net.lane_road()
    n = len(cars)
    lanes = np.array([c[0] for c in cars], dtype=np.int32)
    veh = sc.Vehicles(n=n, route_off=np.arange(n + 1, dtype=np.int32), routes=lr[lanes].astype(np.int32),
                      start_lane=lanes, dep=np.zeros(n, dtype=np.int32), v0f=np.ones(n, dtype=np.float32))
    st = dict(status=np.ones(n, dtype=np.int32), lane=lanes.copy(),
              s=np.array([c[1] for c in cars], dtype=np.float64), v=np.zeros(n), rc=np.zeros(n, dtype=np.int32))
    return veh, st


def check_max_pressure_argmax(libpath=None):
    """R23 with one-step phases (green 1, amber 0): after one step every
    junction of a 3x3 grid shows the phase of maximal pressure of the
    snapshot, for random vehicle counts (brute force against the definition)."""
    net = sc.grid_network(3, length=200.0, lanes=2, green=1, amber=0)
    rng = np.random.default_rng(5)
    for trial in range(12):
        n = int(rng.integers(5, 60))
        lanes = rng.integers(0, net.n_road_lanes, n)
        cars = [(int(l), float(rng.uniform(10.0, 190.0))) for l in lanes]
        veh, st = _parked(net, cars)
        scen = sc.Scenario(net, veh, sc.Params(), "mp")
        t0 = int(rng.integers(0, 40))
        o = _oracle(scen, st, libpath, step=t0)
        o.set_signal(list(range(net.n_junctions)), oracle.POLICY_MAX_PRESSURE)
        counts = np.bincount(lanes, minlength=net.n_lanes)
        before = [o.signal_state(j) for j in range(net.n_junctions)]
        o.step(1)
        for j in range(net.n_junctions):
            exp = _mp_definition(net, counts, j, before[j][0])
            assert o.signal_state(j) == (exp, 1, -1) if exp != before[j][0] else o.signal_state(j) == (exp, 2, -1), \
                (trial, j, o.signal_state(j), exp)


def check_max_pressure_timing(libpath=None):
    """R23 timing, worked by hand: the centre junction of a 3x3 grid (phases of
    30 s green + 3 s amber) is switched to max pressure at step 66, while its
    fixed program shows phase 2; five cars wait on one approach whose
    movements are all red in phase 2.  The junction keeps phase 2 for its 30
    green steps (steps 66-95), shows 3 amber steps (96-98) and turns to the
    phase of maximal pressure at step 99."""
    net = sc.grid_network(3, length=200.0, lanes=1, green=30, amber=3)
    j = 4
    nrl = net.n_road_lanes
    # an approach of the centre junction that is red in phase 2
    lr = net.lane_road()
    lane_in = None
    for l in range(nrl):
        if net.road_to[lr[l]] != j:
            continue
        masks = net.jl_mask[net.jl_off[l] - nrl:net.jl_off[l + 1] - nrl]
        if all(((int(m) >> 2) & 1) == 0 for m in masks):
            lane_in = l
            break
    assert lane_in is not None
    L = float(net.lane_length[lane_in])
    counts = np.zeros(net.n_lanes, dtype=np.int64)
    counts[lane_in] = 5
    best = _mp_definition(net, counts, j, 2)
    assert best != 2
    jl_through = [jl for jl in range(net.jl_off[lane_in], net.jl_off[lane_in + 1])
                  if (int(net.jl_mask[jl - nrl]) >> best) & 1][0]
    # the five cars drive through that movement (a two-road route)
    r_in, r_out = int(lr[lane_in]), int(lr[net.jl_target[jl_through - nrl]])
    n = 5
    veh = sc.Vehicles(n=n, route_off=np.arange(0, 2 * n + 1, 2, dtype=np.int32),
                      routes=np.array([r_in, r_out] * n, dtype=np.int32),
                      start_lane=np.full(n, lane_in, dtype=np.int32), dep=np.zeros(n, dtype=np.int32),
                      v0f=np.ones(n, dtype=np.float32))
    st = dict(status=np.ones(n, dtype=np.int32), lane=np.full(n, lane_in, dtype=np.int32),
              s=np.array([L - 1.0 - 8.0 * k for k in range(n)]), v=np.zeros(n), rc=np.zeros(n, dtype=np.int32))
    scen = sc.Scenario(net, veh, sc.Params(), "mp")
    o = _oracle(scen, st, libpath, step=66)
    o.set_signal([j], oracle.POLICY_MAX_PRESSURE)
    for k in range(40):
        st_k = o.signal_state(j)
        if k <= 29:
            assert st_k == (2, k + 1, -1), (k, st_k)
            assert o.light(jl_through, 66 + k) == oracle.LIGHT_RED
        elif k <= 32:
            assert st_k == (2, k - 29, best), (k, st_k)
            assert o.light(jl_through, 66 + k) == oracle.LIGHT_RED
        elif k == 33:
            assert st_k == (best, 1, -1), (k, st_k)
            assert o.light(jl_through, 66 + k) == oracle.LIGHT_GREEN
        if k <= 33:
            assert (o.state()["lane"] == lane_in).all()  # the queue stays until the green
        elif k == 39:
            assert (o.state()["lane"] != lane_in).any()  # and moves on after it
        o.step(1)


# ---------------------------------------------------------------------------
# Lane / road metrics (reading R24) and lane setters (reading R25)
def check_lane_queue_and_road_speed(libpath=None):
    """R24 worked by hand on one 300 m road of two lanes (and an empty road):
    queued = v < 0.1 m/s within the last 50 m."""
    cars = [(0, 295.0, 0.0),     # queued
            (0, 260.0, 0.05),    # queued (40 m from the end)
            (0, 240.0, 0.0),     # 60 m from the end: not counted
            (0, 200.0, 0.2),     # moving: not counted
            (1, 299.0, 0.0999),  # queued
            (1, 251.0, 0.1)]     # v = 0.1 is not below the threshold
    scen, st = one_road(2, 300.0, cars)
    o = _oracle(scen, st, libpath)
    q = o.lane_queue()
    assert q.tolist() == [2, 1], q
    sp = o.road_speed()
    assert abs(sp[0] - (0.0 + 0.05 + 0.0 + 0.2 + 0.0999 + 0.1) / 6.0) < 1e-12, sp
    # an empty road reports the mean speed limit of its lanes
    scen2 = corridor((300.0, 300.0), [(0, 0)], n_lanes=2)
    o2 = _oracle(scen2, None, libpath)
    sp2 = o2.road_speed()
    assert np.allclose(sp2, np.float32(13.89)), sp2


def check_lane_max_speed(libpath=None):
    """R25: a lane's new speed limit is the v0 of the next step (IDM free road,
    App. B.3 eq. (1): a = a_max (1 - (v/v0)^4))."""
    scen, st = one_road(1, 5000.0, [(0, 10.0, 4.0)])
    o = _oracle(scen, st, libpath)
    o.set_lane_max_speed([0], [5.0])
    o.step(1)
    a = 2.0 * (1.0 - (4.0 / 5.0) ** 4)
    assert abs(o.state()["v"][0] - (4.0 + a)) < 1e-12
    o.set_lane_max_speed([0], [4.0])  # v = v0: ... and a slower limit brakes the car
    v1 = o.state()["v"][0]
    o.step(1)
    assert abs(o.state()["v"][0] - (v1 + 2.0 * (1.0 - (v1 / 4.0) ** 4))) < 1e-12
    assert o.state()["v"][0] < v1


def check_lane_restriction(libpath=None):
    """R25: a restricted next lane stops the car at the end of its lane like a
    red light; a restricted adjacent lane is never the target of a lane
    change; no departure is inserted onto a restricted lane."""
    # (a) stop before a restricted junction lane, go on once it is lifted
    scen = corridor((300.0, 300.0), [(0, 0)])
    o = _oracle(scen, None, libpath)
    o.set_signal([0], oracle.POLICY_NONE)
    jl = scen.net.n_road_lanes
    o.set_lane_restriction([jl], [1])
    L0 = float(scen.net.lane_length[0])
    for t in range(150):
        o.step(1)
        stt = o.state()
        if stt["status"][0] == 1:
            assert stt["lane"][0] == 0 and L0 - stt["s"][0] >= -1e-12
    assert o.state()["v"][0] < 1e-6
    o.set_lane_restriction([jl], [0])
    o.step(60)
    assert o.state()["lane"][0] != 0
    # (b) MOBIL case A wants lane 0; restricted, it never changes
    scen, st = one_road(2, 1000.0, [(1, 100.0, 10.0), (1, 120.0, 5.0)], params=_mobil_params())
    o = _oracle(scen, st, libpath)
    o.set_lane_restriction([0], [1])
    for t in range(20):
        o.step(1)
        assert o.state()["lane"][0] == 1
    o2 = _oracle(scen, st, libpath)
    o2.step(20)
    assert (o2.state()["lane"] == 0).any()  # unrestricted, it does change
    # (c) insertion onto a restricted start lane waits
    scen = corridor((300.0, 300.0), [(0, 0), (1, 0)], n_lanes=2)
    o = _oracle(scen, None, libpath)
    o.set_lane_restriction([0], [1])
    o.step(5)
    stt = o.state()
    assert stt["status"][0] == 0 and stt["status"][1] == 1


def check_reroute(libpath=None):
    """R26 on a corridor of three 300 m roads (route 0-1-2): cut to 0-1 while
    on road 0, or to 1 while on the junction lane into road 1, the car
    arrives at the end of road 1 and never enters road 2; refused: a route not
    starting with the car's road, roads not joined, an arrived car."""
    L = 300.0
    for when in ("road", "junction"):
        scen = corridor((L, L, L), [(0, 0)], turn_len=10.0)
        net = scen.net
        o = _oracle(scen, None, libpath)
        o.set_signal(list(range(net.n_junctions)), oracle.POLICY_NONE)
        lr = net.lane_road()
        t = 0
        while True:
            st = o.state()
            lane = int(st["lane"][0])
            if when == "road" and st["status"][0] == 1 and lane == 0:
                assert not o.set_vehicle_route(0, [1, 2])      # must start with road 0
                assert o.set_vehicle_route(0, [0, 1])
                break
            if when == "junction" and st["status"][0] == 1 and lane >= net.n_road_lanes:
                assert not o.set_vehicle_route(0, [0, 1])      # the junction lane enters road 1
                assert o.set_vehicle_route(0, [1])
                break
            o.step(1)
            t += 1
            assert t < 200
        roads_seen = set()
        for k in range(400):
            o.step(1)
            st = o.state()
            if st["status"][0] == 2:
                break
            if st["lane"][0] < net.n_road_lanes:
                roads_seen.add(int(lr[st["lane"][0]]))
        assert st["status"][0] == 2 and 2 not in roads_seen, (when, roads_seen)
        assert st["rc"][0] == (1 if when == "road" else 1)  # the last road of the stored route
        assert not o.set_vehicle_route(0, [1])                # arrived
    # roads that are not joined
    scen = corridor((L, L, L), [(0, 50)])
    o = _oracle(scen, None, libpath)
    assert not o.set_vehicle_route(0, [0, 2])
    assert o.set_vehicle_route(0, [0])                         # waiting: starts with its start road


# ---------------------------------------------------------------------------
# Lane groups (reading R27)
def _groups_case(lane_idx, turn, cars_extra=(), groups=True, params=None):
    """3x3 grid of 300 m three-lane roads with turn groups; car 0 on lane
    `lane_idx` of an approach of the centre junction, 40 m from its start,
    routed to make `turn` (0 straight, 1 left, 2 right) there.  cars_extra:
    (lane index on the same road, s, v) cars going straight on.  Returns
    (scenario, state, approach lanes, out-road of car 0)."""
    net = sc.grid_network(3, 300.0, 3, 13.89, lane_groups=groups)
    ref = sc.grid_network(3, 300.0, 3, 13.89, lane_groups=True)  # turns are read from the grouped network
    lr = net.lane_road()
    nrl = net.n_road_lanes
    r_in = [r for r in range(net.n_roads) if net.road_to[r] == 4][0]
    lanes = list(range(int(net.road_lane_off[r_in]), int(net.road_lane_off[r_in + 1])))
    # the out-road reached by `turn` (its junction lane leaves lane 0 for a left turn, the last lane for a right)
    def out_road(tn):
        src = lanes[0] if tn != 2 else lanes[-1]
        jls = range(int(ref.jl_off[src]), int(ref.jl_off[src + 1]))
        return [int(lr[ref.jl_target[j - nrl]]) for j in jls if ref.jl_turn[j - nrl] == tn][0]
    r_out, r_straight = out_road(turn), out_road(0)
    cars = [(lanes[lane_idx], 40.0, 8.0)] + [(lanes[o], s_, v_) for o, s_, v_ in cars_extra]
    n = len(cars)
    veh = sc.Vehicles(n=n, route_off=np.arange(0, 2 * n + 1, 2, dtype=np.int32),
                      routes=np.array([r_in, r_out] + [r_in, r_straight] * (n - 1), dtype=np.int32),
                      start_lane=np.array([c[0] for c in cars], dtype=np.int32), dep=np.zeros(n, dtype=np.int32),
                      v0f=np.ones(n, dtype=np.float32))
    st = dict(status=np.ones(n, dtype=np.int32), lane=np.array([c[0] for c in cars], dtype=np.int32),
              s=np.array([c[1] for c in cars]), v=np.array([c[2] for c in cars]), rc=np.zeros(n, dtype=np.int32))
    scen = sc.Scenario(net, veh, params if params is not None else sc.Params(), "groups")
    return scen, st, lanes, r_out


def check_lane_group_mandatory(libpath=None):
    """R27 worked by hand: a car in the right lane that must turn left changes
    one lane to the left in each of the next two steps (free road: the
    changes are safe, no random draw) and then drives on in the left lane; a
    car alongside in the middle lane (gap <= 0) forbids the change, so the
    car stays and stops at the end of its lane."""
    scen, st, lanes, r_out = _groups_case(2, 1)
    o = _oracle(scen, st, libpath)
    o.set_signal(list(range(scen.net.n_junctions)), oracle.POLICY_NONE)
    o.step(1)
    assert o.state()["lane"][0] == lanes[1]
    o.step(1)
    assert o.state()["lane"][0] == lanes[0]
    for _ in range(60):
        o.step(1)
    lr = scen.net.lane_road()
    stt = o.state()
    assert stt["status"][0] == 2 or lr[stt["lane"][0]] == r_out or stt["lane"][0] >= scen.net.n_road_lanes
    # blocked: the middle lane holds a standing queue over its whole length
    # (5.5 m apart: no 5 m car fits) held by a red phase of the approach; the
    # car stays in its lane and stops at its end
    queue = [(1, 295.0 - 5.5 * k, 0.0) for k in range(54)]
    scen, st, lanes, _ = _groups_case(2, 1, cars_extra=queue)
    st["v"][0] = 0.0
    net = scen.net
    nrl = net.n_road_lanes
    masks = [int(net.jl_mask[j - nrl]) for l in lanes for j in range(net.jl_off[l], net.jl_off[l + 1])]
    red = [p for p in range(4) if all(((m >> p) & 1) == 0 for m in masks)][0]
    o = _oracle(scen, st, libpath)
    o.set_signal(list(range(net.n_junctions)), oracle.POLICY_MANUAL, [red] * net.n_junctions)
    # the queue cannot spread out: the outer lanes are not entered (R25)
    o.set_lane_restriction([lanes[0], lanes[2]], [1, 1])
    L = float(scen.net.lane_length[lanes[2]])
    for _ in range(120):
        o.step(1)
        stt = o.state()
        assert stt["lane"][0] == lanes[2] and stt["s"][0] <= L + 1e-12
    assert stt["v"][0] < 1e-6 and L - stt["s"][0] < 2.0 + 1e-6  # at the end of its lane


def check_lane_group_keeps_inside(libpath=None):
    """R27: a car in the left lane that turns left is in its group; behind a
    stopped car, MOBIL wants the middle lane (it does change there without
    lane groups) but the change would leave the group, so it never does."""
    p = _mobil_params()
    for groups, expect_change in ((True, False), (False, True)):
        scen, st, lanes, _ = _groups_case(0, 1, cars_extra=[(0, 60.0, 0.0)], groups=groups, params=p)
        o = _oracle(scen, st, libpath)
        o.set_signal(list(range(scen.net.n_junctions)), oracle.POLICY_NONE)
        changed = False
        for _ in range(15):
            o.step(1)
            changed |= o.state()["lane"][0] == lanes[1]
        assert changed == expect_change, groups


def check_lane_plan_switch(libpath=None):
    """R28 worked by hand: a 3x3 grid of 300 m two-lane roads with two lane
    plans (plan 0: every lane every turn; plan 1: turn groups).  A car in
    the right lane that turns left keeps its lane under plan 0; once its
    road switches to plan 1 it is outside its group and changes to the left
    lane in the next step (free road); under plan 0 again nobody has to."""
    net = sc.grid_network(3, 300.0, 2, 13.89, lane_plans=True)
    lr = net.lane_road()
    nrl = net.n_road_lanes
    r_in = [r for r in range(net.n_roads) if net.road_to[r] == 4][0]
    lanes = list(range(int(net.road_lane_off[r_in]), int(net.road_lane_off[r_in + 1])))
    jls = range(int(net.jl_off[lanes[0]]), int(net.jl_off[lanes[0] + 1]))
    r_left = [int(lr[net.jl_target[j - nrl]]) for j in jls if net.jl_turn[j - nrl] == 1][0]
    veh = sc.Vehicles(n=1, route_off=np.array([0, 2], dtype=np.int32), routes=np.array([r_in, r_left], dtype=np.int32),
                      start_lane=np.array([lanes[1]], dtype=np.int32), dep=np.zeros(1, dtype=np.int32),
                      v0f=np.ones(1, dtype=np.float32))
    st = dict(status=np.ones(1, dtype=np.int32), lane=np.array([lanes[1]], dtype=np.int32), s=np.array([40.0]),
              v=np.array([8.0]), rc=np.zeros(1, dtype=np.int32))
    scen = sc.Scenario(net, veh, sc.Params(p_attempt=0.0), "plans")
    o = _oracle(scen, st, libpath)
    o.set_signal(list(range(net.n_junctions)), oracle.POLICY_NONE)
    for _ in range(3):
        o.step(1)
        assert o.state()["lane"][0] == lanes[1]
    o.set_road_plan([r_in], [1])
    o.step(1)
    assert o.state()["lane"][0] == lanes[0]
    # back in plan 0 the left lane still has access: no change either way
    o.set_road_plan([r_in], [0])
    o.step(3)
    assert o.state()["lane"][0] == lanes[0]


# --------------------------------------------------------------------------
# Lookahead (§3.1 sensing: the first vehicle of the next lane when the own
# lane has no leader; App. B.3; reading R11).  Hand-worked on a one-lane
# corridor of three 300 m roads joined by 10 m junction lanes, all signals
# off (no stop line).  Lane ids: road lanes 0, 1, 2; junction lane 3 joins
# road 0 to road 1, junction lane 4 road 1 to road 2.  Every gap below is
# worked from the geometry: (L_lane - s_ego) + (lengths of the empty lanes
# passed) + s_rear - length, with the REARMOST vehicle of the lane seen.
# --------------------------------------------------------------------------
def _lookahead_case(cars, libpath):
    """cars: list of (lane, s, v); car 0 is the ego.  Route cursor from the
    lane: road lane r -> r, junction lane 3 / 4 -> 0 / 1 (the road just left)."""
    scen = corridor((300.0, 300.0, 300.0), [(0, 0)] * len(cars), turn_len=10.0)
    rc_of = {0: 0, 1: 1, 2: 2, 3: 0, 4: 1}
    st = dict(status=np.ones(len(cars), dtype=np.int32),
              lane=np.array([c[0] for c in cars], dtype=np.int32),
              s=np.array([c[1] for c in cars], dtype=np.float64),
              v=np.array([c[2] for c in cars], dtype=np.float64),
              rc=np.array([rc_of[c[0]] for c in cars], dtype=np.int32))
    o = _oracle(scen, st, libpath)
    o.set_signal([0, 1], oracle.POLICY_NONE)
    return o, o.decision(0)


def _assert_lookahead(o, d, leader, gap, v_ego, v_leader):
    v0 = float(np.float32(13.89))
    assert d["own_stop"] == 0
    assert d["own_has_leader"] == 1 and d["own_leader"] == leader, (d["own_leader"], leader)
    assert d["own_gap"] == gap, (d["own_gap"], gap)
    assert d["a_own"] == o.idm(v_ego, v0, gap, v_ego - v_leader)


def check_lookahead_next_lane(libpath=None):
    """Ego at the front of road 0; the junction lane holds cars at s = 8 and
    s = 1.5: the rearmost (s = 1.5) is the leader, gap (300 - 250) + 1.5 - 5."""
    o, d = _lookahead_case([(0, 250.0, 10.0), (3, 8.0, 6.0), (3, 1.5, 4.0)], libpath)
    _assert_lookahead(o, d, 2, 46.5, 10.0, 4.0)


def check_lookahead_second_lane(libpath=None):
    """Empty junction lane: the rearmost car of road 1 (s = 20 among s = 20,
    60) leads; the gap adds the 10 m junction lane: 50 + 10 + 20 - 5."""
    o, d = _lookahead_case([(0, 250.0, 10.0), (1, 60.0, 9.0), (1, 20.0, 3.0)], libpath)
    _assert_lookahead(o, d, 2, 75.0, 10.0, 3.0)


def check_lookahead_from_junction_lane(libpath=None):
    """Ego on junction lane 3 at s = 4 with road 1 empty: the lane after road
    1 on the route (junction lane 4) is searched: (10 - 4) + 300 + 3 - 5."""
    o, d = _lookahead_case([(3, 4.0, 8.0), (4, 3.0, 2.0)], libpath)
    _assert_lookahead(o, d, 1, 304.0, 8.0, 2.0)


def check_lookahead_bounded(libpath=None):
    """At most two lanes are searched: with the junction lane and road 1 empty,
    a car on junction lane 4 is not seen (free road), nor is anything when
    both next lanes are empty; an own-lane leader is used before any car
    ahead on the next lanes."""
    v0 = float(np.float32(13.89))
    for cars in ([(0, 250.0, 10.0), (4, 5.0, 0.0)], [(0, 250.0, 10.0)]):
        o, d = _lookahead_case(cars, libpath)
        assert d["own_has_leader"] == 0 and d["own_leader"] == -1, d
        assert d["a_own"] == o.idm_free(10.0, v0)
    o, d = _lookahead_case([(0, 250.0, 10.0), (0, 290.0, 7.0), (3, 2.0, 0.0)], libpath)
    _assert_lookahead(o, d, 1, 35.0, 10.0, 7.0)


# --------------------------------------------------------------------------
# Randomized MOBIL draws and direction (App. B.3; readings R3-R6): the
# attempt gate u_att < p_attempt, the change gate u_lc < p_LC(u_T), and the
# side (u_T > 0: left iff u_dir u_T < max(0, u_L); u_T = 0: uniform over the
# feasible sides).  The uniforms are checked against the Philox4x32-10 words
# of counter (vehicle id, step, 0, 0) (the generator is pinned by its known
# answer); u_L, u_R come from states whose utilities the hand cases pin.
# --------------------------------------------------------------------------
def _draws(k0, k1, vid, t):
    w = oracle.philox4x32_10(k0, k1, [vid, t, 0, 0])
    return [float(int(x) >> 8) * 2.0 ** -24 for x in w[:3]]


def _p_lc_reading(p, uT):
    if uT >= 1.0:
        return p.p_hi
    if uT > 0.0:
        return p.p_lo + (p.p_hi - p.p_lo) * uT
    return p.p_lo


def _gate_and_side(d, p):
    """(attempted, candidate, direction) the readings give for decision d."""
    att = d["u_att"] < p.p_attempt
    uLp = d["uL"] if (d["feasL"] and d["uL"] > 0) else 0.0
    uRp = d["uR"] if (d["feasR"] and d["uR"] > 0) else 0.0
    uT = uLp + uRp
    if not att or not d["u_lc"] < _p_lc_reading(p, uT):
        return att, False, 0
    if uT > 0:
        return att, True, -1 if d["u_dir"] * uT < uLp else 1
    sides = [s for s, f in ((-1, d["feasL"]), (1, d["feasR"])) if f]
    if not sides:
        return att, False, 0
    if len(sides) == 2:
        return att, True, -1 if d["u_dir"] < 0.5 else 1
    return att, True, sides[0]


def _scan_gates(cars, p, libpath, steps=300, n_lanes=3):
    scen, st = one_road(n_lanes, 1000.0, cars, params=p)
    o = _oracle(scen, st, libpath)
    k0, k1 = p.seed & 0xFFFFFFFF, (p.seed >> 32) ^ p.scenario
    seen = {"att": 0, "cand": 0, "left": 0, "right": 0}
    last = None
    for t in range(steps):
        o.set_state(st["status"], st["lane"], st["s"], st["v"], st["rc"], t)
        d = o.decision(0)
        assert [d["u_att"], d["u_lc"], d["u_dir"]] == _draws(k0, k1, 0, t), t
        att, cand, dr = _gate_and_side(d, p)
        assert d["attempted"] == att and d["cand"] == cand, (t, d)
        if cand:
            assert d["dir"] == dr, (t, d)
            seen["left" if dr < 0 else "right"] += 1
        seen["att"] += att
        seen["cand"] += cand
        if att:
            last = d
    return seen, last


def check_mobil_draw_gates(libpath=None):
    """Ego in the middle of three lanes behind a slow leader (case A's own
    lane), both adjacent lanes empty: u_L = u_R > 0 (the mirror pin), u_T >=
    1, p_LC = p_hi; over 300 steps of draws every attempt / change / side
    decision is the one the gates give, and both sides occur."""
    p = sc.Params(seed=7)
    seen, d = _scan_gates([(1, 100.0, 10.0), (1, 120.0, 5.0)], p, libpath)
    assert d["uL"] == d["uR"] > 0 and d["feasL"] == d["feasR"] == 1 and d["pLC"] == p.p_hi
    assert seen["left"] > 10 and seen["right"] > 10, seen
    # unequal utilities on both sides (a car 50 m ahead in the right lane
    # lowers u_R, a larger threshold lowers both): 0 < u_R < u_L, u_T in
    # (0, 1), p_LC on its linear branch; left is taken about u_L / u_T of
    # the time, right otherwise
    p2 = sc.Params(seed=11, a_th=1.5)
    seen2, d2 = _scan_gates([(1, 100.0, 10.0), (1, 125.0, 8.0), (2, 150.0, 8.0)], p2, libpath)
    assert d2["feasL"] == d2["feasR"] == 1 and 0.0 < d2["uR"] < d2["uL"] and 0.0 < d2["uT"] < 1.0, d2
    assert p2.p_lo < d2["pLC"] < p2.p_hi
    assert seen2["left"] > seen2["right"] > 3 and seen2["att"] > seen2["cand"], seen2


def check_mobil_uniform_side(libpath=None):
    """u_T = 0 (a lone car on free road: u = -a_th on every side) with p_lo
    raised to 0.3 so that changes occur: a change iff u_lc < 0.3, left iff
    u_dir < 0.5 when both sides are feasible, the only feasible side
    otherwise (ego on the leftmost lane: always right)."""
    p = sc.Params(seed=3, p_lo=0.3, p_attempt=1.0)
    seen, d = _scan_gates([(1, 100.0, 10.0)], p, libpath)
    assert d["uT"] == 0.0 and d["pLC"] == 0.3
    assert seen["left"] > 10 and seen["right"] > 10, seen
    seen2, _ = _scan_gates([(0, 100.0, 10.0)], p, libpath)
    assert seen2["cand"] > 10 and seen2["left"] == 0, seen2


def check_mobil_gate_boundaries(libpath=None):
    """The gates are strict: with p_attempt set to the step's own u_att no
    attempt is made, with p_hi (u_T >= 1) set to the step's own u_lc no change
    is made, and one unit of 2^-24 above each, they pass."""
    cars = [(1, 100.0, 10.0), (1, 120.0, 5.0)]
    base = sc.Params(seed=7, p_attempt=1.0)
    scen, st = one_road(3, 1000.0, cars, params=base)
    d0 = _oracle(scen, st, libpath, step=17).decision(0)
    ua, ul = d0["u_att"], d0["u_lc"]
    assert 0.0 < ua < 1.0 and 0.0 < ul < 0.9
    for p_att, want in ((ua, 0), (ua + 2.0 ** -24, 1)):
        s2, st2 = one_road(3, 1000.0, cars, params=sc.Params(seed=7, p_attempt=p_att))
        assert _oracle(s2, st2, libpath, step=17).decision(0)["attempted"] == want, (p_att, want)
    for p_hi, want in ((ul, 0), (ul + 2.0 ** -24, 1)):
        s2, st2 = one_road(3, 1000.0, cars, params=sc.Params(seed=7, p_attempt=1.0, p_hi=p_hi))
        d = _oracle(s2, st2, libpath, step=17).decision(0)
        assert d["pLC"] == p_hi and d["cand"] == want, (p_hi, want, d)


ALL_CHECKS = [
    check_idm_free_road, check_idm_equilibrium, check_p_lc, check_mobil_case_A,
    check_mobil_case_B, check_mobil_case_C, check_mobil_case_D, check_mobil_mirror, check_neighbours_bruteforce,
    check_free_road_vs_rk4, check_platoon_equilibrium, check_red_light, check_signal_program,
    check_arrival_and_travel_time, check_insertion, check_conflict, check_max_pressure_argmax,
    check_max_pressure_timing, check_lane_queue_and_road_speed, check_lane_max_speed,
    check_lane_restriction, check_reroute, check_lane_group_mandatory, check_lane_group_keeps_inside,
    check_lane_plan_switch, check_lookahead_next_lane, check_lookahead_second_lane,
    check_lookahead_from_junction_lane, check_lookahead_bounded, check_mobil_draw_gates,
    check_mobil_uniform_side, check_mobil_gate_boundaries,
]
