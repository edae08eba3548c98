"""Max-pressure signal policy (reading R23) on the GPU against the FP64
oracle: identical vehicle and signal states over FP64 rollouts, network
speed and completions within 0.5% in FP32."""
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


def _both(scen, precision):
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=precision)
    ora = oracle.Oracle(scen.net, scen.veh, scen.params)
    return sim, ora


def _signal_states_equal(sim, ora, net):
    ids = np.arange(net.n_junctions, dtype=np.int32)
    ph, el, nx = sim.signal_state(ids)
    for j in range(net.n_junctions):
        p, e, q = ora.signal_state(j)
        assert (ph[j], el[j], nx[j]) == (p, e, q), (j, (ph[j], el[j], nx[j]), (p, e, q))


@pytest.mark.parametrize("t_switch", [0, 45])
def test_fp64_rollout_max_pressure_small(t_switch):
    scen = sc.small_scenario()
    sim, ora = _both(scen, 64)
    J = list(range(scen.net.n_junctions))
    sim.step(t_switch); ora.step(t_switch)
    sim.set_signal_policy(J, binding.POLICY_MAX_PRESSURE)
    ora.set_signal(J, oracle.POLICY_MAX_PRESSURE)
    _signal_states_equal(sim, ora, scen.net)
    changes = 0
    prev = sim.signal_state(np.arange(len(J), dtype=np.int32))[0].copy()
    for chunk in range(12):
        sim.step(50); ora.step(50)
        g, r = sim.state(), ora.state()
        assert np.array_equal(g["status"], r["status"])
        act = r["status"] == 1
        assert np.array_equal(g["lane"][act], r["lane"][act])
        assert np.abs(g["s"][act] - r["s"][act]).max(initial=0) < 1e-6
        assert np.abs(g["v"][act] - r["v"][act]).max(initial=0) < 1e-6
        assert np.array_equal(g["flags"], r["flags"])
        _signal_states_equal(sim, ora, scen.net)
        cur = sim.signal_state(np.arange(len(J), dtype=np.int32))[0]
        changes += int((cur != prev).sum())
        prev = cur.copy()
    assert changes > 0  # the policy does switch phases
    gm, rm = sim.metrics(), ora.metrics()
    for k in ("n_active", "n_arrived", "vehicle_updates", "lane_changes", "flagged", "inserted"):
        assert gm[k] == rm[k], (k, gm[k], rm[k])


def test_fp32_rollout_max_pressure_aggregates():
    scen = sc.small_scenario()
    sim, ora = _both(scen, 32)
    J = list(range(scen.net.n_junctions))
    sim.set_signal_policy(J, binding.POLICY_MAX_PRESSURE)
    ora.set_signal(J, oracle.POLICY_MAX_PRESSURE)
    sim.step(600); ora.step(600)
    gm, rm = sim.metrics(), ora.metrics()
    gs, rs = gm["speed_sum"] / gm["vehicle_updates"], rm["speed_sum"] / rm["vehicle_updates"]
    assert abs(gs - rs) <= 0.005 * rs, (gs, rs)
    assert abs(gm["n_arrived"] - rm["n_arrived"]) <= max(1, 0.005 * rm["n_arrived"])
    assert gm["errors"] == 0


def test_signal_state_of_fixed_and_none():
    """The getter on the other policies: the fixed program's phase and amber
    (next phase p+1), and -1 for a junction without signal."""
    scen = sc.small_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=32)
    ids = np.arange(scen.net.n_junctions, dtype=np.int32)
    for t in range(0, 140, 7):
        ph, el, nx = sim.signal_state(ids)
        x = t % 132
        exp_p, exp_amber = x // 33, (x % 33) >= 30
        assert (ph == exp_p).all() and (el == 0).all(), (t, ph)
        assert ((nx == (exp_p + 1) % 4) if exp_amber else (nx == -1)).all(), (t, nx)
        sim.step(7)
    sim.set_signal_policy([0], binding.POLICY_NONE)
    ph, el, nx = sim.signal_state(np.array([0], dtype=np.int32))
    assert ph[0] == -1 and nx[0] == -1
