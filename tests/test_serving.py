"""Serving loop: admission by device-memory budget, overlap of rollouts on the
device, and every rollout's result identical alone and in the mix."""
import numpy as np
import pytest

from paper_2406_10661_gb300 import binding, scenario as sc
from paper_2406_10661_gb300 import serving


def _requests(k=4, horizons=(150, 90, 200, 120)):
    out = []
    for i in range(k):
        scen = sc.small_scenario(seed=i + 1)
        scen.params.scenario = i
        out.append(serving.Request(rid=i, scenario=scen, horizon=horizons[i % len(horizons)],
                                   arrival=0.01 * i, action_seed=100 + i))
    return out


def test_poisson_requests_shape():
    made = []
    reqs = serving.poisson_requests(50, rate_hz=20.0, seed=3,
                                    make=lambda i, G, n, h, s: made.append((G, n, h)) or
                                    sc.Scenario(None, None, sc.Params()))
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) > 0) and 1.0 < arr[-1] < 6.0  # ~50 / 20 s
    G = np.array([m[0] for m in made]); n = np.array([m[1] for m in made]); h = np.array([m[2] for m in made])
    assert G.min() >= 5 and G.max() <= 40 and n.min() >= 5000 and n.max() <= 500_000
    assert h.min() >= 300 and h.max() <= 3600
    reqs2 = serving.poisson_requests(50, rate_hz=20.0, seed=3, make=lambda *a: None)
    assert [r.arrival for r in reqs2] == [r.arrival for r in reqs] and [r.horizon for r in reqs2] == list(h)


def test_actions_reproducible():
    r = _requests(1)[0]
    a = serving.actions_for(r, 10, 16)
    assert np.array_equal(a, serving.actions_for(r, 10, 16)) and a.min() >= 0 and a.max() < 4


def _run_plain(req, every=10):
    """The request on a handle of its own (moss_create), outside any server:
    its actions every `every` steps, then its steps up to the next action."""
    scen = req.scenario
    sim = binding.Simulation(scen.net, scen.veh, scen.params)
    nj = int(scen.net.n_junctions)
    t = 0
    while t < req.horizon:
        sim.set_signal_phase(np.arange(nj, dtype=np.int32), serving.actions_for(req, t, nj))
        k = min(every, req.horizon - t)
        sim.step(k)
        t += k
    m, st = sim.metrics(), sim.state()
    sim.close()
    return m, st


@pytest.mark.gpu
def test_alone_equals_mixed():
    """Requests of different sizes and horizons (not multiples of the action
    interval) share the launches of one slot batch: each result equals the
    request run alone in a one-slot server and on a handle of its own."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    mixed = _requests(6, horizons=(150, 93, 200, 121, 67, 180))
    mixed[4].scenario = sc.medium_scenario(n=20_000)
    mixed[4].scenario.params.scenario = 4
    stats = serving.Server(1 << 34, max_slots=3, keep_state=True).run(mixed, realtime=False)
    assert stats["peak_slots"] >= 2  # the rollouts overlapped
    assert stats["slot_steps"] < sum(r.horizon for r in mixed)  # launches were shared
    for r in mixed:
        alone = _requests(6, horizons=(150, 93, 200, 121, 67, 180))[r.rid]
        if r.rid == 4:
            alone.scenario = mixed[4].scenario
        serving.Server(1 << 34, max_slots=1, keep_state=True).run([alone], realtime=False)
        assert alone.metrics == r.metrics, r.rid
        for k in ("status", "lane", "rc", "s", "v", "flags"):
            assert np.array_equal(alone.state[k], r.state[k]), (r.rid, k)
        assert r.metrics["step"] == r.horizon and len(r.step_ms) == r.horizon
        m, st = _run_plain(r)
        assert m == r.metrics, r.rid
        for k in ("status", "lane", "rc", "s", "v", "flags"):
            assert np.array_equal(st[k], r.state[k]), (r.rid, k)


@pytest.mark.gpu
def test_slot_reuse_and_refusals():
    """A slot is reused after a retire and a step; loading into a busy slot,
    a retired slot before its vehicles left, or a scenario larger than the
    slot is refused, and the slot stays usable."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    a, b = sc.small_scenario(seed=1), sc.small_scenario(seed=2)
    big = sc.medium_scenario(n=20_000)
    caps = binding.slot_caps(a)
    slots = binding.Slots([caps], a.params)
    slots.load(0, a)
    with pytest.raises(binding.MossError):
        slots.load(0, b)  # busy
    slots.step(60)
    m1 = slots.metrics(0)
    slots.retire(0)
    with pytest.raises(binding.MossError):
        slots.load(0, b)  # its vehicles are still there
    slots.step(1)
    with pytest.raises(binding.MossError):
        slots.load(0, big)  # too large
    slots.load(0, b)
    slots.step(60)
    ref = binding.Simulation(b.net, b.veh, b.params)
    ref.step(60)
    assert slots.metrics(0) == ref.metrics() and m1["step"] == 60
    st, rs = slots.state(0), ref.state()
    for k in st:
        assert np.array_equal(st[k], rs[k]), k


@pytest.mark.gpu
def test_budget_admission():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    reqs = _requests()
    one = serving.estimate_slot_bytes(binding.slot_caps(reqs[0].scenario))
    srv = serving.Server(int(2.5 * one), max_slots=8)
    stats = srv.run(reqs, realtime=False)
    assert stats["peak_slots"] <= 2 and all(r.metrics is not None for r in reqs)
    with pytest.raises(binding.MossError) as e:
        serving.Server(one // 2).run(_requests(1), realtime=False)
    assert e.value.code == binding.MOSS_EBUDGET
