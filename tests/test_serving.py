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


@pytest.mark.gpu
def test_alone_equals_mixed():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    mixed = _requests()
    stats = serving.Server(1 << 34, max_slots=8, keep_state=True).run(mixed, realtime=False)
    assert stats["peak_slots"] >= 2  # the rollouts overlapped
    for r in mixed:
        alone = _requests()[r.rid]
        serving.Server(1 << 34, max_slots=1, keep_state=True).run([alone], realtime=False)
        assert alone.metrics == r.metrics, r.rid
        for k in ("status", "lane", "rc", "s", "v", "flags"):
            assert np.array_equal(alone.state[k], r.state[k]), (r.rid, k)
        assert r.metrics["step"] == r.horizon and len(r.step_ms) == r.horizon


@pytest.mark.gpu
def test_budget_admission():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    reqs = _requests()
    one = serving.estimate_device_bytes(reqs[0].scenario)
    srv = serving.Server(int(2.5 * one), max_slots=8)
    stats = srv.run(reqs, realtime=False)
    assert stats["peak_slots"] <= 2 and all(r.metrics is not None for r in reqs)
    with pytest.raises(binding.MossError) as e:
        serving.Server(one // 2).run(_requests(1), realtime=False)
    assert e.value.code == binding.MOSS_EBUDGET
