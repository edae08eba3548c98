"""Metrics read without waiting for the stream (moss_metrics_enqueue /
moss_metrics_read): a slot holds the metrics as they were when it was
enqueued, later steps do not change it, and misuse is refused."""
import numpy as np
import pytest

from paper_2406_10661_gb300 import binding, scenario as sc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    binding.load()


def test_metric_slots_hold_the_enqueued_state():
    scen = sc.small_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params)
    ref = binding.Simulation(scen.net, scen.veh, scen.params)
    sim.step(40)
    sim.metrics_enqueue(0)
    sim.step(25)
    sim.metrics_enqueue(3)
    sim.step(10)
    a, b = sim.metrics_read(0), sim.metrics_read(3)
    ref.step(40)
    assert a == ref.metrics()
    ref.step(25)
    assert b == ref.metrics()
    assert a["step"] == 40 and b["step"] == 65 and sim.metrics()["step"] == 75


def test_pipelined_reads_match_synchronous_reads():
    scen = sc.small_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params)
    ref = binding.Simulation(scen.net, scen.veh, scen.params)
    got, want = [], []
    for k in range(12):
        sim.step(1)
        sim.metrics_enqueue(k % 2)
        if k > 0:
            got.append(sim.metrics_read((k - 1) % 2))
        ref.step(1)
        want.append(ref.metrics())
    got.append(sim.metrics_read(11 % 2))
    assert got == want


def test_batch_slots_per_scenario():
    scens = sc.batched_scenarios(3, n_lo=500, n_hi=3000)
    b = binding.Batch(scens)
    b.step(30)
    for i in range(3):
        b.metrics_enqueue(i, scenario=i)
    for i in range(3):
        assert b.metrics_read(i) == b.metrics(i)


def test_metric_slot_misuse_refused():
    scen = sc.small_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params)
    with pytest.raises(binding.MossError):
        sim.metrics_read(1)          # nothing enqueued
    with pytest.raises(binding.MossError):
        sim.metrics_enqueue(binding.METRIC_SLOTS)
    with pytest.raises(binding.MossError):
        sim.metrics_enqueue(0, scenario=1)
    sim.metrics_enqueue(1)
    sim.metrics_read(1)
    with pytest.raises(binding.MossError):
        sim.metrics_read(1)          # already read
