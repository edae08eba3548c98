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


def test_torch_allocator_backs_the_handle():
    """A handle whose device buffers come from PyTorch's caching allocator
    (moss_batch_create_with_allocator): the bytes torch reports allocated grow
    by at least the handle's size, the rollout equals one on cudaMalloc'd
    buffers (including a re-route, whose device scratch comes from the
    allocator too), and destroying the handle gives the memory back to
    torch's pool."""
    import torch
    scen = sc.small_scenario()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    alloc = binding.torch_allocator()
    sim = binding.Simulation(scen.net, scen.veh, scen.params, allocator=alloc)
    ref = binding.Simulation(scen.net, scen.veh, scen.params)
    assert torch.cuda.memory_allocated() - before >= sim.device_bytes() > 0
    sim.step(150); ref.step(150)
    # a re-route of a waiting vehicle (setter scratch from the allocator)
    st = ref.state()
    waiting = np.nonzero(st["status"] == 0)[0]
    if len(waiting):
        vid = int(waiting[-1])
        r0 = int(scen.veh.routes[scen.veh.route_off[vid]])
        for s_ in (sim, ref):
            s_.set_vehicle_route([vid], [[r0]])
    sim.step(150); ref.step(150)
    a, b = sim.state(), ref.state()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert sim.metrics() == ref.metrics()
    sim.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() <= before + 4096


def test_allocator_with_one_function_is_refused():
    scen = sc.small_scenario()
    bad = binding.MossAllocator(binding.torch_allocator().alloc, binding.RELEASE_FN(), None)
    with pytest.raises(binding.MossError):
        binding.Simulation(scen.net, scen.veh, scen.params, allocator=bad)


@pytest.mark.parametrize("precision", [32, 64])
def test_schedules_give_the_same_results(precision):
    """Every launch schedule (blocks per SM, the road-lane weight of the
    decide runs, the lane-scan tile, the step mode) advances the simulation
    identically; the autotuner steps it normally and reports its choice."""
    scen = sc.medium_scenario(n=15_000)
    ref = binding.Simulation(scen.net, scen.veh, scen.params, precision=precision)
    ref.step(150)
    want_state, want_metrics = ref.state(), ref.metrics()
    schedules = [dict(decide=3, lanescan=1, place=4, road_weight=1, lanes_per_thread=8, step_mode=0,
                      candidates_per_block=0),
                 dict(decide=5, lanescan=2, place=16, road_weight=3, lanes_per_thread=16, step_mode=0,
                      candidates_per_block=1),
                 dict(decide=4, lanescan=4, place=8, road_weight=2, lanes_per_thread=8, step_mode=1,
                      candidates_per_block=256)]
    for sched in schedules:
        sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=precision)
        sim.step(40)
        sim.set_schedule(**sched)
        assert sim.schedule() == sched
        sim.step(110)
        st = sim.state()
        for k in want_state:
            assert np.array_equal(st[k], want_state[k]), (sched, k)
        assert sim.metrics() == want_metrics, sched
        sim.close()
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=precision)
    sim.step(100)
    chosen = sim.autotune(2)  # 32 (or 28) more steps
    assert set(chosen) == set(binding.Simulation.SCHEDULE_KEYS)
    assert chosen["lanes_per_thread"] in (8, 16) and chosen["step_mode"] in (0, 1)
    steps = 150 - sim.metrics()["step"]
    assert steps >= 0
    sim.step(steps)
    st = sim.state()
    for k in want_state:
        assert np.array_equal(st[k], want_state[k]), k
    sim.close()


def test_schedule_out_of_range_refused():
    scen = sc.small_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params)
    before = sim.schedule()
    for bad in (dict(decide=0), dict(road_weight=9), dict(lanes_per_thread=12), dict(step_mode=2),
                dict(place=33), dict(candidates_per_block=257), dict(candidates_per_block=-1)):
        with pytest.raises(binding.MossError):
            sim.set_schedule(**bad)
        assert sim.schedule() == before
    sim.step(5)
    assert sim.metrics()["step"] == 5
