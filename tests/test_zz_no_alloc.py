"""The allocation-free lane-offset entry point (moss_lane_offsets_noalloc).

It serves callers that cannot call cudaMalloc.  The check: for two steps in a
row of a simulation run through the existing entry points (moss_set_state,
moss_step, moss_get_state), feed the per-lane sizes of the state before the
step and the per-lane leave/enter counts of the step to the allocation-free
call, and compare its lane offsets with those of the state moss_step
produced (integers: exact).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2406_10661_gb300 import binding, scenario as sc

pytestmark = pytest.mark.gpu


def _lane_sizes(st, n_lanes):
    act = st["status"] == 1
    return np.bincount(st["lane"][act], minlength=n_lanes).astype(np.int64)


def _leave_enter(a, b, n_lanes):
    """per-lane counts of vehicles that left / entered a lane between states a and b"""
    was = a["status"] == 1
    now = b["status"] == 1
    moved_out = was & (~now | (b["lane"] != a["lane"]))
    moved_in = now & (~was | (b["lane"] != a["lane"]))
    leave = np.bincount(a["lane"][moved_out], minlength=n_lanes)
    enter = np.bincount(b["lane"][moved_in], minlength=n_lanes)
    return leave.astype(np.int64), enter.astype(np.int64)


def test_noalloc_lane_offsets_match_step():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    scen = sc.small_scenario()
    n_lanes = scen.net.n_lanes
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=32)
    sim.step(200)
    before = sim.state()
    dev = torch.device("cuda")
    for call in range(2):  # two calls in a row
        sim.step(1)
        after = sim.state()
        size0 = _lane_sizes(before, n_lanes)
        leave, enter = _leave_enter(before, after, n_lanes)
        off_cur = np.zeros(n_lanes + 1, dtype=np.int32)
        off_cur[1:] = np.cumsum(size0)
        want_off = np.zeros(n_lanes + 1, dtype=np.int64)
        want_off[1:] = np.cumsum(_lane_sizes(after, n_lanes))
        want_lb = np.concatenate([[0], np.cumsum(leave)[:-1]])
        d_cur = torch.tensor(off_cur, device=dev)
        d_leave = torch.tensor(leave.astype(np.int32), device=dev)
        d_enter = torch.tensor(enter.astype(np.int32), device=dev)
        d_next = torch.full((n_lanes + 1,), -7, dtype=torch.int32, device=dev)
        d_lb = torch.full((n_lanes,), -7, dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        rc = binding.moss_lane_offsets_noalloc(n_lanes, d_cur.data_ptr(), d_leave.data_ptr(),
                                               d_enter.data_ptr(), d_next.data_ptr(), d_lb.data_ptr(),
                                               stream)
        assert rc == binding.MOSS_OK
        torch.cuda.synchronize()
        assert np.array_equal(d_next.cpu().numpy().astype(np.int64), want_off), call
        assert np.array_equal(d_lb.cpu().numpy().astype(np.int64), want_lb), call
        before = after


def _noalloc_random(n_lanes, seed, torch):
    """random per-lane sizes, leave <= size and enter counts; the expected
    offsets and leaver prefix by numpy cumsum"""
    rng = np.random.default_rng(seed)
    size = rng.integers(0, 13, n_lanes).astype(np.int64)
    leave = (rng.random(n_lanes) * (size + 1)).astype(np.int64)
    enter = rng.integers(0, 4, n_lanes).astype(np.int64)
    off_cur = np.zeros(n_lanes + 1, dtype=np.int64)
    off_cur[1:] = np.cumsum(size)
    want_off = np.zeros(n_lanes + 1, dtype=np.int64)
    want_off[1:] = np.cumsum(size - leave + enter)
    want_lb = np.concatenate([[0], np.cumsum(leave)[:-1]])
    dev = torch.device("cuda")
    args = [torch.tensor(x.astype(np.int32), device=dev) for x in (off_cur, leave, enter)]
    return args, want_off, want_lb


@pytest.mark.parametrize("n_lanes", [3 * 1024 + 5, 200_003, 362_353, binding.NOALLOC_MAX_LANES])
def test_noalloc_many_tiles(n_lanes):
    """Sizes with many scan tiles (1,024 lanes each): more tiles than the grid
    has blocks, so blocks take several tickets and the look-back walks over
    earlier tiles; up to the largest size accepted.  Two calls in a row on one
    stream with different inputs (each call clears the shared scratch), both
    exact."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    stream = torch.cuda.current_stream().cuda_stream
    dev = torch.device("cuda")
    outs = []
    for call in range(2):
        (d_cur, d_leave, d_enter), want_off, want_lb = _noalloc_random(n_lanes, 17 + call, torch)
        d_next = torch.full((n_lanes + 1,), -7, dtype=torch.int32, device=dev)
        d_lb = torch.full((n_lanes,), -7, dtype=torch.int32, device=dev)
        rc = binding.moss_lane_offsets_noalloc(n_lanes, d_cur.data_ptr(), d_leave.data_ptr(), d_enter.data_ptr(),
                                               d_next.data_ptr(), d_lb.data_ptr(), stream)
        assert rc == binding.MOSS_OK
        outs.append((d_next, d_lb, want_off, want_lb))
    torch.cuda.synchronize()
    for call, (d_next, d_lb, want_off, want_lb) in enumerate(outs):
        assert np.array_equal(d_next.cpu().numpy().astype(np.int64), want_off), call
        assert np.array_equal(d_lb.cpu().numpy().astype(np.int64), want_lb), call


def test_noalloc_flags_negative_size():
    """A lane whose leavers exceed its size plus entrants (a violated
    precondition) is reported: the total offset reads -1."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    n_lanes = 5000
    (d_cur, d_leave, d_enter), _, _ = _noalloc_random(n_lanes, 3, torch)
    d_leave[4321] = int(d_cur[4322] - d_cur[4321]) + int(d_enter[4321]) + 1
    dev = torch.device("cuda")
    d_next = torch.zeros(n_lanes + 1, dtype=torch.int32, device=dev)
    d_lb = torch.zeros(n_lanes, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    assert binding.moss_lane_offsets_noalloc(n_lanes, d_cur.data_ptr(), d_leave.data_ptr(), d_enter.data_ptr(),
                                             d_next.data_ptr(), d_lb.data_ptr(), stream) == binding.MOSS_OK
    torch.cuda.synchronize()
    assert int(d_next[n_lanes]) == -1


def test_noalloc_rejects_oversize():
    binding.load()
    assert binding.moss_lane_offsets_noalloc(binding.NOALLOC_MAX_LANES + 1, 1, 1, 1, 1, 1) == binding.MOSS_EINVAL
