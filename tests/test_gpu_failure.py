"""Failure detection on the GPU without a fault: a bounded device wait on a
flag that nothing sets gives up, the kernel reports it, the host reads
MOSS_ETIMEOUT, and the CUDA context stays usable afterwards."""
import time

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


def test_bounded_wait_gives_up_and_reports():
    t0 = time.perf_counter()
    rc = binding.moss_selftest_bounded_wait()
    dt = time.perf_counter() - t0
    assert rc == binding.MOSS_ETIMEOUT, rc
    assert dt < 30.0
    # the context still works: a small simulation steps and reports no error
    scen = sc.small_scenario()
    sim = binding.Simulation(scen.net, scen.veh, scen.params, precision=32)
    sim.step(50)
    m = sim.metrics()
    assert m["errors"] == 0 and m["step"] == 50 and m["n_active"] > 0
    sim.close()
