"""The C-ABI library: every symbol the header declares is exported, the
binding covers exactly those, and invalid inputs are rejected on the host
(no GPU needed: validation runs before any CUDA call)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2406_10661_gb300 import binding, scenario as sc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "moss.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(moss_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(binding.LIB_PATH)
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    assert sorted(binding.SIGNATURES) == _declared()


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        binding._LIB = None
        try:
            binding.load(str(tmp_path / "nope.so"))
        finally:
            binding._LIB = None


def _scen():
    return sc.small_scenario()


@pytest.mark.parametrize("mutate,what", [
    (lambda s: setattr(s.params, "delta", 2.0), "delta"),
    (lambda s: s.net.lane_length.__setitem__(3, 0.0), "length"),
    (lambda s: s.veh.start_lane.__setitem__(0, (s.veh.start_lane[0] + 2) % s.net.n_road_lanes), "start lane"),
    (lambda s: s.veh.routes.__setitem__(1, s.veh.routes[0]), "route turn"),
    (lambda s: s.veh.dep.__setitem__(5, -1), "departure"),
    (lambda s: s.net.jl_target.__setitem__(0, s.net.n_road_lanes + 5), "jl target"),
])
def test_invalid_inputs_rejected(mutate, what):
    s = _scen()
    mutate(s)
    with pytest.raises(binding.MossError) as e:
        binding.Simulation(s.net, s.veh, s.params)
    assert e.value.code == binding.MOSS_EINVAL, what


def test_bad_precision_rejected():
    s = _scen()
    with pytest.raises(binding.MossError) as e:
        binding.Simulation(s.net, s.veh, s.params, precision=16)
    assert e.value.code == binding.MOSS_EINVAL


def test_batch_needs_equal_model_parameters():
    a, b = _scen(), _scen()
    b.params.T = 1.2
    with pytest.raises(binding.MossError) as e:
        binding.Batch([a, b])
    assert e.value.code == binding.MOSS_EINVAL
