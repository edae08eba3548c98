"""Host helpers of the benchmark that decide which evidence a bench line
carries: the kernel code hash ignores comments and blank space but not code,
and a capture's DRAM traffic is reported only for its own workload and code."""
import os

import pytest

bench = pytest.importorskip("bench")


def _hash_of(tmp_path, texts):
    files = []
    for k, t in enumerate(texts):
        p = tmp_path / f"k{k}.cuh"
        p.write_text(t)
        files.append(str(p))
    old = bench.KERNEL_SOURCES
    try:
        bench.KERNEL_SOURCES = files
        return bench.kernel_source_hash()
    finally:
        bench.KERNEL_SOURCES = old


def test_code_hash_ignores_comments_not_code(tmp_path):
    base = _hash_of(tmp_path, ["int f(int x) { return x + 1; }  // add one\n", "/* two */ int g;\n"])
    assert base == _hash_of(tmp_path, ["// a new comment\nint f(int x) {\n  return x + 1;\n}\n",
                                        "int g;  /* changed\n comment */\n"])
    assert base != _hash_of(tmp_path, ["int f(int x) { return x + 2; }  // add one\n", "/* two */ int g;\n"])


def test_traffic_only_for_matching_workload_and_code(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    (tmp_path / "step_kernels_wl.md").write_text(
        f"# x\n\ntraffic: k_decide 123 sha256:{h}\ntraffic: k_place 456 sha256:{'0' * 64}\n")
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    assert bench.captured_traffic("k_decide", "wl") == 123.0
    assert bench.captured_traffic("k_place", "wl") is None        # captured from other code
    assert bench.captured_traffic("k_decide", "other") is None    # no capture of that workload


def test_committed_profiles_have_traffic_lines():
    """Every committed launch-list summary carries one well-formed traffic line
    (bytes per launch and the SHA-256 of the code it was captured from) for
    each of the three step kernels."""
    import re
    prof = os.path.join(bench.ROOT, "profiles")
    names = [f for f in os.listdir(prof) if f.startswith("step_kernels_")]
    assert "step_kernels_city100x100_2464950.md" in names
    pat = re.compile(r"^traffic: (k_decide|k_lanescan|k_place) [0-9]+ sha256:[0-9a-f]{64}$")
    for f in names:
        with open(os.path.join(prof, f)) as fh:
            kernels = [m.group(1) for m in (pat.match(line.strip()) for line in fh) if m]
        assert sorted(kernels) == ["k_decide", "k_lanescan", "k_place"], f
