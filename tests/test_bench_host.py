"""Host-side arithmetic of bench.py on CPU: the offered serving stream, the
check that ties committed ncu counters to the kernel sources, and the issue
roofline computed from them."""
import hashlib
import json
import os
import shutil
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1603_05143_gb300 import inputs as I  # noqa: E402


def test_offered_stream_offers_the_nominal_rate():
    sizes = [1000, 50_000, 1_000_000, 7]
    for n, rate in ((16, 1e6), (1024, 1.8e8)):
        t, idx = bench.offered_stream(I.rng_for(5), n, rate, sizes)
        assert len(t) == len(idx) == n
        assert t[0] == 0.0 and np.all(np.diff(t) >= 0.0)
        assert idx.min() >= 0 and idx.max() < len(sizes)
        atoms = float(np.sum(np.asarray(sizes)[idx]))
        assert atoms / t[-1] == pytest.approx(rate, rel=1e-12)


def _fake_repo(tmp_path, sources, counters):
    csrc = tmp_path / "paper_1603_05143_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in sources.items():
        (csrc / name).write_bytes(text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / bench.COUNTERS).write_text(json.dumps(counters))


def test_committed_counters_follow_the_source_hash(tmp_path, monkeypatch):
    sources = {"a.cu": b"kernel a\n", "b.cuh": b"kernel b\n"}
    rec = {"sources": ["a.cu", "b.cuh"],
           "source_sha256": hashlib.sha256(b"kernel a\nkernel b\n").hexdigest(),
           "workloads": {"w": {"captured": "w", "kernels": {"k": {"warp_inst_per_atom": 2.0}}}}}
    _fake_repo(tmp_path, sources, rec)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.committed_counters("w")["kernels"]["k"]["warp_inst_per_atom"] == 2.0
    assert bench.committed_counters("other") is None
    # any change to a listed source retires the capture
    (tmp_path / "paper_1603_05143_gb300" / "csrc" / "b.cuh").write_bytes(b"kernel b, changed\n")
    assert bench.committed_counters("w") is None
    shutil.rmtree(tmp_path / "profiles")
    assert bench.committed_counters("w") is None


def test_issue_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "sm_count", lambda local: 152)
    counters = {"captured": "test",
                "kernels": {"k_a": {"warp_inst_per_atom": 1000.0, "thread_inst_per_atom": 16000.0,
                                    "dram_bytes_per_atom": 100.0},
                            "k_b": {"warp_inst_per_atom": 500.0, "thread_inst_per_atom": 16000.0,
                                    "dram_bytes_per_atom": 50.0}}}
    atoms = 1_000_000
    phases = {"k_a": 2.0, "k_b": 1.0}                      # ms
    extra = {"classify_ms": 3.0, "classify_kernels": "k_a + k_b", "more": {}}
    clocks = {"sm_mhz": 2000.0}
    r = bench.roofline(0, clocks, atoms, phases, counters, 3e9, extra)
    slots = 4 * 152 * 2000.0e6                            # warp-instruction issue slots per second
    assert r["bound"] == "alu" and r["kernel"] == "k_a" and r["unit"] == "Twarp-inst/s"
    assert r["peak"] == pytest.approx(slots / 1e12)
    assert r["frac"] == pytest.approx(1000.0 * atoms / 2.0e-3 / slots)
    assert r["lane_issue_frac"] == pytest.approx(r["frac"] * 16.0 / 32.0)
    assert r["traffic"] == pytest.approx(100.0 * atoms)
    assert r["kernels"]["k_b"]["issue_frac"] == pytest.approx(500.0 * atoms / 1.0e-3 / slots)
    assert r["fp32"]["achieved"] == pytest.approx(3e9 / 3.0e-3 / 1e12)
    # without a current capture only the FP32 form is reported, with no traffic
    r0 = bench.roofline(0, clocks, atoms, phases, None, 3e9, extra)
    assert r0["unit"] == "TFLOP/s" and r0["traffic"] is None
    assert r0["frac"] == pytest.approx(r0["achieved"] / r0["peak"])
