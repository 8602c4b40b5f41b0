"""Host-side arithmetic of bench.py's measurement (no GPU): the byte model the roofline
divides by, the launch-shape count it reports, and the committed DRAM figures it reads."""
import json
from types import SimpleNamespace

import pytest

import bench

# The 20k-gate workload's cone (13,203 gates, 1,053 inputs), as the plan reports it.
C2 = {"n_cone_gates": 13203, "n_cone_pi": 1053}


def test_byte_model_per_sample_step():
    """G (2 s_a + 8) + n 28 per sample-step: 240,732 B in FP32 and 187,920 B with 16-bit activations;
    recomputation every k levels adds G s_a (1 + 1/k)."""
    assert bench.algorithmic_bytes_per_step(C2, 1, "f32") == 13203 * 16 + 1053 * 28 == 240732
    assert bench.algorithmic_bytes_per_step(C2, 1, "bf16") == 13203 * 12 + 1053 * 28 == 187920
    assert bench.algorithmic_bytes_per_step(C2, 65536, "f16") == 65536 * 187920
    assert bench.algorithmic_bytes_per_step(C2, 1, "bf16", segment=8) == pytest.approx(187920 + 13203 * 2 * 9 / 8)


def test_resident_byte_model():
    """The resident kernel moves V (and Adam's m, v) once per launch, plus the loss."""
    assert bench.resident_bytes_per_launch(C2, 10, "adam") == 10 * (1053 * 24 + 4)
    assert bench.resident_bytes_per_launch(C2, 10, "gd") == 10 * (1053 * 8 + 4)


def _fake_torch(sms):
    props = SimpleNamespace(multi_processor_count=sms)
    cuda = SimpleNamespace(current_device=lambda: 0, get_device_properties=lambda d: props)
    return SimpleNamespace(cuda=cuda)


@pytest.mark.parametrize("B,launches", [(65536, 2), (18944, 1), (128, 1), (148 * 128 + 77 * 128, 1),
                                        (148 * 128 + 74 * 128, 2), (1024, 1)])
def test_step_kernel_launch_count(B, launches):
    """Whole waves of one-CTA tiles, plus one launch of 2-CTA clusters for a last partial wave of
    at most half the SMs (the library's policy, 148 SMs): 65,536 samples = 444 + 68 tiles."""
    assert bench.step_kernel_launches(B, _fake_torch(148)) == launches
    assert bench.step_kernel_launches(B, _fake_torch(148), "resident") == 1


def test_profile_traffic_reads_only_matching_sources(tmp_path, monkeypatch):
    """Figures taken on another kernel source are not reported; matching ones are, per round when a
    full-size figure of that batch and step count exists."""
    f = tmp_path / "t.json"
    f.write_text(json.dumps({"kernel_source_sha256": "abc", "workloads": {
        "w": {"dram_bytes_per_sample_step": 123.0, "dram_bytes_per_round": {"b64_s5": 9.0e9}}}}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", f)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda text=None: "abc")
    assert bench.profile_traffic("w", "f32") == (123.0, None, "t.json")
    assert bench.profile_traffic("w", "f32", 64, 5) == (123.0, 9.0e9, "t.json")
    assert bench.profile_traffic("other", "f32") == (None, None, None)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda text=None: "def")
    assert bench.profile_traffic("w", "f32") == (None, None, None)


def test_kernel_source_hash_ignores_comments_only():
    a = "int f() { return 1; } // one\n/* block */"
    assert bench.kernel_source_hash(a) == bench.kernel_source_hash("int f() {  return 1; }\n// two")
    assert bench.kernel_source_hash(a) != bench.kernel_source_hash("int f() { return 2; }")


def test_committed_traffic_file_is_consistent():
    """The committed figures name their capture, and their per-sample-step bytes follow from it."""
    d = json.loads(bench.TRAFFIC_FILE.read_text())
    for name, e in d["workloads"].items():
        assert "ncu" in e["capture"] and "--clock-control none" in e["capture"]
        total = e["dram_read_bytes"] + e["dram_write_bytes"]
        assert abs(total / (e["samples"] * e["steps"]) - e["dram_bytes_per_sample_step"]) <= 1.0, name
