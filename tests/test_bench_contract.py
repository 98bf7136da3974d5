"""The reference arm of bench.py (the oracle timed on the host cores) prints
one JSON line with the keys the bench contract asks for (CPU, no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "c1_2d_q2_k1_8", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == "slab solves/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_job_throughput_alone():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(20, 1000.0, 1) == (20.0, 1000.0)


def test_traffic_records_follow_the_kernel_source(tmp_path, monkeypatch):
    """The committed ncu DRAM traffic enters the bench line only while the
    kernel source it was taken on is unchanged: a record with another hash
    gives None, one with the current hash gives its bytes."""
    sys.path.insert(0, ROOT)
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_2303_06742_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in ("stfem.cu", "vanka.cuh", "tc_patch.cuh"):
        with open(os.path.join(ROOT, "paper_2303_06742_gb300", "csrc", name), "rb") as f:
            (csrc / name).write_bytes(f.read())
    key_s, key_t = "w/mixed/patch_apply", "w/tc8/patch_apply"
    (prof / "traffic_k_patch_apply_stream_w.json").write_text(
        json.dumps({key_s: {"bytes_per_launch": 123, "source_hash": bench.kernel_source_hash()}}))
    (prof / "traffic_k_patch_apply_tc_w.json").write_text(
        json.dumps({key_t: {"bytes_per_launch": 456, "source_hash": bench.tc_source_hash()}}))
    assert bench.dram_traffic("w", "mixed") == 123
    assert bench.dram_traffic("w", "mixed", "broken") is None  # another pressure space
    assert bench.dram_traffic_tc("w", 8) == 456
    assert bench.dram_traffic_tc("w", 4) is None
    # a changed kernel invalidates its record, and only its own
    (csrc / "tc_patch.cuh").write_bytes((csrc / "tc_patch.cuh").read_bytes() + b"\n// changed\n")
    assert bench.dram_traffic_tc("w", 8) is None
    assert bench.dram_traffic("w", "mixed") == 123
