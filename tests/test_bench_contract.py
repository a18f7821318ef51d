"""The JSON line of bench.py's reference arm (the FP64 oracle on the host
cores) and its host-only P1 leg, run on a small scale of the headline
workload (no GPU): the keys and types the driver reads."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--steps", "2", "--warmup", "1", "--scale", "0.0625")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_p1_leg_line():
    d = _run("--only", "p1", "--scale", "0.0625")
    assert d["leg"] == "p1" and d["planted_partition_recovered"] is True
    assert d["nnz_s_detected"] == d["nnz_s_planted"] and d["seconds"] > 0


def test_roofline_traffic_is_read_only_for_the_current_sources(tmp_path, monkeypatch):
    """The bench takes a stage kernel's DRAM bytes per launch from an ncu
    summary under profiles/ only if that summary was captured from the
    current kernel sources (their hash); otherwise it reports none."""
    import shutil
    import bench
    src = tmp_path / "paper_2203_16657_gb300" / "csrc"
    src.mkdir(parents=True)
    for name in bench.STAGE_KERNEL_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_2203_16657_gb300", "csrc", name), src / name)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.stage_kernel_source_hash()
    (tmp_path / "profiles" / "k.md").write_text(
        "traffic_per_launch: kernel=cia_window_kernel bytes=6.1e7 source=%s\n"
        "traffic_per_launch: kernel=cia_ring_kernel bytes=5.0e7 source=0000000000000000\n" % h)
    assert bench.measured_traffic("cia_window_kernel") == 6.1e7
    assert bench.measured_traffic("cia_ring_kernel") is None       # stale capture
    (src / "kuramoto.cu").write_text("// changed\n")
    assert bench.measured_traffic("cia_window_kernel") is None     # the kernel changed since
