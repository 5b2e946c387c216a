"""bench.py's command line: the step count defaults per workload (a warm
step replays the whole 1M-trajectory evaluation, so it cannot share the
single scene's 2000), explicit values win, and the timing rules (>= 3 warm-up
steps, >= 1 timed step) are enforced before anything runs."""
import pytest


def test_default_steps_per_workload():
    import bench
    assert bench.parse_args([]).workload == "warm"
    assert bench.parse_args([]).steps == 10
    assert bench.parse_args(["--workload", "scene"]).steps == 2000
    assert bench.parse_args(["--workload", "precision"]).steps == 20
    assert bench.parse_args(["--workload", "batch"]).steps == 100
    assert bench.parse_args(["--workload", "warm"]).steps == 10
    assert bench.parse_args(["--workload", "sweep"]).steps == 2000
    assert bench.parse_args(["--impl", "reference"]).steps == 3


def test_explicit_values_and_limits():
    import bench
    a = bench.parse_args(["--workload", "warm", "--steps", "7", "--warmup", "4"])
    assert (a.steps, a.warmup) == (7, 4)
    for bad in (["--warmup", "2"], ["--steps", "0"]):
        with pytest.raises(SystemExit):
            bench.parse_args(bad)


def test_traffic_figure_only_for_the_measured_source(tmp_path, monkeypatch):
    """roofline.traffic comes from profiles/dram_traffic.json only while the
    kernel sources hash to what the ncu figure was taken with: the committed
    entry matches the committed sources, and any change of a source file (or
    an unknown kernel or workload) gives None."""
    import json
    import os
    import shutil
    import bench
    with open(bench.TRAFFIC_FILE) as f:
        entry = json.load(f)["entries"][0]
    assert bench.measured_traffic(entry["kernel"], entry["workload"]) == entry["bytes_per_launch"]
    assert bench.measured_traffic(entry["kernel"], "another workload") is None
    assert bench.measured_traffic("another_kernel", entry["workload"]) is None
    # a copy of the tree whose first source differs by one byte
    root = tmp_path / "tree"
    for rel in entry["source"] + [os.path.relpath(bench.TRAFFIC_FILE, bench.ROOT)]:
        dst = root / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
    monkeypatch.setattr(bench, "ROOT", str(root))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(root / os.path.relpath(bench.TRAFFIC_FILE, bench.ROOT)))
    assert bench.measured_traffic(entry["kernel"], entry["workload"]) == entry["bytes_per_launch"]
    with open(root / entry["source"][0], "a") as f:
        f.write(" ")
    assert bench.measured_traffic(entry["kernel"], entry["workload"]) is None
