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
