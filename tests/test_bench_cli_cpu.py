"""bench.py's command line on the CPU: which measurement each flag selects,
the default step counts, and the guard that refuses dynamic-training runs
whose Gaussian count could grow past 32M.  The measurements themselves are
replaced by stubs (they need a GPU)."""
import sys

import pytest

import bench


@pytest.fixture
def calls(monkeypatch):
    seen = []
    for name in ("run_ours", "run_reference", "run_dynamic", "run_colour_ablation", "run_density_control",
                 "run_colour_buckets"):
        monkeypatch.setattr(bench, name, lambda args, name=name: seen.append((name, args.steps)))
    return seen


def _main(monkeypatch, *argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    bench.main()


@pytest.mark.parametrize("argv, want", [
    ((), ("run_ours", 300)),
    (("--impl", "reference"), ("run_reference", 300)),
    (("--workload", "dynamic-6M-4x1920x1080"), ("run_dynamic", 20)),
    (("--colour-ablation",), ("run_colour_ablation", 20)),
    (("--density-control",), ("run_density_control", 10)),
    (("--colour-buckets",), ("run_colour_buckets", 10)),
    (("--steps", "7"), ("run_ours", 7)),
])
def test_each_flag_selects_its_measurement(monkeypatch, calls, argv, want):
    _main(monkeypatch, *argv)
    assert calls == [want]


def test_dynamic_runs_that_could_grow_too_far_are_refused(monkeypatch, calls):
    with pytest.raises(SystemExit):
        _main(monkeypatch, "--workload", "dynamic-6M-4x1920x1080", "--steps", "200")
    assert calls == []


def test_fewer_than_three_warmup_steps_are_refused(monkeypatch, calls):
    with pytest.raises(SystemExit):
        _main(monkeypatch, "--warmup", "2")
    assert calls == []
