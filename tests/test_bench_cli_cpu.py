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


def test_fused_backward_bytes_follow_the_records_that_carry_a_gradient():
    """The fused one-view backward + Adam reads and writes every Gaussian's
    parameters and moments but the SH and 2D-gradient record traffic of only
    the Gaussians with a gradient: 1492 B a Gaussian with FP32 SH plus 264 B
    for each with a gradient (192 B of SH read, the record written twice);
    with a 16-bit SH shadow 1588 + 168 B."""
    N, n_grad = 3_000_000, 26_191
    ab32 = bench.algorithmic_bytes(N, 1600 * 1060, 3_000_000, 1_400_000, True, 1, n_grad, False)
    ab16 = bench.algorithmic_bytes(N, 1600 * 1060, 3_000_000, 1_400_000, True, 1, n_grad, True)
    assert ab32["project_bwd_adam"] == 1492 * N + 264 * n_grad
    assert ab16["project_bwd_adam"] == 1588 * N + 168 * n_grad
    # Adam alone writes the shadow only with 16-bit SH storage
    assert ab16["adam"] - ab32["adam"] == 96 * N


def test_deferred_colour_moves_the_sh_read_to_the_listed_records():
    """With the colour deferred the projection reads 44 B of geometry per
    (view, Gaussian) and no SH; the colour stage reads the list entry, the
    mean and the SH of each listed record and writes its colour."""
    N, V, n_col = 3_000_000, 1, 64_932
    now = bench.algorithmic_bytes(N, 1600 * 1060, 3_000_000, 1_400_000, True, V, 0, False, n_col)
    before = bench.algorithmic_bytes(N, 1600 * 1060, 3_000_000, 1_400_000, True, V, 0, False)
    assert before["project"] - now["project"] == V * N * 192
    assert now["colour"] == n_col * (4 + 12 + 192 + 8)
    assert "colour" not in before
