"""bench.py's host-side pieces without a GPU: the default run satisfies the
timing rules, the step-kernel digest covers files that exist, the committed
ncu summary parses, and its DRAM traffic is consistent with the algorithmic
bytes while it matches the current sources."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_defaults_satisfy_the_timing_rules(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    assert args.gpus == 1 and args.warmup >= 3 and args.steps >= 100
    assert args.impl == "ours" and args.store == "f32" and args.n == 4096
    # the FP32 state is far larger than the 129 MB L2: no flush is needed between steps
    assert 9 * 4 * args.n * args.n > 4 * 129e6


def test_step_kernel_digest_covers_existing_files():
    for rel in bench.STEP_KERNEL_SOURCES:
        assert os.path.isfile(os.path.join(ROOT, rel)), rel
    d = bench.source_digest()
    assert len(d) == 16 and int(d, 16) >= 0


def test_committed_profile_summary_parses():
    text = open(bench.PROFILE_SUMMARY).read()
    assert "source digest:" in text
    for store in ("f32", "f16"):
        assert f"traffic_bytes_per_launch[{store}]" in text
    assert "ncu --metrics gpu__time_duration.sum --clock-control none" in text


def test_profiled_traffic_is_consistent_with_the_algorithmic_bytes():
    n = bench.N_DEFAULT
    for store, bytes_per_update in (("f32", 72), ("f16", 36)):
        t = bench.profiled_traffic(store)
        if t is None:
            pytest.skip("the committed ncu summary was taken on other step-kernel sources; recapture it")
        algorithmic = bytes_per_update * n * n
        assert 0.8 * algorithmic <= t <= 1.2 * algorithmic, (store, t, algorithmic)


def test_whole_job_value_counts_every_rank():
    assert bench.whole_job_mlups(1000, 10, 1.0, 1) == pytest.approx(0.01)
    assert bench.whole_job_mlups(1000, 10, 1.0, 4) == pytest.approx(0.04)
    assert bench.max_over_ranks(2.5) == 2.5
