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


def test_digest_ignores_comments_and_layout_but_not_code():
    code = "int f(int a) {\n  return a + 1; // add one\n}\n/* block\n comment */\n"
    assert bench.strip_comments(code) == bench.strip_comments("int f(int a)   { return a + 1; }")
    assert bench.strip_comments(code) != bench.strip_comments("int f(int a) { return a + 2; }")


def test_timed_passes_span_the_minimum_window():
    assert bench.passes_for(1.0) == bench.MIN_PASSES
    assert bench.passes_for(0.004) * 0.004 >= bench.MIN_TIMED_SECONDS
    assert bench.passes_for(10.0) == bench.MIN_PASSES


def test_adjoint_bytes_count_forward_recompute_and_reverse():
    # 2 steps, one checkpoint every 2: forward 2 x 80, recompute 1 x 80, reverse 2 x 132 per node
    assert bench.adjoint_bytes_per_run(1, 2, 2) == 2 * 80 + 80 + 2 * 132
    # a checkpoint every step: nothing is recomputed
    assert bench.adjoint_bytes_per_run(4, 10, 1) == 16 * (10 * 80 + 10 * 132)


def test_both_arms_describe_the_same_workload():
    c = bench.workload_config(4096, "f32")
    assert c["workload"] == "taylor_green_4096x4096_cascaded_f32_store" and c["nodes"] == 4096 ** 2
    assert [k for k, _ in bench.CPU_SAMPLES].count("cavity") == 1


def test_launch_count_of_fused_and_single_steps():
    assert bench.launch_count(0, 20, False) == 20
    assert bench.launch_count(0, 20, True) == 10
    assert bench.launch_count(5, 20, True) == 11  # one single step, nine pairs, one single step
    assert bench.launch_count(1, 1, True) == 1


def test_profile_summary_was_taken_on_the_current_step_kernels():
    """profiles/step_cascaded_tg4096.md records the digest of the step-kernel
    sources its ncu counters were taken on; bench.py reports roofline.traffic
    only while that digest matches.  The committed summary must describe the
    committed kernels (every figure bench.py reads is there)."""
    for key in ("f32", "f16", "f32_two_step"):
        assert bench.profiled_traffic(key) is not None, key
