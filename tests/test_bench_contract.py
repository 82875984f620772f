"""The benchmark's own bookkeeping, on the CPU: the default arguments keep
the timing rules (at least 3 warm-up steps, one GPU), the recorded DRAM
traffic of the force kernel belongs to the current force-kernel source (the
bench reports it only while the source is the one it was measured on), and
the per-stage HBM fractions are the algorithmic bytes over the time."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    import importlib
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        mod = importlib.import_module("bench")
        yield mod
    finally:
        sys.argv = saved


def test_default_arguments_keep_the_timing_rules(bench):
    sys.argv = ["bench.py"]
    args = bench.parse()
    assert args.gpus == 1 and args.warmup >= 3 and args.steps >= 1
    assert args.n == 1 << 24 and args.theta == 0.5 and not args.mono
    assert args.impl == "ours" and not args.no_other


def test_force_traffic_record_matches_the_current_kernel_source(bench):
    """A change to csrc/force.cu must come with a new ncu traffic capture
    (and its SHA-256 prefix): otherwise the bench line's traffic is null."""
    sys.argv = ["bench.py"]
    args = bench.parse()
    assert bench.force_traffic(bench.workload_name(args)) is not None


def test_stage_hbm_fractions(bench):
    stages = {"ms_box_keys": 1.0, "ms_sort": 2.0, "ms_walk": 5.0}
    n, nodes, peak = 1000, 300, 1000.0
    out = bench.stage_hbm(stages, n, nodes, peak)
    bp, bn = bench.STAGE_BYTES["ms_box_keys"]
    want = (bp * n + bn * nodes) / (1.0 * 1e6)
    assert out["box_keys"]["gb_s"] == pytest.approx(want)
    assert out["box_keys"]["frac"] == pytest.approx(want / peak)
    assert "walk" not in out  # not an HBM-bound stage
    coh = bench.stage_hbm(stages, n, nodes, peak, coherent=True)
    assert coh["sort"]["bytes"] == bench.STAGE_BYTES_COHERENT["ms_sort"][0] * n
