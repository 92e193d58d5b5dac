"""The benchmark's reference arm (the CPU oracle timed on the host) produces
the contract's JSON line without a GPU: same metric and unit as the GPU arm,
impl "reference", a cpu_baseline block and an e2e block with zero copies."""
import argparse

import bench


def test_reference_arm_line_on_cpu(monkeypatch):
    monkeypatch.setattr(bench, "REF_STEP_BUDGET_S", 0.2)
    args = argparse.Namespace(workload="c1", steps=2, warmup=1)
    line = bench.run_reference(args, rank=0, world=1)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "butterflies/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["butterflies_per_step"] == 2 * 10 * 512  # forward + inverse of one 2^10 transform


def test_reference_arm_other_ranks_do_no_work():
    args = argparse.Namespace(workload="c1", steps=1, warmup=0)
    assert bench.run_reference(args, rank=1, world=2) is None
