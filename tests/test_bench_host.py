"""Host-side arithmetic of the benchmark lines: algorithmic work per launch, the
committed ncu summaries it pairs with, and the clock-record parser."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        import bench as b
    finally:
        sys.argv = saved
    return b


def test_algorithmic_work_counts_literals_and_nodes(bench):
    from paper_2308_15020_gb300 import gen

    # two 3-clauses, one XOR of 4, one at-least-2 of 5 literals (node path: J = (5 + 1) // 2 + 1 = 4 nodes)
    inst = gen.from_lists(6, [(gen.OR, 0, [1, -2, 3]), (gen.OR, 0, [2, 4, -5]), (gen.XOR, 1, [1, 2, 3, 4]),
                              (gen.ATLEAST, 2, [1, 2, 3, 4, 5])])
    st = bench.instance_stats(inst)
    B, T = 7, 11
    flops, bytes_, node_dominates, smem = bench.algorithmic_work(st, B, T, elem=4)
    closed = 3 + 3 + 4
    assert flops == (4 * 5 * bench.NODE_FLOPS + closed * bench.CLOSED_FLOPS) * B * T
    assert smem == 2 * 4 * closed * B * T
    assert bytes_ == 2 * B * 6 * 4 + inst.nnz * 4 + inst.m * 16 + B * 5
    assert node_dominates  # 20 (node, literal) units against 10 closed-form literals


def test_constant_cardinality_is_not_node_work(bench):
    from paper_2308_15020_gb300 import gen

    inst = gen.from_lists(4, [(gen.ATLEAST, 0, [1, 2, 3]), (gen.ATLEAST, 5, [1, 2, 3]), (gen.OR, 0, [1, 4])])
    flops, _, node_dominates, smem = bench.algorithmic_work(bench.instance_stats(inst), 1, 1)
    assert not node_dominates
    assert flops == (3 + 3 + 2) * bench.CLOSED_FLOPS


@pytest.mark.parametrize("kernel,workload,family", [
    ("ffsat_fused", "cnf_xor_n2000", "fused"),
    ("ffsat_fused", "cnf_card_n20000", "fused"),
    ("ffsat_batch", "uneven_batch", "fused"),
    ("ffsat_cluster", "3sat_n100", "cluster"),
])
def test_committed_summaries_pair_with_their_sources(bench, kernel, workload, family):
    """Each committed ncu summary names the command and the source hash it was
    taken on; the bench lines report its DRAM traffic and counters while the
    hash matches the kernel's sources, and nothing once they have changed."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    text = open(path).read()
    assert "--clock-control none" in text and "command:" in text
    taken = [ln.split(":", 1)[1].strip() for ln in text.splitlines() if ln.startswith("kernel_source_hash:")]
    assert len(taken) == 1
    traffic = bench.profile_traffic(kernel, workload)
    counters = bench.profile_counters(kernel, workload)
    if taken[0] == bench.kernel_source_hash(family):
        assert traffic is not None and traffic > 0
        assert counters and "issue_active_pct" in counters
    else:
        assert traffic is None and counters is None
    assert bench.profile_traffic(kernel, "no_such_workload") is None


def test_clock_parser_keeps_the_timed_region(bench, tmp_path):
    s = bench.ClockSampler("0")
    s.path = str(tmp_path / "clk.csv")
    rows = [
        # timestamp, index, sm, max, power, active, hw, hw_thermal, sw_thermal, sw_power
        "2026/01/01 00:00:00.000, 0, 1200, 2070, 300, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/01/01 00:00:01.000, 0, 2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/01/01 00:00:01.050, 0, 2055, 2070, 950, 0x4, Not Active, Not Active, Not Active, Active",
    ]
    open(s.path, "w").write("\n".join(rows) + "\n")
    import datetime

    s.t_mark = datetime.datetime.strptime("2026/01/01 00:00:01.000", "%Y/%m/%d %H:%M:%S.%f").timestamp()

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s.proc = Done()
    s.fh = open(os.devnull, "w")
    out = s.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == pytest.approx(2062.5) and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert np.isfinite(out["sm_mhz"])
    # a window that ends before the last sample (the end of the timed region)
    t1 = datetime.datetime.strptime("2026/01/01 00:00:01.000", "%Y/%m/%d %H:%M:%S.%f").timestamp()
    w = s.window(t1 - 0.01, t1 - 0.01)  # samples within 50 ms of the window count
    assert w["samples"] == 1 and w["sm_mhz"] == 2070.0 and w["reasons"] == []
