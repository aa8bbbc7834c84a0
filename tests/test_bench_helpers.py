"""bench.py's host-side helpers (no GPU): the root level's well-separated pair count that the
mixed roofline takes off the refined-pair work equals the library's own count on a tree whose
only refined subgrid is the root; the per-kernel traffic table parses; the CPU name is found."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2101_08226_gb300 import api, synth  # noqa: E402


@pytest.mark.parametrize("theta", [0.34, 0.5, 0.7])
def test_root_pairs_equal_library_count(theta):
    t = api.Tree(1, synth.uniform_flags(1))  # refined root, leaf level 1
    assert t.counts_by_type(theta)["m2l_refined_refined"] == bench.root_pairs(theta)


def test_traffic_table_parses():
    for workload in ("binary_q0.7_L5", "binary_q0.6_L7"):
        tr = bench.measured_traffic(workload)
        assert isinstance(tr, dict)
        # empty once the kernel sources differ from the captured ones; otherwise every kernel
        # the rooflines name is there
        if tr:
            for k in ("k_m2l_ref<double>", "k_m2l_stage", "k_m2l_leaf<double>"):
                assert tr[k] > 0


def test_cpu_model_is_named():
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
