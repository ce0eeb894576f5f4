"""Host arithmetic of bench.py's roofline and iteration accounting on CPU: the algorithmic bytes of
the two operator kernels written out for one Q3 element and one Q1 element (circulant-diagonal
rows of (n_e/2 + 1) n_e entries), the achieved bandwidth and fraction of a launch from the
sampled family timing (one apply = one launch per order class), the dominant-kernel choice, and
the operators' share of an iteration."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def problem(ps):
    return types.SimpleNamespace(p=list(ps), nelx=len(ps), nely=1)


def test_operator_bytes_by_hand():
    # one Q3 element: n_e = 32 rows of 17 diagonals = 544 entries; 16 node ids; 10 DOFs of vectors
    pr = problem([3])
    assert bench.operator_bytes(pr, 10) == 544 * 8 + 16 * 4 + 10 * 16
    assert bench.lead_bytes(pr, 10) == 544 * 4 + 16 * 4 + 10 * 8
    # one Q1 element: n_e = 8, 5 diagonals = 40 entries, 4 node ids
    pr1 = problem([1])
    assert bench.operator_bytes(pr1, 8) == 40 * 8 + 4 * 4 + 8 * 16
    assert bench.lead_bytes(pr1, 8) == 40 * 4 + 4 * 4 + 8 * 8


def test_roofline_fraction_and_traffic_scaling():
    pr = problem([3] * 524288)
    fams = {"applydf64": (10, 10 * 0.5), "applylead": (40, 40 * 0.25)}   # (launches, total ms)
    split = bench.roofline(fams, "applydf64", 2.5e9, pr, 6250.0, lead=False)
    assert abs(split["avg_launch_us"] - 500.0) < 1e-9
    assert abs(split["achieved"] - 5000.0) < 1e-6          # 2.5 GB in 0.5 ms
    assert abs(split["frac"] - 0.8) < 1e-12
    # the stored capture is per element, scaled to the launch's elements (rows above 64 MB)
    assert abs(split["traffic"] - bench.TMA_TRAFFIC_PER_ELEMENT["split"] * 524288) < 1.0
    lead = bench.roofline(fams, "applylead", 1.25e9, pr, 6250.0, lead=True)
    assert abs(lead["frac"] - 0.8) < 1e-12
    assert "false,float" in lead["kernel"] and "true,double" in split["kernel"]
    # no sampled launches: no roofline; a class too small for the staged kernel: no stored traffic
    assert bench.roofline({}, "applylead", 1.0, pr, 6250.0, lead=True) is None
    small = bench.roofline(fams, "applydf64", 1e6, problem([3] * 100), 6250.0, lead=False)
    assert small["traffic"] is None and "pipe" in small["kernel"]
    # two order classes: one apply is two launches, so the apply's time is twice a launch's
    two = bench.roofline({"applydf64": (20, 20 * 0.25)}, "applydf64", 2.5e9, problem([3, 2] * 262144), 6250.0,
                         lead=False)
    assert abs(two["avg_launch_us"] - 500.0) < 1e-9


def test_iteration_share():
    bd = {"applydf64": {"ms": 150.0}, "applylead": {"ms": 700.0}, "precond": {"ms": 580.0},
          "vector": {"ms": 70.0}, "indicator": {"ms": 200.0}}
    sh = bench.iteration_share(bd, 340)
    assert abs(sh["operator_ms_per_iter"] - 850.0 / 340) < 1e-12
    assert abs(sh["solve_ms_per_iter"] - 1500.0 / 340) < 1e-12
    assert abs(sh["ratio"] - 1500.0 / 850.0) < 1e-12
    assert bench.iteration_share({}, 10)["ratio"] is None


def test_multigrid_operator_choice():
    """The single-instance workloads run the FP32 cycle unless told otherwise; the batched workload
    (binary instances) leaves the choice to the library (AUTO); an explicit choice wins in both."""
    import pytest
    mto = pytest.importorskip("paper_1811_09821_gb300")
    args = types.SimpleNamespace(mg_operator=None)
    assert bench.mg_operator_of(args) == mto.MG_OP_LEAD
    assert bench.mg_operator_of(args, batched=True) == mto.MG_OP_AUTO
    for name, op in (("lead", mto.MG_OP_LEAD), ("split", mto.MG_OP_SPLIT), ("auto", mto.MG_OP_AUTO)):
        args.mg_operator = name
        assert bench.mg_operator_of(args) == op and bench.mg_operator_of(args, batched=True) == op
