"""Host logic of bench.py (no GPU): the roofline's traffic figures come from the committed
ncu summary, the batch split covers every system once, and the profiling-cases module
imports without a device."""
import importlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_traffic_per_element_read_from_the_profile_summary():
    import bench
    t = bench.ncu_traffic_per_element("f32")
    assert set(t) == {"basis_dot", "basis_axpy"}
    # a launch reads every code once plus w's planes: a little above 4 bytes per element
    for v in t.values():
        assert 4.0 < v < 4.5
    assert bench.ncu_traffic_per_element("e4m3") == {}


def test_shard_units_cover_every_unit_once():
    import bench
    for n in (0, 1, 7, 512):
        for world in (1, 2, 3, 8):
            shares = [list(bench.shard_units(n, world, r)) for r in range(world)]
            flat = [i for s in shares for i in s]
            assert flat == list(range(n))                       # contiguous, in rank order
            sizes = [len(s) for s in shares]
            assert max(sizes) - min(sizes) <= 1


def test_profile_cases_module_imports_without_a_gpu():
    pc = importlib.import_module("paper_2009_12101_gb300.profile_cases")
    for name in ("case_gemv", "case_spmv", "case_mlp", "main"):
        assert callable(getattr(pc, name))


def test_kernel_class_table_shares_and_rates():
    import bench
    prof = {"basis_dot": {"ms": 30.0, "bytes": 1.5e11, "launches": 1000},
            "spmv": {"ms": 10.0, "bytes": 4.0e10, "launches": 500},
            "store": {"ms": 0.0, "bytes": 0.0, "launches": 0}}
    t = bench.kernel_class_table(prof)
    assert set(t) == {"basis_dot", "spmv"}                     # classes never launched left out
    assert abs(t["basis_dot"]["share"] - 0.75) < 1e-12
    assert t["spmv"]["us_per_launch"] == 20.0
    assert t["basis_dot"]["gbs"] == 5000.0 and t["spmv"]["gbs"] == 4000.0


def test_clock_record_from_nvidia_smi_lines():
    import bench
    lines = [
        "0, 2070, 2070, 850.10, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 900.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",     # unreadable sample: skipped
        "index, clocks.sm",                                              # stray header: skipped
    ]
    r = bench.parse_clock_lines(lines)
    assert r["samples"] == 3 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["power_w_max"] == 1390.0 and r["reasons"] == ["sw_power_cap"]
    r = bench.parse_clock_lines(lines[:1] + [
        "0, 1500, 2070, 700.0, 0x0000000000000008, Active, Not Active, Active, Not Active"])
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.parse_clock_lines([])["sm_mhz"] is None
