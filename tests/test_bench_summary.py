"""bench.py's compact summary (the last key of its JSON line, the part kept
when only the end of the output is read): built from full variant records,
from records of variants that failed, and from none, without a GPU."""
import json

import bench


def _variants():
    sweep = {"targets": list(range(10))}
    for kind in ("H", "U", "T", "CZ", "MCPF"):
        for prec in (64, 128):
            sweep[f"{kind}_c{prec}_GBps_by_target"] = [1000.0 + t for t in range(10)]
    return {
        "sv12_c128": {"us_per_circuit": 135.4},
        "sv30_c64": {"gates_per_s": 14808.2, "pass_kernel_hbm_frac_of_measured": 0.661,
                     "error_vs_fp64": {"max_abs_err": 1.7e-10, "one_minus_fidelity": 4.8e-13}},
        "sv33_c128": {"gates_per_s": 77.8},
        "dm14_c128": {"ops_per_s": 2631.6},
        "single_gate_sweep": sweep,
        "batch4096_c64": {"circuits_per_s": 65800.0, "plain_c128_circuits_per_s": 547.0, "tile_qubits": 13,
                          "schedule": "persistent launch",
                          "error_vs_fp64_all_registers": {"max_abs_err": 8.1e-8, "max_one_minus_fidelity": 2.2e-13}},
        "multi_target_passes": {"c64_m5": {"ms": 2.75, "GBps": 6239.4}},
        "serving": {"10_req_per_s": {"served": {"circuits_per_s": 10.7, "p50_ms": 7.1, "p99_ms": 273.0},
                                     "plain_c128_one_at_a_time": {"circuits_per_s": 10.2}}},
        "partitioned_28q_4parts": {"gates_per_s": 15200.0},
    }


def test_summary_of_full_records_is_short_and_carries_the_figures():
    s = bench.compact_summary(_variants())
    text = json.dumps({"summary": s})
    assert len(text) < 1500
    assert s["sv30_c64"] == [14800.0, 0.66, 1.7e-10, 4.8e-13]
    assert s["sv33_c128"][0] == 77.8 and s["sv12_us"] == 135.0
    # per-target sweeps: min and median over the bits from 5 up, the last
    # three excluded
    assert s["sweep30_bits5up_min_med_GBps"]["U64"] == [1005, 1006]
    assert s["batch"]["sched"] == "persist" and s["batch"]["c_s"] == 65800.0
    assert s["multi_GBps"] == {"c64_m5": 6239}
    assert s["serve_c_s_p50ms_p99ms_p99shedms_plainc128"]["10"] == [10.7, 7.1, 273.0, None, 10.2]
    assert s["part28_4_gates_s"] == 15200.0


def test_summary_of_failed_or_missing_variants():
    assert bench.compact_summary({}) == {}
    s = bench.compact_summary({"sv30_c64": {"error": "out of memory"}, "batch4096_c64": {"error": "x"},
                               "serving": {"error": "x"}, "single_gate_sweep": {"error": "x"}})
    assert s["sv30_c64"] == [None, None, None, None]
    assert "batch" not in s and "sweep30_bits5up_min_med_GBps" not in s
    assert s["serve_c_s_p50ms_p99ms_p99shedms_plainc128"] == {}
