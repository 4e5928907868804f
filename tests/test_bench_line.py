"""bench.py's result line (the last stdout line) stays short and complete.

The tables go out as earlier detail lines; the last line carries only the keys
a result needs.  Built here from worst-case values on the CPU (no GPU).
"""
import json

import bench


def _worst_line():
    roof = {"bound": "alu", "kernel": "star", "achieved": 0.123456789, "peak": 1.19876543, "unit": "TFLOP/s",
            "frac": 0.1029876, "traffic": 123456789.0, "kernel_launches_per_step": 1234.56}
    cpu = {"value": 103022.919992, "unit": "unknowns/s", "cores": 144, "kind": "oracle",
           "sample": bench.sample_text(912673 * 12, 123.456)}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 999,
              "reasons": ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]}
    return bench.result_line(value=190316000.885, steps=20, warmup=5, ms_total=2536.5789, unknowns=24137569, p0=2,
                             world=8, iterations=3, mixed=("mixed_fp32_tc", 562357770.71, 4), e2e=183456789.123,
                             roof=roof, peak_measured=True, cpu=cpu, clocks=clocks,
                             sweep={"fp64": 407123456.78, "mixed": 666123456.78})


def test_result_line_is_short():
    text = json.dumps(_worst_line())
    assert "\n" not in text
    assert len(text.encode()) <= bench.MAX_LINE, len(text)


def test_result_line_has_the_required_keys():
    line = _worst_line()
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "roofline", "cpu_baseline", "clocks"):
        assert k in line, k
    assert line["config"]["workload"] == bench.HEADLINE
    assert set(line["e2e"]) == {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(line["roofline"])
    assert {"value", "unit", "cores", "kind", "sample"} <= set(line["cpu_baseline"])
    assert line["mixed"]["speedup_vs_fp64"] > 1.0
