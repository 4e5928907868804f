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


def _kst(**classes):
    base = {"ms": 0.0, "launches": 0, "flops": 0.0, "bytes": 0.0, "xflops": 0.0}
    return {k: {**base, **v} for k, v in classes.items()}


PEAKS = {"fp64": (1.25, "fp64 probe"), "hbm": (6792.4, "copy")}


def test_roofline_executed_count_against_the_star_peak():
    kst = _kst(star=dict(ms=100.0, launches=10, flops=3e12, bytes=1e9, xflops=1e11),
               vector=dict(ms=1.0, launches=5, bytes=1e9))
    r = bench.roofline(kst, (1.25, "fp64 probe"), PEAKS, steps=2)
    assert r["kernel"] == "star" and r["bound"] == "alu"
    assert abs(r["achieved"] - 1.0) < 1e-12 and abs(r["frac"] - 0.8) < 1e-12
    assert abs(r["paper_count_tflops"] - 30.0) < 1e-9 and r["launches_per_step"] == 5


def test_roofline_without_executed_count_reports_no_fraction():
    # tensor-core star: the library's count covers the CUDA-core levels only
    kst = _kst(star=dict(ms=100.0, launches=10, flops=3e12, xflops=1e9))
    r = bench.roofline(kst, (78.0, "fp32 probe"), PEAKS, steps=1, tc=True)
    assert r["achieved"] is None and r["frac"] is None and r["peak"] == 78.0
    # an FP64 element class with only the paper count is measured against the FP64 peak
    kst = _kst(elem_schur=dict(ms=10.0, launches=3, flops=1e10), star=dict(ms=1.0, launches=1, xflops=1e6))
    r = bench.roofline(kst, (78.0, "fp32 probe"), PEAKS, steps=1)
    assert r["kernel"] == "elem_schur" and r["bound"] == "alu" and r["peak"] == 1.25 and r["frac"] is None


def test_roofline_of_the_float_float_classes():
    # float-float forms: the element class mixes the FP64 outer residual with float-float level
    # residuals (no single peak); condensation runs on the FP32 pipes
    fp32 = (78.0, "fp32 probe")
    kst = _kst(elem_schur=dict(ms=10.0, launches=3, flops=1e10), star=dict(ms=1.0, launches=1, xflops=1e6))
    r = bench.roofline(kst, fp32, PEAKS, steps=1, class_peaks=bench.ff_class_peaks(fp32))
    assert r["peak"] is None and r["frac"] is None and "outer residual" in r["note"]
    kst = _kst(condense=dict(ms=10.0, launches=1, flops=1e10), star=dict(ms=1.0, launches=1, xflops=1e6))
    r = bench.roofline(kst, fp32, PEAKS, steps=1, class_peaks=bench.ff_class_peaks(fp32))
    assert r["kernel"] == "condense" and r["peak"] == 78.0 and "FP32 pipes" in r["note"]


def test_roofline_data_movement_class_against_measured_hbm():
    kst = _kst(star_gather=dict(ms=2.0, launches=4, bytes=6.7924e9))
    r = bench.roofline(kst, (1.25, "fp64 probe"), PEAKS, steps=1)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 3396.2) < 1e-6 and abs(r["frac"] - 0.5) < 1e-12


def test_measured_hbm_reads_the_peaks_file():
    v, src = bench.measured_hbm()
    assert v > 1000.0 and isinstance(src, str)
