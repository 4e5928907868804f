"""Benchmark: unknowns/s per solve to a 1e-10 relative residual reduction.

Headline workload: Poisson on the unit cube, 6 x 6 x 6 stretched elements
(per-axis aspect ratios drawn log-uniform in [1, 8]), degree p = 48,
289^3 = 24,137,569 unknowns, manufactured right-hand side, coarse degree
p0 = 2.  One step = one whole solve: condensation, Algorithm 4 (V-cycles) to
a 1e-10 reduction of the condensed residual, interior recovery.  `value` is
the plain FP64 GPU form; `mixed` the fastest mixed-precision form on the same
workload (FP32 smoother and transfers, TF32 tensor-core transforms where the
form has them, FP64 residuals and outer iteration).

Timing: CUDA events on the solving stream around each solve, L2 flushed (a
256 MiB write) before every solve, W untimed warm-up steps, then K timed
steps with per-kernel timing OFF; max over ranks.  `e2e` times the same steps
through the host-buffer entry point (pinned host f in, u out, copies inside
the timed region).  The roofline line comes from a separate pass of the same
steps with the library's per-kernel CUDA events on: the dominant kernel's
executed operations (counted by the library from the kernel's loop trip
counts) over its event time, against the FP64 peak measured in the same run.

Every table (forms, kernels, the 8^3 degree sweep, the 64-solve batch, the
other workloads) goes to stdout as `{"detail": ...}` lines BEFORE the last
line; the last line is the short result line.  Multi-GPU runs are replicas
(the path has no exchange step on one mesh).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

HEADLINE = "poisson_6x6x6_p48_stretched"
CPU_SAMPLE = "poisson_2x2x2_p48_stretched"
SWEEP = [4, 8, 16, 32]
METRIC = "unknowns/s per solve to 1e-10 residual (FP64 vs mixed); smoother HBM GB/s"
# timed forms: name -> (precision, outer iteration, smoother)
FORMS = {"fp64": ("fp64", "mg", "star"), "mixed": ("mixed", "mg", "star"), "mixed_tc": ("mixed_tc", "mg", "star"),
         "mixed_bf16": ("mixed_bf16", "mg", "star"), "mixed_ff_tc": ("mixed_ff_tc", "mg", "star"),
         "mixed_ff": ("mixed_ff", "mg", "star"), "kmg_mixed_ff_tc": ("mixed_ff_tc", "kmg", "star"),
         "mixed_fp32": ("mixed_fp32", "mg", "star"), "mixed_fp32_tc": ("mixed_fp32_tc", "mg", "star"),
         "kmg_fp64": ("fp64", "kmg", "star"), "kmg_mixed": ("mixed", "kmg", "star"),
         "kmg_mixed_tc": ("mixed_tc", "kmg", "star"), "eblock_fp64": ("fp64", "mg", "element"),
         "eblock_mixed": ("mixed", "mg", "element")}
MIXED_FORMS = ("mixed", "mixed_tc", "mixed_bf16", "mixed_ff_tc")  # candidates for the result line's `mixed`
DETAIL_FORMS = ("kmg_fp64", "kmg_mixed", "kmg_mixed_tc", "kmg_mixed_ff_tc", "mixed_fp32", "mixed_fp32_tc",
                "mixed_ff")
TC_FORMS = ("mixed_tc", "mixed_bf16", "mixed_fp32_tc", "mixed_ff_tc")  # star on the tensor cores at n_S >= 31
SWEEP_FORMS = ("fp64", "mixed", "mixed_tc", "mixed_ff_tc")  # forms of the 8^3 degree sweep
FF_PRECISIONS = ("mixed_ff", "mixed_ff_tc")  # level residuals, condensation and recovery in float-float
BATCH_MIXED = "mixed_ff_tc"  # precision of the batch's mixed graphs
FP64_NOMINAL_TFLOPS = 1.25  # 2 FP64 FMA / clock / SM x 152 SMs x 2.07 GHz: fallback when the probe fails
# DRAM bytes (read + write) per k_star<double> launch of the timed FP64 region of the headline
# workload (all levels, every launch of two steps), from an ncu capture of that region
# (dram__bytes_read.sum + dram__bytes_write.sum); null once the star kernel's source changed since
# (hash below).  Mostly the per-class 1/D tables (6.9 MB per star at p = 48).
STAR_TRAFFIC = {"bytes_per_launch": 5.941e8, "source": "723cf972005e1ba7"}
STAR_SOURCES = ("star_kernel.cuh", "kernels_star_f64.cu")
MAX_LINE = 1400  # bytes of the result line (the last stdout line)


def star_source_hash():
    """First 16 hex digits of the SHA-256 of the FP64 star-kernel sources (None if one is missing)."""
    import hashlib
    hsh = hashlib.sha256()
    for name in STAR_SOURCES:
        path = os.path.join(ROOT, "paper_1808_03595_gb300", "csrc", name)
        if not os.path.exists(path):
            return None
        with open(path, "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:16]


def r4(x):
    """x rounded to 4 significant digits (None and non-finite values pass through as None)."""
    if x is None:
        return None
    x = float(x)
    if not math.isfinite(x):
        return None
    return float(f"{x:.4g}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 3.0:  # first sample before the timed region
            time.sleep(0.05)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, value):
    if pg is None:
        return value
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def emit(name, payload, sink):
    """One detail line on stdout (before the result line) and into the optional detail file."""
    sink[name] = payload
    print(json.dumps({"detail": name, **payload}), flush=True)


# ---------------------------------------------------------------- the oracle on the host (CPU baseline)

def oracle_sample():
    """One whole oracle solve (numpy FP64: condensation, Algorithm 4 to 1e-10, recovery) of the 2^3-element
    sample of the headline workload; returns (unknowns, seconds, iterations)."""
    from oracle import dense, matfree
    h, p, lam, f, p0 = workloads.config(CPU_SAMPLE)
    mesh = dense.Mesh(h, p, lam)
    t0 = time.perf_counter()
    _, it, _ = matfree.solve(mesh, f, p0=p0)
    dt = time.perf_counter() - t0
    return int(f.size), dt, it


def sample_text(n_unknowns, seconds):
    return (f"whole oracle solves (numpy FP64, Alg. 4) of the 2x2x2-element sample of the 6^3 workload "
            f"(p=48, same width law and f): {n_unknowns} unknowns in {seconds:.1f} s")


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample()
    tot_n, tot_t = 0, 0.0
    for _ in range(args.steps):
        n, dt, _ = oracle_sample()
        tot_n += n
        tot_t += dt
    v = tot_n / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": r4(v), "unit": "unknowns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r4(1e3 * tot_t / args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": HEADLINE, "sample": CPU_SAMPLE, "parallelism": "host cores"},
        "cpu_baseline": {"value": r4(v), "unit": "unknowns/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample_text(tot_n, tot_t)},
        "e2e": {"value": r4(v), "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def timed_solves(ctx, f, u, steps, flush, stream, host=None):
    """Sum of the CUDA-event times of `steps` solves (L2 flushed before each) and the last info."""
    import torch
    ms, info = 0.0, None
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if host is not None:
            _, info = ctx.solve_host(host[0], host[1], rtol=1e-10)
        else:
            _, info = ctx.solve(f, rtol=1e-10, out=u)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        assert info.res_final <= 1e-10 * info.res0, (info.res_final, info.res0)
    return ms, info


def roofline(kst, star_peak, peaks, steps, tc=False, class_peaks=None):
    """Roofline of the dominant kernel class of a timing pass (kst: class -> totals over `steps` solves).

    star_peak: (TFLOP/s, source) of the precision the form's star kernel runs in; peaks: "fp64" and
    "hbm" (value, source).  tc: the form runs its star on the tensor cores at the upper levels, where
    the library keeps no executed-operation count.  class_peaks: class -> ((TFLOP/s, source) or None,
    note) for the classes whose kernels do not run on the FP64 pipe in this form (None: kernels of
    several precisions in one class, no single peak)."""
    dom = max(kst, key=lambda k: kst[k]["ms"])
    d = kst[dom]
    total_ms = sum(v["ms"] for v in kst.values())
    launches = sum(v["launches"] for v in kst.values())
    sec = d["ms"] / 1e3
    out = {"kernel": dom, "share": d["ms"] / total_ms, "launches_per_step": d["launches"] / steps,
           "ms_per_launch": 1e3 * sec / max(1, d["launches"]), "kernel_launches_per_step": launches / steps}
    if d["xflops"] > 0 and not (tc and dom == "star"):
        achieved = d["xflops"] / sec / 1e12
        out.update({"bound": "alu", "achieved": achieved, "peak": star_peak[0], "unit": "TFLOP/s",
                    "frac": achieved / star_peak[0] if star_peak[0] else None, "peak_source": star_peak[1],
                    "ops_per_launch": d["xflops"] / max(1, d["launches"]),
                    "paper_count_tflops": d["flops"] / sec / 1e12, "hbm_gbs": d["bytes"] / sec / 1e9})
    elif d["flops"] > 0:
        # arithmetic-bound class without an executed-operation count: the paper count only
        pk, note = star_peak if dom == "star" else peaks["fp64"], "no executed-operation count for this kernel class"
        if class_peaks and dom in class_peaks:
            pk, why = class_peaks[dom]
            note = f"{note}; {why}"
        out.update({"bound": "alu", "achieved": None, "peak": pk[0] if pk else None, "unit": "TFLOP/s",
                    "frac": None, "peak_source": pk[1] if pk else None,
                    "paper_count_tflops": d["flops"] / sec / 1e12, "note": note})
    else:
        achieved = d["bytes"] / sec / 1e9
        out.update({"bound": "hbm", "achieved": achieved, "unit": "GB/s", "peak": peaks["hbm"][0],
                    "frac": achieved / peaks["hbm"][0] if peaks["hbm"][0] else None, "peak_source": peaks["hbm"][1]})
    return out


def ff_class_peaks(fp32):
    """Kernel classes of the float-float forms that leave the FP64 pipe (see `roofline`)."""
    ff = (fp32, "float-float arithmetic on the FP32 pipes")
    return {"elem_schur": (None, "FP64 outer residual and float-float level residuals in one class"),
            "condense": ff, "recover": ff}


def measured_hbm():
    """(GB/s, source): the copy bandwidth measured on this GPU type, else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s)"


def kernel_table(kst, steps, tc=False):
    """Per-class event times and rates; tc: the star's executed count covers only its CUDA-core levels."""
    return {k: {"ms_per_step": r4(v["ms"] / steps), "launches_per_step": r4(v["launches"] / steps),
                "paper_tflops": r4(v["flops"] / (v["ms"] / 1e3) / 1e12) if v["flops"] and v["ms"] else None,
                "exec_tflops": (r4(v["xflops"] / (v["ms"] / 1e3) / 1e12)
                                if v["xflops"] and v["ms"] and not (tc and k == "star") else None),
                "hbm_gbs": r4(v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["bytes"] and v["ms"] else None}
            for k, v in kst.items() if v["launches"]}


def timing_pass(ctx, f, u, steps):
    """Per-kernel CUDA-event statistics of `steps` solves (a pass separate from the timed ones)."""
    ctx.set_timing(True)
    for _ in range(steps):
        ctx.solve(f, rtol=1e-10, out=u)
    kst = ctx.kstats()
    ctx.set_timing(False)
    return kst


def run_semmg(args, world, rank, local, pg):
    import torch
    from paper_1808_03595_gb300 import Context
    from paper_1808_03595_gb300 import build as _build
    from paper_1808_03595_gb300.solver import peak_tflops
    _build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    details = {}
    K, W = args.steps, args.warmup

    try:
        fp64_peak, fp64_src = peak_tflops(torch.float64), "measured (FP64 FMA chains, this run)"
        fp32_peak = peak_tflops(torch.float32)
    except Exception:  # pragma: no cover - a probe failure falls back to the nominal rate
        fp64_peak, fp64_src, fp32_peak = FP64_NOMINAL_TFLOPS, "nominal (probe failed)", None
    emit("peaks", {"fp64_tflops": r4(fp64_peak), "fp32_tflops": r4(fp32_peak), "source": fp64_src}, details)

    # ---- headline workload
    h, p, lam, f, p0 = workloads.config(HEADLINE)
    fd = torch.as_tensor(f, dtype=torch.float64, device=dev)
    ud = torch.empty_like(fd)
    unknowns = int(fd.numel())
    forms = ["fp64"] + list(MIXED_FORMS) + ([] if args.quick else list(DETAIL_FORMS))
    ctx = {}
    for form in forms:
        prec, solver, sm = FORMS[form]
        ctx[form] = Context(h, p, lam, p0=p0, precision=prec, solver=solver, smoother=sm)
        if args.autotune:
            ctx[form].autotune()
    for form in forms:
        for _ in range(W):
            ctx[form].solve(fd, rtol=1e-10, out=ud)
    torch.cuda.synchronize()

    # timed region of `value`: per-kernel timing off
    barrier(pg)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.nvtx.range_push("fp64_timed")  # NVTX ranges name the timed regions for profilers
    t64, info64 = timed_solves(ctx["fp64"], fd, ud, K, flush, stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(pg)
    tform, iters, infos = {}, {"fp64": info64.iters}, {"fp64": info64}
    for form in forms[1:]:
        torch.cuda.nvtx.range_push(f"{form}_timed")
        tform[form], inf = timed_solves(ctx[form], fd, ud, K, flush, stream)
        torch.cuda.nvtx.range_pop()
        iters[form], infos[form] = inf.iters, inf
    # end to end through the host-buffer entry point (pinned host f in, u out)
    te2e = float("nan")
    if not args.no_e2e:
        fh = torch.as_tensor(f, dtype=torch.float64).pin_memory()
        uh = torch.empty_like(fh).pin_memory()
        ctx["fp64"].solve_host(fh, uh, rtol=1e-10)
        te2e, _ = timed_solves(ctx["fp64"], None, None, K, flush, stream, host=(fh, uh))
    # roofline pass: the same solves with the per-kernel events on
    npass = max(1, min(K, 5))
    kst = timing_pass(ctx["fp64"], fd, ud, npass)
    emit("kernels_fp64", {"workload": HEADLINE, "solves": npass, "kernels": kernel_table(kst, npass)}, details)
    kst_m = {}
    for form in MIXED_FORMS:
        kst_m[form] = timing_pass(ctx[form], fd, ud, npass)
        emit(f"kernels_{form}", {"workload": HEADLINE, "solves": npass,
                                 "kernels": kernel_table(kst_m[form], npass, tc=form in TC_FORMS)}, details)
    torch.cuda.synchronize()

    t64 = max_over_ranks(pg, t64)
    te2e = max_over_ranks(pg, te2e)
    tform = {k: max_over_ranks(pg, v) for k, v in tform.items()}
    value = world * unknowns * K / (t64 / 1e3)
    vforms = {k: world * unknowns * K / (v / 1e3) for k, v in tform.items()}
    e2e = world * unknowns * K / (te2e / 1e3) if te2e == te2e else None
    emit("forms", {"workload": HEADLINE, "unknowns": unknowns,
                   "forms": {k: {"value": r4(v), "speedup_vs_fp64": r4(v / value), "iterations": iters[k],
                                 "reduction": r4(infos[k].res_final / infos[k].res0), "rho": r4(infos[k].rho),
                                 "us_per_unknown": r4(1e6 / v), "precision": FORMS[k][0], "solver": FORMS[k][1]}
                             for k, v in [("fp64", value)] + list(vforms.items())}}, details)
    peaks = {"fp64": (fp64_peak, fp64_src), "hbm": measured_hbm()}
    roof = roofline(kst, peaks["fp64"], peaks, npass)
    h_now = star_source_hash()
    roof["traffic"] = (STAR_TRAFFIC["bytes_per_launch"] if roof["kernel"] == "star" and h_now is not None
                       and h_now == STAR_TRAFFIC["source"] else None)
    emit("roofline", {k: (r4(v) if isinstance(v, float) else v) for k, v in roof.items()}, details)
    fp32 = (fp32_peak, "measured (FP32 FMA chains, this run)")
    for form in MIXED_FORMS:
        rm = roofline(kst_m[form], fp32, peaks, npass, tc=form in TC_FORMS,
                      class_peaks=ff_class_peaks(fp32) if FORMS[form][0] in FF_PRECISIONS else None)
        emit(f"roofline_{form}", {k: (r4(v) if isinstance(v, float) else v) for k, v in rm.items()}, details)
    best = max(MIXED_FORMS, key=lambda k: vforms[k])
    for c in ctx.values():
        c.close()

    # ---- secondary: the 8^3 Helmholtz degree sweep (one step = the four solves)
    sweep = run_sweep(args, dev, stream, flush, details)

    if not args.quick and rank == 0:
        run_batch(args, dev, stream, flush, details)
        run_configs(args, dev, stream, flush, details)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n, dt = 0, 0.0
        while dt < 10.0:  # about 10 s or more of CPU work: whole oracle solves of the sample
            n1, dt1, _ = oracle_sample()
            n, dt = n + n1, dt + dt1
        cpu = {"value": r4(n / dt), "unit": "unknowns/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": sample_text(n, dt)}
        emit("cpu_baseline", {**cpu, "us_per_unknown": r4(1e6 * dt / n)}, details)

    line = result_line(value=value, steps=K, warmup=W, ms_total=t64, unknowns=unknowns, p0=p0, world=world,
                       iterations=info64.iters, mixed=(best, vforms[best], iters[best]), e2e=e2e, roof=roof,
                       peak_measured=fp64_src.startswith("measured"), cpu=cpu, clocks=clk, sweep=sweep)
    if args.detail_json and rank == 0:
        with open(args.detail_json, "w") as fh:
            json.dump({"result": line, **details}, fh, indent=1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def result_line(value, steps, warmup, ms_total, unknowns, p0, world, iterations, mixed, e2e, roof, peak_measured,
                cpu, clocks, sweep):
    """The last stdout line: the headline and the keys the result needs, nothing else (it stays under
    MAX_LINE bytes; the tables went out as detail lines before it)."""
    best, vbest, itbest = mixed
    return {
        "metric": METRIC, "value": r4(value), "unit": "unknowns/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": r4(ms_total / steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": HEADLINE, "unknowns": unknowns, "solver": "alg4", "p0": p0,
                   "l2": "flushed (256 MiB write) before every solve",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "iterations": iterations,
        "mixed": {"value": r4(vbest), "form": best, "speedup_vs_fp64": r4(vbest / value), "iterations": itbest},
        "e2e": {"value": r4(e2e), "unit": "unknowns/s", "h2d_bytes_per_step": 8 * unknowns,
                "d2h_bytes_per_step": 8 * unknowns},
        "gpu_launches": int(round(roof["kernel_launches_per_step"] * steps)),
        "roofline": {"bound": roof["bound"],
                     "kernel": "k_star<double>" if roof["kernel"] == "star" else roof["kernel"],
                     "achieved": r4(roof["achieved"]), "peak": r4(roof["peak"]), "unit": roof["unit"],
                     "frac": r4(roof["frac"]), "traffic": roof["traffic"],
                     "peak_kind": "measured" if peak_measured else "nominal"},
        "cpu_baseline": cpu,
        "clocks": {k: clocks.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons", "samples")},
        "sweep_8x8x8": sweep,
    }


def run_sweep(args, dev, stream, flush, details):
    """Helmholtz lambda = 1 on 8^3 uniform elements, p in {4, 8, 16, 32}: FP64 and two mixed forms (CUDA-core
    and tensor-core smoother), one step = the four solves; unknowns/s over the K timed steps."""
    import torch
    from paper_1808_03595_gb300 import Context
    out = {}
    cases = []
    for q in SWEEP:
        h, q, lam, f, p0 = workloads.config(f"helmholtz_8x8x8_p{q}")
        fd = torch.as_tensor(f, dtype=torch.float64, device=dev)
        cases.append((q, fd, torch.empty_like(fd), {form: Context(h, q, lam, p0=p0, precision=FORMS[form][0])
                                                    for form in SWEEP_FORMS}))
    n = sum(int(c[1].numel()) for c in cases)
    table = {}
    for form in SWEEP_FORMS:
        for q, fd, ud, cx in cases:
            if args.autotune:
                cx[form].autotune()
            for _ in range(args.warmup):
                cx[form].solve(fd, out=ud)
        ms, its = 0.0, {}
        for q, fd, ud, cx in cases:
            t, info = timed_solves(cx[form], fd, ud, args.steps, flush, stream)
            ms += t
            its[q] = info.iters
        out[form] = r4(n * args.steps / (ms / 1e3))
        table[form] = {"value": out[form], "ms_per_step": r4(ms / args.steps), "iterations": its}
    for _, _, _, cx in cases:
        for c in cx.values():
            c.close()
    emit("sweep_8x8x8", {"workload": "helmholtz_8x8x8_p4-8-16-32", "unknowns_per_step": n, **table}, details)
    # the result line carries FP64 and the fastest mixed form (the table above names each form)
    return {"fp64": out["fp64"], "mixed": max(v for f, v in out.items() if f != "fp64")}


def run_configs(args, dev, stream, flush, details):
    """The other workloads of the paper's shape, one solve per step per form (not part of `value`):
    Helmholtz 16^3 at p = 16 (lambda 0 and 100, Dirichlet; lambda 1 with Neumann faces and periodic),
    Helmholtz 8^3 at p = 16 with the element-centred block smoother (Sec. 3.4), and the Sec. 5.2
    problem (8^3, k = 5, Dirichlet data) at p = 16 and 32."""
    import torch
    from paper_1808_03595_gb300 import Context
    plan = [("helmholtz_16x16x16_p16", 0.0, None, ["fp64", "mixed", "mixed_tc", "mixed_ff_tc", "kmg_mixed"]),
            ("helmholtz_16x16x16_p16", 100.0, None, ["fp64", "mixed"]),
            ("helmholtz_16x16x16_p16", 1.0, ("N",) * 6, ["fp64", "mixed"]),
            ("helmholtz_16x16x16_p16", 1.0, ("P",) * 6, ["fp64", "mixed"]),
            ("helmholtz_8x8x8_p16", None, None, ["eblock_fp64", "eblock_mixed"]),
            ("paper_sec52_8x8x8_p16", 0.0, None, ["fp64", "mixed", "mixed_ff_tc", "kmg_mixed"]),
            ("paper_sec52_8x8x8_p32", 0.0, None, ["fp64", "mixed", "mixed_ff_tc", "kmg_mixed"])]
    for name, lam, bc, forms in plan:
        gd = ue = None
        if name.startswith("paper_sec52"):
            p, p0 = int(name.rsplit("_p", 1)[1]), 2
            h = workloads.uniform_widths(8, 2 * math.pi)
            ue, f = workloads.paper_solution(h, p, 5.0, lam)
            gd = torch.as_tensor(ue, dtype=torch.float64, device=dev)
        else:
            h, p, lam0, f, p0 = workloads.config(name, lam=lam)
            lam = lam0 if lam is None else lam
        fd = torch.as_tensor(f, dtype=torch.float64, device=dev)
        ud = torch.empty_like(fd)
        n = int(fd.numel())
        key = f"{name}_lambda{lam:g}" + ({"N": "_neumann", "P": "_periodic"}[bc[0]] if bc else "")
        res = {"unknowns": n}
        for form in forms:
            prec, solver, sm = FORMS[form]
            with Context(h, p, lam, p0=p0, precision=prec, solver=solver, bc=bc, smoother=sm) as c:
                if args.autotune:
                    c.autotune()
                for _ in range(args.warmup):
                    c.solve(fd, out=ud, g=gd)
                ms = 0.0
                for _ in range(args.steps):
                    flush.fill_(1.0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    _, info = c.solve(fd, out=ud, g=gd)
                    e1.record(stream)
                    e1.synchronize()
                    ms += e0.elapsed_time(e1)
                    assert info.res_final <= 1e-10 * info.res0, (key, form)
            res[form] = {"value": r4(n * args.steps / (ms / 1e3)), "ms": r4(ms / args.steps),
                         "iterations": info.iters}
            if ue is not None:
                res[form]["max_error_vs_exact"] = r4(float(torch.max(torch.abs(ud - gd))))
        emit(f"config_{key}", res, details)


def run_batch(args, dev, stream, flush, details):
    """64 independent Helmholtz solves (n ~ U{2..12}, p ~ U{4..24}, lambda = 10^U(-2,3)) in one CUDA graph
    launch, in the mixed form with the tensor-core smoother (Algorithms 4 and 5) and in the plain FP64
    form (the same graph, and sequential solve calls); throughput = total unknowns / time per batch."""
    import torch
    from paper_1808_03595_gb300 import Batch, Context
    cases = workloads.batch64()
    fs = [torch.as_tensor(f, dtype=torch.float64, device=dev) for _, _, _, f in cases]
    us = [torch.empty_like(f) for f in fs]
    unknowns = sum(int(f.numel()) for f in fs)
    out = {"workload": "batch64 (n~U{2..12}, p~U{4..24}, lambda=10^U(-2,3), f~U(-1,1), seed 1808035955)",
           "solves": len(cases), "unknowns": unknowns}

    def graph(prec, solver):
        ctxs = [Context(h, p, lam, p0=2, precision=prec, solver=solver) for h, p, lam, _ in cases]
        if args.autotune:
            for c in ctxs:
                c.autotune()
        b = Batch(ctxs, fs, us)
        for _ in range(args.warmup):
            b.solve()
        ms, iters = 0.0, []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, infos = b.solve()
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            assert rc == 0 and all(i.res_final <= 1e-10 * i.res0 for i in infos)
            iters = [i.iters for i in infos]
        res = {"value": r4(unknowns * args.steps / (ms / 1e3)), "ms_per_batch": r4(ms / args.steps),
               "graph_nodes": b.graph_nodes(), "iterations": {"min": min(iters), "max": max(iters),
                                                              "mean": r4(sum(iters) / len(iters))}}
        b.close()
        for c in ctxs:
            c.close()
        return res

    out["mixed_mg"] = graph(BATCH_MIXED, "mg")
    out["mixed_kmg"] = graph(BATCH_MIXED, "kmg")
    out["fp64_mg"] = graph("fp64", "mg")
    # the plain FP64 form as a user without the batched entry point runs it: one solve call after another
    ctxs = [Context(h, p, lam, p0=2, precision="fp64", solver="mg") for h, p, lam, _ in cases]
    if args.autotune:
        for c in ctxs:
            c.autotune()
    for _ in range(args.warmup):
        for c, f, u in zip(ctxs, fs, us):
            c.solve(f, out=u)
    ms = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for c, f, u in zip(ctxs, fs, us):
            _, info = c.solve(f, out=u)
            assert info.res_final <= 1e-10 * info.res0
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    for c in ctxs:
        c.close()
    out["fp64_sequential"] = {"value": r4(unknowns * args.steps / (ms / 1e3)), "ms_per_batch": r4(ms / args.steps)}
    out["speedup_mixed_vs_fp64_graph"] = r4(out["mixed_mg"]["value"] / out["fp64_mg"]["value"])
    out["speedup_mixed_kmg_vs_fp64_graph"] = r4(out["mixed_kmg"]["value"] / out["fp64_mg"]["value"])
    out["speedup_mixed_vs_fp64_sequential"] = r4(out["mixed_mg"]["value"] / out["fp64_sequential"]["value"])
    emit("batch64", out, details)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="semmg", choices=["semmg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer timing (profiling runs)")
    ap.add_argument("--quick", action="store_true",
                    help="headline, its mixed forms and the 8^3 sweep only (no batch, other workloads or "
                         "Krylov / all-FP32 forms)")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="tune launch shapes per level before the warm-up (outside the timed region)")
    ap.add_argument("--detail-json", default=None, help="also write the result and every detail table here")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local, pg = dist_setup()
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    else:
        rc = run_semmg(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
