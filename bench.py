"""Benchmark: unknowns/s per solve to a 1e-10 relative residual reduction.

Workload (default): Helmholtz lambda = 1 on the unit cube, 8x8x8 uniform
elements, degree sweep p in {4, 8, 16, 32}, f = manufactured solution plus
seeded N(0, 1e-2) noise at the GLL nodes, plain FP64 GPU form, coarse degree
p0 = 2.  One step solves all four degrees (condensation, V-cycles to 1e-10,
interior recovery); unknowns = sum of (8p+1)^3.  The mixed-precision form
(FP32 smoother and transfers, FP64 residual arithmetic, inside FP64 iterative
refinement) is timed on the same workload and reported under "mixed"; "forms"
adds the all-FP32 V-cycle and the Krylov-accelerated iteration (Algorithm 5)
in FP64 and mixed precision, and "batched" 64 independent solves in one CUDA
graph.

Timing: CUDA events on the solving stream around each solve, L2 flushed
(256 MiB write) before every solve, W untimed warm-up steps, then K timed
steps; max over ranks.  "e2e" repeats the timed steps through the host-buffer
entry point (pinned host f in, u out, copies inside the timed region).
Multi-GPU runs are replicas (the path has no exchange step on one mesh).
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

SWEEP = [4, 8, 16, 32]
WORKLOAD = "helmholtz_8x8x8_p4-8-16-32"
METRIC = "unknowns/s per solve to 1e-10 residual (FP64 vs mixed); smoother HBM GB/s"
# timed forms: name -> (precision, outer iteration).  "fp64" is the headline value,
# "mixed" the mixed-precision line (FP32 smoother and transfers, FP64 residuals).
FORMS = {"fp64": ("fp64", "mg"), "mixed": ("mixed", "mg"), "mixed_fp32": ("mixed_fp32", "mg"),
         "mixed_tc": ("mixed_tc", "mg"), "kmg_fp64": ("fp64", "kmg"), "kmg_mixed": ("mixed", "kmg"),
         "kmg_mixed_tc": ("mixed_tc", "kmg"), "eblock_fp64": ("fp64", "mg"), "eblock_mixed": ("mixed", "mg"),
         "eblock_mult_mixed": ("mixed", "mg"), "mixed_fp32_tc": ("mixed_fp32_tc", "mg"),
         "kmg_mixed_fp32_tc": ("mixed_fp32_tc", "kmg")}
# forms with the element-centred block smoother (Sec. 3.4) instead of the vertex stars
ELEMENT_FORMS = {"eblock_fp64": "element", "eblock_mixed": "element", "eblock_mult_mixed": "element_mult"}
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate (no measured FP64 entry in the peaks file)
# DRAM bytes (read + write) per k_star<double> launch of the timed FP64 sweep: ncu
# --metrics dram__bytes_read.sum,dram__bytes_write.sum per launch of `bench.py --forms fp64
# --no-e2e --no-batch --no-configs --no-cpu-baseline --steps 1 --warmup 3`, averaged per degree and
# weighted by the sweep's star launches per degree (28 at p = 4, 20 at 8, 12 at 16, 6 at 32);
# profiles/k_star_f64_dram_helmholtz_8x8x8.md.  Valid only for the star-kernel source it was
# measured on (hash below).
STAR_TRAFFIC_BYTES = 7.771e6
STAR_TRAFFIC_SOURCE = "fb81d2dbe05b46a3"
# Executed FP64 operations (2 DFMA + DMUL + DADD thread instructions, ncu sass counters) per
# k_star<double> launch, per level degree, from `bench.py --degrees 32 --forms fp64 --no-e2e --no-batch
# --no-configs --no-cpu-baseline --no-autotune --steps 1 --warmup 3` (the first launch at each of
# p = 32, 16, 8, 4; profiles/k_star_f64_executed_ops_helmholtz_8x8x8.md), weighted like the traffic:
# the kernel executes 32-44 % of the paper's 37 n_S^3 count, so this rate measures the FP64 pipe.
STAR_EXEC_FLOPS = {4: 0.004116e9, 8: 0.032777e9, 16: 0.264593e9, 32: 2.158269e9}
STAR_EXEC_WEIGHTS = {4: 28, 8: 20, 16: 12, 32: 6}
STAR_EXEC_SOURCE = "fb81d2dbe05b46a3"
STAR_SOURCES = ("star_kernel.cuh", "kernels_star_f64.cu")


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


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


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

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
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


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
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


# ---------------------------------------------------------------- reference arm: the oracle on the host

def oracle_sample(p=16):
    """One O2 (oracle) solve of the 8x8x8 Helmholtz workload at degree p; returns (unknowns, seconds, iters)."""
    from oracle import dense, matfree
    h, p, lam, f, p0 = workloads.config(f"helmholtz_8x8x8_p{p}")
    mesh = dense.Mesh(h, p, lam)
    t0 = time.perf_counter()
    _, it, _ = matfree.solve(mesh, f, p0=p0)
    dt = time.perf_counter() - t0
    return (8 * p + 1) ** 3, dt, it


def run_reference(args, world, rank, pg):
    if rank != 0:
        return 0
    sample_p = args.cpu_sample_p
    for _ in range(args.warmup):
        oracle_sample(sample_p)
    tot_n, tot_t = 0, 0.0
    for _ in range(args.steps):
        n, dt, _ = oracle_sample(sample_p)
        tot_n += n
        tot_t += dt
    v = tot_n / tot_t
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "unknowns/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"p={sample_p} solve per step", "parallelism": "none"},
        "cpu_baseline": {"value": v, "unit": "unknowns/s", "cores": cores, "kind": "oracle",
                         "sample": f"one matrix-free oracle (numpy FP64) solve of helmholtz_8x8x8 at p={sample_p} "
                                   f"({(8 * sample_p + 1) ** 3} unknowns) per step"},
        "e2e": {"value": v, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm

def run_semmg(args, world, rank, local, pg):
    import torch
    from paper_1808_03595_gb300 import Context
    from paper_1808_03595_gb300 import build as _build
    _build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    degrees = [int(x) for x in args.degrees.split(",")]

    forms = args.forms.split(",")
    if "fp64" not in forms:
        forms = ["fp64"] + forms
    for form in forms:
        if form not in FORMS:
            raise SystemExit(f"unknown form {form}; choose from {sorted(FORMS)}")
    cases = []
    for p in degrees:
        h, p, lam, f, p0 = workloads.config(f"helmholtz_8x8x8_p{p}")
        fd = torch.as_tensor(f, dtype=torch.float64, device=dev)
        ud = torch.empty_like(fd)
        fh = torch.as_tensor(f, dtype=torch.float64).pin_memory()
        uh = torch.empty_like(fh).pin_memory()
        c = {"p": p, "n": int(fd.numel()), "f": fd, "u": ud, "fh": fh, "uh": uh}
        for form in forms:
            prec, solver = FORMS[form]
            c[form] = Context(h, p, lam, p0=p0, precision=prec, solver=solver,
                              smoother=ELEMENT_FORMS.get(form, "star"))
        cases.append(c)
    tuned = {}
    if args.autotune:
        for c in cases:
            for form in forms:
                ctx = c[form]
                ctx.autotune()
                dts = torch.float32 if FORMS[form][0] in ("mixed_fp32", "mixed_fp32_tc") else torch.float64
                dt = torch.float64 if FORMS[form][0] == "fp64" else torch.float32
                tuned.setdefault(form, {})[c["p"]] = {
                    "star": ctx.launch_shape(ctx.L, "star", dt), "schur": ctx.launch_shape(ctx.L, "schur", dts)}
    torch.cuda.synchronize()

    per_p_ms = {form: {} for form in forms}

    def solve_all(form, timed, host=False):
        ms, iters = 0.0, {}
        for c in cases:
            ctx = c[form]
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if host:
                _, info = ctx.solve_host(c["fh"], c["uh"], rtol=1e-10)
            else:
                _, info = ctx.solve(c["f"], rtol=1e-10, out=c["u"])
            e1.record(stream)
            e1.synchronize()
            if timed:
                dt = e0.elapsed_time(e1)
                ms += dt
                if not host:
                    per_p_ms[form][c["p"]] = per_p_ms[form].get(c["p"], 0.0) + dt / args.steps
            iters[c["p"]] = info.iters
            assert info.res_final <= 1e-10 * info.res0, (form, c["p"], info.res_final, info.res0)
        return ms, iters

    for form in forms:
        for _ in range(args.warmup):
            solve_all(form, False)
    # timed region (device-resident inputs)
    for c in cases:
        c["fp64"].set_timing(True)
    barrier(pg)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t64, it64 = 0.0, {}
    for _ in range(args.steps):
        ms, it64 = solve_all("fp64", True)
        t64 += ms
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(pg)
    kst = {}
    for c in cases:
        for k, v in c["fp64"].kstats().items():
            acc = kst.setdefault(k, {"ms": 0.0, "launches": 0, "flops": 0.0, "bytes": 0.0})
            for kk in acc:
                acc[kk] += v[kk]
        c["fp64"].set_timing(False)
    te2e = float("nan")
    tform, itform, kstform = {}, {}, {}
    for form in forms:
        if form == "fp64":
            continue
        for c in cases:
            c[form].set_timing(True)
        tf = 0.0
        for _ in range(args.steps):
            ms, itform[form] = solve_all(form, True)
            tf += ms
        tform[form] = tf
        kk = kstform.setdefault(form, {})
        for c in cases:
            for k, v in c[form].kstats().items():
                acc = kk.setdefault(k, {"ms": 0.0, "launches": 0, "flops": 0.0})
                acc["ms"] += v["ms"]
                acc["launches"] += v["launches"]
                acc["flops"] += v["flops"]
            c[form].set_timing(False)
    t32 = tform.get("mixed", float("nan"))
    it32 = itform.get("mixed", {})
    kst32 = kstform.get("mixed", {})
    if not args.no_e2e:
        # end to end through the host-buffer entry point
        solve_all("fp64", False, host=True)
        te2e = 0.0
        for _ in range(args.steps):
            ms, _ = solve_all("fp64", True, host=True)
            te2e += ms
    torch.cuda.synchronize()

    t64 = max_over_ranks(pg, t64)
    t32 = max_over_ranks(pg, t32)
    te2e = max_over_ranks(pg, te2e)
    tform = {k: max_over_ranks(pg, v) for k, v in tform.items()}
    unknowns = sum(c["n"] for c in cases)
    value = world * unknowns * args.steps / (t64 / 1e3)
    value32 = world * unknowns * args.steps / (t32 / 1e3)
    e2e = world * unknowns * args.steps / (te2e / 1e3)
    forms_out = {"fp64": {"precision": "fp64", "solver": "mg", "value": value, "ms_per_step": t64 / args.steps,
                          "iterations": it64}}
    for form, tf in tform.items():
        v = world * unknowns * args.steps / (tf / 1e3)
        forms_out[form] = {"precision": FORMS[form][0], "solver": FORMS[form][1],
                           "smoother": ELEMENT_FORMS.get(form, "star"), "value": v,
                           "ms_per_step": tf / args.steps, "iterations": itform[form], "speedup_vs_fp64": v / value,
                           "kernels": {k: {"ms_per_step": x["ms"] / args.steps,
                                           "launches_per_step": x["launches"] / args.steps,
                                           "tflops": (x["flops"] / (x["ms"] / 1e3) / 1e12) if x["flops"] else None}
                                       for k, x in kstform[form].items()}}

    # roofline of the dominant kernel (FP64 form): FP64-ALU bound
    dom = max(kst, key=lambda k: kst[k]["ms"])
    d = kst[dom]
    total_ms = sum(v["ms"] for v in kst.values())
    launches = sum(v["launches"] for v in kst.values())
    peaks = load_peaks()
    traffic = None
    if dom == "star":
        if star_source_hash() == STAR_TRAFFIC_SOURCE:
            traffic = STAR_TRAFFIC_BYTES
    executed = None
    if dom == "star" and star_source_hash() == STAR_EXEC_SOURCE and degrees == SWEEP:
        per_launch = sum(STAR_EXEC_FLOPS[q] * STAR_EXEC_WEIGHTS[q] for q in SWEEP) / sum(STAR_EXEC_WEIGHTS.values())
        rate = per_launch * d["launches"] / (d["ms"] / 1e3) / 1e12
        executed = {"flops_per_launch": per_launch, "achieved": rate, "frac": rate / FP64_PEAK_TFLOPS}
    if d["flops"] > 0:
        achieved = d["flops"] / (d["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "kernel": dom, "executed": executed,
                "algorithmic_bytes_per_launch": d["bytes"] / max(1, d["launches"]),
                "peak_source": "nominal FP64 1.25 TFLOP/s (2 FP64 FMA/clk/SM x 152 SMs at 2.07 GHz)",
                "launches": d["launches"], "share_of_kernel_time": d["ms"] / total_ms,
                "hbm_gbs": d["bytes"] / (d["ms"] / 1e3) / 1e9}
    else:
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        pk = peaks.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk, "unit": "GB/s", "frac": achieved / pk,
                "traffic": None, "kernel": dom, "launches": d["launches"]}

    line = {
        "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t64 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "degrees": degrees, "elements": [8, 8, 8], "lambda": 1.0, "p0": 2,
                   "rtol": 1e-10, "l2": "flushed (256 MiB write) before every solve",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "iterations": {"fp64": it64, "mixed": it32},
        "mixed": {"value": value32, "unit": "unknowns/s", "dtype": "f64+f32", "ms_per_step": t32 / args.steps,
                  "speedup_vs_fp64": value32 / value},
        "e2e": {"value": e2e, "unit": "unknowns/s", "h2d_bytes_per_step": 8 * unknowns,
                "d2h_bytes_per_step": 8 * unknowns},
        "gpu_launches": int(launches // max(1, args.steps)) * args.steps,
        "kernels_fp64": {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps}
                         for k, v in kst.items()},
        "kernels_mixed": {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps}
                          for k, v in kst32.items()},
        "forms": forms_out,
        "ms_per_degree": per_p_ms,
        "launch_shapes_finest_level": tuned,
        "roofline": roof,
        "clocks": clk,
    }
    if args.batch and rank == 0:
        line["batched"] = run_batch(args, dev, stream, flush)
        line["batched_kmg"] = run_batch(args, dev, stream, flush, solver="kmg")
        if "fp64_plain" in line["batched"]:
            line["batched_kmg"]["speedup_vs_fp64_plain"] = (line["batched_kmg"]["value"] /
                                                            line["batched"]["fp64_plain"]["value"])
    if args.configs and rank == 0:
        line["configs"] = run_configs(args, dev, stream, flush)
    if rank == 0 and not args.no_cpu_baseline:
        n, dt = 0, 0.0
        while dt < 10.0:  # about 10 s of CPU work: whole oracle solves until then
            n1, dt1, _ = oracle_sample(args.cpu_sample_p)
            n, dt = n + n1, dt + dt1
        line["cpu_baseline"] = {"value": n / dt, "unit": "unknowns/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"matrix-free oracle (numpy FP64) solves of helmholtz_8x8x8 at "
                                          f"p={args.cpu_sample_p} ({n} unknowns in all), {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for c in cases:
        for form in forms:
            c[form].close()
    return 0


def run_configs(args, dev, stream, flush):
    """The other workloads of the paper's shape, one solve per form each (not part of `value`):
    Helmholtz 16^3 at p = 16 (lambda 0 and 100, Dirichlet; lambda 1 with Neumann faces and periodic) and
    Poisson on 6^3 stretched elements at p = 48."""
    import torch
    from paper_1808_03595_gb300 import Context
    out = {}
    plan = [("helmholtz_16x16x16_p16", 0.0, None, ["fp64", "mixed", "mixed_tc", "kmg_mixed"]),
            ("helmholtz_16x16x16_p16", 100.0, None, ["fp64", "mixed"]),
            ("helmholtz_16x16x16_p16", 1.0, ("N",) * 6, ["fp64", "mixed", "kmg_mixed"]),
            ("helmholtz_16x16x16_p16", 1.0, ("P",) * 6, ["fp64", "mixed", "kmg_mixed"]),
            ("poisson_6x6x6_p48_stretched", None, None, ["fp64", "mixed", "mixed_tc", "kmg_fp64", "kmg_mixed"]),
            ("paper_sec52_8x8x8_p16", 0.0, None, ["fp64", "mixed", "kmg_mixed"]),
            ("paper_sec52_8x8x8_p32", 0.0, None, ["fp64", "mixed", "kmg_mixed"])]
    for name, lam, bc, forms in plan:
        gd = ue = None
        if name.startswith("paper_sec52"):
            # the runtime tests' problem: (0, 2 pi)^3, k = 5, lambda = 0, inhomogeneous Dirichlet data
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
        out[key] = {"unknowns": n}
        for form in forms:
            prec, solver = FORMS[form]
            with Context(h, p, lam, p0=p0, precision=prec, solver=solver, bc=bc) as c:
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
            out[key][form] = {"value": n * args.steps / (ms / 1e3), "ms": ms / args.steps, "iterations": info.iters}
            if ue is not None:
                out[key][form]["max_error_vs_exact"] = float(torch.max(torch.abs(ud - gd)))
    return out


def run_batch(args, dev, stream, flush, solver="mg"):
    """64 independent Helmholtz solves (n ~ U{2..12}, p ~ U{4..24}, lambda = 10^U(-2,3), mixed form) in one
    CUDA graph launch; throughput = total unknowns / graph time."""
    import torch
    from paper_1808_03595_gb300 import Batch, Context
    cases = workloads.batch64()
    ctxs, fs, us = [], [], []
    for h, p, lam, f in cases:
        ctxs.append(Context(h, p, lam, p0=2, precision="mixed", solver=solver))
        fs.append(torch.as_tensor(f, dtype=torch.float64, device=dev))
        us.append(torch.empty_like(fs[-1]))
    t0 = time.perf_counter()
    if args.autotune:
        for c in ctxs:
            c.autotune()
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = Batch(ctxs, fs, us)
    t_capture = time.perf_counter() - t0
    for _ in range(args.warmup):
        b.solve()
    ms = 0.0
    iters = []
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
    unknowns = sum(int(f.numel()) for f in fs)
    out = {"workload": "batch64 (n~U{2..12}, p~U{4..24}, lambda=10^U(-2,3), f~U(-1,1), seed 1808035955)",
           "solver": solver, "value": unknowns * args.steps / (ms / 1e3), "unit": "unknowns/s", "dtype": "f64+f32",
           "solves": len(cases), "unknowns": unknowns, "ms_per_batch": ms / args.steps,
           "graph_nodes": b.graph_nodes(), "capture_s": t_capture, "autotune_s": t_tune,
           "iterations": {"min": min(iters), "max": max(iters), "mean": sum(iters) / len(iters)}}
    b.close()
    for c in ctxs:
        c.close()
    if solver == "mg":
        # the plain FP64 GPU form on the same 64 solves, one solve call after another
        ctxs = [Context(h, p, lam, p0=2, precision="fp64", solver="mg") for h, p, lam, _ in cases]
        if args.autotune:
            for c in ctxs:
                c.autotune()
        for _ in range(args.warmup):
            for c, f, u in zip(ctxs, fs, us):
                c.solve(f, out=u)
        ms64 = 0.0
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
            ms64 += e0.elapsed_time(e1)
        v64 = unknowns * args.steps / (ms64 / 1e3)
        out["fp64_plain"] = {"value": v64, "ms_per_batch": ms64 / args.steps,
                             "note": "same 64 solves, FP64 form, sequential semmg_solve calls"}
        out["speedup_vs_fp64_plain"] = out["value"] / v64
        for c in ctxs:
            c.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="semmg", choices=["semmg", "reference"])
    ap.add_argument("--degrees", default=",".join(str(p) for p in SWEEP))
    ap.add_argument("--cpu-sample-p", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", default=",".join(FORMS),
                    help="forms to time, from " + ", ".join(FORMS) + " (fp64 is always timed: the headline)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer timing (profiling runs)")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="tune launch shapes per degree before the warm-up (outside the timed region)")
    ap.add_argument("--configs", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the 16^3 p=16, 6^3 p=48 stretched and Sec. 5.2 workloads (under configs)")
    ap.add_argument("--batch", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the 64-solve batched graph workload")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        rc = run_reference(args, world, rank, pg)
    else:
        rc = run_semmg(args, world, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
