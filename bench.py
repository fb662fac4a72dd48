#!/usr/bin/env python
"""Benchmark of the BF-MHT apply on GB300: transforms/s (synthesis + adjoint) and roofline.

Workload (default): the unit sphere, n = 65536 jittered-Fibonacci points, m = 65536 real
spherical harmonics up to degree 255, eps = 1e-6, leaf size 128, FP32 apply, analysis
weights 4 pi / n.  One step = one synthesis f = Phi c plus one weighted analysis
c = Phi^T W f of `--nrhs` vectors; value = vectors transformed (both directions) per second
over all ranks.  Inputs are resident in HBM; the packed factors (GBs) are far larger than
L2, so every step streams them from HBM (no flush needed).

`--impl reference` times the FP64 CPU oracle on the same workload: its butterfly apply (Sec. 2,
stage by stage, numpy/BLAS on the host cores) of the plan's exported factors, one whole
transform pair per step.

`--gpus N` (N > 1) without a launcher starts N replicas itself (torch.distributed.run on this
node, one rank per GPU); under a launcher (WORLD_SIZE set) every rank runs one replica.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "transforms/s (synthesis + weighted adjoint)"
# DRAM bytes (read + write) per algorithmic byte of the per-stage kernel, from ncu's
# dram__bytes_read.sum + dram__bytes_write.sum over every stage launch of one timed step on the
# 16384-point sphere (the launch shapes the autotuner chose there).  Traffic grows in proportion
# to the bytes a launch streams (1.001 on the largest 16384-point stages), so a full-size
# launch's traffic is this ratio times its algorithmic bytes.  None: not captured for the
# current kernel.
NCU_DRAM_PER_ALG_BYTE = {
    "k_rowdot synthesis (transfer levels 0..L)": 0.9998,
    "k_rowdot adjoint (transfer levels L..0)": 1.0034,
}
WORKLOADS = {
    # name: (n, lmax, leaf, eps)
    "sphere65536": (65536, 255, 128, 1e-6),
    "sphere16384": (16384, 127, 128, 1e-6),   # small case for profiler captures
    "sphere4096": (4096, 63, 128, 1e-6),
}
# the deformed-sphere FEM configuration at its stated size: its plan comes from a file written by
# tests/c3_plan.py (the eigenpairs take half an hour of host time), named by --plan-cache or
# the environment variable MHT_C3_PLAN
C3 = "c3"
C3_DESC = {"workload": "deformed-sphere mesh: icosphere level 6 (40962 vertices, 81920 triangles), radius "
                       "1 + 0.2 h / max|h|, P1 cotangent stiffness + lumped mass, the 4096 lowest generalized "
                       "eigenpairs (FP64 host spectral slicing), eps=1e-6, leaf 128, patch-rule Fiedler tree, "
                       "FP32 factors, lumped-mass weights",
           "n": 40962, "m": 4096, "eps": 1e-6, "leaf_size": 128,
           "l2": "packed factors (0.2 GB) > 129 MB L2 (streamed from HBM every step; no flush needed)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--multi-rhs", type=int, default=64, help="extra measurement at this many RHS (0: off)")
    ap.add_argument("--workload", default="sphere65536", choices=sorted(WORKLOADS) + [C3, "batch64", "torus_sweep", "peaks", "ranks"],
                    help="batch64: 64 ragged instances (torus / sphere / deformed sphere, n in [2000, 40000], "
                         "m = n/4, 1-128 RHS each) in one persistent launch per direction; torus_sweep: the flat-torus "
                         "memory law (m = ceil(n/25), eps 1e-3 and 1e-6) with single-RHS apply times; peaks: "
                         "the GEMM rates the multi-RHS rooflines divide by (TF32, FP32, FP64, BF16); ranks: "
                         "the rank layout of a replica launch (gloo, no GPU work)")
    ap.add_argument("--plan-cache", default=os.environ.get("MHT_PLAN_CACHE", ""))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the FP64 error check of the multi-RHS forms")
    ap.add_argument("--no-autotune", action="store_true", help="time the default launch shapes")
    ap.add_argument("--path", default="auto", choices=["auto", "fused", "staged"],
                    help="apply path: one persistent launch per direction, or one launch per stage")
    return ap.parse_args()


def workload_desc(name):
    if name == C3:
        return dict(C3_DESC)
    n, lmax, leaf, eps = WORKLOADS[name]
    return {"workload": f"unit sphere: n={n} jittered-Fibonacci points, m={(lmax + 1) ** 2} real spherical "
                        f"harmonics (degree <= {lmax}), eps={eps:g}, leaf {leaf}, FP32 factors, weights 4pi/n",
            "n": n, "m": (lmax + 1) ** 2, "eps": eps, "leaf_size": leaf,
            "l2": ("packed factors >> 129 MB L2 (streamed from HBM every step; no flush needed)" if n >= 16384 else
                   "packed factors may fit in the 129 MB L2 (L2-resident small case; not a bench line)")}


# ------------------------------------------------------------------ reference arm (oracle)
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def blas_threads(k):
    """Sets the thread count of numpy's bundled OpenBLAS (when its control symbol is found);
    returns the previous count, or None when it cannot be set."""
    import ctypes
    import glob

    import numpy as np
    libdir = os.path.join(os.path.dirname(np.__file__), "..", "numpy.libs")
    for lib in glob.glob(os.path.join(libdir, "*openblas*")):
        try:
            h = ctypes.CDLL(lib)
        except OSError:
            continue
        for prefix in ("scipy_openblas", "openblas"):
            for suffix in ("64_", ""):
                get = getattr(h, f"{prefix}_get_num_threads{suffix}", None)
                put = getattr(h, f"{prefix}_set_num_threads{suffix}", None)
                if get is not None and put is not None:
                    prev = int(get())
                    put(ctypes.c_int(int(k)))
                    return prev
    return None


def analysis_weights(plan, workload):
    """The plan's analysis weights: quadrature 4 pi / n on the sphere; on the mesh the lumped
    mass stored in the plan file."""
    import numpy as np
    if workload == C3:
        return plan.export()["weights"]
    return np.full(plan.n, 4 * np.pi / plan.n)


def oracle_factors(plan):
    """The plan's FP64 factors in the oracle's form (array reshaping only)."""
    from tests._bridge import arrays_to_oracle
    return arrays_to_oracle(plan.export())


def oracle_step(F, c, w):
    """One step of the reference: the oracle's FP64 butterfly apply (Sec. 2, stage by stage) of
    synthesis f = Phi c and weighted analysis Phi^T W f.  Returns (wall, process CPU) seconds."""
    from oracle import butterfly as B
    t0, p0 = time.perf_counter(), time.process_time()
    f = B.synthesize(F, c)
    B.analyze(F, f, w)
    return time.perf_counter() - t0, time.process_time() - p0


def cpu_baseline(F, c, w, steps, warmup=1):
    """The oracle's butterfly apply of the same plan on the host: whole transforms, numpy/BLAS
    on every core the process may use; plus one transform with BLAS limited to a single thread."""
    for _ in range(max(1, warmup)):
        oracle_step(F, c, w)
    runs = [oracle_step(F, c, w) for _ in range(max(1, steps))]
    wall = sum(r[0] for r in runs)
    used = sum(r[1] for r in runs) / max(wall, 1e-9)
    single = None
    prev = blas_threads(1)
    if prev is not None:
        single = 1.0 / oracle_step(F, c, w)[0]
        blas_threads(prev)
    avail = len(os.sched_getaffinity(0))
    meta = {"kind": "oracle", "cores": max(1, round(used)), "cpu_time_per_wall_time": round(used, 2),
            "cores_available": avail, "cpu_model": cpu_model(), "single_core_transforms_per_s": single,
            "sample": f"{len(runs)} whole transforms (synthesis + weighted analysis of one vector): the oracle's "
                      f"FP64 butterfly apply of the plan's exported factors, numpy with BLAS on up to {avail} "
                      f"threads"}
    return len(runs) / wall, meta, [r[0] for r in runs]


def direct_summation_sample(name, budget_s=15.0):
    """The exact transform by direct summation (rows of Phi by the normalized Legendre
    recurrence) on a random sample of rows, scaled to whole transforms by n / rows."""
    import numpy as np

    import workloads as W
    from oracle import harmonics as H
    n, lmax, leaf, eps = WORKLOADS[name]
    X = W.fibonacci_points(n)
    m = (lmax + 1) ** 2
    c = W.sphere_coefficients(m)[:, 0]
    w = np.full(n, 4 * np.pi / n)
    rng = np.random.default_rng(0)

    def rows_step(rows):
        t0 = time.perf_counter()
        Phi = H.sphere_phi(X[rows], lmax)
        f = Phi @ c
        _ = Phi.T @ (w[rows] * f)
        return time.perf_counter() - t0

    rows = np.sort(rng.choice(n, 256, replace=False))
    per_row = rows_step(rows) / len(rows)
    s = int(min(n, max(256, budget_s / max(per_row, 1e-9))))
    rows = np.sort(rng.choice(n, s, replace=False))
    t = rows_step(rows)
    return {"value": 1.0 / (t * n / s), "unit": "transforms/s", "sample": f"{s} of {n} rows, scaled by n/{s}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload not in WORKLOADS and args.workload != C3:
        raise SystemExit("--impl reference times the oracle on the single-plan workloads only")
    import numpy as np

    import workloads as W
    from paper_2605_21828_gb300.build import build_library
    build_library()
    desc = workload_desc(args.workload)
    plan, setup_s, _ = get_plan(args, None, 0)  # the library's host build of the factors (not timed)
    F = oracle_factors(plan)
    n, m = plan.n, plan.m
    c = W.sphere_coefficients(m)[:, 0]
    w = analysis_weights(plan, args.workload)
    steps = max(1, args.steps)
    value, cb, times = cpu_baseline(F, c, w, steps, warmup=args.warmup)
    ms = 1000.0 / value
    cb["value"] = value
    cb["unit"] = "transforms/s"
    desc.update({"nrhs": 1, "plan_setup_s": round(setup_s, 1)})
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "transforms/s", "n_gpus": args.gpus, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": desc,
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = [[x.strip() for x in line.split(",")] for line in open(self.path)]
        rows = [r for r in rows if len(r) >= 9]
        if len({r[0] for r in rows}) > 1:  # several GPUs visible: keep this rank's
            rows = [r for r in rows if r[0] == str(gpu_index)]
        for p in rows:
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(x, dist, device="cpu"):
    """The largest value of x over all ranks (identity without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def get_plan(args, dist, rank):
    import numpy as np

    import workloads as W
    from paper_2605_21828_gb300 import Plan
    t0 = time.time()
    if args.workload == C3:
        path = args.plan_cache or os.environ.get("MHT_C3_PLAN", "")
        if not path or not os.path.exists(path):
            raise SystemExit("--workload c3 reads a saved plan (--plan-cache or MHT_C3_PLAN; "
                             "written by python tests/c3_plan.py OUT.plan)")
        return Plan.load(path, mode="fp32"), time.time() - t0, False
    n, lmax, leaf, eps = WORKLOADS[args.workload]
    m = (lmax + 1) ** 2
    cache = args.plan_cache or os.path.join(tempfile.gettempdir(), f"mht_{args.workload}.plan")
    built = False
    if rank == 0 and not os.path.exists(cache):
        X = W.fibonacci_points(n)
        plan = Plan.build(n=n, m=m, eigenvalues=W.sphere_eigenvalues(m), evaluator="sphere", points=X, eps=eps,
                          leaf_size=leaf, mode="fp32", weights=np.full(n, 4 * np.pi / n))
        built = True
        if dist is not None or args.plan_cache:
            plan.save(cache)
    if dist is not None:
        dist.barrier()
    if not built:
        plan = Plan.load(cache, mode="fp32")
    return plan, time.time() - t0, built


MODES_MULTI = {
    # mode: (kernel description, tensor products per useful product, tensor dtype)
    "fp32": ("k_rowdot (SIMT FP32, Kahan-compensated)", 0, None),
    "3xtf32": ("k_tcs (tcgen05 kind::tf32: two-way split, 3 products, FP32 accumulation)", 3, "tf32"),
    "6xbf16": ("k_tcs (tcgen05 kind::f16 BF16: exact three-way split, 6 products, FP32 accumulation)", 6, "bf16"),
}


def tensor_peak_tflops(dtype, peaks):
    """Dense tensor peak for a kernel timed inside a long step: the driver's sustained bf16 GEMM
    rate, and for TF32 that rate times the nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)."""
    bf16 = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
    return bf16 if dtype == "bf16" else bf16 * 1.1 / 2.25


def multi_rhs_measure(args, plan, dev, stream, world, step, K):
    """The same step with --multi-rhs vectors: plain FP32 SIMT products against the split
    tensor-core products (3xTF32, 6xBF16), each timed, with its error against the FP64 apply of
    the same factors and, for the tensor-core forms, the roofline of the block-product kernel."""
    import torch

    import workloads as W
    km = args.multi_rhs
    m = plan.m
    plan.set_path("auto")  # wide RHS counts take the per-stage kernels
    C = torch.from_numpy(W.sphere_coefficients(m, km)).float().to(dev)
    multi = {"nrhs": km}
    outs = {}
    L = plan.levels
    stages = [plan.level_info(s) for s in range(L + 2)]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    for mode, (kdesc, prods, tdt) in MODES_MULTI.items():
        plan.set_mode(mode)
        tuned = plan.autotune(km) if not args.no_autotune else []
        for _ in range(3):
            step(C)
        torch.cuda.synchronize()
        reps = max(3, K // 4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            step(C)
        e1.record(stream)
        torch.cuda.synchronize()
        mms = e0.elapsed_time(e1) / reps
        outs[mode] = (plan.synthesize_raw(C), step(C))
        r = {"ms_per_step": mms, "transforms_per_s": world * km / (mms / 1e3), "kernels": kdesc}
        if prods:
            # per-stage times of the same steps; the stages the tensor cores ran
            plan.profile(True)
            for _ in range(reps):
                step(C)
            torch.cuda.synchronize()
            sm, _ = plan.stage_times(0)
            am, _ = plan.stage_times(1)
            plan.profile(False)
            tens = {(t["direction"], t["stage"]) for t in tuned if t["tensor"]} if tuned else \
                {(d, s) for d in (0, 1) for s in range(L + 2)}
            t_ms, flops, nbytes = 0.0, 0.0, 0.0
            for d, times in ((0, sm), (1, am)):
                for s in range(L + 2):
                    if (d, s) not in tens:
                        continue
                    E = stages[s]["transfer_entries"]
                    t_ms += times[s] / reps
                    flops += 2.0 * E * km  # useful: one multiply-add per stored entry and RHS
                    # stored entries once per launch, vectors (gathered in + written out) per RHS
                    nbytes += 4.0 * E + km * (stages[s]["algorithmic_bytes"] - 4.0 * E)
            tpk = tensor_peak_tflops(tdt, peaks)
            achieved = flops / (t_ms / 1e3) / 1e12 if t_ms > 0 else 0.0
            bound = min(hbm * 1e9 * flops / max(nbytes, 1.0) / 1e12, tpk / prods)
            r["stage_ms"] = {"synthesis": [round(x / reps, 5) for x in sm], "adjoint": [round(x / reps, 5) for x in am]}
            r["roofline"] = {"bound": "hbm" if hbm * 1e9 * flops / max(nbytes, 1.0) / 1e12 < tpk / prods else "tensor",
                             "kernel": "k_tcs (both directions, tensor-core stages)", "achieved": achieved,
                             "peak": bound, "unit": "TFLOP/s (useful, 2 flop per stored entry and RHS)",
                             "frac": achieved / bound if bound > 0 else 0.0,
                             "tensor_peak_tflops": tpk, "tensor_frac": achieved * prods / tpk,
                             "hbm_GBps": nbytes / (t_ms / 1e3) / 1e9 if t_ms > 0 else 0.0,
                             "hbm_frac": nbytes / (t_ms / 1e3) / 1e9 / hbm if t_ms > 0 else 0.0,
                             "kernel_ms_per_step": t_ms, "intensity_flop_per_byte": flops / max(nbytes, 1.0),
                             "peak_source": "min(MEASURED_PEAKS.json hbm_gbs x intensity, sustained "
                                            f"{'bf16' if tdt == 'bf16' else 'bf16 x 1.1/2.25 (TF32)'} tensor peak / "
                                            f"{prods} products) (of measured)"}
        multi[mode] = r
    plan.set_mode("fp32")
    for mode in ("3xtf32", "6xbf16"):
        multi[f"speedup_{mode}_vs_fp32"] = multi["fp32"]["ms_per_step"] / multi[mode]["ms_per_step"]
    if not args.no_accuracy:
        # rounding error of every FP32 form against the FP64 apply of the same factors (max over
        # RHS of the relative l2 error per RHS)
        ref = plan.clone("fp64").bind(device=dev, max_nrhs=km)
        C64 = C.double()
        r_syn = ref.synthesize_raw(C64)
        r_rt = ref.analyze_raw(r_syn, weighted=True)
        torch.cuda.synchronize()
        for mode in MODES_MULTI:
            for i, (nm, r) in enumerate((("synthesis", r_syn), ("round_trip", r_rt))):
                e = torch.linalg.norm(outs[mode][i].double() - r, dim=0) / torch.linalg.norm(r, dim=0)
                multi[mode][f"rel_err_{nm}_vs_fp64"] = float(e.max())
        ref.close()
        del ref, r_syn, r_rt, C64
        torch.cuda.empty_cache()
    return multi


def run_ours(args):
    import numpy as np
    import torch

    import workloads as W
    from paper_2605_21828_gb300.build import build_library
    build_library()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    plan, setup_s, built = get_plan(args, dist, rank)
    info = plan.info()
    K, Wm = args.steps, args.warmup
    nrhs = args.nrhs
    max_nrhs = max(nrhs, args.multi_rhs or 1)
    plan.bind(device=dev, max_nrhs=max_nrhs)
    plan.set_path(args.path)
    tune = None
    if not args.no_autotune and args.path != "fused":
        t0 = time.time()
        cfgs = plan.autotune(nrhs)
        tune = {"seconds": round(time.time() - t0, 2),
                "stages [dir, stage, tensor, rhs_tile, slot_KB, slots, CTAs/SM]": [
                    [t["direction"], t["stage"], t["tensor"], t["rhs_tile"], t["slot_kb"], t["slots"],
                     t["ctas_per_sm"]] for t in cfgs],
                "grouped_stages {dir: head, tail}": {d: [g["head"], g["tail"]] for d, g in plan.grouping.items()}}
    n, m = plan.n, plan.m
    c = torch.from_numpy(W.sphere_coefficients(m, nrhs)).float().to(dev)
    c = c[:, 0].contiguous() if nrhs == 1 else c
    stream = torch.cuda.current_stream(dev)

    def step(x):
        f = plan.synthesize_raw(x)
        return plan.analyze_raw(f, weighted=True)

    clocks = ClockSampler()
    clocks.start()
    for _ in range(max(Wm, 3)):
        step(c)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_steps")  # profilers can select these launches
    ev0.record(stream)
    for _ in range(K):
        step(c)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    # the same K steps again with CUDA events around every kernel launch (per-stage times)
    plan.profile(True)
    for _ in range(K):
        step(c)
    torch.cuda.synchronize()
    syn_ms, syn_n = plan.stage_times(0)
    adj_ms, adj_n = plan.stage_times(1)
    plan.profile(False)
    clk = clocks.stop(local)
    status = plan.check()
    ms_total = max_over_ranks(ms_total, dist, dev)
    ms_step = ms_total / K
    value = world * K * nrhs / (ms_total / 1000.0)

    # per-stage roofline: the dominant kernel is the one with the most device time
    L = plan.levels
    stages = [plan.level_info(s) for s in range(L + 2)]
    all_bytes = sum(st_["algorithmic_bytes"] for st_ in stages)
    nst = L + 2

    def fused_bytes(d):
        """Algorithmic bytes one step streams through the persistent launches of direction d: all
        stages on the fused path, else the stages grouped at both ends by the autotuner."""
        if args.path == "fused":
            return all_bytes
        g = plan.grouping.get(d, {"head": 0, "tail": 0}) if tune is not None else {"head": 0, "tail": 0}
        ks = set(range(g["head"])) | set(range(nst - g["tail"], nst)) if (g["head"] or g["tail"]) else set()
        return sum(stages[k if d == 0 else nst - 1 - k]["algorithmic_bytes"] for k in ks)
    kern = {
        "k_rowdot synthesis (transfer levels 0..L)": (
            syn_ms[:L + 1].sum(), syn_n[:L + 1].sum(),
            sum(stages[s]["algorithmic_bytes"] * syn_n[s] for s in range(L + 1))),
        "k_rowdot adjoint (transfer levels L..0)": (
            adj_ms[:L + 1].sum(), adj_n[:L + 1].sum(),
            sum(stages[s]["algorithmic_bytes"] * adj_n[s] for s in range(L + 1))),
        "k_rowdot synthesis (column bases U)": (syn_ms[L + 1], syn_n[L + 1],
                                                stages[L + 1]["algorithmic_bytes"] * syn_n[L + 1]),
        "k_rowdot adjoint (column bases U)": (adj_ms[L + 1], adj_n[L + 1],
                                              stages[L + 1]["algorithmic_bytes"] * adj_n[L + 1]),
        "k_fused synthesis (grouped stages, persistent launches)": (syn_ms[L + 2], syn_n[L + 2], K * fused_bytes(0)),
        "k_fused adjoint (grouped stages, persistent launches)": (adj_ms[L + 2], adj_n[L + 2], K * fused_bytes(1)),
    }
    name, (kms, kl, kbytes) = max(kern.items(), key=lambda kv: kv[1][0])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = (kbytes / 1e9) / (kms / 1e3) if kms > 0 else 0.0
    ratio = NCU_DRAM_PER_ALG_BYTE.get(name)
    traffic = ratio * kbytes / max(kl, 1) if ratio else None  # bytes per launch, like achieved
    step_bytes = 2 * all_bytes  # one synthesis + one adjoint (factor bytes dominate)
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else
                "fallback 6800 GB/s", "traffic": traffic, "launches": int(kl), "avg_launch_ms": kms / max(kl, 1),
                "step_algorithmic_GB": step_bytes / 1e9,
                "step_frac": (step_bytes / 1e9) / (ms_step / 1e3) / peak}
    per_stage = {"path": args.path, "launches_per_step": int((syn_n.sum() + adj_n.sum()) // K),
                 "synth_ms": [round(x / K, 5) for x in syn_ms], "adjoint_ms": [round(x / K, 5) for x in adj_ms],
                 "algorithmic_MB": [round(s["algorithmic_bytes"] / 1e6, 3) for s in stages]}

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        import ctypes as Cc

        from paper_2605_21828_gb300 import _lib
        lib = _lib.load()
        ch = torch.from_numpy(W.sphere_coefficients(m, nrhs)).float().pin_memory()
        fh = torch.empty((nrhs, n), dtype=torch.float32).pin_memory()
        ch2 = torch.empty((nrhs, m), dtype=torch.float32).pin_memory()
        chc = ch.t().contiguous().pin_memory()  # column-major m x nrhs
        s = Cc.c_void_p(stream.cuda_stream)

        def host_step():
            _lib.check(lib.mht_synthesize_host(plan._h, Cc.c_void_p(chc.data_ptr()), m, Cc.c_void_p(fh.data_ptr()),
                                               n, nrhs, s))
            _lib.check(lib.mht_analyze_host(plan._h, Cc.c_void_p(fh.data_ptr()), n, Cc.c_void_p(ch2.data_ptr()),
                                            m, nrhs, 1, s))
        for _ in range(3):
            host_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            host_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, dist, dev)
        e2e = {"value": world * K * nrhs / dt, "unit": "transforms/s",
               "h2d_bytes_per_step": (m + n) * 4 * nrhs, "d2h_bytes_per_step": (n + m) * 4 * nrhs,
               "api": "mht_synthesize_host + mht_analyze_host (pinned host buffers)"}

    # multi-RHS measurement (same step, more vectors per launch): plain FP32 SIMT products
    # against the 3xTF32 tensor-core products, with the relative difference of their results
    multi = None
    if args.multi_rhs and args.multi_rhs > 1:
        multi = multi_rhs_measure(args, plan, dev, stream, world, step, K)

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's FP64 butterfly apply of this plan on the host cores (a bounded number of
        # whole transforms), and the exact transform by direct summation on sampled rows
        F = oracle_factors(plan)
        c0 = W.sphere_coefficients(m)[:, 0]
        wv = analysis_weights(plan, args.workload)
        t_one = oracle_step(F, c0, wv)[0]
        v, meta, _ = cpu_baseline(F, c0, wv, steps=int(max(1, min(8, 12.0 / max(t_one, 1e-3)))), warmup=0)
        del F
        cb = dict(meta, value=v, unit="transforms/s")
        if args.workload in WORKLOADS:  # the sphere's Phi has a closed form to sum directly
            cb["direct_summation"] = direct_summation_sample(args.workload, budget_s=10.0)

    launches = int(syn_n.sum() + adj_n.sum())  # launches of the K profiled steps = K steps' launches
    desc = workload_desc(args.workload)
    desc.update({"nrhs": nrhs, "levels": L, "stored_entries": info["stored_entries"],
                 "factor_GB": info["factor_bytes"] / 1e9, "compression_vs_dense": n * m / info["stored_entries"],
                 "plan_setup_s": round(setup_s, 1), "plan_built_here": built, "parallelism": f"replicas x{world}"})
    line = {"metric": METRIC, "value": value,
            "unit": "transforms/s", "n_gpus": world, "steps": K, "warmup": max(Wm, 3), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": desc, "roofline": roofline, "per_stage": per_stage,
            "multi_rhs": multi, "e2e": e2e, "cpu_baseline": cb, "clocks": clk, "gpu_launches": launches,
            "autotune": tune,
            "device_status": status}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def batch_plans(args):
    """The 64 instances of the batched ragged workload.  Built four at a time (four threads each;
    the C build releases the GIL); kept as plan files only when --plan-cache names a folder."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np

    import workloads as W
    from paper_2605_21828_gb300 import Plan
    specs = W.batched_instances(64, seed=2)
    cache = args.plan_cache or ""
    if cache:
        os.makedirs(cache, exist_ok=True)
    t0 = time.time()
    threads = max(1, (os.cpu_count() or 4) // 4)

    def one(i):
        sp = specs[i]
        path = os.path.join(cache, f"inst{i:02d}.plan") if cache else ""
        if path and os.path.exists(path):
            return Plan.load(path, mode="fp32"), False
        n, m = sp["n"], sp["m"]
        kw = dict(n=n, m=m, eps=1e-6, leaf_size=64, mode="fp32", num_threads=threads)
        if sp["kind"] == "torus":
            K = W.torus_modes_lowest(m)
            p = Plan.build(eigenvalues=W.torus_eigenvalues(K), evaluator="torus", points=W.torus_points(n, seed=i),
                           torus_modes=K, weights=np.full(n, 4 * np.pi ** 2 / n), **kw)
        else:
            X = W.fibonacci_points(n, seed=i) if sp["kind"] == "sphere" else W.deformed_sphere_points(n, seed=i)
            p = Plan.build(eigenvalues=W.sphere_eigenvalues(m), evaluator="sphere", points=X,
                           weights=np.full(n, 4 * np.pi / n), **kw)
        if path:
            p.save(path)
        return p, True

    order = sorted(range(len(specs)), key=lambda i: -specs[i]["n"])  # largest first
    with ThreadPoolExecutor(4) as ex:
        done = dict(zip(order, ex.map(one, order)))
    plans = [done[i][0] for i in range(len(specs))]
    built = sum(1 for i in done if done[i][1])
    return specs, plans, time.time() - t0, built


def run_batch(args):
    """Batched ragged workload: one persistent launch per direction (CUDA graph) for all 64
    instances, against the plain FP32 per-instance apply (one mht_synthesize / mht_analyze
    per instance) on the same inputs."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2605_21828_gb300 import Batch
    from paper_2605_21828_gb300.build import build_library
    build_library()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    specs, plans, setup_s, built = batch_plans(args)
    ks = [sp["nrhs"] for sp in specs]
    total_rhs = sum(ks)
    bt = Batch(plans, ks).bind(device=dev)
    for i, p in enumerate(plans):
        C_ = W.gaussian_columns(p.m, ks[i], 100 + i, complex_=p.complex)
        bt.c[i].copy_(torch.from_numpy(C_).to(bt.c[i].dtype))
    stream = torch.cuda.current_stream(dev)
    t0 = time.time()
    tune_ms = bt.autotune() if not args.no_autotune else None
    tune_s = time.time() - t0
    for i, p in enumerate(plans):  # the autotuner overwrote the vectors
        C_ = W.gaussian_columns(p.m, ks[i], 100 + i, complex_=p.complex)
        bt.c[i].copy_(torch.from_numpy(C_).to(bt.c[i].dtype))

    def step():
        bt.synthesize()
        bt.analyze(weighted=True)

    clocks = ClockSampler()
    clocks.start()
    K, Wm = args.steps, max(args.warmup, 3)
    for _ in range(Wm):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    status = bt.check()
    # one more synthesis from the original inputs, kept for the comparison below
    cin = []
    for i, p in enumerate(plans):
        C_ = W.gaussian_columns(p.m, ks[i], 100 + i, complex_=p.complex)
        bt.c[i].copy_(torch.from_numpy(C_).to(bt.c[i].dtype))
        cin.append(bt.c[i].clone())
    f_batch = [f.clone() for f in bt.synthesize()]

    # plain FP32 per-instance apply of the same vectors (per-stage kernels, one call per instance)
    for p, k in zip(plans, ks):
        p.bind(device=dev, max_nrhs=k).set_path("staged")

    def step_plain():
        for i, p in enumerate(plans):
            f = p.synthesize_raw(cin[i])
            p.analyze_raw(f, weighted=True)

    for _ in range(Wm):
        step_plain()
    torch.cuda.synchronize()
    reps = max(3, K // 4)
    e0.record(stream)
    for _ in range(reps):
        step_plain()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1) / reps
    clk = clocks.stop(0)
    # the batch and the per-instance apply run the same row arithmetic: compare exactly
    same = all(torch.equal(p.synthesize_raw(cin[i]).reshape(f_batch[i].shape), f_batch[i])
               for i, p in enumerate(plans))

    # multi-RHS SIMT: bound by FP32 issue, not by HBM; algorithmic flops = one multiply-add per
    # stored entry and RHS (complex entries: four), both directions
    flops = sum(2 * 2 * p.info()["stored_entries"] * k * (4 if p.complex else 1) for p, k in zip(plans, ks))
    peak = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 FMA lanes x 2 flop x max SM clock, TFLOP/s
    achieved = flops / 1e12 / (ms / 1e3)
    factor_bytes = sum(2 * sum(p.level_info(s)["algorithmic_bytes"] for s in range(p.levels + 2)) for p in plans)

    # the tensor-core form: every instance's own apply (6xBF16 block products from 16 real / 8
    # complex RHS on) on forked streams, replayed from one CUDA graph; its difference from the
    # FP32 results
    bt.set_mode("6xbf16")
    for i in range(len(plans)):
        bt.c[i].copy_(cin[i])
    for _ in range(Wm):
        step()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_tc = e0.elapsed_time(e1) / K
    for i in range(len(plans)):
        bt.c[i].copy_(cin[i])
    f_tc = bt.synthesize()
    torch.cuda.synchronize()
    diff = max(float(torch.linalg.norm((f_tc[i] - f_batch[i]).to(torch.complex128 if plans[i].complex else
                                                                   torch.float64)) /
                     torch.linalg.norm(f_batch[i].to(torch.complex128 if plans[i].complex else torch.float64)))
               for i in range(len(plans)))
    status_tc = bt.check()
    bt.set_mode("fp32")
    info = bt.info()
    line = {"metric": "transforms/s (synthesis + weighted adjoint), batched ragged", "value": total_rhs / (ms / 1e3),
            "unit": "transforms/s", "n_gpus": 1, "steps": K, "warmup": Wm, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched ragged: 64 instances cycling flat torus / unit sphere / deformed sphere, "
                                   "n uniform in [2000, 40000] (seed 2), m = n/4, 1-128 RHS each, eps=1e-6, leaf 64",
                       "instances": len(plans), "total_rhs": total_rhs, "n_total": sum(sp["n"] for sp in specs),
                       "factor_GB": sum(p.info()["factor_bytes"] for p in plans) / 1e9,
                       "items_per_direction": [info["items_synthesis"], info["items_analysis"]],
                       "persistent_ctas": info["grid"], "plan_setup_s": round(setup_s, 1), "plans_built_here": built,
                       "deformed_basis": "spherical harmonics of the radial direction at deformed-sphere points",
                       "l2": "factors (GBs) > 129 MB L2"},
            "per_instance_fp32": {"ms_per_step": ms_plain, "transforms_per_s": total_rhs / (ms_plain / 1e3),
                                  "launches_per_step": 2 * sum(p.levels + 2 for p in plans),
                                  "identical_results": bool(same)},
            "speedup_vs_per_instance": ms_plain / ms,
            "tensor_core_form": {"ms_per_step": ms_tc, "transforms_per_s": total_rhs / (ms_tc / 1e3),
                                 "speedup_vs_per_instance_fp32": ms_plain / ms_tc,
                                 "max_rel_diff_synthesis_vs_fp32_form": diff, "device_status": status_tc,
                                 "kernels": "k_tcs 6xBF16 (instances with >= 16 real / 8 complex RHS) and "
                                            "k_rowdot, 8 forked streams in one CUDA graph"},
            "roofline": {"bound": "alu", "kernel": "k_batch (both directions, all instances)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                         "hbm_GBps_of_algorithmic_bytes": factor_bytes / 1e9 / (ms / 1e3),
                         "note": "one multiply-add per stored entry and RHS; the compensated sums issue about "
                                 "twice that; RHS tiles beyond the first re-read an item's rows from L2"},
            "autotune": {"seconds": round(tune_s, 2), "best_ms_both_directions": tune_ms},
            "gpu_launches": 2 * (K + Wm), "clocks": clk, "device_status": status}
    print(json.dumps(line), flush=True)


def run_torus_sweep(args):
    """Flat torus, m = ceil(n/25) lowest modes, eps in {1e-3, 1e-6}, leaf 64 (the memory-scaling
    experiment of Sec. 6.1): stored entries, compression against dense Phi, and the FP32
    single-RHS synthesis + analysis time of each plan."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2605_21828_gb300 import Plan
    from paper_2605_21828_gb300.build import build_library
    build_library()
    dev = torch.device("cuda", 0)
    sizes = [int(x) for x in os.environ.get("MHT_SWEEP_SIZES", "4096,16384,65536,262144").split(",")]
    points = []
    for eps in (1e-3, 1e-6):
        for n in sizes:
            m = -(-n // 25)
            K = W.torus_modes_lowest(m)
            t0 = time.time()
            p = Plan.build(n=n, m=m, eigenvalues=W.torus_eigenvalues(K), evaluator="torus",
                           points=W.torus_points(n), torus_modes=K, eps=eps, leaf_size=64, mode="fp32")
            build_s = time.time() - t0
            p.bind(device=dev, max_nrhs=1)
            p.autotune(1)
            c = torch.from_numpy(W.gaussian(m, 1, True)).to(torch.complex64).to(dev)
            for _ in range(3):
                p.analyze_raw(p.synthesize_raw(c), weighted=False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 50
            e0.record()
            for _ in range(reps):
                p.analyze_raw(p.synthesize_raw(c), weighted=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            info = p.info()
            alg = 2 * sum(p.level_info(s_)["algorithmic_bytes"] for s_ in range(p.levels + 2))
            points.append({"eps": eps, "n": n, "m": m, "levels": p.levels, "stored_entries": info["stored_entries"],
                           "compression_vs_dense": n * m / info["stored_entries"], "build_s": round(build_s, 1),
                           "ms_per_step": ms, "GBps_algorithmic": alg / 1e9 / (ms / 1e3)})
            p.close()
            del p
            torch.cuda.empty_cache()
    fit = {}
    for eps in (1e-3, 1e-6):
        pts = [q for q in points if q["eps"] == eps]
        if len(pts) >= 2:
            x = np.log([q["n"] for q in pts])
            fit[str(eps)] = {"stored_exponent": float(np.polyfit(x, np.log([q["stored_entries"] for q in pts]), 1)[0]),
                             "time_exponent": float(np.polyfit(x, np.log([q["ms_per_step"] for q in pts]), 1)[0])}
    print(json.dumps({"metric": "flat-torus memory law and apply time (synthesis + adjoint, complex64, 1 RHS)",
                      "unit": "ms per step", "n_gpus": 1, "data": "synthetic", "dtype": "c64",
                      "config": {"workload": "flat torus, uniform points in [-pi,pi]^2, m = ceil(n/25) lowest modes, "
                                             "leaf 64"},
                      "points": points, "loglog_fit": fit}), flush=True)


def run_peaks(args):
    """Dense GEMM rates of this GPU for the rooflines of the multi-RHS forms, measured like the
    bf16 peak beside them: torch.matmul of 8192^3 (2 N^3 flops) in each type, best of 10 (burst)
    and back to back for 4 s (sustained), CUDA events.  TF32 = float32 inputs with TF32 tensor
    cores allowed; FP32 = float32 with TF32 off (SIMT FMA); FP64 = double."""
    import torch
    dev = torch.device("cuda", 0)
    out = {}
    for name, dt, tf32, N in (("bf16", torch.bfloat16, False, 8192), ("tf32", torch.float32, True, 8192),
                              ("fp32", torch.float32, False, 8192), ("fp64", torch.float64, False, 4096)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        torch.backends.cudnn.allow_tf32 = tf32
        a = torch.randn(N, N, device=dev, dtype=dt)
        b = torch.randn(N, N, device=dev, dtype=dt)
        c = a @ b
        torch.cuda.synchronize()
        best = 1e30
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(10):
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        reps, t_end = 0, time.time() + 4.0
        e0.record()
        while time.time() < t_end:
            torch.matmul(a, b, out=c)
            reps += 1
            if reps % 8 == 0:
                torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        sus = e0.elapsed_time(e1) / reps
        out[name] = {"N": N, "tflops_burst": 2 * N ** 3 / (best / 1e3) / 1e12,
                     "tflops_sustained": 2 * N ** 3 / (sus / 1e3) / 1e12}
        del a, b, c
    torch.backends.cuda.matmul.allow_tf32 = False
    print(json.dumps({"metric": "dense GEMM peaks", "gpu": torch.cuda.get_device_name(dev), "torch": torch.__version__,
                      "how": "torch.matmul N^3 (2 N^3 flops): best of 10 (burst), back to back for 4 s (sustained)",
                      "peaks": out}), flush=True)


def replica_command(gpus, argv, port):
    """The command that starts `gpus` replicas of this script on this node, one rank per GPU."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
            "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *argv]


def free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_ranks(args):
    """Each rank reports (rank, world size, local rank) and rank 0 prints the gathered layout."""
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    me = [rank, world, int(os.environ.get("LOCAL_RANK", "0"))]
    if world > 1:
        dist.init_process_group("gloo")
        got = [None] * world
        dist.all_gather_object(got, me)
        dist.destroy_process_group()
    else:
        got = [me]
    if rank == 0:
        print(json.dumps({"workload": "ranks", "n_gpus": args.gpus, "ranks": got}), flush=True)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # no launcher: start the replicas here (the same command line on every rank)
        sys.exit(subprocess.call(replica_command(args.gpus, sys.argv[1:], free_port())))
    if args.workload == "ranks":
        run_ranks(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "torus_sweep":
        run_torus_sweep(args)
    elif args.workload == "peaks":
        run_peaks(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
