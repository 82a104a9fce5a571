"""Benchmark: ACR setup + preconditioned Krylov solve to relative residual 1e-8.

Workload (default): the nonsymmetric convection-diffusion operator
-Lap u + beta . grad u at n = 128 (2,097,152 unknowns), beta =
(50,50,50)(1 + 0.5 sin 2 pi x sin 2 pi y), first-order upwind, f ~ U(-1,1)
(seed 20); ACR with eps = 1e-2, eta = 2, leaf 64, factors in FP32 (the mixed
form: FP64 leaf inverses, recompression cores and Krylov); FP64
GMRES(30), right-preconditioned, rtol 1e-8.

One step = acr_setup (coefficients already on the device) + acr_krylov_solve
+ acr_destroy.  `value` is seconds per solve for the whole job: with N
replicas (one process per GPU, independent solves), value = step time / N.

The JSON line also carries: the FP64 plain form (--fp64-steps, default 1),
an end-to-end measurement through the public API with host buffers, the
roofline of the dominant setup kernel (from one extra profiled step), the
apply's HBM roofline, and the CPU oracle timed on a bounded sample.

--impl reference times the CPU oracle instead (the only reference this
method has), each step one bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ACR setup+Krylov s to rel-res 1e-8 at n=128; mixed vs FP64 plain, same GB300"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def load_peaks():
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


# FP32 CUDA-core peak of the part: SMs (queried) x 128 FP32 lanes x 2 flop/FMA
def fp32_alu_peak_tflops(mhz, sms=152):
    return sms * 128 * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle arm
def oracle_sample(n_sample=32):
    """Oracle ACR setup + GMRES(30) on the n_sample instance of the workload.

    Returns (seconds, iterations)."""
    import numpy as np
    from inputs import workload
    from oracle.assembly import stencil_codi, stencil_matrix, plane_blocks
    from oracle.cr import cr_setup, cr_apply
    from oracle.hstructure import Structure
    from oracle.krylov import gmres
    spec, beta, f = workload("codi_n128", n=n_sample)
    t0 = time.perf_counter()
    st = stencil_codi(beta, n_sample)
    A = stencil_matrix(st, n_sample)
    D, Ld, Ud = plane_blocks(st, n_sample)
    F = cr_setup(D, Ld, Ud, Structure(n_sample, 2.0, spec["leaf"]), spec["eps"])
    u, it, hist = gmres(lambda v: A @ v, f, lambda v: cr_apply(F, v), rtol=spec["rtol"],
                        restart=spec["restart"])
    dt = time.perf_counter() - t0
    assert hist[-1] <= spec["rtol"] * 1.0001
    return dt, it


def oracle_scale():
    """Scale an n=32 oracle time to the n=128 workload.  The oracle keeps
    every plane block as a dense n^2 x n^2 array, so its setup costs
    O(n planes x (n^2)^3) = O(n^7); the factor (128/32)^7 is applied."""
    return (128.0 / 32.0) ** 7


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "grouped_gemm_dram_codi_n64.md")
# the grouped-GEMM family's sources: its kernels and the device helpers they inline
GEMM_SOURCES = [os.path.join(ROOT, "paper_1712_08872_gb300", "csrc", f)
                for f in ("acr_gemm_kernels.cu", "acr_gemm_tc.cu", "acr_device.h", "acr_tc.h")]


def gemm_source_sha():
    """SHA-256 over the grouped-GEMM family's source files, in order."""
    import hashlib
    h = hashlib.sha256()
    for f in GEMM_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def gemm_traffic_per_flop():
    """DRAM bytes per algorithmic flop of the grouped-GEMM kernels, from the
    committed ncu summary, or None when the kernel source has changed since
    those counters were taken."""
    try:
        txt = open(TRAFFIC_FILE).read()
        sha = gemm_source_sha()
    except OSError:
        return None, "no capture"
    bpf = rec = None
    for ln in txt.splitlines():
        ln = ln.strip()
        if ln.startswith("bytes_per_flop:"):
            bpf = float(ln.split(":")[1])
        elif ln.startswith("source_sha256:"):
            rec = ln.split(":")[1].strip()
    if bpf is None or rec != sha:
        return None, "kernel changed since the capture"
    return bpf, "profiles/grouped_gemm_dram_codi_n64.md, scaled by flops per launch"


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest of every rank's value (the job's time is its slowest
    replica's); the value itself on one process."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def seconds_per_solve(step_ms, world):
    """Whole-job time per solve: `world` independent replicas each finish one
    solve per step of step_ms (the max over ranks)."""
    return step_ms / 1000.0 / world


def cpu_cores():
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return os.cpu_count()


SAMPLE_DESC = ("full oracle ACR setup + GMRES(30) to 1e-8 on the n=32 instance of the same "
               "recipe (beta field, eps 1e-2, eta 2, leaf 64, seed 20), scaled to n=128 by "
               "the oracle's O(n^7) dense-plane cost, (128/32)^7")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    times = []
    for i in range(args.warmup + args.steps):
        dt, it = oracle_sample()
        if i >= args.warmup:
            times.append(dt)
    t = sum(times) / len(times)
    value = t * oracle_scale()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1000.0, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "codi_n128_acr_gmres30", "n": 128, "eps": 1e-2, "eta": 2.0,
                       "leaf": 64, "sample": "n=32 oracle solve per step",
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": SAMPLE_DESC, "sample_seconds": t},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def profile_setup(args):
    """One setup of the benchmark recipe at --n with CUDA events around every
    setup launch; prints the time and device-counted flops per kernel class,
    per GEMM stage and per CR level.  Used for the ncu captures under
    profiles/ (a small n keeps a capture short)."""
    import torch
    import paper_1712_08872_gb300 as acr
    from inputs import workload
    dev = torch.device("cuda", 0)
    acr.load_library()
    n = args.n
    spec, beta, _ = workload("codi_n128", n=n)
    coef = torch.empty(7 * n ** 3, dtype=torch.float64, device=dev)
    acr.acr_stencil_codi(n, torch.tensor(beta.ravel(), dtype=torch.float64, device=dev), coef)
    prec = acr.ACR_FP64 if args.fp64 else acr.ACR_FP32
    stream = torch.cuda.current_stream()
    table = None
    if args.gemm_table:
        table = [int(v) for v in args.gemm_table.split(",")] + [0] * 16
        table = table[:16]
    elif args.tuned:
        table, *shape_ms = acr.acr_autotune_gemm(n, coef, spec["eps"], 2.0, spec["leaf"], prec,
                                                 args.rank_cap, stream)
        for v, ms in enumerate(shape_ms):
            print("  shape %d stage ms:" % v, [round(x, 1) for x in ms[:13]])
    if table is not None:
        print("kernel shapes per stage:", ",".join(str(v) for v in table[:13]))
    h = acr.acr_setup(n, coef, spec["eps"], 2.0, spec["leaf"], prec, args.rank_cap, stream,
                      acr.ACR_FLAG_PROFILE, table)
    p = acr.acr_get_profile(h)
    inf = acr.acr_get_setup_info(h)
    acr.acr_destroy(h)
    print("n=%d %s setup %.1f ms (host issue %.1f ms), levels %d, max rank %d, factors %.3f GB"
          % (n, "FP64" if args.fp64 else "FP32", inf.setup_ms, inf.host_issue_ms, inf.levels,
             inf.max_rank, inf.factor_bytes / 1e9))
    for k in ("gemm", "orth", "eig", "leaf_inv", "other"):
        st = getattr(p, k)
        print("  %-9s launches %7d  %9.1f ms  %8.3f TFLOP/s  %.4f GFLOP"
              % (k, st.launches, st.ms, st.flops / max(st.ms, 1e-9) / 1e9, st.flops / 1e9))
    for i, nm in enumerate(p.STAGES):
        print("    %-14s %9.1f ms  %10.3f GFLOP  %8.3f TFLOP/s"
              % (nm, p.stage_ms[i], p.stage_flops[i] / 1e9,
                 p.stage_flops[i] / max(p.stage_ms[i], 1e-9) / 1e9))
    print("  leaf inverses by the FP64 fallback: %d" % inf.leaf_fp64_fallbacks)
    print("  inversion ms per level", [round(x, 1) for x in p.inv_ms[:inf.levels + 1]])
    print("  update ms per level   ", [round(x, 1) for x in p.upd_ms[:inf.levels]])
    return 0


def profile_apply(args):
    """One setup of the benchmark recipe at --n (FP32 factors) and three
    applies of --nrhs right-hand sides at once (32: the tensor-core path;
    1: the single-vector path); prints the CUDA-event time per apply.  Used
    for the ncu captures of the apply kernels."""
    import torch
    import paper_1712_08872_gb300 as acr
    from inputs import workload
    dev = torch.device("cuda", 0)
    acr.load_library()
    n = args.n
    spec, beta, f = workload("codi_n128", n=n)
    coef = torch.empty(7 * n ** 3, dtype=torch.float64, device=dev)
    acr.acr_stencil_codi(n, torch.tensor(beta.ravel(), dtype=torch.float64, device=dev), coef)
    stream = torch.cuda.current_stream()
    h = acr.acr_setup(n, coef, spec["eps"], 2.0, spec["leaf"], acr.ACR_FP32, args.rank_cap, stream)
    nr = args.nrhs
    R = torch.tensor(f, dtype=torch.float64, device=dev).repeat(nr)
    Z = torch.empty_like(R)
    acr.acr_apply(h, R, Z, nr, stream)
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(3):
        acr.acr_apply(h, R, Z, nr, stream)
    eb.record(stream)
    torch.cuda.synchronize()
    info = acr.acr_get_setup_info(h)
    acr.acr_destroy(h)
    ms = ea.elapsed_time(eb) / 3
    print("n=%d %d-vector apply %.3f ms (%.4f ms per vector), factor bytes per pass %.3f GB, "
          "%.0f GB/s" % (n, nr, ms, ms / nr, info.apply_bytes / 1e9,
                         info.apply_bytes / (ms / 1000.0) / 1e9))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="acr", choices=["acr", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--bf16-steps", type=int, default=3)
    ap.add_argument("--no-gemm-autotune", action="store_true",
                    help="default GEMM kernel shapes instead of the autotuned table")
    ap.add_argument("--no-config1", action="store_true",
                    help="skip the n=64 high-contrast boxes comparison of the three forms")
    ap.add_argument("--no-mixed-batch", action="store_true",
                    help="skip the 12-instance mixed batch under a captured graph")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the multi-right-hand-side measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rank-cap", type=int, default=24)
    ap.add_argument("--profile-apply", "--profile-apply32", dest="profile_apply",
                    action="store_true",
                    help="one setup at --n and three applies of --nrhs vectors, timed")
    ap.add_argument("--nrhs", type=int, default=32,
                    help="with --profile-apply: right-hand sides per apply (1, 8 or 32)")
    ap.add_argument("--profile-setup", action="store_true",
                    help="run one profiled setup (ACR_FLAG_PROFILE) at --n and print its "
                         "per-class, per-stage and per-level times; no benchmark line")
    ap.add_argument("--fp64", action="store_true", help="with --profile-setup: FP64 factors")
    ap.add_argument("--tuned", action="store_true",
                    help="with --profile-setup: GEMM kernel shapes from acr_autotune_gemm")
    ap.add_argument("--gemm-table", default="",
                    help="with --profile-setup: GEMM kernel shape per stage, comma-separated")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_setup:
        return profile_setup(args)
    if args.profile_apply:
        return profile_apply(args)

    import numpy as np
    import torch
    import paper_1712_08872_gb300 as acr
    from inputs import workload

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    acr.load_library()

    n = args.n
    spec, beta, f = workload("codi_n128", n=n)
    eps, eta, leaf = spec["eps"], 2.0, spec["leaf"]
    rtol, restart = spec["rtol"], spec["restart"]
    N = n ** 3
    beta_d = torch.tensor(beta.ravel(), dtype=torch.float64, device=dev)
    f_d = torch.tensor(f, dtype=torch.float64, device=dev)
    coef = torch.empty(7 * N, dtype=torch.float64, device=dev)
    acr.acr_stencil_codi(n, beta_d, coef)
    u = torch.zeros(N, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    # GEMM kernel shapes per setup stage, tuned once on this operator (outside
    # the timed region) for the float forms
    tune = None
    table = None
    if not args.no_gemm_autotune:
        try:
            table, *shape_ms = acr.acr_autotune_gemm(n, coef, eps, eta, leaf, acr.ACR_FP32,
                                                     args.rank_cap, stream)
            tune = {"table": table[:13]}
            for v, ms in enumerate(shape_ms):
                tune["stage_ms_shape%d" % v] = [round(x, 1) for x in ms[:13]]
        except acr.AcrError as e:   # the default shapes still give a valid step
            table = None
            tune = {"error": str(e)}

    def step(prec, flags=0):
        var = table if prec != acr.ACR_FP64 else None
        h = acr.acr_setup(n, coef, eps, eta, leaf, prec, args.rank_cap, stream, flags, var)
        u.zero_()
        info, st = acr.acr_krylov_solve(h, coef, acr.ACR_GMRES, restart, rtol, 1000, f_d, u,
                                        stream, check=False)
        sinfo = acr.acr_get_setup_info(h)
        prof = acr.acr_get_profile(h) if flags else None
        acr.acr_destroy(h)
        if st != 0:
            raise RuntimeError("solve failed: " + acr.acr_status_string(st))
        return info, sinfo, prof

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(prec, steps):
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = acr.acr_launch_count()
        e0.record(stream)
        infos = [step(prec) for _ in range(steps)]
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / steps
        launches = (acr.acr_launch_count() - l0) // steps
        ms = max_over_ranks(ms, dist, dev)
        return ms, infos, launches

    # warm-up (mixed form)
    for _ in range(args.warmup):
        step(acr.ACR_FP32)
    with ClockSampler(local) as clk:
        ms, infos, launches = timed(acr.ACR_FP32, args.steps)
    clocks = clk.summary()
    solve_info, setup_info, _ = infos[-1]

    # FP64 plain form on the same GPU
    fp64 = None
    if args.fp64_steps > 0:
        step(acr.ACR_FP64)                       # warm-up
        ms64, inf64, _ = timed(acr.ACR_FP64, args.fp64_steps)
        fp64 = {"s": ms64 / 1000.0, "iterations": inf64[-1][0].iterations,
                "setup_ms": inf64[-1][1].setup_ms, "max_rank": inf64[-1][1].max_rank,
                "factor_gb": inf64[-1][1].factor_bytes / 1e9}

    # BF16-stored factors (setup as FP32, factors rounded to bfloat16)
    bf16 = None
    if args.bf16_steps > 0:
        step(acr.ACR_BF16)                       # warm-up
        msb, infb, _ = timed(acr.ACR_BF16, args.bf16_steps)
        bf16 = {"s": msb / 1000.0, "iterations": infb[-1][0].iterations,
                "rel_residual": infb[-1][0].rel_residual, "setup_ms": infb[-1][1].setup_ms,
                "factor_gb": infb[-1][1].factor_bytes / 1e9}

    # end to end through the public API: pinned host inputs -> device,
    # assembly, setup, solve, solution -> host
    e2e = None
    if args.e2e_steps > 0:
        beta_h = torch.tensor(beta.ravel(), dtype=torch.float64).pin_memory()
        f_h = torch.tensor(f, dtype=torch.float64).pin_memory()
        u_h = torch.empty(N, dtype=torch.float64).pin_memory()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for it in range(args.e2e_steps + 1):     # the first pass is a warm-up
            if it == 1:
                e0.record(stream)
            bd = beta_h.to(dev, non_blocking=True)
            fd = f_h.to(dev, non_blocking=True)
            cf = torch.empty(7 * N, dtype=torch.float64, device=dev)
            acr.acr_stencil_codi(n, bd, cf)
            h = acr.acr_setup(n, cf, eps, eta, leaf, acr.ACR_FP32, args.rank_cap, stream, 0,
                              table)
            uu = torch.zeros(N, dtype=torch.float64, device=dev)
            acr.acr_krylov_solve(h, cf, acr.ACR_GMRES, restart, rtol, 1000, fd, uu, stream)
            acr.acr_destroy(h)
            u_h.copy_(uu, non_blocking=True)
        e1.record(stream)
        barrier()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.e2e_steps, dist, dev)
        e2e = {"value": seconds_per_solve(e2e_ms, world), "unit": "s",
               "h2d_bytes_per_step": 4 * N * 8,
               "d2h_bytes_per_step": N * 8}

    # roofline: one extra profiled step (CUDA events around every setup launch)
    _, _, prof = step(acr.ACR_FP32, acr.ACR_FLAG_PROFILE)
    peaks, peak_src = load_peaks()
    stats = {k: getattr(prof, k) for k in ("gemm", "orth", "eig", "leaf_inv", "other")}
    dom = max(stats, key=lambda k: stats[k].ms)
    mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    ds = stats[dom]
    if dom == "gemm":
        achieved = ds.flops / (ds.ms / 1000.0) / 1e12
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0), sms)
        bpf, tsrc = gemm_traffic_per_flop()
        traffic = bpf * ds.flops / ds.launches if (bpf is not None and ds.launches) else None
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                "traffic_source": tsrc, "kernel": "k_ggemm/k_gdot<float> (grouped GEMM family)",
                "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 x max SM clock" % sms,
                "launches": ds.launches, "ms_total": ds.ms}
    else:
        achieved = ds.flops / (ds.ms / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": None, "unit": "TFLOP/s",
                "frac": None, "traffic": None, "kernel": dom, "launches": ds.launches,
                "ms_total": ds.ms}
    roof["setup_breakdown_ms"] = {k: round(v.ms, 1) for k, v in stats.items()}
    roof["gemm_stage_ms"] = {nm: round(prof.stage_ms[i], 1) for i, nm in enumerate(prof.STAGES)}
    roof["gemm_stage_tflops"] = {nm: round(prof.stage_flops[i] / max(prof.stage_ms[i], 1e-9) / 1e9, 3)
                                 for i, nm in enumerate(prof.STAGES)}

    # apply (hot loop of the solve): HBM roofline
    def apply_roofline(prec):
        h = acr.acr_setup(n, coef, eps, eta, leaf, prec, args.rank_cap, stream)
        z = torch.empty_like(f_d)
        for _ in range(3):
            acr.acr_apply(h, f_d, z, 1, stream)
        torch.cuda.synchronize()
        ea = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(10):
            acr.acr_apply(h, f_d, z, 1, stream)
        eb.record(stream)
        torch.cuda.synchronize()
        apply_ms = ea.elapsed_time(eb) / 10
        ainfo = acr.acr_get_setup_info(h)
        acr.acr_destroy(h)
        apply_gbs = ainfo.apply_bytes / (apply_ms / 1000.0) / 1e9
        return {"bound": "hbm", "achieved": apply_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": apply_gbs / peaks["hbm_gbs"], "ms": apply_ms,
                "bytes_per_apply": ainfo.apply_bytes, "peak_source": peak_src}

    apply_roof = apply_roofline(acr.ACR_FP32)
    if args.bf16_steps > 0:
        apply_roof["bf16"] = apply_roofline(acr.ACR_BF16)

    # batching: the multi-RHS apply at the benchmark size (factors streamed
    # once per group of 8 right-hand sides), and the indefinite Helmholtz
    # recipe's 32 right-hand sides solved in lockstep vs one at a time
    batch = None
    if not args.no_batch:
        h = acr.acr_setup(n, coef, eps, eta, leaf, acr.ACR_FP32, args.rank_cap, stream)
        nr = 8
        Rm = f_d.repeat(nr)
        Zm = torch.empty_like(Rm)
        for _ in range(2):
            acr.acr_apply(h, Rm, Zm, nr, stream)
        torch.cuda.synchronize()
        ea = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        for _ in range(5):
            acr.acr_apply(h, Rm, Zm, nr, stream)
        eb.record(stream)
        torch.cuda.synchronize()
        multi_ms = ea.elapsed_time(eb) / 5
        acr.acr_destroy(h)
        hs, sig, Fh = workload("helmholtz_n64")
        nh, nrh = hs["n"], Fh.shape[0]
        Nh = nh ** 3
        ch = torch.empty(7 * Nh, dtype=torch.float64, device=dev)
        acr.acr_stencil_helmholtz(nh, torch.tensor(sig, dtype=torch.float64, device=dev), ch)
        Fd = torch.tensor(Fh.ravel(), dtype=torch.float64, device=dev)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hh = acr.acr_setup(nh, ch, hs["eps"], hs["eta"], hs["leaf"], acr.ACR_FP32, 48, stream)
        e1.record(stream)
        Ub = torch.zeros(nrh * Nh, dtype=torch.float64, device=dev)
        ib, sb = acr.acr_krylov_solve(hh, ch, acr.ACR_GMRES, hs["restart"], hs["rtol"], 500, Fd,
                                      Ub, stream, check=False, nrhs=nrh)
        e2.record(stream)
        Us = torch.zeros(nrh * Nh, dtype=torch.float64, device=dev)
        its_seq = 0
        for k in range(nrh):
            ik, _ = acr.acr_krylov_solve(hh, ch, acr.ACR_GMRES, hs["restart"], hs["rtol"], 500,
                                         Fd[k * Nh:(k + 1) * Nh], Us[k * Nh:(k + 1) * Nh],
                                         stream, check=False)
            its_seq = max(its_seq, ik.iterations)
        e3.record(stream)
        torch.cuda.synchronize()
        acr.acr_destroy(hh)
        batch = {"apply_8rhs_ms": multi_ms, "apply_ms_per_rhs_of_8": multi_ms / nr,
                 "apply_single_ms": apply_roof["ms"],
                 "helmholtz": {"workload": "helmholtz_n64 (8-layer medium, 10 points per "
                                           "wavelength, eps 1e-5, FP32 factors)",
                               "nrhs": nrh, "setup_s": e0.elapsed_time(e1) / 1000.0,
                               "lockstep_solve_s": e1.elapsed_time(e2) / 1000.0,
                               "lockstep_iterations": ib.iterations,
                               "lockstep_converged": bool(ib.converged),
                               "max_rel_residual": ib.rel_residual,
                               "one_at_a_time_solve_s": e2.elapsed_time(e3) / 1000.0,
                               "one_at_a_time_max_iterations": its_seq}}

    # config 1: high-contrast boxes at n = 64, the three forms, PCG to 1e-8
    config1 = None
    if not args.no_config1:
        cs, kap, fb = workload("poisson_boxes_n64")
        nb = cs["n"]
        cb = torch.empty(7 * nb ** 3, dtype=torch.float64, device=dev)
        acr.acr_stencil_poisson(nb, torch.tensor(kap, dtype=torch.float64, device=dev), cb)
        fbd = torch.tensor(fb, dtype=torch.float64, device=dev)
        config1 = {"workload": "poisson_boxes_n64 (40 boxes kappa 1e4, eps 1e-2, leaf 64, "
                               "PCG to 1e-8, maxit 1000)"}
        for name, prec in (("fp64", acr.ACR_FP64), ("fp32", acr.ACR_FP32), ("bf16", acr.ACR_BF16)):
            res = None
            for rep in range(2):                 # warm-up, then the timed run
                barrier()
                ea, eb, ec = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                ea.record(stream)
                hb = acr.acr_setup(nb, cb, cs["eps"], 2.0, cs["leaf"], prec, args.rank_cap, stream)
                eb.record(stream)
                ub = torch.zeros(nb ** 3, dtype=torch.float64, device=dev)
                ib, sb = acr.acr_krylov_solve(hb, cb, acr.ACR_PCG, 0, cs["rtol"], 1000, fbd, ub,
                                              stream, check=False)
                ec.record(stream)
                torch.cuda.synchronize()
                acr.acr_destroy(hb)
                res = {"s": ea.elapsed_time(ec) / 1000.0, "setup_s": ea.elapsed_time(eb) / 1000.0,
                       "solve_s": eb.elapsed_time(ec) / 1000.0, "iterations": ib.iterations,
                       "converged": bool(ib.converged), "rel_residual": ib.rel_residual}
            config1[name] = res

    # config 3 (second half): 12 kappa-Poisson instances at n in {32, 48, 64}
    # in one batch; the setup + apply of all 12 captured in a CUDA graph
    mixed = None
    if not args.no_mixed_batch:
        from inputs import gaussian_field_kappa, uniform_rhs
        ns = [32, 48, 64] * 4
        cfs = []
        for i, nn in enumerate(ns):
            c = torch.empty(7 * nn ** 3, dtype=torch.float64, device=dev)
            acr.acr_stencil_poisson(nn, torch.tensor(gaussian_field_kappa(nn, 40 + i),
                                                     dtype=torch.float64, device=dev), c)
            cfs.append(c)
        rb = torch.tensor(np.concatenate([uniform_rhs(nn, 100 + i) for i, nn in enumerate(ns)]),
                          dtype=torch.float64, device=dev)
        zb = torch.empty_like(rb)
        gs = torch.cuda.Stream(device=dev)
        barrier()
        t0 = time.perf_counter()
        bt = acr.acr_batch_create(ns, cfs, 1e-2, 2.0, 64, acr.ACR_FP32, args.rank_cap, gs)
        create_s = time.perf_counter() - t0
        acr.acr_batch_capture(bt, rb, zb, gs)
        acr.acr_batch_replay(bt, gs)             # warm-up
        acr.acr_batch_status(bt, gs)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        ea.record(gs)
        for _ in range(reps):
            acr.acr_batch_replay(bt, gs)
        eb.record(gs)
        acr.acr_batch_status(bt, gs)
        graph_ms = ea.elapsed_time(eb) / reps
        acr.acr_batch_destroy(bt)
        # the same 12 problems as separate handles (setup + one apply each)
        barrier()
        ea.record(stream)
        o = 0
        for i, nn in enumerate(ns):
            hs_ = acr.acr_setup(nn, cfs[i], 1e-2, 2.0, 64, acr.ACR_FP32, args.rank_cap, stream)
            acr.acr_apply(hs_, rb[o:o + nn ** 3], zb[o:o + nn ** 3], 1, stream)
            acr.acr_destroy(hs_)
            o += nn ** 3
        eb.record(stream)
        torch.cuda.synchronize()
        mixed = {"workload": "12 kappa-Poisson instances (Gaussian field, seeds 40-51), "
                             "n = 32, 48, 64 x 4, FP32, eps 1e-2, leaf 64",
                 "create_s": create_s, "graph_setup_apply_s": graph_ms / 1000.0,
                 "separate_handles_setup_apply_s": ea.elapsed_time(eb) / 1000.0}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        dt, it = oracle_sample()
        # the GPU on the very same sample (n = 32 instance of the recipe),
        # measured in this run: the like-for-like comparison
        sp, sb_, sf = workload("codi_n128", n=32)
        c32 = torch.empty(7 * 32 ** 3, dtype=torch.float64, device=dev)
        acr.acr_stencil_codi(32, torch.tensor(sb_.ravel(), dtype=torch.float64, device=dev), c32)
        f32d = torch.tensor(sf, dtype=torch.float64, device=dev)
        gpu32 = []
        for rep in range(4):
            barrier()
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            h32 = acr.acr_setup(32, c32, eps, eta, leaf, acr.ACR_FP32, args.rank_cap, stream)
            u32 = torch.zeros(32 ** 3, dtype=torch.float64, device=dev)
            acr.acr_krylov_solve(h32, c32, acr.ACR_GMRES, restart, rtol, 1000, f32d, u32, stream)
            acr.acr_destroy(h32)
            eb.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                gpu32.append(ea.elapsed_time(eb) / 1000.0)
        g32 = statistics.median(gpu32)
        cpu = {"value": dt * oracle_scale(), "unit": "s", "cores": cpu_cores(), "kind": "oracle",
               "sample": SAMPLE_DESC, "sample_seconds": dt,
               "same_sample": {"n": 32, "oracle_s": dt, "gpu_fp32_s": g32,
                               "oracle_over_gpu": dt / g32}}

    value = seconds_per_solve(ms, world)
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "codi_n128_acr_gmres30", "n": n, "unknowns": N, "eps": eps,
                       "eta": eta, "leaf": leaf, "rank_cap": args.rank_cap,
                       "form": "FP32 factors; FP64 leaf inverses, cores and GMRES",
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (factors tens of GB)"},
            "iterations": solve_info.iterations, "rel_residual": solve_info.rel_residual,
            "setup_s": setup_info.setup_ms / 1000.0,
            "setup_host_issue_s": setup_info.host_issue_ms / 1000.0,
            "leaf_fp64_fallbacks": setup_info.leaf_fp64_fallbacks,
            "solve_s": solve_info.solve_ms / 1000.0,
            "max_rank": setup_info.max_rank, "factor_gb": setup_info.factor_bytes / 1e9,
            "fp64_plain": fp64, "bf16_factors": bf16,
            "speedup_vs_fp64": (fp64["s"] / (ms / 1000.0)) if fp64 else None,
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
            "roofline": roof, "apply_roofline": apply_roof, "batching": batch,
            "config1_boxes_n64": config1, "mixed_batch": mixed, "gemm_autotune": tune,
            "cpu_baseline": cpu}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
