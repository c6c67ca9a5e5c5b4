"""Benchmark of the block staircase sweep on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                    [--workload qbd_L32768_m64] [--apply inverse|coupled]

A step is one sweep of Algorithm 2 over the whole chain (both half-sweeps and
the normalisation of Eq. (2)) on the workload's synthetic generator, whose
FP64 blocks (3.2 GB for L=32768, m=64) stay resident in HBM and exceed L2, so
no L2 flush is needed between steps.  `value` is sweeps/s over all ranks
(each rank sweeps its own replica: weak scaling, no collective on the data
path).  `e2e` is the same metric through the host-buffer entry point
mc_sweep_host (H2D of x, the sweep, D2H of the new iterate, every step).
`--impl reference` times the CPU oracle on this host's cores on a bounded
sample of the same workload instead.
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

METRIC = "sweeps/s and HBM GB/s per sweep; batched solves/s and p99 at resid <=1e-10"
UNIT = "sweeps/s"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src = 6800.0, "fallback"
    if os.path.exists(p):
        with open(p) as f:
            hbm, src = float(json.load(f)["hbm_gbs"]), "measured"
    return hbm, src


# FP64 peak of a GB300: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz (maximum
# SM clock) = 1.2586 TFLOP/s.  The 2 DFMA lanes/clk/SM pipe rate is what
# ncu's FP64-pipe utilisation of the sweep kernel implies (95 % busy at
# 1.215 TFLOP/s); the independent FMA-loop probe (--measure-fp64-peak) and
# cuBLAS DGEMM are reported beside it.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def gpu_id(local):
    """nvidia-smi selector of the CUDA device `local` of this process.

    nvidia-smi numbers GPUs in its own (PCI) order and ignores
    CUDA_VISIBLE_DEVICES, so a CUDA ordinal is not an nvidia-smi index: the
    device is named by its UUID (from torch, else from a UUID entry of
    CUDA_VISIBLE_DEVICES); an index is used only when neither is known."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(local).uuid)
        if u and u != "None":
            return u if u.startswith(("GPU-", "MIG-")) else "GPU-" + u
    except Exception:
        pass
    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    if local < len(vis) and vis[local].startswith(("GPU-", "MIG-")):
        return vis[local]
    if local < len(vis) and vis[local].isdigit():
        return vis[local]
    return str(local)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 100 ms in a thread."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = str(gpu)       # nvidia-smi selector: UUID (gpu_id) or index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "gpu": self.gpu}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[4 + k].lower() == "active"})
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows), "power_w_max": max(pw) if pw else None,
                "gpu": self.gpu}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(ms, e2e_s, steps, e2e_steps, ws, device="cpu"):
    """Whole-job numbers of a multi-rank run: every rank sweeps its own replica
    (weak scaling, no collective on the data path); the timed region counts as
    long as the slowest rank.  Returns (ms_max, e2e_s_max, value, e2e_value)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms), float(e2e_s)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, e2e_s = float(t[0]), float(t[1])
    return ms, e2e_s, ws * steps / (ms * 1e-3), ws * e2e_steps / e2e_s


def oracle_sample_rate(name, seconds=15.0, max_levels=None, threads=0, oc=None):
    """CPU oracle sweeps/s on the workload (whole by default; the first
    max_levels levels scaled by the level ratio otherwise), timed for about
    `seconds` after one untimed sweep.  oc: an oracle chain of the workload
    already built (reused between calls)."""
    import numpy as np

    import oracle
    import synth

    L, m = synth.workload_shape(name)
    Ls = L if max_levels is None else min(L, max_levels)
    if oc is None:
        blocks = synth.workload(name, 0, Ls)
        oc = oracle.Chain(*blocks)
        del blocks
    cores = oracle.threads(threads)
    N = Ls * m
    x = np.full(N, 1.0 / N)
    t0 = time.perf_counter()
    x = oc.sweeps(x, 1)
    t1 = time.perf_counter() - t0
    k = max(1, int(seconds / max(t1, 1e-6)))
    t0 = time.perf_counter()
    oc.sweeps(x, k)
    t = time.perf_counter() - t0
    rate = k / t * (Ls / L)
    what = (f"all {L} levels" if Ls == L else f"the first {Ls} of {L} levels, scaled by {Ls}/{L}")
    return rate, cores, f"{k} oracle sweeps (Algorithm 2 + Eq. (2) normalisation) of {what} " \
                        f"(m={m}), {cores} threads", k, t, oc


def oracle_threads_restore():
    """Back to every host core for the oracle (after a single-thread sample)."""
    import oracle
    oracle.threads(os.cpu_count() or 1)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synth

    name = args.workload
    L, m = synth.workload_shape(name)
    # one step = one oracle sweep of the whole chain (about 30 ms on 16 cores
    # for 32768 levels of 64); chains too large for a few-minute run are
    # sampled by their first levels, scaled by the level ratio
    Ls = L if L * m * m <= 32768 * 256 * 256 else 4096
    blocks = synth.workload(name, 0, Ls)
    oc = oracle.Chain(*blocks)
    del blocks
    cores = oracle.threads(0)
    N = Ls * m
    x = np.full(N, 1.0 / N)
    for _ in range(args.warmup):
        x = oc.sweeps(x, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x = oc.sweeps(x, 1)
    t = time.perf_counter() - t0
    value = args.steps / t * (Ls / L)
    what = (f"all {L} levels" if Ls == L else f"the first {Ls} of {L} levels, sweeps/s scaled "
            f"by {Ls}/{L}")
    sample = f"each step = 1 oracle sweep of {what} (m={m}), {cores} threads"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t / args.steps / (Ls / L), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": name, "L": L, "m": m, "sample_levels": Ls},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def src_hash(sources):
    """First 16 hex digits of the SHA-256 of the named csrc files, in order."""
    import hashlib
    hs = hashlib.sha256()
    for src in sources:
        with open(os.path.join(ROOT, "paper_2302_07551_gb300", "csrc", src), "rb") as f:
            hs.update(f.read())
    return hs.hexdigest()[:16]


def run_mine(args):
    import numpy as np
    import torch

    import synth
    import paper_2302_07551_gb300 as mcl

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    name = args.workload
    L, m = synth.workload_shape(name)
    N = L * m

    # inputs: synthetic generator blocks built on the host, copied once to HBM
    t0 = time.perf_counter()
    blocks = synth.workload(name)
    banded = isinstance(blocks, dict)
    n_diags = len(blocks) if banded else 3
    if banded:
        d = {e: torch.from_numpy(b).to(dev) for e, b in blocks.items()}
    else:
        d = [torch.from_numpy(b).to(dev) for b in blocks]
    del blocks
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(dev)
    # paired pentadiagonal workloads: skip the structurally zero quadrants
    paired = synth.WORKLOADS[name]["kind"] == "penta" and args.apply == "inverse" and m % 64 == 0
    with torch.cuda.stream(stream):
        if banded:
            ch = mcl.Chain.banded(d, apply=args.apply, stream=stream, dtype=args.dtype)
        else:
            ch = mcl.Chain(*d, apply=args.apply, stream=stream, dtype=args.dtype, paired=paired)
    del d
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0

    x = torch.full((N,), 1.0 / N, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    # set-up (untimed): the library's autotuner picks the fused launches'
    # blocks per SM (and, for low-precision storage, levels per unit)
    tuning = None
    if not args.no_tune:
        bps, lpu, tms = ch.tune(x, min(64, args.steps, 1024))
        tuning = {"blocks_per_sm": bps, "levels_per_unit": lpu, "tuned_ms": tms}
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_id(local))
    sampler.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        ch.sweep(x, y, 1)
        x, y = y, x
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # timed region: K sweeps as the solve loop runs them -- chunks of
    # --check-every sweeps, each one fused launch that ends with the residual
    # of its result (formed from the splitting), the scale reduction and the
    # normalisation, then a host read of [e^T z, step, residual] (the stopping
    # test); CUDA events on the chain's stream around the whole region
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    check = max(1, args.refine_every)
    resid_checks = []
    if args.dtype == "f64":
        st = torch.zeros(3, dtype=torch.float64, device=dev)
        sth = torch.zeros(3, dtype=torch.float64).pin_memory()
        e0.record(stream)
        with torch.cuda.stream(stream):
            for done in range(0, args.steps, check):
                ch.sweep(x, x, min(check, args.steps - done), stats=st)
                sth.copy_(st, non_blocking=True)
                stream.synchronize()
                resid_checks.append(float(sth[2]))
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        # per-kernel device times of one launch of the same size (at most 1024
        # sweeps per fused launch) with its residual units
        prof_steps = min(args.steps, check, 1024)
        _, prof = ch.profile(x, y, prof_steps)
        torch.cuda.synchronize()
        x, y = y, x
    else:
        # a step = one correction sweep of mixed-precision refinement, with the
        # FP64 outer step (residual, q, update, renormalisation) every
        # --refine-every sweeps inside the timed region
        with torch.cuda.stream(stream):
            e0.record(stream)
            ch.solve(x0=x, tol=0.0, eps=0.0, maxit=args.steps, check_every=args.refine_every, pi=y)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        _, prof = ch.profile(x, y, min(args.steps, 200))
        prof_steps = min(args.steps, 200)
    if ws > 1:
        torch.distributed.barrier()
    x, y = y, x

    # end to end through host buffers (pinned): every step one mc_sweep_host
    # call, which reads x from pinned host memory and returns pi there; the
    # stats with the residual every --check-every steps, as the solve loop
    xh = torch.empty(N, dtype=torch.float64).pin_memory()
    yh = torch.empty(N, dtype=torch.float64).pin_memory()
    xh.copy_(x.cpu())
    ke = max(3, min(args.steps, 200))
    ch.sweep_host(xh, yh, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(ke):
        ch.sweep_host(xh, yh, 1, stats=(i % check == check - 1 or i == ke - 1))
        xh, yh = yh, xh
    e2e_s = time.perf_counter() - t0
    clocks = sampler.stop()
    ms, e2e_s, value, e2e_value = aggregate(ms, e2e_s, args.steps, ke, ws, device=dev)

    # algorithmic bytes and flops (FP64): per level, the stored blocks streamed
    # once (3 m^2 doubles inverse mode, 2 m^2 coupled) plus the neighbour
    # vector read once and z written once (16 m bytes); per sweep add reading
    # x and writing pi (16 N bytes) as counted for the whole step.
    nmat = 3 if args.apply == "inverse" else 2
    if banded:
        nmat = n_diags       # every off-diagonal block of Q^T plus (-T_dd)^{-1}
    tail_bytes = tail_flops = 0
    if args.dtype == "f64":
        # paired chains stream 3/4 of each off-diagonal block
        mats = (2.5 if paired else nmat)
        bytes_level = int(8 * mats * m * m) + 16 * m
        sweep_bytes = L * int(8 * mats * m * m) + 16 * N
        if not banded:
            # residual units of the last launch: T_lo and T_up of every
            # diagonal-only level (3/4 of each when paired) and z_K, z_{K-1}
            # at its two neighbours
            offd = 1.5 if paired else 2.0
            p0 = (L + 1) // 2
            tail_bytes = p0 * (int(8 * offd * m * m) + 32 * m)
            tail_flops = p0 * int(2 * offd * m * m)
    else:
        # FP32 vectors: neighbour d read, q read, d written (16 m bytes / level)
        es = 4 if args.dtype == "f32" else 2
        mat = 2 * es * m * m + (4 * m * m if args.apply == "inverse" else 0)
        bytes_level = mat + 16 * m
        sweep_bytes = L * bytes_level
    flops_level = int(2 * (2.5 if (paired and args.dtype == "f64") else nmat) * m * m)
    # dominant kernel: the fused sweep kernel (one launch runs all timed
    # sweeps or correction sweeps, up to 1024 per launch)
    fused = prof["fused"]
    sweeps_per_launch = min(prof_steps, 1024) if fused else 1
    n_launch = -(-prof_steps // sweeps_per_launch)
    # kernels of this library launched inside the timed region: per chunk the
    # fused sweeps (+ residual units), the scale reduction and the
    # normalisation; mixed precision: the start (scale check, residual with
    # q) and per refinement step the fused correction sweeps, the update, the
    # normalisation and the residual with q
    n_chunks = -(-args.steps // check)
    n_kernels = 3 * n_chunks if args.dtype == "f64" else 2 + 4 * n_chunks
    kern_ms = prof["sweeps_ms"] / n_launch
    kern_bytes = bytes_level * L * sweeps_per_launch + tail_bytes
    kern_flops = flops_level * L * sweeps_per_launch + tail_flops
    kern_ms_per_sweep = {"sweeps": prof["sweeps_ms"] / prof_steps,
                         "scale": prof["scale_ms"] / prof_steps,
                         "normalise": prof["norm_ms"] / prof_steps}
    hbm_peak, hbm_src = peaks()
    achieved_gbs = kern_bytes / (kern_ms * 1e-3) / 1e9
    achieved_tf = kern_flops / (kern_ms * 1e-3) / 1e12
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        rate, cores, sample, _, _, oc = oracle_sample_rate(name, seconds=args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        # the same oracle on one host thread (a shorter run on the same chain)
        r1, c1, s1, _, _, _ = oracle_sample_rate(name, seconds=args.cpu_seconds / 3, threads=1,
                                                 oc=oc)
        cpu["single_thread"] = {"value": r1, "unit": UNIT, "cores": c1, "sample": s1}
        del oc
        oracle_threads_restore()
    if args.dtype == "f64":
        kname = ("k_sweeps_banded" if banded else "k_sweeps") if fused else "k_phase"
        key = f"{name}:{args.apply}"
    else:
        kname = "k_sweeps_lp"
        key = f"{name}:{args.apply}:{args.dtype}"
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        with open(tp) as f:
            tk = json.load(f).get("kernels", {}).get(kname)
        # counters taken on an older kernel source do not describe this one
        if tk and key in tk["workloads"] and tk["kernel_src_sha256"] == src_hash(tk["sources"]):
            w = tk["workloads"][key]
            traffic = (w["bytes_per_sweep"] * sweeps_per_launch + w.get("tail_bytes", 0)
                       if fused else w["bytes_per_launch"])
    if args.dtype == "f64":
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved_tf / FP64_PEAK_TFLOPS,
                "traffic": traffic,
                "kernel": f"{kname} (fused: {sweeps_per_launch} sweeps + residual units per launch)",
                "peak_source": "derived: 152 SMs x 2 FP64 lanes/clk x 2 flop x 2.07 GHz; the fma-loop probe (--measure-fp64-peak) measures 1.2558 TFLOP/s = 1.996 lanes/clk/SM",
                "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                        "frac": achieved_gbs / hbm_peak, "peak_source": hbm_src}}
    else:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved_gbs / hbm_peak, "traffic": traffic,
                "kernel": f"k_sweeps_lp (fused: {sweeps_per_launch} correction sweeps per launch)",
                "peak_source": hbm_src}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.dtype == "f64" else f"{args.dtype} blocks, f32 sweeps, f64 refinement",
        "data": "synthetic (seeded QBD generator, level-dependent blocks)",
        "config": {"workload": name, "L": L, "m": m, "N": N, "apply": args.apply, "stair": 1,
                   "check_every": check if args.dtype == "f64" else None,
                   "tuning": tuning,
                   "paired_zero_quadrants_skipped": bool(paired),
                   "block_bytes": sweep_bytes - 16 * N,
                   "refine_every": args.refine_every if args.dtype != "f64" else None,
                   "l2": "no flush: the streamed blocks exceed L2 (129 MB) every step",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "gbs_per_sweep": sweep_bytes / (ms / args.steps * 1e-3) / 1e9,
        "roofline": roof,
        "kernel_ms_per_sweep": kern_ms_per_sweep,
        "residual_checks": resid_checks[-3:],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * N,
                "d2h_bytes_per_step": 8 * N + 8 * 3,
                "how": "mc_sweep_host per step: x read from pinned host memory by the "
                       "kernels, pi stored into pinned host memory by the normalisation"},
        "gpu_launches": n_kernels,
        "clocks": clocks,
        "setup_s": setup_s,
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)
    ch.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_solve(args):
    """Time to solution: one full solve of the workload to ||Q^T pi||_1 <= tol
    for FP64 and the mixed-precision forms, with the result's distance to the
    FP64 solution (the FP64 GPU path itself matches the CPU oracle to 1e-10 on
    every oracle-sized case of the test suite)."""
    import numpy as np
    import torch

    import synth
    import paper_2302_07551_gb300 as mcl

    torch.cuda.set_device(0)
    name = args.workload
    L, m = synth.workload_shape(name)
    blocks = synth.workload(name)
    d = [torch.from_numpy(b).cuda() for b in blocks]
    del blocks
    torch.cuda.synchronize()
    rows = []
    ref = None
    # paired pentadiagonal workloads: the FP64 inverse-mode form skips the
    # structurally zero quadrants (as in the throughput line)
    penta = synth.WORKLOADS[name]["kind"] == "penta" and m % 64 == 0
    for dtype in args.solve_dtypes.split(","):
        paired = penta and dtype == "f64" and args.apply == "inverse"
        ch = mcl.Chain(*d, apply=args.apply, dtype=dtype, paired=paired)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pi, res = ch.solve(tol=args.tol, maxit=10_000_000, check_every=args.refine_every)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        p = pi.cpu().numpy()
        if ref is None and dtype == "f64":
            ref = p
        rows.append({"dtype": dtype, "paired": paired, "seconds": t, "sweeps": res["sweeps"],
                     "residual": res["residual"], "converged": res["converged"],
                     "rel_l1_vs_f64": (float(np.abs(p - ref).sum() / np.abs(ref).sum())
                                       if ref is not None else None),
                     "ms_per_sweep": 1e3 * t / max(res["sweeps"], 1)})
        ch.close()
    print(json.dumps({"mode": "time_to_solution", "workload": name, "L": L, "m": m,
                      "apply": args.apply, "tol": args.tol, "refine_every": args.refine_every,
                      "results": rows}), flush=True)


def kernel_summary(trials, hbm_peak, hbm_src):
    """HBM rate of the batched fused sweep launches from the autotuner's timed
    chunks (CUDA events around the launches, algorithmic bytes of the live
    requests): over the kept configurations and over all trials."""
    if not trials:
        return None
    kept = [t for t in trials if t["chosen"]]

    def rate(ts):
        ms = sum(t["sweep_ms"] for t in ts)
        return sum(t["sweep_bytes"] for t in ts) / (ms * 1e-3) / 1e9 if ms > 0 else None

    best = max(t["sweep_bytes"] / (t["sweep_ms"] * 1e-3) / 1e9 for t in trials if t["sweep_ms"] > 0)
    kg = rate(kept)
    return {"kept_gbs": kg, "kept_frac": kg / hbm_peak if kg else None,
            "all_trials_gbs": rate(trials), "best_trial_gbs": best,
            "best_trial_frac": best / hbm_peak, "peak_gbs": hbm_peak, "peak_source": hbm_src,
            "n_trials": len(trials), "n_signatures": len({t["signature"] for t in trials})}


def run_serve(args):
    """Continuous-batching serving on the seeded request stream (first K
    requests): closed-loop capacity, then Poisson arrivals at --load x that
    capacity; solves/s and p50/p99 latency per form."""
    import numpy as np
    import torch

    import synth
    import paper_2302_07551_gb300 as mcl

    torch.cuda.set_device(0)
    reqs = synth.request_stream(args.requests)
    t0 = time.perf_counter()
    blocks = [synth.qbd(r["L"], r["m"], r["ratio"], r["seed"], True) for r in reqs]
    gen_s = time.perf_counter() - t0
    budget = int(args.budget_gb * (1 << 30))
    # batched forms separate the gains of precision (BF16 vs FP64 blocks),
    # coupling (W = (-T_dd)^{-1} T_lo, ... vs the explicit inverse) and
    # packing (all requests in shared launches vs one request at a time)
    forms = {
        "batched_bf16_coupled": dict(dtype="bf16", apply="coupled", max_active=1024, autotune=True),
        "batched_bf16_inverse": dict(dtype="bf16", apply="inverse", max_active=1024, autotune=True),
        "batched_f64_coupled": dict(dtype="f64", apply="coupled", max_active=1024, autotune=True),
        "fp64_one_at_a_time": dict(dtype="f64", apply="inverse", max_active=1, autotune=False),
    }
    hbm_peak, hbm_src = peaks()
    out = {"mode": "serve", "requests": args.requests, "tol": args.serve_tol,
           "budget_gb": args.budget_gb, "load": args.load, "check_every": args.refine_every,
           "stream": "first %d of the seeded stream (L log-uniform [128,16384], m in "
                     "{16,32,64,128}, ratio U(0.5,0.95))" % args.requests,
           "host_generation_s": gen_s, "forms": {}}
    for name, f in forms.items():
        if args.serve_forms and name not in args.serve_forms.split(","):
            continue
        srv = mcl.Server(budget, dtype=f["dtype"], apply=f["apply"], tol=args.serve_tol,
                         check_every=args.refine_every, max_active=f["max_active"],
                         autotune=f["autotune"])

        def drive(arrivals):
            """Submit request i once time >= arrivals[i] (and it fits); step
            until all finish.  Returns per-request (arrival, finish, sweeps)."""
            start = time.perf_counter()
            nxt, done, fin = 0, 0, {}
            queue = []
            while done < len(reqs):
                now = time.perf_counter() - start
                while nxt < len(reqs) and arrivals[nxt] <= now:
                    queue.append(nxt)
                    nxt += 1
                while queue and srv.submit(queue[0], *blocks[queue[0]]):
                    queue.pop(0)
                na, _ = srv.step()
                while True:
                    r = srv.fetch()
                    if r is None:
                        break
                    tag, _, res, st = r
                    fin[tag] = (time.perf_counter() - start, res["sweeps"], st, res["residual"])
                    done += 1
                if na == 0 and not queue and nxt < len(reqs):
                    time.sleep(max(0.0, min(arrivals[nxt] - (time.perf_counter() - start), 0.05)))
            return fin

        fin = drive([0.0] * len(reqs))                 # closed loop: capacity
        t_cap = max(v[0] for v in fin.values())
        cap = len(reqs) / t_cap
        trials = srv.trials()
        lam = args.load * cap
        gaps = np.array([r["gap"] for r in reqs]) / lam
        arr = np.cumsum(gaps) - gaps[0]
        fin = drive(list(arr))
        lat = np.array([fin[i][0] - arr[i] for i in range(len(reqs))])
        span = max(v[0] for v in fin.values()) - arr[0]
        out["forms"][name] = {
            "dtype": f["dtype"], "apply": f["apply"], "capacity_solves_s": cap,
            "arrival_rate": lam, "solves_s": len(reqs) / span,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_s": float(lat.max()), "sweeps_total": int(sum(v[1] for v in fin.values())),
            "all_converged": all(v[2] == 0 for v in fin.values()),
            "max_residual": float(np.nanmax([v[3] for v in fin.values()])),
            "grid": srv.grid(),
            "batched_kernel": kernel_summary(trials, hbm_peak, hbm_src),
            "tuner_trials": trials,
            "per_request": [[i, reqs[i]["L"], reqs[i]["m"], round(reqs[i]["ratio"], 3),
                             fin[i][1], fin[i][3], round(float(lat[i]), 4), fin[i][2]]
                            for i in range(len(reqs))]}
        srv.close()
    print(json.dumps(out), flush=True)


def run_contraction(args):
    """Observed contraction factor (step_k / step_{k-w})^(1/w), w = the check
    window, of the stair splittings of type 1 and 2, block Gauss-Seidel (one
    wavefront-ordered fused launch per window) and block Jacobi on one
    workload from the uniform start, recorded every --segment sweeps up to
    --steps (block Jacobi: --bj-steps) so that the approach to the asymptotic
    rate is visible, with the GPU sweeps/s of each (Sect. 2: on
    block-tridiagonal Q^T the staircase and block Gauss-Seidel share their
    spectrum; block Jacobi has the eigenvalue -1 and does not converge)."""
    import torch

    import synth
    import paper_2302_07551_gb300 as mcl

    torch.cuda.set_device(0)
    name = args.workload
    L, m = synth.workload_shape(name)
    blocks = synth.workload(name)
    d = [torch.from_numpy(b).cuda() for b in blocks]
    del blocks
    torch.cuda.synchronize()
    N = L * m
    rows = {}
    w = min(args.refine_every, 1024)
    # --warm-start S: every splitting starts from the type-1 stair iterate after
    # S sweeps from uniform, so that all are timed over the same late window
    x_start = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    if args.warm_start > 0:
        ch = mcl.Chain(*d, stair=1)
        x_start, _ = ch.solve(tol=0.0, eps=0.0, maxit=args.warm_start,
                              check_every=min(w, args.warm_start), raise_on_maxit=False)
        torch.cuda.synchronize()
        ch.close()
    for stair, label, nsw in ((1, "stair1", args.steps), (2, "stair2", args.steps),
                              (4, "block_gauss_seidel", args.steps),
                              (3, "block_jacobi", args.bj_steps)):
        ch = mcl.Chain(*d, stair=stair)
        x = x_start.clone()
        pi = torch.empty_like(x)
        torch.cuda.synchronize()
        traj, done, t = [], 0, 0.0
        while done < nsw:
            seg = min(args.segment, nsw - done)
            t0 = time.perf_counter()
            _, res = ch.solve(x0=x, tol=0.0, eps=0.0, maxit=seg, check_every=min(w, seg), pi=pi,
                              raise_on_maxit=False)
            torch.cuda.synchronize()
            t += time.perf_counter() - t0
            done += seg
            x, pi = pi, x
            traj.append([done, res["contraction"], res["step"], res["residual"]])
        rows[label] = {"sweeps": done, "contraction": traj[-1][1], "step": traj[-1][2],
                       "residual": traj[-1][3], "sweeps_s": done / t,
                       "trajectory": traj}
        ch.close()
    print(json.dumps({"mode": "contraction", "workload": name, "L": L, "m": m,
                      "window": w, "segment": args.segment, "warm_start": args.warm_start,
                      "results": rows}), flush=True)


def run_batch_classes(args):
    """Batched correction sweeps by block size: for m = 128, 64, 32, 16 the
    single-chain fused launch (mc_tune's choice) and the solve server's
    batched launch on requests of that size alone (the autotuner's trials),
    then on a four-size mix; HBM rate of the sweep launches against the
    measured copy rate."""
    import torch

    import synth
    import paper_2302_07551_gb300 as mcl

    torch.cuda.set_device(0)
    dtype = args.dtype if args.dtype != "f64" else "bf16"
    apply = args.apply
    hbm_peak, hbm_src = peaks()
    e = 2 if dtype == "bf16" else 4

    def level_bytes(m):
        return 2 * e * m * m + (0 if apply == "coupled" else 4 * m * m) + 16 * m

    def single(L, m):
        b = synth.qbd(L, m, 0.9, seed=7, level_dependent=True)
        ch = mcl.Chain(*(torch.from_numpy(x).cuda() for x in b), dtype=dtype, apply=apply)
        del b
        N = L * m
        x = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
        bps, lpu, ms = ch.tune(x, 64)
        ch.close()
        gbs = level_bytes(m) * L * 64 / ms / 1e6
        return dict(L=L, m=m, blocks_per_sm=bps, levels_per_unit=lpu, ms_per_64_sweeps=ms,
                    gbs=gbs, frac=gbs / hbm_peak)

    def server(mix):
        srv = mcl.Server(48 << 30, dtype=dtype, apply=apply, tol=1e-30, check_every=64,
                         maxit=10 ** 9)
        for i, (L, m) in enumerate(mix):
            assert srv.submit(i, *synth.qbd(L, m, 0.85, seed=100 + i, level_dependent=True))
        for _ in range(14):      # the autotuner's trials, then kept-configuration chunks
            srv.step()
        tr = srv.trials()
        srv.close()
        rows = [dict(blocks_per_sm=t["blocks_per_sm"], levels_per_unit=t["levels_per_unit"],
                     split64=t["split64"], deep=t["deep"], chosen=t["chosen"],
                     sweep_ms=t["sweep_ms"], gbs=t["sweep_bytes"] / t["sweep_ms"] / 1e6)
                for t in tr]
        best = max(rows, key=lambda r: r["gbs"])
        return dict(mix=[list(x) for x in mix], best_gbs=best["gbs"],
                    best_frac=best["gbs"] / hbm_peak, trials=rows)

    out = {"mode": "batch_classes", "dtype": dtype, "apply": apply,
           "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src, "single": {}, "batched": {}}
    for L, m in ((16384, 128), (32768, 64), (32768, 32), (32768, 16)):
        out["single"]["m%d" % m] = single(L, m)
    for name, mix in (("m128", [(4096, 128)] * 8), ("m64", [(8192, 64)] * 8),
                      ("m32", [(8192, 32)] * 16), ("m16", [(8192, 16)] * 16),
                      ("mix", [(4096, 128)] * 4 + [(8192, 64)] * 4 + [(8192, 32)] * 4
                       + [(8192, 16)] * 4)):
        out["batched"][name] = server(mix)
    print(json.dumps(out), flush=True)


def run_host_transfer(args):
    """Where the end-to-end step's time goes: per call, a one-sweep device call
    with its sync, the host-buffer call (x read in place from pinned memory by
    the kernels, pi stored into pinned memory by the normalisation), the same
    step through the copy engine (16 MB H2D, device sweep, 16 MB D2H), the
    device sweep followed by the D2H copy, and each 16 MB copy alone."""
    import torch

    import synth
    import paper_2302_07551_gb300 as mcl

    torch.cuda.set_device(0)
    blocks = synth.workload(args.workload)
    d = [torch.from_numpy(b).cuda() for b in blocks]
    del blocks
    ch = mcl.Chain(*d)
    del d
    N = ch.N
    xd = torch.full((N,), 1.0 / N, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    xh = torch.empty(N, dtype=torch.float64).pin_memory()
    xh.copy_(xd.cpu())
    yh = torch.empty(N, dtype=torch.float64).pin_memory()
    s = ch.stream
    out = {}

    def run(name, f, n=60):
        for _ in range(5):
            f()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            f()
        torch.cuda.synchronize()
        out[name] = 1e3 * (time.perf_counter() - t0) / n

    def on(fn):
        def g():
            with torch.cuda.stream(s):
                fn()
            s.synchronize()
        return g

    run("device_sweep_ms", on(lambda: ch.sweep(xd, yd, 1)))
    run("host_buffer_sweep_ms", lambda: ch.sweep_host(xh, yh, 1, stats=False))
    run("copy_engine_h2d_sweep_d2h_ms", on(lambda: (xd.copy_(xh, non_blocking=True),
                                                   ch.sweep(xd, yd, 1),
                                                   yh.copy_(yd, non_blocking=True))))
    run("device_sweep_then_d2h_ms", on(lambda: (ch.sweep(xd, yd, 1),
                                               yh.copy_(yd, non_blocking=True))))
    run("h2d_copy_ms", on(lambda: xd.copy_(xh, non_blocking=True)))
    run("d2h_copy_ms", on(lambda: yh.copy_(yd, non_blocking=True)))
    mb = 8 * N / 1e6
    out["bytes_each_way"] = 8 * N
    out["h2d_gbs"] = mb / out["h2d_copy_ms"]
    out["d2h_gbs"] = mb / out["d2h_copy_ms"]
    # the link's rate on copies long enough that the per-call sync does not count
    big = 1 << 27
    bh = torch.empty(big, dtype=torch.float64).pin_memory()
    bd = torch.empty(big, dtype=torch.float64, device="cuda")
    run("h2d_copy_1GiB_ms", on(lambda: bd.copy_(bh, non_blocking=True)), n=10)
    run("d2h_copy_1GiB_ms", on(lambda: bh.copy_(bd, non_blocking=True)), n=10)
    out["h2d_1GiB_gbs"] = 8 * big / 1e6 / out["h2d_copy_1GiB_ms"]
    out["d2h_1GiB_gbs"] = 8 * big / 1e6 / out["d2h_copy_1GiB_ms"]
    print(json.dumps({"mode": "host_transfer", "workload": args.workload, "results": out}),
          flush=True)
    ch.close()


def measure_fp64_peak():
    """FP64 multiply-add peak of this GPU: the probe library's fma loop
    (libmcprobe.so: 8, 16 or 32 independent chains per thread, unrolled 4x,
    1-8 blocks of 128-1024 threads per SM, best of the grid shapes) and cuBLAS
    DGEMM 8192^3 (best of 10), with the SM clock sampled meanwhile; the per-SM
    rate follows from the loop's TFLOP/s, the SM count and the median SM
    clock."""
    import ctypes

    import torch

    from paper_2302_07551_gb300 import build as pbuild
    torch.cuda.set_device(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if not os.path.exists(pbuild.PROBE_LIB):
        raise RuntimeError(f"{pbuild.PROBE_LIB} not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(pbuild.PROBE_LIB)
    lib.mcprobe_fp64_rate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double)]
    lib.mcprobe_fp64_rate.restype = ctypes.c_int
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    loop = []
    sampler = ClockSampler(gpu_id(0))
    sampler.start()
    for chains in (8, 16, 32):
        for reg in (1, 0):
            for per_sm in (1, 2, 4, 8):
                for threads in (128, 256, 512, 1024):
                    v = ctypes.c_double(0.0)
                    iters = (1 << 18) // chains
                    rc = lib.mcprobe_fp64_rate(stream, per_sm * sms, threads, iters, chains, reg,
                                               ctypes.byref(v))
                    if rc == 1:        # block too large for this variant's registers
                        continue
                    if rc != 0:
                        raise RuntimeError(f"mcprobe_fp64_rate failed ({rc})")
                    loop.append({"chains": chains, "blocks": per_sm * sms, "threads": threads,
                                 "reg_operands": reg, "tflops": v.value})
    loop_clocks = sampler.stop()
    best = max(loop, key=lambda r: r["tflops"])
    best_loop = best["tflops"]
    mhz = loop_clocks.get("sm_mhz") or 0.0
    n = 8192
    a = torch.rand(n, n, dtype=torch.float64, device="cuda")
    b = torch.rand(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_id(0))
    sampler.start()
    dgemm = 0.0
    for _ in range(10):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        c = a @ b
        e1.record()
        torch.cuda.synchronize()
        dgemm = max(dgemm, 2 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    clocks = sampler.stop()
    per_sm_clk = best_loop * 1e12 / (2 * sms * mhz * 1e6) if mhz else None
    print(json.dumps({"fp64_fma_loop_tflops": best_loop, "best_shape": best,
                      "fma_loop_clocks": loop_clocks, "sms": sms,
                      "dfma_lanes_per_clk_per_sm": per_sm_clk,
                      "fp64_dgemm_tflops": dgemm, "n": n, "clocks": clocks,
                      "fma_loop_grid": loop}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="qbd_L32768_m64")
    ap.add_argument("--apply", default="inverse", choices=["inverse", "coupled"])
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16"])
    ap.add_argument("--refine-every", "--check-every", dest="refine_every", type=int, default=64,
                    help="sweeps per residual check (FP64) / correction sweeps per refinement step")
    ap.add_argument("--solve", action="store_true",
                    help="time one full solve to --tol per dtype instead of sweeps")
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--solve-dtypes", default="f64,f32,bf16",
                    help="comma list of storage types for --solve (f64 first for the distances)")
    ap.add_argument("--serve", action="store_true", help="serving benchmark on the request stream")
    ap.add_argument("--contraction", action="store_true",
                    help="contraction factors of stair / block Jacobi / block Gauss-Seidel")
    ap.add_argument("--bj-steps", type=int, default=20000)
    ap.add_argument("--warm-start", type=int, default=0,
                    help="contraction mode: start every splitting from the type-1 stair iterate "
                         "after this many sweeps from uniform")
    ap.add_argument("--segment", type=int, default=16384,
                    help="contraction mode: sweeps between recorded contraction factors")
    ap.add_argument("--requests", type=int, default=16)
    ap.add_argument("--serve-tol", type=float, default=1e-10)
    ap.add_argument("--serve-forms", default="",
                    help="comma list of forms to run (batched_bf16_coupled, batched_bf16_inverse, "
                         "batched_f64_coupled, fp64_one_at_a_time); default all")
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch configuration (skip mc_tune at set-up)")
    ap.add_argument("--measure-fp64-peak", action="store_true")
    ap.add_argument("--host-transfer", action="store_true",
                    help="time the parts of the end-to-end (host-buffer) step")
    ap.add_argument("--batch-classes", action="store_true",
                    help="low-precision sweep rate by block size, single chain and batched")
    args = ap.parse_args()
    if args.measure_fp64_peak:
        measure_fp64_peak()
        return
    if args.host_transfer:
        run_host_transfer(args)
        return
    if args.batch_classes:
        run_batch_classes(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.solve:
        run_solve(args)
    elif args.serve:
        run_serve(args)
    elif args.contraction:
        run_contraction(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
