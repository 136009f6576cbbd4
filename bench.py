"""Benchmark: lattice site-updates/s of the region-scheduled evolution on one GB300.

Workload (one "step" = one pass of the whole hot path over one batch): the
128^3 matter-era string field (nu = 2, tau0 = 10, tau_ref = tau0 + 256 dt,
lambda = 2, eta = 1, dx = 1, dt = 0.25), random-phase initial field from
seed 0, evolved 256 leapfrog steps in FP32 with the Kahan-compensated drift,
region base B = 16 (8 steps per band, 32 bands, 131072 regions).  Every step
starts from the same initial state (restored on the device before the step,
outside the timed region) and L2 is flushed between steps.

Printed (rank 0, one JSON line): value = site-updates/s from CUDA events on
the library's stream around each sp_evolve call; the monolithic GPU sweep on
the same inputs; roofline of the region kernel (algorithmic bytes per
site-update x updates / kernel time from events around that kernel, against
the measured HBM copy bandwidth); e2e through the C ABI with host buffers;
the FP64 CPU oracle timed on the host cores (bounded sample); SM clocks
sampled with nvidia-smi during the timed region.

--impl reference times the FP64 CPU oracle on the same workload instead
(bounded sample per step), as the reference arm.

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the method needs no collective), value = all ranks' updates / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, STEPS, B = 128, 256, 16  # the benchmark workload (options below resize it for profiling only)
NU, TAU0, LAM, ETA, DX, DT = 2.0, 10.0, 2.0, 1.0, 1.0, 0.25
SEED = 0
# Algorithmic HBM bytes per site-update of the region path at B = 16: band-top
# state plus sloped faces, counted by brute force over one steady-state band
# (13.8 read + 11.4 written, each face cell written once, read by every
# consumer).
ALG_BYTES_PER_UPDATE = {8: 42.8, 16: 25.3, 32: 13.8}
MONO_BYTES_PER_UPDATE = 48.0
# On-chip (shared-memory) bytes per site-update of the region kernel: seven
# phi reads (8 B) and one phi write, one (pi, c) read and write (16 B each).
SMEM_BYTES_PER_UPDATE = 7 * 8 + 8 + 2 * 16
# Shared-memory bandwidth of one GB300, nominal: 128 B per clock per SM.
SMS, SMEM_BYTES_PER_CLOCK = 152, 128
WORKLOAD = (f"{N}^3 matter era (nu=2, tau0=10, tau_ref=74), lambda=2, eta=1, dx=1, dt=0.25, random-phase "
            f"init seed 0, {STEPS} leapfrog steps, region base B={B}")
METRIC = "lattice site-updates/s"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the region kernel and everything that shapes what it moves (tables, launch)
KERNEL_SOURCES = ["paper_1011_4046_gb300/csrc/sp_kernels.cu", "paper_1011_4046_gb300/csrc/sp_device.cuh",
                  "paper_1011_4046_gb300/csrc/sp_update.h", "paper_1011_4046_gb300/csrc/sp_api.cu",
                  "paper_1011_4046_gb300/csrc/planner.cpp", "paper_1011_4046_gb300/csrc/planner.h"]


def ncu_traffic(workload_is_default):
    """DRAM bytes per region-kernel launch from the committed ncu record, or
    None when the kernel sources changed since it was taken (or the workload
    differs from the one it was taken on)."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "region_kernel_traffic.json")) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for s in KERNEL_SOURCES:
            with open(os.path.join(ROOT, s), "rb") as f:
                h.update(f.read())
        if not workload_is_default or h.hexdigest()[:16] != rec["kernel_sources_sha256_16"]:
            return None
        return rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]
    except Exception:
        return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        import tempfile

        self.path = os.path.join(tempfile.gettempdir(), f"sp_bench_clocks_{os.getpid()}_{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def smem_roofline(updates, kernel_ms, clk):
    """On-chip line of the region kernel: its shared-memory bytes per launch
    over the launch time, against the nominal bandwidth at the SM clock
    sampled during the timed region (or the maximum clock)."""
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    peak = SMS * SMEM_BYTES_PER_CLOCK * mhz * 1e6 / 1e9
    achieved = SMEM_BYTES_PER_UPDATE * updates / (kernel_ms / 1e3) / 1e9
    return {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": f"nominal (152 SMs x 128 B/clock at {mhz:.0f} MHz)",
            "bytes_per_update": SMEM_BYTES_PER_UPDATE}


def trace_utilisation(trace, ctas):
    """GPU analogues of the paper's CPU utilisation and degree of parallelism
    (Sec. 6) from per-region (start, end) globaltimer stamps: the fraction of
    the persistent CTAs' time spent inside regions, and the mean number of
    regions in flight."""
    tr = np.asarray(trace, dtype=np.int64)
    start, end = tr[:, 0], tr[:, 1]
    span = float(end.max() - start.min())
    busy = float((end - start).sum())
    return {"regions": int(len(tr)), "cta_busy_fraction": busy / (ctas * span),
            "mean_regions_in_flight": busy / span, "mean_region_us": busy / len(tr) / 1e3,
            "makespan_ms": span / 1e6}


def whole_job_rate(local_ms, units_per_rank, ws, device=None):
    """Whole-job throughput of independent replicas: every rank processed
    units_per_rank units in local_ms; the job took the slowest rank's time.
    Returns (units/s over all ranks, max ms).  With ws > 1 this needs an
    initialised process group (NCCL on the GPUs, gloo on the host)."""
    t = float(local_ms)
    if ws > 1:
        import torch
        import torch.distributed as dist

        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return ws * units_per_rank / (t / 1e3), t


def flush_l2(buf):
    buf.zero_()


def run_ours(args):
    import torch

    global N, STEPS, WORKLOAD
    if args.grid != N or args.leapfrog_steps != STEPS:
        WORKLOAD = WORKLOAD.replace(f"{N}^3", f"{args.grid}^3").replace(f"{STEPS} leapfrog", f"{args.leapfrog_steps} leapfrog")
        WORKLOAD = WORKLOAD.replace("tau_ref=74", f"tau_ref={TAU0 + args.leapfrog_steps * DT:g}")
        N, STEPS = args.grid, args.leapfrog_steps

    from paper_1011_4046_gb300 import inputs, sp

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)  # a capturable stream (the sweep is replayed as a CUDA graph)
    torch.cuda.set_stream(stream)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    p = sp.make_params(N, dx=DX, dt=DT, lam=LAM, eta=ETA, nu=NU, tau0=TAU0, tau_ref=TAU0 + STEPS * DT)
    phi0, pi0, c0 = inputs.initial_state((N, N, N), SEED, "phase", eta=ETA)
    host_init = sp.pack_state(phi0, pi0, c0)                    # library state layout, 24 B/site
    init_dev = torch.from_numpy(host_init).to(dev)              # resident copy to restore from
    g = sp.Grid([p], stream=stream)
    g.plan(base_B=args.base, threads=args.threads)
    info = g.plan_info(0)
    updates = N ** 3 * STEPS
    l2_flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    init_bytes = init_dev.numel() * 8

    def restore():
        rc = sp.sp_write_surface(g.h, 0, sp.SP_SURF_STATE, init_dev.data_ptr(), init_bytes, 1)
        assert rc == 0, sp.sp_strerror(rc)

    def one_step(flags):
        restore()
        flush_l2(l2_flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = sp.sp_evolve(g.h, STEPS, sp.SP_ASYNC | sp.SP_RESTART | sp.SP_TIMING | flags)
        e1.record(stream)
        if rc != 0:
            raise sp.SpError(rc, "sp_evolve")
        e1.synchronize()
        kernel = g.timing()
        return e0.elapsed_time(e1), kernel

    # ---- region path ----
    for _ in range(args.warmup):
        one_step(0)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    t_wall0 = time.perf_counter()
    step_ms, kern_ms = [], []
    for _ in range(args.steps):
        ms, kt = one_step(0)
        step_ms.append(ms)
        kern_ms.append(kt[1])
    barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    value, total_ms = whole_job_rate(sum(step_ms), updates * args.steps, ws, dev)
    ms_per_step = total_ms / args.steps

    # correctness guard on the benchmarked result: finite field
    phi_end = g.read_state(0)[0]
    finite = bool(np.all(np.isfinite(phi_end)))

    # the paper's utilisation figures (Sec. 6), from one traced call outside the timed region
    restore()
    rc = sp.sp_evolve(g.h, STEPS, sp.SP_RESTART | sp.SP_TRACE)
    if rc != 0:
        raise sp.SpError(rc, "sp_evolve (trace)")
    utilisation = trace_utilisation(g.trace(0, int(info["regions_per_band"] * (STEPS // (info["base_B"] // 2)))),
                                    info["grid"])

    # ---- monolithic sweep on the same inputs (the comparator) ----
    for _ in range(max(1, args.warmup // 2)):
        one_step(sp.SP_MONOLITHIC)
    mono_ms = [one_step(sp.SP_MONOLITHIC)[0] for _ in range(args.steps)]
    mono_value = updates * args.steps / (sum(mono_ms) / 1e3)

    # ---- e2e through the C ABI with host buffers ----
    pinned_in = torch.from_numpy(host_init.view(np.float32).copy()).pin_memory()  # phi | (pi, c)
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    nbytes = pinned_in.numel() * 4
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        barrier()
        t0 = time.perf_counter()
        rc = sp.sp_write_surface(g.h, 0, sp.SP_SURF_STATE, pinned_in.data_ptr(), nbytes, 0)
        rc = rc or sp.sp_evolve(g.h, STEPS, sp.SP_ASYNC | sp.SP_RESTART)
        rc = rc or sp.sp_read_surface(g.h, 0, sp.SP_SURF_STATE, pinned_out.data_ptr(), nbytes, 0)
        t1 = time.perf_counter()
        if rc != 0:
            raise sp.SpError(rc, "e2e")
        if it >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_value = ws * updates * len(e2e_ms) / (sum(e2e_ms) / 1e3)
    g.close()

    if rank != 0:
        return None
    hbm, peak_kind = peaks()
    kern_mean = sum(kern_ms) / len(kern_ms)
    base = info["base_B"]
    alg_bytes = ALG_BYTES_PER_UPDATE[base] * updates
    achieved = alg_bytes / (kern_mean / 1e3) / 1e9
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "site-updates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded random-phase field)",
        "config": {"workload": WORKLOAD if base == B else WORKLOAD.replace(f"B={B}", f"B={base}"), "grid": N,
                   "leapfrog_steps": STEPS, "region_base": base,
                   "regions": int(info["regions_per_band"] * (STEPS // (base // 2))),
                   "threads_per_cta": info["threads"], "ctas": info["grid"],
                   "mailbox_slots": info["mailbox_slots"], "mailbox_bytes": info["mailbox_bytes"],
                   "l2": "flushed (512 MiB write) before every step; state restored on device outside timing",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "monolithic": {"value": mono_value, "unit": "site-updates/s", "ms_per_step": sum(mono_ms) / len(mono_ms),
                       "speedup_of_regions": value / ws / mono_value},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": peak_kind,
                     "traffic": ncu_traffic(N == 128 and STEPS == 256 and base == B and args.threads == 0),
                     "kernel": "region_kernel", "kernel_ms": kern_mean,
                     "alg_bytes_per_update": ALG_BYTES_PER_UPDATE[base],
                     "design_bytes_per_update": info["bytes_per_update"]},
        "roofline_smem": smem_roofline(updates, kern_mean, clk),
        "e2e": {"value": e2e_value, "unit": "site-updates/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes, "ms_per_step": sum(e2e_ms) / len(e2e_ms)},
        "gpu_launches": 2 * args.steps,
        "utilisation": utilisation,
        "clocks": clk,
        "wall_s_timed_region": wall,
        "field_finite": finite,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    return out


def run_batched(args):
    """The batched workload: 64 simulations, N drawn from the multiples of 8 in
    [48, 160], nu in {0, 1, 2} (seeds 0-63), 192 steps each, in one autotuned
    persistent launch replayed from a CUDA graph; the monolithic sweep of the
    same batch beside it.  One JSON line (1 GPU)."""
    import torch

    from paper_1011_4046_gb300 import inputs, sp

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    steps = 192
    params, inits = [], []
    for seed, n, nu in inputs.batched_workload(64):
        tau0 = 10.0 if nu > 0 else 1.0
        params.append(sp.make_params(n, dx=DX, dt=DT, lam=LAM, eta=ETA, nu=float(nu), tau0=tau0,
                                     tau_ref=tau0 + steps * DT))
        st = inputs.initial_state((n, n, n), seed, "phase" if nu > 0 else "gaussian", sigma=0.3)
        inits.append(torch.from_numpy(sp.pack_state(*st)).to(dev))
    updates = sum(p.n[0] * p.n[1] * p.n[2] for p in params) * steps
    g = sp.Grid(params, stream=stream)
    t0 = time.perf_counter()
    g.plan(base_B=sp.SP_AUTOTUNE, threads=sp.SP_AUTOTUNE)
    tune_s = time.perf_counter() - t0
    infos = [g.plan_info(i) for i in range(len(params))]
    l2_flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_step(flags):
        for i, buf in enumerate(inits):
            rc = sp.sp_write_surface(g.h, i, sp.SP_SURF_STATE, buf.data_ptr(), buf.numel() * 8, 1)
            assert rc == 0, sp.sp_strerror(rc)
        flush_l2(l2_flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = sp.sp_evolve(g.h, steps, sp.SP_ASYNC | sp.SP_RESTART | flags)
        e1.record(stream)
        if rc != 0:
            raise sp.SpError(rc, "sp_evolve")
        e1.synchronize()
        return e0.elapsed_time(e1)

    res = {}
    for name, flags in (("regions", 0), ("monolithic", sp.SP_MONOLITHIC)):
        for _ in range(args.warmup):
            one_step(flags)
        ms = [one_step(flags) for _ in range(args.steps)]
        res[name] = (updates * len(ms) / (sum(ms) / 1e3), sum(ms) / len(ms))
    g.close()
    bases = sorted({i["base_B"] for i in infos})
    return {"metric": METRIC, "value": res["regions"][0], "unit": "site-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["regions"][1],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded random-phase / Gaussian fields)",
            "config": {"workload": "batched: 64 simulations, N uniform over multiples of 8 in [48,160], "
                                   "nu in {0,1,2}, seeds 0-63, 192 steps each, one autotuned persistent launch "
                                   "per region base, replayed from a CUDA graph",
                       "site_updates": updates, "region_bases": bases,
                       "threads_per_cta": {str(b): next(i["threads"] for i in infos if i["base_B"] == b)
                                           for b in bases},
                       "ctas": {str(b): next(i["grid"] for i in infos if i["base_B"] == b) for b in bases},
                       "mailbox_slots": {str(b): next(i["mailbox_slots"] for i in infos if i["base_B"] == b)
                                         for b in bases},
                       "autotune_s": tune_s, "autotune_candidates": infos[0]["tune_candidates"],
                       "l2": "flushed (512 MiB write) before every step; states restored on device outside timing",
                       "parallelism": "1 GPU"},
            "monolithic": {"value": res["monolithic"][0], "unit": "site-updates/s",
                           "ms_per_step": res["monolithic"][1],
                           "speedup_of_regions": res["regions"][0] / res["monolithic"][0]},
            "gpu_launches": 2 * len(bases) * args.steps}  # per base: queue reset + region kernel


def cpu_baseline(budget_s, n_steps_cap=STEPS):
    """The FP64 oracle, as it stands, on the host cores: the same workload,
    bounded to about budget_s seconds of steps."""
    import oracle
    from paper_1011_4046_gb300 import inputs

    oracle.build()
    p = oracle.make_params(N, dx=DX, dt=DT, lam=LAM, eta=ETA, nu=NU, tau0=TAU0, tau_ref=TAU0 + STEPS * DT)
    phi0, pi0, _ = inputs.initial_state((N, N, N), SEED, "phase", eta=ETA)
    phi = phi0.astype(np.complex128)
    pi = pi0.astype(np.complex128)
    done, chunk = 0, 8  # steps per oracle call
    t0 = time.perf_counter()
    while done < n_steps_cap and (time.perf_counter() - t0) < budget_s:
        k = min(chunk, n_steps_cap - done)
        phi, pi = oracle.run(p, phi, pi, done, k)
        done += k
    el = time.perf_counter() - t0
    return {"value": N ** 3 * done / el, "unit": "site-updates/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"first {done} of {STEPS} steps of the {N}^3 workload in calls of 8 steps "
                      f"({N ** 3 * done:.3g} site-updates, {el:.1f} s, FP64, OpenMP over z-planes)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle
    from paper_1011_4046_gb300 import inputs

    oracle.build()
    p = oracle.make_params(N, dx=DX, dt=DT, lam=LAM, eta=ETA, nu=NU, tau0=TAU0, tau_ref=TAU0 + STEPS * DT)
    phi0, pi0, _ = inputs.initial_state((N, N, N), SEED, "phase", eta=ETA)
    per_step = max(1, args.ref_levels)
    times = []
    phi = phi0.astype(np.complex128)
    pi = pi0.astype(np.complex128)
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        phi, pi = oracle.run(p, phi0, pi0, 0, per_step)
        el = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(el)
    value = N ** 3 * per_step * len(times) / sum(times)
    sample = (f"each step: the first {per_step} of {STEPS} leapfrog steps of the {N}^3 workload "
              f"(FP64 oracle, OpenMP over z-planes)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random-phase field)",
            "config": {"workload": WORKLOAD, "grid": N, "leapfrog_steps": STEPS, "region_base": B},
            "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-levels", type=int, default=4, help="leapfrog steps per reference-arm step")
    ap.add_argument("--base", type=int, default=B, help="region base (the workload's is 16)")
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0 = library default)")
    ap.add_argument("--grid", type=int, default=N, help="grid side (profiling of smaller cases only)")
    ap.add_argument("--leapfrog-steps", type=int, default=STEPS, help="steps per run (profiling only)")
    ap.add_argument("--workload", default="grid", choices=["grid", "batched"],
                    help="grid: the 128^3 workload (default); batched: the 64-simulation batch")
    args = ap.parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    elif args.workload == "batched":
        out = run_batched(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
