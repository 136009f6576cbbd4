"""Benchmark: lattice site-updates/s of the region-scheduled evolution on one GB300.

Workload (the largest single-GPU configuration): the 1280^3 matter-era string
field (nu = 2, tau0 = 10, tau_ref = tau0 + 2048 dt, lambda = 2, eta = 1,
dx = 1, dt = 0.25), random-phase initial field from seed 0, 2048 leapfrog
steps in FP32 with the Kahan-compensated drift, evolved as the paper's
lattice of 4-cube regions (edge 16: 4096 site-updates over 16 levels per
region, the state read and written in place).  One bench "step" is one pass of
the whole hot path over a slice of that run: one sp_evolve call of 128
leapfrog steps (ticket reset, persistent lattice kernel), continuing from
where the previous step stopped; when a pass reaches level 2048 the initial
field is restored (outside the timed region) and the run starts over.  Every
call of the run has the same regions, so the rate over any slice is the rate
of the whole run.  The state (50 GB) is far larger than L2, so no flush is
needed.  --shape split measures the split tiling (base 16, 64-step calls of
whole bands, mailboxes) instead.

Printed (rank 0, one JSON line): value = site-updates/s from CUDA events on
the library's stream around each sp_evolve call; the monolithic GPU sweep on
the same field (its own grid, after the region grid is freed); the roofline
of the region kernel (algorithmic bytes per site-update x updates / kernel
time from events around that kernel, against the measured HBM copy
bandwidth); e2e through the C ABI with the state in host memory (copied in
and out inside the timed region); the FP64 CPU oracle timed on the host cores
on a bounded sample; SM clocks sampled with nvidia-smi during the timed
region; and, as an extra key, the 128^3 x 256 L2-resident workload.

--impl reference times the FP64 CPU oracle on the same workload's bounded
sample instead, as the reference arm.  --workload batched runs the
64-simulation batch.

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the method needs no collective), value = all ranks' updates / max time.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NU, TAU0, LAM, ETA, DX, DT = 2.0, 10.0, 2.0, 1.0, 1.0, 0.25
SEED = 0
# The workloads: grid side, leapfrog steps of the whole run, steps per bench
# step (one sp_evolve call), region base.
# Default region geometry: the paper's 4-cube lattice (edge B = 4s = 16), one
# bench step = one 128-step call (each call pays once for the layers its first
# and last levels cut).  --shape split: the split tiling at base 16, 64-step
# calls (whole bands).
BIG = dict(N=1280, STEPS=2048, PER_STEP=128, B=16, SHAPE="lattice")
SMALL = dict(N=128, STEPS=256, PER_STEP=256, B=16, SHAPE="lattice")
SPLIT_PER_STEP = 64
# Sample of the big workload that the FP64 oracle times on the host cores: the
# first SAMPLE_Z planes of its initial field as a periodic slab.
SAMPLE_Z = 32
# Algorithmic HBM bytes per site-update of the region path, by region base:
# band-top state plus sloped faces, counted by brute force over one
# steady-state band (each face cell written once, read by every consumer).
ALG_BYTES_PER_UPDATE = {8: 42.8, 16: 25.3, 32: 13.8}
MONO_BYTES_PER_UPDATE = 48.0
# On-chip (shared-memory) bytes per site-update of the region kernel: seven
# phi reads (8 B) and one phi write, one (pi, c) read and write (16 B each).
SMEM_BYTES_PER_UPDATE = 7 * 8 + 8 + 2 * 16
# the lattice kernel also reads its cell entry (4 B) and row record (8 B)
SMEM_BYTES_PER_UPDATE_LATTICE = SMEM_BYTES_PER_UPDATE + 4 + 8
# Shared-memory bandwidth of one GB300, nominal: 128 B per clock per SM (the
# fallback when the measured peak is not available).
SMS, SMEM_BYTES_PER_CLOCK = 152, 128
# FP32 flops of one site update (the Laplacian sums, force, kick and
# Kahan-compensated drift of both components; a fused multiply-add counts 2).
FLOP_PER_UPDATE = 41
METRIC = "lattice site-updates/s"


def workload_name(w):
    n, steps = w["N"], w["STEPS"]
    regions = (f"4-cube lattice regions of edge B={w['B']}" if w.get("SHAPE") == "lattice"
               else f"region base B={w['B']}")
    return (f"{n}^3 matter era (nu=2, tau0=10, tau_ref={TAU0 + steps * DT:g}), lambda=2, eta=1, dx=1, dt=0.25, "
            f"random-phase init seed 0, {steps} leapfrog steps, {regions}")


def lattice_layers(B, steps):
    """Layers of lattice regions a call of `steps` levels meets (lattice.h)."""
    return (steps - 1) // (B // 4) + 4


def shape_const(shape):
    from paper_1011_4046_gb300 import sp

    return sp.SP_SHAPE_LATTICE if shape == "lattice" else sp.SP_SHAPE_SPLIT


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the region kernels and everything that shapes what they move (tables, launch)
KERNEL_SOURCES = {
    "split": ["paper_1011_4046_gb300/csrc/sp_kernels.cu", "paper_1011_4046_gb300/csrc/sp_device.cuh",
              "paper_1011_4046_gb300/csrc/sp_update.h", "paper_1011_4046_gb300/csrc/sp_api.cu",
              "paper_1011_4046_gb300/csrc/planner.cpp", "paper_1011_4046_gb300/csrc/planner.h",
              "paper_1011_4046_gb300/csrc/sp_region_common.cuh"],
    "lattice": ["paper_1011_4046_gb300/csrc/sp_lattice.cu", "paper_1011_4046_gb300/csrc/sp_device.cuh",
                "paper_1011_4046_gb300/csrc/sp_update.h", "paper_1011_4046_gb300/csrc/sp_api.cu",
                "paper_1011_4046_gb300/csrc/lattice.cpp", "paper_1011_4046_gb300/csrc/lattice.h"],
}
TRAFFIC_RECORD = {"split": "region_kernel_traffic.json", "lattice": "lattice_kernel_traffic.json"}


def kernel_sources_hash(shape):
    import hashlib

    h = hashlib.sha256()
    for s in KERNEL_SOURCES[shape]:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(base, updates_per_launch, shape="split"):
    """DRAM bytes (read + written) per region-kernel launch, from the committed
    ncu record of that kernel: its bytes per site-update, measured on a
    smaller grid of the same kernel and base whose state (and mailboxes) are
    far larger than L2, times the site-updates of this launch.  None when the
    kernel sources changed since the record was taken or the base differs."""
    try:
        with open(os.path.join(ROOT, "profiles", TRAFFIC_RECORD[shape])) as f:
            rec = json.load(f)
        if kernel_sources_hash(shape) != rec["kernel_sources_sha256_16"] or int(rec["region_base"]) != int(base):
            return None
        per_update = (rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]) / rec["site_updates"]
        return per_update * updates_per_launch
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
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
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
        return parse_clocks(open(self.path).read().splitlines())


def parse_clocks(lines):
    """Median SM clock, maximum clock and the throttle reasons seen, from
    nvidia-smi csv lines (the FIELDS order, no header, no units)."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
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
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


def smem_roofline(updates, kernel_ms, clk, measured_gbs=None, bytes_per_update=SMEM_BYTES_PER_UPDATE):
    """On-chip line of the region kernel: its shared-memory bytes per launch
    over the launch time, against the device's measured shared-memory read
    bandwidth (sp_measure_peaks) when given, else the nominal bandwidth at the
    SM clock sampled during the timed region (or the maximum clock)."""
    achieved = bytes_per_update * updates / (kernel_ms / 1e3) / 1e9
    if measured_gbs:
        peak, kind = measured_gbs, "measured (sp_measure_peaks: conflict-free 16-byte shared-memory reads, all SMs)"
    else:
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        peak = SMS * SMEM_BYTES_PER_CLOCK * mhz * 1e6 / 1e9
        kind = f"nominal (152 SMs x 128 B/clock at {mhz:.0f} MHz)"
    return {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": kind, "bytes_per_update": bytes_per_update}


def alu_roofline(updates, kernel_ms, measured_tflops):
    """FP32 line of the region kernel: FLOP_PER_UPDATE flops per site-update
    (fused multiply-adds counted as two) over the launch time, against the
    measured FP32 FMA throughput."""
    achieved = FLOP_PER_UPDATE * updates / (kernel_ms / 1e3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": measured_tflops, "unit": "TFLOP/s",
            "frac": achieved / measured_tflops, "peak_kind": "measured (sp_measure_peaks: FP32 FMA chains)",
            "flop_per_update": FLOP_PER_UPDATE}


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


def pass_schedule(n_calls, per_step, run_steps):
    """Start level of each of n_calls consecutive bench steps of per_step
    leapfrog steps over a run of run_steps: the run continues from call to
    call and starts over at level 0 when a pass is complete (a restore)."""
    out, lvl = [], 0
    for _ in range(n_calls):
        if lvl + per_step > run_steps:
            lvl = 0
        out.append(lvl)
        lvl += per_step
    return out


def host_available_bytes():
    try:
        return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        return 0


def fill_random_phase(phi, n, seed, slab=16):
    """The random-phase field into the device tensor phi (nz, ny, nx), made on
    the host slab by slab (the same values as the whole-field generator)."""
    import torch

    from paper_1011_4046_gb300 import inputs

    workers = max(1, min(16, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as pool:
        jobs = {pool.submit(inputs.random_phase_slab, n, seed, z, min(z + slab, n[2])): z
                for z in range(0, n[2], slab)}
        for fut in cf.as_completed(jobs):
            z = jobs[fut]
            s = torch.from_numpy(fut.result())
            phi[z:z + s.shape[0]].copy_(s, non_blocking=False)


def setup_dist():
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def run_grid(args, w, extra=None):
    """The region path, the sweep and e2e on one grid workload ``w``."""
    import torch

    from paper_1011_4046_gb300 import sp

    ws, rank, local = dist_env()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    N, STEPS, PER, B = w["N"], w["STEPS"], w["PER_STEP"], w["B"]
    peaks_onchip = sp.sp_measure_peaks(stream.cuda_stream)
    n = (N, N, N)
    sites = N ** 3
    p = sp.make_params(N, dx=DX, dt=DT, lam=LAM, eta=ETA, nu=NU, tau0=TAU0, tau_ref=TAU0 + STEPS * DT)
    shape = (N, N, N)
    phi = torch.empty(shape, dtype=torch.complex64, device=dev)
    pic = torch.zeros(shape + (2,), dtype=torch.complex64, device=dev)
    t0 = time.perf_counter()
    fill_random_phase(phi, n, SEED)
    phi0 = phi.clone()  # pi = c = 0 at the start: phi alone restores the initial state
    init_s = time.perf_counter() - t0
    updates = sites * PER

    def restore(g):
        phi.copy_(phi0)
        pic.zero_()
        g.set_level(0, 0)

    shape = w.get("SHAPE", "split")
    lattice = shape == "lattice"
    # the e2e leg's host copy of the state, allocated (pinned) before the other
    # legs: allocated just before the leg, late in a long run, its copies
    # measured about half as fast (0.40 / 0.78 s against 0.26 / 0.39 s for
    # the 50 GB in / out at 1280^3)
    # (every rank of the node holds one: pinned only with room for all of them
    # and two more, and no e2e leg without room for them all)
    e2e_host = None
    e2e_nbytes = 24 * sites
    local_ranks = int(os.environ.get("LOCAL_WORLD_SIZE", "1"))
    e2e_room = host_available_bytes()
    e2e_skip = None
    if not args.no_e2e and e2e_room < (local_ranks + 1) * e2e_nbytes:
        e2e_skip = (f"host memory: {e2e_room / 1e9:.0f} GB available for {local_ranks} rank(s) of "
                    f"{e2e_nbytes / 1e9:.0f} GB state each")
    if not args.no_e2e and e2e_skip is None:
        e2e_pinned = e2e_room > (local_ranks + 2) * e2e_nbytes
        e2e_host = torch.empty(e2e_nbytes // 4, dtype=torch.float32, pin_memory=e2e_pinned)
    g = sp.Grid([p], states=[(phi, pic)], stream=stream)
    g.plan(base_B=B if args.base == 0 else args.base, threads=args.threads, shape=shape_const(shape))
    info = g.plan_info(0)
    base = info["base_B"]
    regions_per_call = int(info["regions_per_band"] * (lattice_layers(base, PER) if lattice else PER // (base // 2)))
    if lattice:
        c_upd, c_rd, c_wr = sp.sp_lattice_call_bytes(base, PER)
        alg_bytes = (c_rd + c_wr) / c_upd
    else:
        alg_bytes = ALG_BYTES_PER_UPDATE[base]
    calls = args.warmup + args.steps
    sched = pass_schedule(calls, PER, STEPS)

    def one_step(start_level):
        if start_level == 0 and g.level(0) != 0:
            restore(g)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = sp.sp_evolve(g.h, PER, sp.SP_ASYNC | sp.SP_TIMING)
        e1.record(stream)
        if rc != 0:
            raise sp.SpError(rc, "sp_evolve")
        e1.synchronize()
        return e0.elapsed_time(e1), g.timing()[1]

    for lvl in sched[:args.warmup]:
        one_step(lvl)
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    t_wall0 = time.perf_counter()
    step_ms, kern_ms = [], []
    for lvl in sched[args.warmup:]:
        ms, kt = one_step(lvl)
        step_ms.append(ms)
        kern_ms.append(kt)
    barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    value, total_ms = whole_job_rate(sum(step_ms), updates * args.steps, ws, dev)
    finite = bool(torch.isfinite(torch.view_as_real(phi)).all().item())
    end_level = g.level(0)

    # the paper's utilisation figures (Sec. 6), from one traced call outside the timed region
    utilisation = None
    if not args.no_trace:
        if end_level + PER > STEPS:
            restore(g)
        rc = sp.sp_evolve(g.h, PER, sp.SP_TRACE)
        if rc != 0:
            raise sp.SpError(rc, "sp_evolve (trace)")
        utilisation = trace_utilisation(g.trace(0, regions_per_call), info["grid"])

    # ---- e2e through the C ABI: state in host memory, copied in and out every step ----
    e2e = None if e2e_skip is None else {"unavailable": e2e_skip}
    if e2e_host is not None:
        nbytes = e2e_nbytes
        if g.level(0) + PER * (args.e2e_steps + 1) > STEPS:
            restore(g)
        pinned, host = e2e_pinned, e2e_host
        rc = sp.sp_read_surface(g.h, 0, sp.SP_SURF_STATE, host.data_ptr(), nbytes, 0)
        if rc != 0:
            raise sp.SpError(rc, "sp_read_surface")
        e2e_ms = []
        for it in range(1 + args.e2e_steps):
            barrier()
            t0 = time.perf_counter()
            rc = sp.sp_write_surface(g.h, 0, sp.SP_SURF_STATE, host.data_ptr(), nbytes, 0)
            rc = rc or sp.sp_evolve(g.h, PER, sp.SP_ASYNC)
            rc = rc or sp.sp_read_surface(g.h, 0, sp.SP_SURF_STATE, host.data_ptr(), nbytes, 0)
            t1 = time.perf_counter()
            if rc != 0:
                raise sp.SpError(rc, "e2e")
            if it:
                e2e_ms.append((t1 - t0) * 1e3)
        del host, e2e_host
        e2e = {"value": ws * updates * len(e2e_ms) / (sum(e2e_ms) / 1e3), "unit": "site-updates/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": sum(e2e_ms) / len(e2e_ms), "steps": len(e2e_ms),
               "host_buffer": "pinned" if pinned else "pageable",
               "how": "per step: sp_write_surface (host -> device), sp_evolve, sp_read_surface (device -> host), "
                      "host wall clock"}
    g.close()

    # ---- monolithic sweep on the same field (its own grid, after the mailboxes are freed) ----
    mono = None
    if args.mono_steps > 0:
        restore_level = 0
        phi.copy_(phi0)
        pic.zero_()
        gm = sp.Grid([p], states=[(phi, pic)], stream=stream)
        try:
            gm.set_level(0, restore_level)
            ms = []
            for it in range(1 + args.mono_steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rc = sp.sp_evolve(gm.h, PER, sp.SP_ASYNC | sp.SP_MONOLITHIC)
                e1.record(stream)
                if rc != 0:
                    raise sp.SpError(rc, "sp_evolve (sweep)")
                e1.synchronize()
                if it:
                    ms.append(e0.elapsed_time(e1))
        finally:
            gm.close()
        mv = updates * len(ms) / (sum(ms) / 1e3)
        mono = {"value": mv, "unit": "site-updates/s", "ms_per_step": sum(ms) / len(ms), "steps": len(ms),
                "speedup_of_regions": value / ws / mv,
                "roofline_frac": MONO_BYTES_PER_UPDATE * mv / 1e9 / peaks()[0]}
    del phi, pic, phi0
    torch.cuda.empty_cache()

    hbm, peak_kind = peaks()
    kern_mean = sum(kern_ms) / len(kern_ms)
    achieved = alg_bytes * updates / (kern_mean / 1e3) / 1e9
    wl = dict(w, B=base)
    kernel_name = "lattice_kernel" if lattice else "region_kernel"
    smem_bytes = SMEM_BYTES_PER_UPDATE_LATTICE if lattice else SMEM_BYTES_PER_UPDATE
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "site-updates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded random-phase field)",
        "config": {"workload": workload_name(wl), "grid": N, "leapfrog_steps": STEPS,
                   "leapfrog_steps_per_bench_step": PER, "region_base": base, "region_shape": shape,
                   "bench_step": f"one sp_evolve call of {PER} leapfrog steps continuing the run "
                                 f"(start levels {sched[args.warmup]}..{sched[-1]} timed); the initial field is "
                                 f"restored when a pass reaches level {STEPS}",
                   "regions_per_bench_step": regions_per_call,
                   "threads_per_cta": info["threads"], "ctas": info["grid"],
                   "mailbox_slots": info["mailbox_slots"], "mailbox_bytes": info["mailbox_bytes"],
                   "l2": ("inputs larger than L2 (state 24 B/site = "
                          f"{24 * sites / 1e9:.1f} GB plus " + ("the odd-level phi array" if lattice else "mailboxes")
                          + "), no flush" if N >= 512 else "state partly L2-resident (see extra key)"),
                   "init_s": init_s, "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "monolithic": mono,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": peak_kind,
                     "traffic": ncu_traffic(base, updates, shape),
                     "kernel": kernel_name, "kernel_ms": kern_mean,
                     "alg_bytes_per_update": alg_bytes,
                     "design_bytes_per_update": alg_bytes if lattice else info["bytes_per_update"],
                     "traffic_from": f"profiles/{TRAFFIC_RECORD[shape]} scaled by site-updates per launch"},
        "roofline_smem": smem_roofline(updates, kern_mean, clk, peaks_onchip[0], smem_bytes),
        "roofline_alu": alu_roofline(updates, kern_mean, peaks_onchip[1]),
        "measured_onchip_peaks": {"smem_gbs": peaks_onchip[0], "fp32_tflops": peaks_onchip[1]},
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,  # per bench step: ticket / queue reset + persistent region kernel
        "utilisation": utilisation,
        "clocks": clk,
        "wall_s_timed_region": wall,
        "field_finite": finite,
    }
    if extra:
        out.update(extra)
    return out


def run_small(args):
    """The 128^3 x 256 workload, whose state and mailboxes are largely
    L2-resident (the sweep runs at L2 speed there): region path and sweep,
    L2 flushed (512 MiB write) before every step, state restored on the device
    outside the timed region."""
    import torch

    from paper_1011_4046_gb300 import inputs, sp

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    w = dict(SMALL, SHAPE=args.shape)
    N, STEPS = w["N"], w["STEPS"]
    p = sp.make_params(N, dx=DX, dt=DT, lam=LAM, eta=ETA, nu=NU, tau0=TAU0, tau_ref=TAU0 + STEPS * DT)
    st = inputs.initial_state((N, N, N), SEED, "phase", eta=ETA)
    init_dev = torch.from_numpy(sp.pack_state(*st)).to(dev)
    g = sp.Grid([p], stream=stream)
    g.plan(base_B=w["B"], shape=shape_const(w["SHAPE"]))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    updates = N ** 3 * STEPS
    res = {}
    for name, flags in (("regions", 0), ("monolithic", sp.SP_MONOLITHIC)):
        ms, kms = [], []
        for it in range(args.small_warmup + args.small_steps):
            rc = sp.sp_write_surface(g.h, 0, sp.SP_SURF_STATE, init_dev.data_ptr(), init_dev.numel() * 8, 1)
            assert rc == 0, sp.sp_strerror(rc)
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = sp.sp_evolve(g.h, STEPS, sp.SP_ASYNC | sp.SP_RESTART | sp.SP_TIMING | flags)
            e1.record(stream)
            if rc != 0:
                raise sp.SpError(rc, "sp_evolve")
            e1.synchronize()
            if it >= args.small_warmup:
                ms.append(e0.elapsed_time(e1))
                kms.append(g.timing()[1])
        res[name] = (updates * len(ms) / (sum(ms) / 1e3), sum(ms) / len(ms), sum(kms) / len(kms))
    g.close()
    hbm, _ = peaks()
    kern = res["regions"][2]
    if w["SHAPE"] == "lattice":
        c_upd, c_rd, c_wr = sp.sp_lattice_call_bytes(w["B"], STEPS)
        alg = (c_rd + c_wr) / c_upd
    else:
        alg = ALG_BYTES_PER_UPDATE[w["B"]]
    return {"workload": workload_name(w), "value": res["regions"][0], "unit": "site-updates/s",
            "ms_per_step": res["regions"][1], "steps": args.small_steps,
            "monolithic": {"value": res["monolithic"][0], "ms_per_step": res["monolithic"][1],
                           "speedup_of_regions": res["regions"][0] / res["monolithic"][0]},
            "roofline_frac": alg * updates / (kern / 1e3) / 1e9 / hbm,
            "l2": "flushed (512 MiB write) before every step; state restored on device outside timing"}


def run_batched(args):
    """The batched workload: 64 simulations, N drawn from the multiples of 8 in
    [48, 160], nu in {0, 1, 2} (seeds 0-63), 192 steps each, in one persistent
    launch per region size replayed from a CUDA graph (lattice regions: edge 16
    where it divides a simulation's sides, else 8; split tiling: the autotuned
    base and block shape); the monolithic sweep of the same batch beside it.
    One JSON line (1 GPU)."""
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
    if args.shape == "lattice":
        g.plan(base_B=0, threads=0, shape=sp.SP_SHAPE_LATTICE)
    else:
        g.plan(base_B=sp.SP_AUTOTUNE, threads=sp.SP_AUTOTUNE)
    tune_s = time.perf_counter() - t0
    infos = [g.plan_info(i) for i in range(len(params))]
    l2_flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_step(flags):
        for i, buf in enumerate(inits):
            rc = sp.sp_write_surface(g.h, i, sp.SP_SURF_STATE, buf.data_ptr(), buf.numel() * 8, 1)
            assert rc == 0, sp.sp_strerror(rc)
        l2_flush.zero_()
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
                                   "nu in {0,1,2}, seeds 0-63, 192 steps each, one persistent launch per "
                                   "region base, replayed from a CUDA graph",
                       "region_shape": args.shape,
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


def oracle_sample(w, z_planes=SAMPLE_Z):
    """The bounded sample of workload ``w`` the FP64 oracle is timed on: the
    first z_planes planes of its initial field, as a periodic slab, with the
    workload's physics.  Returns (oracle params, phi, pi)."""
    import oracle
    from paper_1011_4046_gb300 import inputs

    N = w["N"]
    nz = min(N, z_planes)
    phi = inputs.random_phase_slab((N, N, N), SEED, 0, nz, eta=ETA).astype(np.complex128)
    p = oracle.make_params((N, N, nz), dx=DX, dt=DT, lam=LAM, eta=ETA, nu=NU, tau0=TAU0,
                           tau_ref=TAU0 + w["STEPS"] * DT)
    return p, phi, np.zeros_like(phi)


def cpu_baseline(budget_s, w=BIG):
    """The FP64 oracle, as it stands, on the host cores: the bounded sample
    of the workload, stepped in calls of 4 steps for about budget_s seconds."""
    import oracle

    oracle.build()
    p, phi, pi = oracle_sample(w)
    sites = p.n[0] * p.n[1] * p.n[2]
    done, chunk = 0, 4
    t0 = time.perf_counter()
    while done < w["STEPS"] and (time.perf_counter() - t0) < budget_s:
        phi, pi = oracle.run(p, phi, pi, done, chunk)
        done += chunk
    el = time.perf_counter() - t0
    return {"value": sites * done / el, "unit": "site-updates/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"the first {p.n[2]} z-planes of the {w['N']}^3 workload's initial field as a periodic "
                      f"{p.n[0]}x{p.n[1]}x{p.n[2]} slab with the workload's physics, {done} leapfrog steps in "
                      f"calls of 4 ({sites * done:.3g} site-updates, {el:.1f} s, FP64, OpenMP over z-planes)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle

    oracle.build()
    w = BIG
    p, phi0, pi0 = oracle_sample(w)
    sites = p.n[0] * p.n[1] * p.n[2]
    per_step = max(1, args.ref_levels)
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.run(p, phi0, pi0, 0, per_step)
        el = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(el)
    value = sites * per_step * len(times) / sum(times)
    sample = (f"each step: {per_step} leapfrog steps of the first {p.n[2]} z-planes of the {w['N']}^3 workload "
              f"as a periodic {p.n[0]}x{p.n[1]}x{p.n[2]} slab (FP64 oracle, OpenMP over z-planes)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "site-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random-phase field)",
            "config": {"workload": workload_name(w), "grid": w["N"], "leapfrog_steps": w["STEPS"],
                       "region_base": w["B"]},
            "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="1280", choices=["1280", "batched"],
                    help="1280: the 1280^3 x 2048 workload (default, with the 128^3 x 256 workload as an "
                         "extra key); batched: the 64-simulation batch")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-levels", type=int, default=4, help="leapfrog steps per reference-arm step")
    ap.add_argument("--base", type=int, default=0, help="region base (0: the workload's)")
    ap.add_argument("--shape", default=None, choices=["split", "lattice"],
                    help="region geometry: the paper's 4-cube lattice or the split tiling (pyramids and "
                         "wedges); default: the lattice for the grid workloads, the split tiling for the "
                         "batch (each measured the faster there)")
    ap.add_argument("--threads", type=int, default=0, help="threads per CTA (0 = library default)")
    ap.add_argument("--grid", type=int, default=0, help="grid side (profiling of smaller cases only)")
    ap.add_argument("--per-step", type=int, default=0, help="leapfrog steps per bench step (profiling only)")
    ap.add_argument("--mono-steps", type=int, default=3, help="timed sweep steps (after one warm-up)")
    ap.add_argument("--e2e-steps", type=int, default=2, help="timed e2e steps (after one warm-up)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-trace", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 128^3 extra key")
    ap.add_argument("--small-steps", type=int, default=5)
    ap.add_argument("--small-warmup", type=int, default=3)
    args = ap.parse_args()
    if args.shape is None:
        args.shape = "split" if args.workload == "batched" else "lattice"
    if args.impl == "reference":
        out = run_reference(args)
    elif args.workload == "batched":
        out = run_batched(args)
    else:
        setup_dist()
        ws, rank, _ = dist_env()
        w = dict(BIG, SHAPE=args.shape)
        if args.shape == "split":
            w["PER_STEP"] = SPLIT_PER_STEP
        if args.grid:
            w["N"] = args.grid
        if args.per_step:
            w["PER_STEP"] = args.per_step
        extra = {}
        if not args.no_extra and not args.grid:
            import torch

            extra["extra_128cubed_l2_resident"] = run_small(args)
            torch.cuda.empty_cache()
        out = run_grid(args, w, extra)
        if rank != 0:
            out = None
        elif not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, w)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
