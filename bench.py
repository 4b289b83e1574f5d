"""Benchmark of the dust drag-coupling step (gather + exponential-midpoint push
+ feedback deposit) on the 3-D shearing-box workload: 128^3 zones, 16.8M
grains (8 per zone), TSC weights, St = 0.1, dust-to-gas ratio 0.02, feedback
applied, mixed precision (FP32 push and gather, FP64 positions, int64
fixed-point deposit).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` = grain-updates/s over all ranks (each rank
steps its own independent instance: weak scaling, no collective on the data
path); the FP64 GPU path is measured beside it.  `--impl reference` times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1908_10793_gb300 import inputs as I  # noqa: E402

METRIC = "grain-updates/s (gather+push+deposit) mixed vs FP64 on 1 GB300; % HBM roofline"
UNIT = "grain-updates/s"
WORKLOAD_NAME = ("sbox3d: 3-D shearing box (orbital-advection frame) 128^3 zones, 16,777,216 "
                 "grains (8/zone), St=0.1, dust/gas 0.02, TSC, feedback on")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sort-interval", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-disks", action="store_true")
    ap.add_argument("--disk-steps", type=int, default=10)
    ap.add_argument("--disk-scale", default="full", choices=["full", "mid"],
                    help="mid: the cylindrical disk at an eighth of its size (profiling runs)")
    ap.add_argument("--disk-legs", default="cyldisk,sphdisk,cyldisk_gas_predictor,cyldisk_volume_weighting")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--small", action="store_true", help="16^3 grid (profiling runs)")
    ap.add_argument("--grid", type=int, default=0, help="zones per side (profiling runs)")
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 per-grain, 2 tiled")
    ap.add_argument("--tile", type=str, default="0,0,0")
    ap.add_argument("--gas-predictor", action="store_true",
                    help="main leg with the gas half-step predictor (profiling runs)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# Sources the shearing-box step kernel is compiled from (its translation
# unit and the headers it includes); the profiled traffic is dropped when one
# of them changes.
STEP_KERNEL_SOURCES = [
    "include/dust.h",
    "paper_1908_10793_gb300/csrc/dust_internal.h",
    "paper_1908_10793_gb300/csrc/dust_device.cuh",
    "paper_1908_10793_gb300/csrc/dust_step_kernels.cuh",
    "paper_1908_10793_gb300/csrc/dust_tiled.cuh",
    "paper_1908_10793_gb300/csrc/dust_slab.cuh",
    "paper_1908_10793_gb300/csrc/dust_geom_sb.cu",
]


# string and character literals (kept), line and block comments (dropped)
_C_TOKENS = re.compile(r'"(?:\\.|[^"\\])*"|\'(?:\\.|[^\'\\])*\'|//[^\n]*|/\*.*?\*/', re.S)


def _code_only(text):
    """C/C++ source without its comments, whitespace runs collapsed: edits of
    comments or layout do not change the compiled kernel."""
    kept = _C_TOKENS.sub(lambda m: " " if m.group(0).startswith("/") else m.group(0), text)
    return " ".join(kept.split())


def source_digest(root=None, read=None):
    """Digest of the step kernel's sources (code only).  read(path) -> text
    can supply another revision's files."""
    root = ROOT if root is None else root
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(root, f), encoding="utf-8") as fh:
                text = fh.read()
        else:
            text = read(f)
        h.update(os.path.basename(f).encode() + _code_only(text).encode())
    return h.hexdigest()[:16]


def profiled_record():
    """The committed ncu figures of the step kernel (per grain), if they were
    taken on the current sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic_step_sbox3d.txt")
    try:
        rec = {}
        with open(path) as f:
            for line in f:
                if line.strip() and not line.startswith("#"):
                    k, v = line.split(None, 1)
                    rec[k] = v.strip()
        return rec if rec.get("source_digest") == source_digest() else None
    except Exception:
        return None


def profiled_traffic(ngrains):
    """DRAM bytes per launch of the step kernel from the committed ncu summary
    (None when it is not for the current sources)."""
    rec = profiled_record()
    try:
        return float(rec["dram_bytes_per_grain"]) * ngrains if rec else None
    except (KeyError, ValueError):
        return None


# Warp-instruction issue of one GB300: 152 SMs x 4 schedulers x 2.07 GHz.
ISSUE_PEAK_PER_S = 152 * 4 * 2.07e9


def issue_rate(ngrains, kernel_s):
    """The step kernel against the instruction-issue ceiling that bounds it:
    warp instructions per grain from the committed ncu summary (same source
    check as the traffic) times the grains of a launch, over the measured
    launch time."""
    rec = profiled_record()
    try:
        per = float(rec["warp_instructions_per_grain"]) if rec else None
    except (KeyError, ValueError):
        per = None
    if per is None or kernel_s <= 0:
        return None
    achieved = per * ngrains / kernel_s
    return {"bound": "instruction issue", "achieved": achieved, "peak": ISSUE_PEAK_PER_S,
            "unit": "warp instructions/s", "frac": achieved / ISSUE_PEAK_PER_S,
            "warp_instructions_per_grain": per,
            "source": "profiles/traffic_step_sbox3d.txt (ncu), peak from unit counts and clock"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = max(smax, float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, device):
    """Largest value of x over all ranks (x itself with one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world, units_per_rank, seconds):
    """Whole-job throughput: every rank processed units_per_rank in at most
    `seconds` (the slowest rank's time)."""
    return world * units_per_rank / seconds


def algorithmic_bytes(w, precision_bytes):
    """Bytes one step (gather + push + deposit) must move at minimum: every
    grain's state read and written once (3 FP64 coordinates + 3 momentum-like
    values, and the species index and stopping-time value where the workload
    has them), each zone's gas (rho + 3 velocities) read once and its
    4-channel int64 deposit written once.  The zone sort is not part of it
    (reported as sort_overhead).  Shearing box 128^3, mixed: 72 B per grain
    + 48 B per zone at 8 grains per zone = 78 B per grain."""
    per_grain = 2 * (3 * 8 + 3 * precision_bytes)
    if w.species is not None:
        per_grain += 2 * 1
    if w.param is not None:
        per_grain += 2 * precision_bytes
    per_zone = 4 * precision_bytes + 4 * 8
    return w.ngrains * per_grain + w.ncell * per_zone, per_grain, per_zone


def sort_overhead(w, kt, steps):
    """The zone sort, beside the roofline: the step kernel finishes it (reads
    each grain through the permutation, reads the sorted id and writes the
    id column, 12 B per grain beyond the algorithmic bytes), and the sort's
    own kernels run before the step (key counts, scan, pair scatter, id sort
    inside each zone)."""
    extra = 3 * 4 * w.ngrains
    return {"step_kernel_bytes_per_grain": 12, "step_kernel_bytes_per_launch": extra,
            "sort_kernels_ms_per_step": kt.sort_ms / max(1, steps),
            "sort_kernel_launches_per_step": kt.sort_launches / max(1, steps)}


def run_ours(args):
    import torch
    from paper_1908_10793_gb300 import dust as D

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = I.sbox3d(args.grid if args.grid else ("small" if args.small else "full"))
    # a real stream (not the legacy default stream) shared by the library and
    # the timing events
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    def make(precision, timing, **kw):
        ctx = D.Context(w, precision=precision, stream=stream.cuda_stream,
                        sort_interval=args.sort_interval, timing=timing, device=local,
                        kernel=args.kernel, tile=[int(x) for x in args.tile.split(",")], **kw)
        ctx.set_gas(w.rho, w.vgas)
        ctx.load(w.q, w.v)
        return ctx

    def timed(ctx, steps, warmup, sample_clocks=False):
        for _ in range(warmup):
            ctx.step(w.dt)
        ctx.sync()
        ctx.kernel_times(reset=True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        clocks = ClockSampler(local) if sample_clocks else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.step(w.dt)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ck = clocks.stop() if clocks else None
        ms = max_over_ranks(e0.elapsed_time(e1), dev)
        rc, st = ctx.sync(check=False)
        kt = ctx.kernel_times(reset=True)
        return ms, rc, st, kt, ck

    # ---- mixed path, inputs resident in HBM
    ctx = make(D.DUST_MIXED, 1, gas_predictor=int(args.gas_predictor))
    ms, rc, st, kt, clocks = timed(ctx, args.steps, args.warmup, sample_clocks=True)
    ngr = w.ngrains
    value = weak_value(world, ngr * args.steps, ms / 1e3)
    step_ms_avg = kt.step_ms / max(1, kt.step_launches)
    ab, per_grain, per_zone = algorithmic_bytes(w, 4)
    achieved = ab / (step_ms_avg / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    sort_over = sort_overhead(w, kt, args.steps)
    launches = int(kt.step_launches + kt.sort_launches + kt.other_launches)
    ctx.close()

    # ---- FP64 GPU path beside it
    fp64 = None
    if not args.no_fp64:
        ctx = make(D.DUST_FP64, 1)
        k64 = max(2, args.steps // 4)
        ms64, rc64, _, kt64, _ = timed(ctx, k64, min(args.warmup, 3))
        fp64 = {"value": weak_value(world, ngr * k64, ms64 / 1e3), "ms_per_step": ms64 / k64,
                "steps": k64, "status": rc64,
                "step_kernel_ms": kt64.step_ms / max(1, kt64.step_launches)}
        ctx.close()

    # ---- end to end through the C interface with host buffers: every step
    # loads the grains and the gas from pinned host memory, steps, and reads
    # the grains (with ids) and the deposit back.  Headline: a context with
    # dust_options.host_io_async, where one step's read-back, the next
    # step's load and the steps overlap (dust_sync at the end waits for the
    # last copies), with the velocities as float32 host arrays (the mixed
    # store's own precision: dust_load_particles_v32 / _get_particles_v32);
    # beside it the same calls with synchronous copies, and the float64
    # velocity calls.
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        hq = [pin(x) for x in w.q]
        hv = [pin(x) for x in w.v]
        hv32 = [pin(np.asarray(x, dtype=np.float32)) for x in w.v]
        hrho = pin(w.rho)
        hg = [pin(x) for x in w.vgas]
        outs = [([pin(np.empty(ngr)) for _ in range(6)],
                 torch.empty(ngr, dtype=torch.int64).pin_memory().numpy(),
                 torch.empty((w.ncell, 4), dtype=torch.int64).pin_memory().numpy(),
                 [pin(np.empty(ngr, np.float32)) for _ in range(3)])
                for _ in range(2)]
        ke = max(2, min(args.steps, 20))

        def run_e2e(async_io, v32=True):
            ctx = make(D.DUST_MIXED, 0, host_io_async=async_io)

            def one(k):
                o, oid, odep, o32 = outs[k % 2]
                if v32:
                    D.dust_load_particles_v32(ctx.handle, *hq, *hv32)
                else:
                    D.dust_load_particles(ctx.handle, *hq, *hv)
                D.dust_set_gas(ctx.handle, hrho, *hg)
                D.dust_step(ctx.handle, w.dt)
                if v32:
                    D.dust_get_particles_v32(ctx.handle, ngr, *o[:3], *o32, ids=oid)
                else:
                    D.dust_get_particles(ctx.handle, ngr, *o, ids=oid)
                D.dust_get_deposit(ctx.handle, fixed=odep)

            one(0)
            ctx.sync(check=False)
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for k in range(ke):
                one(k)
            ctx.sync(check=False)
            torch.cuda.synchronize(dev)
            te = max_over_ranks(time.perf_counter() - t0, dev)
            return ctx, te

        ctx, te_f64 = run_e2e(1, v32=False)
        ctx.close()
        ctx, te_async = run_e2e(1)
        ctx.close()
        ctx, te_sync = run_e2e(0)
        h2d, d2h = e2e_bytes_per_step(ngr, w.ncell, v32=True)
        h2d64, d2h64 = e2e_bytes_per_step(ngr, w.ncell, v32=False)
        e2e = {"value": weak_value(world, ngr * ke, te_async), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ke,
               "host_io": "asynchronous (dust_options.host_io_async = 1), pinned buffers; "
                          "coordinates float64, velocities float32 (dust_load_particles_v32, "
                          "dust_get_particles_v32)",
               "synchronous_calls": {"value": weak_value(world, ngr * ke, te_sync),
                                     "ms_per_step": te_sync / ke * 1e3},
               "float64_velocities": {"value": weak_value(world, ngr * ke, te_f64),
                                      "ms_per_step": te_f64 / ke * 1e3,
                                      "h2d_bytes_per_step": h2d64, "d2h_bytes_per_step": d2h64},
               "ms_per_step": te_async / ke * 1e3,
               "breakdown": e2e_breakdown(ctx, D, torch, dev, w, hq, hv32, hrho, hg, outs[0][0][:3],
                                          outs[0][3], outs[0][1], outs[0][2])}
        ctx.close()

    # ---- batched instances (64 streaming-instability boxes, one graph launch
    # per two steps) against the same instances stepped one at a time
    batch = None
    if not args.no_batch:
        batch = run_batch(args, D, torch, dev, stream)

    # ---- the global disk workloads (cylindrical and spherical, mixed)
    disks = None
    if not args.no_disks:
        disks = run_disks(args, D, torch, dev, stream)

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baselines(w, steps=2)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Philox; shapes of the paper's shearing-box setup)",
            "config": {"workload": WORKLOAD_NAME if w.ncell == 128 ** 3 else
                       "sbox3d %d^3 (profiling size)" % round(w.ncell ** (1 / 3)),
                       "precision": "mixed: f32 push/gather, f64 positions, int64 deposit",
                       "grains": ngr, "zones": w.ncell, "sort_interval": args.sort_interval or 1,
                       "l2": "inputs larger than L2 (grain store %d MB)" % (ngr * 36 // 2**20),
                       "parallelism": "independent instance per GPU",
                       "gas_predictor": int(args.gas_predictor)},
            "status": rc,
            "kernel_ms_per_step": {"step": kt.step_ms / args.steps, "sort": kt.sort_ms / args.steps,
                                   "other": kt.other_ms / args.steps},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_kind,
                         "kernel": "step (gather+push+deposit)",
                         "algorithmic_bytes_per_launch": ab,
                         "bytes_per_grain": per_grain, "bytes_per_zone": per_zone,
                         "bytes_per_grain_amortised": ab / ngr,
                         "traffic": profiled_traffic(ngr)},
            "sort_overhead": sort_over,
            "issue": issue_rate(ngr, kt.step_ms / max(1, kt.step_launches) / 1e3),
            "gpu_launches": launches,
            "fp64": fp64,
            "batch": batch,
            "disks": disks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch(args, D, torch, dev, stream):
    """64 independent 2-D shearing boxes (32^2 .. 512^2 zones, 1-16 grains per
    zone, St in {0.01, 0.1, 1}), mixed precision.  Each dust_batch_step call
    is one persistent launch for all instances and steps.  The autotuner
    times candidate configurations (a tile shape for every instance, and the
    batch's sort interval) in the batch itself, a few steps each; the chosen
    configuration is then timed over the leg's steps.  Beside it: the default
    configuration, the earlier graph of per-instance kernels, and dust_step
    on each context in turn on one stream."""
    from paper_1908_10793_gb300 import autotune
    ws = I.si2d_batch("full")
    ngr = sum(w.ngrains for w in ws)
    K = max(2, args.batch_steps)
    best, tried = autotune.tune_batch(ws, steps=4, device=dev.index)
    policy, kint, mode = best
    Kb = K - K % 2 if mode else K
    ms_best = autotune.time_batch(ws, policy, kint, steps=Kb, device=dev.index, batch_mode=mode)
    ms_def = autotune.time_batch(ws, None, 1, steps=K, device=dev.index)
    ms_graph = autotune.time_batch(ws, None, 1, steps=K - K % 2, device=dev.index, batch_mode=1)
    cs = []
    try:
        for w in ws:
            c = D.Context(w, precision=D.DUST_MIXED, sort_interval=1, device=dev.index,
                          stream=stream.cuda_stream)
            c.set_gas(w.rho, w.vgas)
            c.load(w.q, w.v)
            cs.append(c)
        for _ in range(2):
            for c, w in zip(cs, ws):
                c.step(w.dt)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for c, w in zip(cs, ws):
            for _ in range(K):
                c.step(w.dt)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_s = e0.elapsed_time(e1) / K
        rc = min(c.sync(check=False)[0] for c in cs)
    finally:
        for c in cs:
            c.close()
    label = lambda cfg: "%s, sort every %d, %s" % (  # noqa: E731
        "default tiles" if cfg[0] is None else "tile %s" % list(cfg[0]), cfg[1],
        "graph of per-instance kernels" if cfg[2] else "one persistent launch")
    return {"value": ngr / (ms_best / 1e3), "unit": UNIT, "ms_per_step": ms_best,
            "config_chosen": label(best), "instances": len(ws), "grains": ngr,
            "zones": sum(w.ncell for w in ws), "steps": Kb,
            "path": "graph of per-instance kernels" if mode else
                    "one persistent cooperative launch per call",
            "tuner": {label(k): v for k, v in tried.items()},
            "default_config": {"value": ngr / (ms_def / 1e3), "ms_per_step": ms_def,
                               "config": "default tiles, sort every 1, one persistent launch"},
            "graph_of_per_instance_kernels": {"value": ngr / (ms_graph / 1e3),
                                              "ms_per_step": ms_graph},
            "one_at_a_time": {"value": ngr / (ms_s / 1e3), "ms_per_step": ms_s},
            "status": rc,
            "workload": "64 2-D (x,z) orbital-advection shearing boxes, 32^2..512^2 zones, "
                        "1-16 grains/zone, St 0.01/0.1/1, dust/gas 0.01/0.02/0.1, TSC, "
                        "feedback on, mixed precision"}


def e2e_bytes_per_step(ngrains, ncell, v32=True):
    """Host-link bytes of one end-to-end step: in, the grains' coordinates
    (float64) and velocities (float32 with v32, else float64) and the gas
    (density and three velocity components, float64); out, the grains'
    coordinates, velocities and int64 ids and the int64 deposit (four
    channels per zone)."""
    vb = 4 if v32 else 8
    h2d = ngrains * (3 * 8 + 3 * vb) + ncell * 4 * 8
    d2h = ngrains * (3 * 8 + 3 * vb + 8) + ncell * 4 * 8
    return h2d, d2h


def e2e_breakdown(ctx, D, torch, dev, w, hq, hv, hrho, hg, oq, ov, oid, odep):
    """Untimed by the headline: two more end-to-end steps of the headline's
    calls (float32 velocities) with a device synchronise around every call
    (ms per call, the faster of the two), and the bandwidth of plain
    pinned-memory copies of the grains' size in each direction and in both
    at once, which bound the end-to-end figure."""
    ngr = w.ngrains

    def timed(f):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        f()
        torch.cuda.synchronize(dev)
        return (time.perf_counter() - t0) * 1e3

    calls = {}
    for _ in range(2):
        one = {
            "load_particles_v32": timed(lambda: D.dust_load_particles_v32(ctx.handle, *hq, *hv)),
            "set_gas": timed(lambda: D.dust_set_gas(ctx.handle, hrho, *hg)),
            "step": timed(lambda: D.dust_step(ctx.handle, w.dt)),
            "get_particles_v32": timed(lambda: D.dust_get_particles_v32(ctx.handle, ngr, *oq, *ov, ids=oid)),
            "get_deposit": timed(lambda: D.dust_get_deposit(ctx.handle, fixed=odep)),
        }
        calls = {k: min(v, calls.get(k, v)) for k, v in one.items()}
    nb = ngr * 6
    host = torch.empty(nb, dtype=torch.float64).pin_memory()
    host2 = torch.empty(nb, dtype=torch.float64).pin_memory()
    devb = torch.empty(nb, dtype=torch.float64, device=dev)
    devb2 = torch.empty(nb, dtype=torch.float64, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    link = {}
    for _ in range(2):
        link["h2d_gbs"] = nb * 8 / timed(lambda: devb.copy_(host, non_blocking=True)) / 1e6
        link["d2h_gbs"] = nb * 8 / timed(lambda: host.copy_(devb, non_blocking=True)) / 1e6

        def both():
            with torch.cuda.stream(s1):
                devb.copy_(host, non_blocking=True)
            with torch.cuda.stream(s2):
                host2.copy_(devb2, non_blocking=True)
        link["both_directions_gbs"] = 2 * nb * 8 / timed(both) / 1e6
    link["bytes_each"] = nb * 8
    del host, host2, devb, devb2
    return {"ms_per_call": calls, "link": link}


def run_disks(args, D, torch, dev, stream):
    """Cylindrical (384 x 1024 x 64, 50M grains, 4 species) and spherical
    (256 x 128 x 512, 33M grains, St log-uniform in [1e-4, 10]) disks, mixed
    precision, sort every step; grain-updates/s over the timed steps.  The
    spherical disk keeps its gas fixed: far from the midplane its gas density
    falls to ~1e-9 of the midplane value, where a single grain makes the local
    dust-to-gas ratio 1e4 or more, and neither the explicit feedback nor the
    predictor-corrector coupling is stable for grains as stiff as St = 1e-4
    there.  Two more lines run the cylindrical disk with the gas half-step
    drag predictor and with the traditional volume weighting (Eq. CIC_vol)
    instead of TSC."""
    out = {}
    peak, _ = measured_peaks()
    legs = (("cyldisk", I.cyldisk, 1, {}, None),
            ("sphdisk", I.sphdisk, 0, {}, None),
            ("cyldisk_gas_predictor", I.cyldisk, 1, {"gas_predictor": 1}, None),
            ("cyldisk_volume_weighting", I.cyldisk, 1, {}, I.VOLUME))
    wanted = args.disk_legs.split(",")
    for name, make, feedback, extra, weight in legs:
        if name not in wanted or (args.disk_scale == "mid" and make is not I.cyldisk):
            continue
        w = make(args.disk_scale)
        if weight is not None:
            w.weight = weight
        ctx = D.Context(w, precision=D.DUST_MIXED, stream=stream.cuda_stream, timing=1,
                        device=dev.index, feedback=feedback, **extra)
        try:
            ctx.set_gas(w.rho, w.vgas)
            ctx.load(w.q, w.v, w.species, w.param)
            for _ in range(3):
                ctx.step(w.dt)
            ctx.sync(check=False)
            ctx.kernel_times(reset=True)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.disk_steps):
                ctx.step(w.dt)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            rc, st = ctx.sync(check=False)
            kt = ctx.kernel_times(reset=True)
        finally:
            ctx.close()
        ab, per_grain, per_zone = algorithmic_bytes(w, 4)
        step_ms = kt.step_ms / max(1, kt.step_launches)
        out[name] = {"value": w.ngrains * args.disk_steps / (ms / 1e3), "unit": UNIT,
                     "ms_per_step": ms / args.disk_steps, "grains": w.ngrains, "zones": w.ncell,
                     "kernel_ms_per_step": {"step": kt.step_ms / args.disk_steps,
                                            "sort": kt.sort_ms / args.disk_steps,
                                            "other": kt.other_ms / args.disk_steps},
                     "step_roofline_frac": ab / (step_ms / 1e3) / 1e9 / peak,
                     "status": rc, "removed": st.n_removed, "feedback": feedback,
                     "weight": ("cic", "tsc", "volume")[w.weight],
                     "gas_predictor": int(extra.get("gas_predictor", 0))}
    return out


def _momentum_like(w, q, v):
    """Physical grain velocities -> the momentum-like variables the oracle
    steps (cylindrical l = R v_phi; spherical r v_theta, r sin(theta) v_phi)."""
    p = [x.copy() for x in v]
    if w.geom == I.CYLINDRICAL:
        p[1] = q[0] * v[1]
    elif w.geom == I.SPHERICAL:
        p[1] = q[0] * v[1]
        p[2] = q[0] * np.sin(q[1]) * v[2]
    return p


def _zone_volumes(w):
    e = w.edges
    d = [np.diff(x) for x in e]
    if w.geom == I.CYLINDRICAL:
        d[0] = 0.5 * np.diff(e[0] ** 2)
    elif w.geom == I.SPHERICAL:
        d[0] = np.diff(e[0] ** 3) / 3.0
        d[1] = -np.diff(np.cos(e[1]))
    Z, Y, X = np.meshgrid(d[2], d[1], d[0], indexing="ij")
    return (X * Y * Z).ravel()


def host_threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:
        return max(1, os.cpu_count() or 1)


def cpu_baseline(w, steps=2, ngrains=None, threads=1, return_state=False):
    """The FP64 oracle as it stands on the full grid and a seeded subset
    (default: all) of the grains, `steps` steps.  threads > 1: the grains are
    cut into that many contiguous ranges, each stepped by the oracle on its
    own host thread into its own dense deposit (the oracle's C function runs
    without the interpreter lock), the deposits are summed in range order and
    the feedback is applied to the gas after the sum."""
    import concurrent.futures as cf

    import oracle as O
    O.build()
    s = w if ngrains is None else I.subsample(w, ngrains)
    fb = bool(s.feedback)
    prob = O.Problem(geom=s.geom, edges=s.edges, bc=s.bc, weight=s.weight,
                     species_mass=s.species_mass, species_tau_mode=s.species_tau_mode,
                     species_tau=s.species_tau, fargo=s.fargo, omega=s.omega, q=s.qshear,
                     gm=s.gm, vertical_gravity=s.vertical_gravity,
                     feedback_apply=int(fb and threads == 1))
    q = [x.copy() for x in s.q]
    p = _momentum_like(s, q, s.v)
    pg = O.gas_momentum(prob, s.vgas)
    rho = s.rho.copy()
    active = np.ones(s.ngrains, np.uint8)
    bounds = np.linspace(0, s.ngrains, threads + 1).astype(np.int64)
    sp, par = s.species, s.param
    dV = _zone_volumes(s) if (fb and threads > 1) else None

    def part(i, t):
        r = slice(int(bounds[i]), int(bounds[i + 1]))
        dep, _ = O.step(prob, [x[r] for x in q], [x[r] for x in p], active[r], t, s.dt, rho, pg,
                        None if sp is None else sp[r], None if par is None else par[r])
        return dep

    ex = cf.ThreadPoolExecutor(max_workers=threads) if threads > 1 else None
    t0 = time.perf_counter()
    for k in range(steps):
        if ex is None:
            O.step(prob, q, p, active, k * s.dt, s.dt, rho, pg, sp, par)
        else:
            deps = list(ex.map(lambda i: part(i, k * s.dt), range(threads)))
            dep = deps[0]
            for d in deps[1:]:
                dep += d
            if fb:
                for c in range(3):
                    pg[c] += dep[:, c] / (rho * dV)
    el = time.perf_counter() - t0
    if ex is not None:
        ex.shutdown()
    out = {"value": s.ngrains * steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": "%d grains x %d steps of the same workload (full grid), %s"
                     % (s.ngrains, steps, "single thread" if threads == 1 else
                        "%d host threads over grain ranges" % threads), "seconds": el}
    if return_state:
        out["state"] = (q, p, pg, active)
    return out


def cpu_baselines(w, steps=2):
    """The oracle on all host cores (the line's cpu_baseline) with the
    single-thread figure beside it."""
    nt = host_threads()
    one = cpu_baseline(w, steps=steps, threads=1)
    allc = cpu_baseline(w, steps=steps, threads=nt) if nt > 1 else dict(one)
    allc["single_thread"] = one
    return allc


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = I.sbox3d("small" if args.small else "full")
    nt = host_threads()
    # a bounded sample per step: about 1.5e8 grain-steps per host thread for
    # the whole warm-up + timed run (a minute or two)
    budget = 150_000_000 * nt
    n = int(min(w.ngrains, max(1 << 16, budget // max(1, args.steps + args.warmup))))
    cpu_baseline(w, steps=1, ngrains=1024)  # build + warm the library
    times = []
    for _ in range(args.warmup):
        cpu_baseline(w, steps=1, ngrains=n, threads=nt)
    for _ in range(args.steps):
        r = cpu_baseline(w, steps=1, ngrains=n, threads=nt)
        times.append(r["seconds"])
    tot = sum(times)
    value = n * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD_NAME, "grains_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                         "sample": "%d of the %d grains (full grid) per step, %d host threads "
                                   "over grain ranges" % (n, w.ngrains, nt)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
