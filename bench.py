"""Benchmark: MLUPS and HBM-roofline fraction of the fused fluctuating-LB step.

Default workload: D3Q19 Taylor-Green vortex, 256^3 periodic, Re = 100,
Wi = 1, beta = 0.5, u0 = 0.02, FP32 storage and arithmetic, fused kernel.
One step = one fused collide-stream-stress launch over all 16.8 M sites.
The state (18.7 GB) is far larger than L2, so no L2 flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --forms          # every other form, one subprocess each
    python bench.py --form NAME      # one form alone

The default run prints one JSON line (rank 0): the headline, its roofline,
the end-to-end figure through the public API with page-locked host buffers,
and the CPU oracle timed on the host cores (one core, and all cores as
independent processes).  With N > 1 (torchrun) every rank runs an
independent replica of the workload on its own GPU (the method's single
grid does not shard here) and `value` counts the updates of all ranks.

The other forms (precisions, the D2Q9 four-roll mill, the split kernels,
the original scheme, other constitutive models, the batched grids and the
learned closure) run only under --forms, each in a process of its own, so
that one form's memory or failure cannot touch the headline.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import resource
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline per form at <=1e-3 rel-L2 vs FP64 oracle"
UNIT = "MLUPS"
WORKLOAD = dict(lattice="D3Q19", n=256, Re=100.0, Wi=1.0, beta=0.5, U0=0.02)
KERNEL_SOURCES = ["paper_2506_13072_gb300/csrc/fvlb_kernels.cuh",
                  "paper_2506_13072_gb300/csrc/fvlb_lattice.cuh",
                  "paper_2506_13072_gb300/csrc/fvlb_launch.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def maxrss_mb() -> float:
    """Peak resident host memory of this process so far (MB)."""
    return round(resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 1024.0, 1)


def log(msg: str):
    sys.stderr.write(f"[bench {time.strftime('%H:%M:%S')}] {msg} (maxrss {maxrss_mb()} MB)\n")
    sys.stderr.flush()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def traffic_record(kernel_key: str):
    """DRAM bytes per launch from a committed ncu summary, valid only while
    the kernel sources are unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    r = rec.get(kernel_key)
    if not r or r.get("kernel_hash") != kernel_hash():
        return None
    return r


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, each sample stamped with the
    host's monotonic clock when it arrives, so that the samples of a window
    (the timed region) can be picked out afterwards."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, period_ms: int = 50):
        self.dev = device_index
        self.period = period_ms
        self.proc = None
        self.rows = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.period)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    self.rows.append((time.monotonic(), parts))

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread is not None:
                self.thread.join(timeout=5)

    def wait_for_samples(self, n: int, step_fn, limit_s: float = 4.0) -> int:
        """Run step_fn() until n samples have arrived (at most limit_s);
        returns how many times it ran."""
        calls = 0
        t0 = time.monotonic()
        while (self.proc is not None and len(self.rows) < n
               and time.monotonic() - t0 < limit_s):
            step_fn()
            calls += 1
        return calls

    def summary(self, t0: float, t1: float):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [r for (t, r) in self.rows if t0 <= t <= t1]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = sorted(v for v in (num(r[1]) for r in rows) if v is not None)
        mx = max((v for v in (num(r[2]) for r in rows) if v is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        pw = [v for v in (num(r[3]) for r in rows) if v is not None]
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(pw) if pw else None}


def tgv_problem(n, fields=True, out_u=None, out_p=None):
    from paper_2506_13072_gb300 import workloads as W

    w = WORKLOAD
    return W.taylor_green_3d(n=n, U0=w["U0"], Re=w["Re"], Wi=w["Wi"], beta=w["beta"],
                             fields=fields, out_u=out_u, out_p=out_p)


def main_problem(args, fields=True):
    """The timed workload: the default D3Q19 Taylor-Green box, or (for
    profiling) another size or the D2Q9 four-roll mill (at rest)."""
    from paper_2506_13072_gb300 import workloads as W

    if args.lattice == "d2q9":
        return W.four_roll(n=args.n or 2048, Wi=0.5, beta=0.5)
    return tgv_problem(args.n or WORKLOAD["n"], fields=fields)


# ---------------------------------------------------------------------------
# CPU oracle, timed on a bounded sample of the workload
# ---------------------------------------------------------------------------

def _oracle_worker(seconds: float, n: int):
    """One single-threaded FP64 oracle on an n^3 Taylor-Green box with the
    workload's physics, stepped for about `seconds`; returns (steps, sites,
    elapsed)."""
    import oracle as O

    pr = tgv_problem(n)
    o = O.Oracle(pr.lattice, **pr.oracle_kwargs())
    o.init(u=pr.u0, p=pr.p0, A=pr.A0)
    o.step(1)
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        o.step(1)
        steps += 1
    return steps, pr.sites, time.perf_counter() - t0


def cpu_baseline(seconds: float = 8.0, n: int = 32):
    """The oracle as it stands, on the host cores: one process alone, then
    one independent process per core at once (the oracle is single-threaded;
    the processes are started with `spawn`, never forked from this CUDA
    process).  Returns the cpu_baseline object (value = all cores)."""
    import multiprocessing as mp

    import oracle as O

    O.build()
    steps1, sites, dt1 = _oracle_worker(seconds, n)
    one = sites * steps1 / dt1 / 1e6
    cores = os.cpu_count() or 1
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            res = pool.starmap(_oracle_worker, [(seconds, n)] * cores)
        allc = sum(s * m / t for (s, m, t) in res) / 1e6
        used = cores
        note = (f"{cores} independent single-threaded oracle processes at once, "
                f"each on its own {n}^3 box for ~{seconds:g} s "
                f"({sum(r[0] for r in res)} steps in all)")
    except Exception as e:          # a host that cannot spawn: report the one-core figure
        allc, used = one, 1
        note = f"all-core leg failed ({type(e).__name__}); single process only"
    return {"value": round(allc, 3), "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"FP64 CPU oracle (plain C, gcc -O2), D3Q19 Taylor-Green {n}^3 "
                      f"({sites} sites, the workload's Re, Wi, beta): {note}",
            "single_core": {"value": round(one, 4), "unit": UNIT, "cores": 1,
                            "sample": f"one process, {steps1} steps in {dt1:.1f} s"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    per_step = []
    import oracle as O

    pr = tgv_problem(32)
    o = O.Oracle(pr.lattice, **pr.oracle_kwargs())
    o.init(u=pr.u0, p=pr.p0, A=pr.A0)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s0 = time.perf_counter()
        o.step(1)
        per_step.append(time.perf_counter() - s0)
    dt = time.perf_counter() - t0
    value = pr.sites * args.steps / dt / 1e6
    sample = f"FP64 CPU oracle, single thread, D3Q19 Taylor-Green 32^3 (same Re, Wi, beta), {args.steps} steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(args, "oracle sample 32^3"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def kernel_label(lattice: str, precision: str) -> str:
    """The fused-step kernel instance the library launches for this workload."""
    S = {"fp64": "double", "fp32": "float", "fp16_dev": "__half", "bf16_dev": "__nv_bfloat16",
         "fp16_dev_sr": "half_sr", "bf16_dev_sr": "bf16_sr"}[precision]
    minb = 1 if precision == "fp64" else 2
    if lattice == "d2q9":
        if precision == "fp64":
            return (f"k_step_fused<D2Q9,double,GX=4,TY=1,MINB=1,periodic> "
                    f"(128 nodes x 3 stress components per block, in-warp halo fill)")
        nfw = 5 if precision == "fp32" else 4
        return (f"k_step_fused<D2Q9,{S},GX=4,TY=1,MINB=2,periodic,fill warps> "
                f"(128 nodes x 3 stress components + {nfw} halo fill warps per block, "
                f"bulk tensor copies into the stage)")
    if precision == "fp32":
        return (f"k_step_fused<D3Q19,float,GX=1,TY=1,MINB=2,periodic,fill warps,XN=2> "
                f"(64 nodes x 6 stress components + 7 halo fill warps per block, "
                f"bulk tensor copies into the stage)")
    if precision == "fp64":
        return (f"k_step_fused<D3Q19,double,GX=1,TY=1,MINB=1,periodic,fill warps> "
                f"(32 nodes x 6 stress components + 4 halo fill warps per block)")
    return (f"k_step_fused<D3Q19,{S},GX=1,TY=1,MINB=2,periodic,fill warps,XN=2> "
            f"(64 nodes x 6 stress components + 4 halo fill warps per block, "
            f"bulk tensor copies into the stage)")


def config_dict(args=None, note=""):
    w = WORKLOAD
    prec = args.precision if args else "fp32"
    if args is not None and args.lattice == "d2q9":
        n = args.n or 2048
        return {"workload": f"D2Q9 four-roll mill {n}^2 periodic, Wi=0.5, beta=0.5, {prec} fused step",
                "lattice": "D2Q9", "grid": [n, n], "precision": prec, "kernel": "fused",
                "parallelism": "replicas", "note": note}
    n = (args.n if args is not None and args.n else w["n"])
    return {"workload": f"D3Q19 Taylor-Green vortex {n}^3 periodic, Re={w['Re']:g}, "
                        f"Wi={w['Wi']:g}, beta={w['beta']:g}, u0={w['U0']:g}, {prec} fused step",
            "lattice": w["lattice"], "grid": [n] * 3, "precision": prec,
            "kernel": "fused", "l2": "state 18.7 GB >> 129 MB L2; no flush needed",
            "parallelism": "replicas", "note": note}


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------

def aggregate(dt_local, units_local, dist):
    """Whole-job rate of weakly scaled replicas: the units of all ranks over
    the slowest rank's time (max over ranks).  Returns (dt_max, units_total)."""
    if dist is None:
        return dt_local, units_local
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([dt_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def time_steps(sim, steps, stream):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def pinned_f64(shape):
    """A page-locked host float64 array (torch's pinned host allocator)."""
    import torch

    n = 1
    for s in shape:
        n *= s
    return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy().reshape(shape)


def run_ours(args, rank, world, dist):
    import torch

    from paper_2506_13072_gb300 import fvlb as F

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    F.use_torch_allocator()
    stream = torch.cuda.current_stream()
    prec = F.PRECISIONS[args.precision]
    scheme = F.FVLB_SCHEME_ORIGINAL if args.scheme == "original" else F.FVLB_SCHEME_PRESENT
    launches = 3 if scheme == F.FVLB_SCHEME_ORIGINAL else 1     # per step

    # The initial fields live in page-locked host buffers, written in place
    # by the workload generator; the same buffers feed the end-to-end leg.
    pr = main_problem(args, fields=False)
    u0 = pinned_f64(pr.shape + (pr.D,))
    p0 = pinned_f64(pr.shape)

    def fill_inputs():
        if args.lattice == "d3q19":
            tgv_problem(pr.nx, out_u=u0, out_p=p0)
        else:
            u0[...] = 0.0           # the four-roll mill starts at rest
            p0[...] = 0.0

    fill_inputs()
    log("fields built")
    sim = F.Simulation.from_problem(pr, precision=prec, kernel=F.FVLB_KERNEL_FUSED,
                                    stream=stream, scheme=scheme)
    sim.init_fields(u0, p0, None)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    log("warm")

    sites = pr.sites
    with ClockSampler(local) as clk:
        # more identical untimed steps until the clock sampler is reporting,
        # so that its samples cover the timed region and the steps just before
        preroll = clk.wait_for_samples(2, lambda: (sim.step(10), torch.cuda.synchronize()))
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        w0 = time.monotonic()
        dt = time_steps(sim, args.steps, stream)
        torch.cuda.synchronize()
        w1 = time.monotonic()
        time.sleep(0.06)
    clocks = clk.summary(min(w0, w1 - 0.3), w1 + 0.02)
    clocks["window"] = "timed region and the identical steps just before it"
    dt, units = aggregate(dt, sites * args.steps, dist)
    if dist is not None:
        dist.barrier()
    log(f"timed {args.steps} steps: {1e3 * dt / args.steps:.3f} ms/step")
    diag = sim.reduce(check_finite=False)
    bpu = sim.bytes_per_update()

    # End to end through the public API with host buffers: upload of the
    # initial fields (u, p; A = I is the library's rest default), K steps,
    # download of the velocity field, all inside the timed region.  The same
    # handle and page-locked buffers as above; the velocity is read back into
    # the u buffer (the upload has completed when fvlb_init_fields returns).
    sim.fields(F.FVLB_FIELD_U, u0.reshape(-1))      # first call allocates its buffer
    fill_inputs()
    sim.init_fields(u0, p0, None)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    sim.init_fields(u0, p0, None)
    sim.step(args.steps)
    sim.fields(F.FVLB_FIELD_U, u0.reshape(-1))
    e2e_dt = time.perf_counter() - t0
    sim.close()
    e2e_dt, e2e_units = aggregate(e2e_dt, sites * args.steps, dist)
    h2d = (u0.nbytes + p0.nbytes) / args.steps
    d2h = u0.nbytes / args.steps
    log("end to end done")

    value = units / dt / 1e6
    launch_s = dt / args.steps                 # one fused launch per step
    achieved = bpu * sites / launch_s / 1e9    # GB/s, algorithmic bytes
    peaks, which = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    tr = (traffic_record(f"{args.lattice}_{args.n or 'default'}_{args.precision}_fused")
          if launches == 1 else None)

    if rank != 0:
        return
    del u0, p0
    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = cpu_baseline()
        log("cpu baseline done")
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32"}.get(args.precision, "f32 (16-bit storage)"),
        "data": "synthetic (seeded Taylor-Green initial field of Sec. 3.4)",
        "config": config_dict(args, "" if launches == 1 else "original scheme"),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": tr["dram_bytes_per_launch"] if tr else None,
                     "algorithmic_bytes_per_launch": bpu * sites,
                     "bytes_per_update": bpu, "peak_source": f"{which} hbm_gbs (copy)",
                     "kernel": kernel_label(args.lattice, args.precision)
                               + ("" if launches == 1 else
                                  "; original scheme: k_taup + k_fdiv + this kernel "
                                  "(ORIG) per step, state bytes over the step time")},
        "e2e": {"value": round(e2e_units / e2e_dt / 1e6, 1), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "fvlb_init_fields(u, p) from page-locked host memory + K steps + "
                        "fvlb_fields(U) to page-locked host memory, one handle"},
        "gpu_launches": args.steps * launches,
        "clocks": clocks,
        "preroll_steps": 10 * preroll,
        "diagnostics": {"KE": diag["KE"], "PE": diag["PE"], "nonfinite": diag["nonfinite"]},
        "host_maxrss_mb": maxrss_mb(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# The other forms (--forms / --form NAME), each in a process of its own
# ---------------------------------------------------------------------------

# name -> (lattice, n, precision, kernel, scheme, model, model parameter)
FORMS = {
    "d3q19_256_fp16_dev": ("d3q19", 256, "fp16_dev", 0, 0, 0, 0.0),
    "d3q19_256_bf16_dev": ("d3q19", 256, "bf16_dev", 0, 0, 0, 0.0),
    "d3q19_256_fp64": ("d3q19", 256, "fp64", 0, 0, 0, 0.0),
    "d3q19_256_fp32_split": ("d3q19", 256, "fp32", 1, 0, 0, 0.0),
    "d3q19_256_fp32_original": ("d3q19", 256, "fp32", 0, 1, 0, 0.0),
    "d3q19_256_fp32_original_split": ("d3q19", 256, "fp32", 1, 1, 0, 0.0),
    "d3q19_256_fp32_giesekus": ("d3q19", 256, "fp32", 0, 0, 1, 0.3),
    "d3q19_256_fp32_ptt_exp": ("d3q19", 256, "fp32", 0, 0, 3, 0.25),
    "d2q9_2048_fp32": ("d2q9", 2048, "fp32", 0, 0, 0, 0.0),
    "d2q9_2048_fp16_dev": ("d2q9", 2048, "fp16_dev", 0, 0, 0, 0.0),
    "d2q9_2048_fp32_split": ("d2q9", 2048, "fp32", 1, 0, 0, 0.0),
    "d2q9_2048_fp32_original": ("d2q9", 2048, "fp32", 0, 1, 0, 0.0),
    "d2q9_2048_fp32_original_split": ("d2q9", 2048, "fp32", 1, 1, 0, 0.0),
}
SPECIAL_FORMS = ["batched_fp32", "batched_fp16", "one_by_one_fp32", "closure"]


def form_rate(F, pr, precision, steps, warmup, stream, kernel=0, scheme=0):
    import torch

    s = F.Simulation.from_problem(pr, precision=precision, kernel=kernel, stream=stream,
                                  scheme=scheme)
    s.init_fields(pr.u0, pr.p0, None)
    s.step(warmup)
    torch.cuda.synchronize()
    dt = time_steps(s, steps, stream)
    bpu = s.bytes_per_update()
    s.close()
    mlups = pr.sites * steps / dt / 1e6
    return {"mlups": round(mlups, 1), "gbs_algorithmic": round(bpu * pr.sites * steps / dt / 1e9, 1),
            "bytes_per_update": bpu, "ms_per_step": round(1e3 * dt / steps, 4)}


def batch_rate(F, precision, stream, steps=40):
    """512 uneven D2Q9 instances (four-roll / Poiseuille, n log-uniform in
    [32, 512], seed 0) in one persistent launch per step, graph-replayed,
    tile shape autotuned (the tuning steps run before the timed region)."""
    import torch

    from paper_2506_13072_gb300 import workloads as W

    probs = W.batch_instances(count=512, seed=0)
    stream = torch.cuda.Stream()      # graph capture needs a non-legacy stream
    bt = F.Batch(probs, precision=precision, stream=stream)
    bt.step(1 + 18 + 2)        # first step, autotuning, one graph replay
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bt.step(steps)
    e1.record(stream)
    e1.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    info = bt.info()
    bt.close()
    sites = info["sites"]
    return {"mlups": round(sites * steps / dt / 1e6, 1),
            "gbs_algorithmic": round(info["bytes_per_update"] * sites * steps / dt / 1e9, 1),
            "bytes_per_update": info["bytes_per_update"], "ms_per_step": round(1e3 * dt / steps, 4),
            "sites": sites, "instances": 512, "tile": [32 * info["gx"], info["rows"]],
            "launches_per_step": 1}


def one_by_one_rate(F, precision, stream, steps=10):
    """The same 512 instances as batch_rate, each its own handle stepped by
    its own fused launch through the public API (512 launches a step): the
    baseline the batched form replaces."""
    import torch

    from paper_2506_13072_gb300 import workloads as W

    probs = W.batch_instances(count=512, seed=0)
    sims = [F.Simulation.from_problem(p, precision=precision, stream=stream) for p in probs]
    for s in sims:
        s.init_fields()
        s.step(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        for s in sims:
            s.step(1)
    e1.record(stream)
    e1.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    sites = sum(p.sites for p in probs)
    bpu = sims[0].bytes_per_update()
    for s in sims:
        s.close()
    return {"mlups": round(sites * steps / dt / 1e6, 1),
            "gbs_algorithmic": round(bpu * sites * steps / dt / 1e9, 1),
            "bytes_per_update": bpu, "ms_per_step": round(1e3 * dt / steps, 4),
            "sites": sites, "instances": 512, "launches_per_step": 512}


def closure_rate(F, stream, steps=10, n=None):
    """D3Q19 Taylor-Green 256^3 (or n^3) FP32 with the learned closure: the network is
    trained on pairs from Taylor-Green 32^3 runs of the plain method (Wi 1 and
    0.2; relative loss), then replaces chi where its per-node residual is
    within 1e-2."""
    import torch

    from paper_2506_13072_gb300 import workloads as W

    net = F.Mlp(F.FVLB_D3Q19, capacity=1 << 20, seed=0)
    for Wi in (1.0, 0.2):
        small = W.taylor_green_3d(n=32, U0=0.02, Re=100, Wi=Wi, beta=0.5)
        s = F.Simulation.from_problem(small, precision=F.FVLB_FP32)
        s.init_fields(small.u0, small.p0, small.A0)
        for _ in range(8):
            s.step(100)
            net.collect(s, stride=5)
        s.close()
    net.set_loss(1e-3)
    for nt, b, lr in ((10000, 1024, 2e-3), (10000, 2048, 5e-4), (10000, 4096, 1e-4)):
        net.train(nt, batch=b, lr=lr)
    pr = tgv_problem(n or WORKLOAD["n"])
    sim = F.Simulation.from_problem(pr, precision=F.FVLB_FP32, stream=stream)
    sim.init_fields(pr.u0, pr.p0, None)
    pr.u0 = pr.p0 = None
    sim.set_closure(net, tol=1e-2)
    sim.step(3)
    torch.cuda.synchronize()
    dt = time_steps(sim, steps, stream)
    st = sim.closure_stats()
    bpu = sim.bytes_per_update()
    sim.close()
    net.close()
    tot = st["network"] + st["fallback"]
    return {"mlups": round(pr.sites * steps / dt / 1e6, 1),
            "gbs_algorithmic": round(bpu * pr.sites * steps / dt / 1e9, 1),
            "bytes_per_update": bpu, "ms_per_step": round(1e3 * dt / steps, 4),
            "network_share_of_node_updates": round(st["network"] / max(1, tot), 4),
            "tol": 1e-2}


def run_form(args):
    """One form alone (single GPU); prints its JSON line."""
    import torch

    from paper_2506_13072_gb300 import fvlb as F
    from paper_2506_13072_gb300 import workloads as W

    torch.cuda.set_device(0)
    F.use_torch_allocator()
    stream = torch.cuda.current_stream()
    name = args.form
    steps = max(5, args.steps)
    if name in FORMS:
        lat, n, precision, kernel, scheme, model, mpar = FORMS[name]
        n = args.n or n
        if lat == "d3q19":
            pr = tgv_problem(n)
            work = f"D3Q19 Taylor-Green {n}^3 (Re 100, Wi 1, beta 0.5)"
        else:
            pr = W.four_roll(n=n, Wi=0.5, beta=0.5)
            work = f"D2Q9 four-roll mill {n}^2 (Wi 0.5, beta 0.5)"
        pr.model, pr.mpar = model, mpar
        work += (f", {precision}, {'split' if kernel else 'fused'} kernel, "
                 f"{'original' if scheme else 'present'} scheme"
                 + (f", model {model} ({mpar:g})" if model else ""))
        r = form_rate(F, pr, F.PRECISIONS[precision], steps, 3, stream, kernel=kernel,
                      scheme=scheme)
    elif name.startswith("batched"):
        prec = F.FVLB_FP32 if name == "batched_fp32" else F.FVLB_FP16_DEV
        r = batch_rate(F, prec, stream, steps=max(steps, 40))
        work = "512 uneven D2Q9 grids (n log-uniform in [32, 512]), one launch per step"
    elif name == "one_by_one_fp32":
        r = one_by_one_rate(F, F.FVLB_FP32, stream, steps=10)
        work = "the same 512 D2Q9 grids, one handle and one fused launch each per step"
    else:
        r = closure_rate(F, stream, steps=steps, n=args.n or None)
        work = f"D3Q19 Taylor-Green {args.n or WORKLOAD['n']}^3 FP32 with the learned closure"
    peaks, which = measured_peaks()
    r["frac_of_hbm_peak"] = round(r["gbs_algorithmic"] / float(peaks.get("hbm_gbs", 6800.0)), 3)
    r["peak_source"] = f"{which} hbm_gbs (copy)"
    print(json.dumps({"form": name, "workload": work, "unit": UNIT, **r,
                      "host_maxrss_mb": maxrss_mb()}), flush=True)


def run_forms(args):
    """Every form, each in a subprocess of its own; prints one JSON line per
    form (a failed form prints its exit status instead)."""
    for name in list(FORMS) + SPECIAL_FORMS:
        cmd = [sys.executable, os.path.abspath(__file__), "--form", name,
               "--steps", str(args.steps)]
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
            lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
            if r.returncode == 0 and lines:
                print(lines[-1], flush=True)
            else:
                print(json.dumps({"form": name, "failed": r.returncode,
                                  "stderr_tail": r.stderr[-600:]}), flush=True)
        except subprocess.TimeoutExpired:
            print(json.dumps({"form": name, "failed": "timeout"}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="(accepted; forms run only with --forms)")
    ap.add_argument("--forms", action="store_true", help="time every other form, one process each")
    ap.add_argument("--lattice", default="d3q19", choices=["d3q19", "d2q9"])
    ap.add_argument("--n", type=int, default=0, help="grid nodes per axis (0: the default workload)")
    ap.add_argument("--precision", default="fp32",
                    choices=["fp64", "fp32", "fp16_dev", "bf16_dev", "fp16_dev_sr", "bf16_dev_sr"])
    ap.add_argument("--scheme", default="present", choices=["present", "original"],
                    help="original: the comparison scheme of Tables 1-2 (profiling)")
    ap.add_argument("--form", default="", choices=[""] + list(FORMS) + SPECIAL_FORMS,
                    help="time only this form and print its line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.forms:
        run_forms(args)
        return
    if args.form:
        run_form(args)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
