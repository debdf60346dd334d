#!/usr/bin/env python3
"""Benchmark of the exponential-integrator Fourier pseudospectral Maxwell step on GB300.

Headline workload: 512^3 grid on [0, 2pi]^3, eps = mu = 1, seeded random
divergence-free fields (Gaussian spectrum, sigma = 16), h = 0.02, K steps
(default 500) with the invariants reduced after every step, in the FP32
precision form (FFTs and update in FP32, phase c|k|h in FP64, invariant sums
in FP64).  One step is the whole method: forward 3D R2C of the six real
fields, the exact exponential update with the invariant sums, inverse 3D C2R
back to the six real fields.  Beside it the same workload is timed in FP64,
and in the spectral-resident form (state kept as the spectrum at load, step n
writes R(t_n) applied to it: one HBM pass per step), FP32 and FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Rank 0 prints one JSON line.  Under torchrun (N > 1) every rank runs an
independent replica of the workload on its own GPU (the path needs no data
exchange); value = all ranks' field-point-steps / max-over-ranks time.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "field-point-steps/s + %HBM roofline at 512^3 (FP32 vs FP64); serve p50/p99"
UNIT = "field-point-steps/s"
GRID = (512, 512, 512)
H = 0.02
SIGMA = 16.0
SEED = 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=512, help="cubic grid size (default 512)")
    ap.add_argument("--shape", type=int, nargs=3, default=None, metavar=("NX", "NY", "NZ"),
                    help="a non-cubic grid for the headline form only (small profiling cases; implies "
                         "--no-secondary)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the FP64 and literal-form lines")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline")
    ap.add_argument("--only", choices=["dft8", "batch"], default=None,
                    help="dft8: only the tensor-core DFT-as-GEMM evaluation; batch: only the batched form "
                         "(64 uneven FP32 instances, spectral form; --steps steps); one JSON line, for profiling")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6800.0, "fallback (6.8 TB/s)"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thr.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {
            "sm_mhz": float(np.median(sm)) if sm else None,
            "sm_max_mhz": float(max(smax)) if smax else None,
            "reasons": sorted(reasons),
            "samples": len(sm),
        }


def gpu_smi_id(torch, dev):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if dev < len(ids):
            return ids[dev]
    try:
        return f"GPU-{torch.cuda.get_device_properties(dev).uuid}"
    except Exception:
        return dev


# ------------------------------------------------------------------ timing
def timed_steps(torch, solver, stream, h, steps, warmup, dist=None, clocks=None):
    """Warm up, then time `steps` steps with CUDA events on the solver's stream."""
    solver.step(h, warmup, 1)
    solver.sync()
    solver.profile(True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    ncu_range = bool(os.environ.get("MX_NCU_RANGE"))  # profiler range around the timed steps (ncu --profile-from-start off)
    if ncu_range:
        torch.cuda.profiler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(h, steps, 1)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    if ncu_range:
        torch.cuda.profiler.stop()
    ck = clocks.stop() if clocks else None
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    prof = solver.profile_read()
    solver.profile(False)
    return ms, prof, ck


def max_over_ranks(torch, dist, v):
    """Largest value over ranks (the slowest rank's time); NCCL reduces on the GPU, gloo on the host."""
    if dist is None:
        return v
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, units_per_rank, ms):
    """Replicas: every rank processes units_per_rank; throughput = all units / slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


# kernel kind (as profiled by the library) -> kernel template and the sources it is built from
KERNEL_NAMES = {
    "x_r2c": "k_x_r2c_tma (x-direction R2C, six fields)",
    "x_c2r": "k_x_c2r_tma (x-direction C2R, six fields)",
    "y_fft": "k_fft_strided_tma2 / k_fft_strided_tma (y-direction, six components, two-stage or one-stage "
             "tensor-copy variant as scheduled; forward and inverse launches)",
    "z_fft": "k_fft_strided (z-direction, six components)",
    "z_fused": "k_z_fused_tma (z forward + exponential update + invariants + z inverse, tensor-copy prefetch)",
    "spectral": "k_spectral_grp / k_spectral_tma (exponential update + invariants; rows sharing |k|^2 grouped when Mx is a multiple of 128)",
}
KERNEL_SOURCES = {
    "x_r2c": ["mx_fft.cuh", "mx_tma.cuh", "mx_kernels.cuh", "mx_xpass_tma.cuh", "mx_fft_launch.cuh", "mx_fft_f32.cu"],
    "x_c2r": ["mx_fft.cuh", "mx_tma.cuh", "mx_kernels.cuh", "mx_xpass_tma.cuh", "mx_fft_launch.cuh", "mx_fft_f32.cu"],
    "y_fft": ["mx_fft.cuh", "mx_tma.cuh", "mx_kernels.cuh", "mx_strided_tma.cuh", "mx_tmap.h", "mx_fft_launch.cuh",
              "mx_fft_f32s.cu"],
    "z_fft": ["mx_fft.cuh", "mx_tma.cuh", "mx_kernels.cuh", "mx_strided_tma.cuh", "mx_tmap.h", "mx_fft_launch.cuh",
              "mx_fft_f32s.cu"],
    "z_fused": ["mx_fft.cuh", "mx_tma.cuh", "mx_kernels.cuh", "mx_tmap.h", "mx_fft_launch.cuh", "mx_zfused.cuh",
                "mx_zfused_f32b.cu"],
    "spectral": ["mx_fft.cuh", "mx_tma.cuh", "mx_kernels.cuh", "mx_spectral_tma.cuh", "mx_spectral.cu"],
}


def npoints(grid):
    """Grid points of a cubic size or an (nx, ny, nz) shape."""
    return int(np.prod(grid)) if isinstance(grid, (tuple, list)) else grid ** 3


def pass_bytes(kind, grid, es):
    """Algorithmic bytes of one launch of a pass over all six components: read and write six components'
    worth of the packed half spectrum (N_S / 2 complex values each), equal to six real fields."""
    return 12 * (npoints(grid) // 2) * 2 * es


def traffic_for(key):
    """dram bytes per launch from the committed ncu summary, if it matches the current sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(key)
    if not ent:
        return None
    if ent.get("source_sha") != source_sha(key.split("_fp")[0]):
        return None
    return ent.get("bytes_per_launch")


def source_sha(kind):
    """Hash of the sources the kernel of this kind is built from."""
    import hashlib

    hsh = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2210_06232_gb300", "csrc")
    for f in KERNEL_SOURCES.get(kind, sorted(os.listdir(csrc))):
        hsh.update(open(os.path.join(csrc, f), "rb").read())
    return hsh.hexdigest()[:16]


# ------------------------------------------------------------------ forms
def run_form(torch, mx, grid, precision, form, steps, warmup, stream, dist=None, clocks=None, keep=False):
    n = tuple(grid) if isinstance(grid, (tuple, list)) else (grid, grid, grid)
    lo, hi = (0.0, 0.0, 0.0), (2 * np.pi,) * 3
    s = mx.Solver(n, lo, hi, 1.0, 1.0, precision, form, stream=stream)
    s.autotune()  # kernel variant and grid per pass of this shape (cached per process)
    s.load_random(SEED, SIGMA)
    ms, prof, ck = timed_steps(torch, s, stream, H, steps, warmup, dist, clocks)
    inv = s.invariants()
    if not keep:
        s.close()
        s = None
    return s, ms, prof, ck, inv


def drift(inv):
    e0 = inv[0]["E1"]
    return float(max(abs(r["E1"] - e0) for r in inv) / abs(e0))


# flops per k-point (one of the N_S/2 points of the packed half spectrum) of the exponential update
# (Apply: k.H, k.E, k x E, k x H and the six updated components) and of the fifteen invariant sums
UPDATE_FLOPS_PER_K = 116
INVARIANT_FLOPS_PER_K = 90


def step_flops(grid, form):
    """Algorithmic flops of one step: 2.5 N log2 N per real 3D transform of N = grid^3 points (half the
    classic 5 N log2 N of a complex one), six fields forward and inverse in the literal form (none in the
    spectral-resident form, the z transforms in the xy-resident one), plus the update and the invariant
    sums at every k-point."""
    ns = npoints(grid)
    nz = grid[2] if isinstance(grid, (tuple, list)) else grid
    # xy-resident form: the z share of those transforms only (30 N log2 N splits as 30 N log2 of each axis)
    fft = {0: 6 * 2 * 2.5 * ns * np.log2(ns), 1: 0.0, 2: 6 * 2 * 2.5 * ns * np.log2(nz)}[form]
    return fft + (ns / 2) * (UPDATE_FLOPS_PER_K + INVARIANT_FLOPS_PER_K)


def form_entry(name, grid, precision, form, ms, steps, prof, peak, inv, world, alu_peak=None):
    ns = npoints(grid)
    es = 8 if precision == 0 else 4
    step_ms = ms / steps
    value = world * ns * steps / (ms / 1e3)
    min_bytes = 12 * ns * es
    passes = sum(v[1] for k, v in prof.items() if k not in ("table", "gen")) / steps
    e = {
        "value": value,
        "unit": UNIT,
        "ms_per_step": step_ms,
        "dtype": "f64" if precision == 0 else "f32",
        "form": {0: "literal (3D R2C -> update -> 3D C2R per step)", 1: "spectral-resident (absolute time)",
                 2: "xy-resident (state: x-y spectrum; z forward -> update -> z inverse per step)"}[form],
        "hbm_passes_per_step": passes,
        "step_hbm_roofline_frac": (min_bytes / (step_ms / 1e3) / 1e9) / peak,
        "energy_rel_drift": drift(inv),
        "kernels_ms_per_step": {k: v[0] / steps for k, v in prof.items() if v[1]},
    }
    if alu_peak:
        fl = step_flops(grid, form)
        ach = fl / (step_ms / 1e3)
        e["alu_roofline"] = {"bound": "alu", "pipe": "fp64" if precision == 0 else "fp32",
                             "algorithmic_flops_per_step": fl, "achieved_flops": ach, "peak_flops": alu_peak,
                             "peak_source": "measured in this run (mx_fma_peak: FMA chains on every SM, "
                                            "an FMA counting two flops)", "frac": ach / alu_peak}
    return name, e


BATCH_SHAPES = [(32, 32, 32), (48, 64, 80), (64, 64, 64), (96, 96, 64), (128, 128, 128)]


def batch_run(torch, mx, peak, steps, warmup, stream, ninst=64, seed=4, form=None):
    """Batched form: 64 FP32 instances of uneven grids, eps, mu in [1, 4], h in [0.01, 0.1], sigma = 8.
    Spectral form: every step of every instance in one persistent cooperative launch per mx_batch_step
    call.  Literal form: each instance's autotuned x, y, fused z, y, x passes per step, all instances as
    parallel branches of one CUDA graph per call."""
    form = mx.MX_FORM_SPECTRAL if form is None else form
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(ninst):
        n = BATCH_SHAPES[rng.integers(len(BATCH_SHAPES))]
        specs.append(dict(n=n, eps=float(rng.uniform(1, 4)), mu=float(rng.uniform(1, 4)), h=float(rng.uniform(0.01, 0.1))))
    b = mx.Batch(specs, mx.MX_FP32, stream=stream, form=form)
    b.load_random(seed, 8.0)
    b.step(steps, 1)  # warm-up call: captures the graph for this step count
    b.sync()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps, 1)
    e1.record(stream)
    e1.synchronize()
    b.sync()
    ms = e0.elapsed_time(e1)
    pts = sum(int(np.prod(sp["n"])) for sp in specs)
    drift = 0.0
    for i in range(ninst):
        inv = b.instance(i).invariants()
        e = [r["E1"] for r in inv]
        drift = max(drift, (max(e) - min(e)) / e[0])
    used = b.graph_used()
    shape = b.launch_shape()
    b.close()
    min_bytes = 12 * pts * 4
    return {
        "form": "literal (graph of per-instance pass chains)" if form == mx.MX_FORM_LITERAL
                else "spectral-resident (one persistent launch)",
        "value": pts * steps / (ms / 1e3),
        "unit": UNIT,
        "ms_per_step": ms / steps,
        "instances": ninst,
        "field_points": pts,
        "shapes": {"x".join(map(str, sh)): sum(1 for sp in specs if tuple(sp["n"]) == sh) for sh in BATCH_SHAPES},
        "launches_per_call": 1 if form != mx.MX_FORM_LITERAL else None,
        "persistent_launch": {"blocks": shape[0], "threads_per_block": shape[1]} if shape[0] else None,
        "graph_replayed": used,
        "step_hbm_roofline_frac": (min_bytes / (ms / steps / 1e3) / 1e9) / peak,
        "energy_rel_drift_max": drift,
        "dtype": "f32",
    }


SERVE_SHAPES = [(32, 32, 32), (64, 64, 64), (96, 96, 96), (128, 128, 128), (192, 192, 192)]
# offered rate of the multi-step scenario (mean ~650 steps per request): about what one GB300 sustains
SERVE_MULTISTEP_RATE = 8.0


def serve_run(torch, mx, duration=5.0, rate=200.0, seed=5, budget=32 << 30, multistep=False):
    """Serving form: Poisson arrivals (mean `rate`/s) of solves with grids from SERVE_SHAPES, t_end ~ U[1, 50],
    eps, mu ~ U[1, 4], FP32 or FP64 (50/50), random divergence-free initial fields; p50/p99 latency (submission
    to completion), solves/s and the device concurrency the server recorded.  multistep=False: each request is
    the paper's single step of size t_end; True: ceil(t_end / h) steps with h ~ U[0.01, 0.1]."""
    import threading

    rng = np.random.default_rng(seed)
    inputs, outs = {}, {}
    for sh in SERVE_SHAPES:
        for prec in (mx.MX_FP32, mx.MX_FP64):
            dt = torch.float64 if prec == mx.MX_FP64 else torch.float32
            g = mx.Solver(sh, (0, 0, 0), (2 * np.pi,) * 3, 1.0, 1.0, prec, mx.MX_FORM_SPECTRAL)
            g.load_random(seed + sh[0], 8.0)
            E = torch.empty((3,) + sh, dtype=dt).pin_memory()
            H = torch.empty_like(E).pin_memory()
            g.read(E, H)
            g.close()
            inputs[(sh, prec)] = (E, H)
            outs[(sh, prec)] = [(torch.empty_like(E).pin_memory(), torch.empty_like(H).pin_memory()) for _ in range(6)]
    srv = mx.Server(budget, max_active=64)
    free = {k: list(v) for k, v in outs.items()}
    lock = threading.Lock()

    def submit(sh, prec, t_end, eps, mu, nsteps=1):
        E0, H0 = inputs[(sh, prec)]
        with lock:
            pool = free[(sh, prec)]
            Eo, Ho = pool.pop() if pool else (torch.empty_like(E0).pin_memory(), torch.empty_like(H0).pin_memory())
        rid = srv.submit(sh, E0, H0, Eo, Ho, t_end, eps, mu, prec, nsteps, 0)
        return rid, (sh, prec, Eo, Ho)

    def release(tag):
        sh, prec, Eo, Ho = tag
        with lock:
            free[(sh, prec)].append((Eo, Ho))

    # warm-up: one request per class (creates and tunes the pooled contexts)
    for sh in SERVE_SHAPES:
        for prec in (mx.MX_FP32, mx.MX_FP64):
            rid, tag = submit(sh, prec, 1.0, 1.0, 1.0)
            srv.wait(rid)
            srv.result(rid)
            release(tag)
    # arrivals
    n = int(duration * rate)
    gaps = rng.exponential(1.0 / rate, size=n)
    plan = []
    for _ in range(n):
        sh = SERVE_SHAPES[rng.integers(len(SERVE_SHAPES))]
        prec = mx.MX_FP32 if rng.random() < 0.5 else mx.MX_FP64
        t_end, eps, mu = float(rng.uniform(1, 50)), float(rng.uniform(1, 4)), float(rng.uniform(1, 4))
        nsteps = int(np.ceil(t_end / rng.uniform(0.01, 0.1))) if multistep else 1
        plan.append((sh, prec, t_end, eps, mu, nsteps))
    import queue as _q

    pending = _q.Queue()
    lat, done_t = [], []

    def collector():  # waits in submission order, returns output buffers to the pool
        while True:
            item = pending.get()
            if item is None:
                return
            rid, tag = item
            if srv.wait(rid, 120.0) == 2:
                _, l = srv.result(rid)
                lat.append(l)
                done_t.append(time.perf_counter())
            release(tag)

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    due = t0
    for gap, (sh, prec, t_end, eps, mu, nsteps) in zip(gaps, plan):
        due += gap
        now = time.perf_counter()
        if due > now:
            time.sleep(due - now)
        pending.put(submit(sh, prec, t_end, eps, mu, nsteps))
    t_sub = time.perf_counter()
    pending.put(None)
    th.join()
    ok = len(lat)
    t1 = max(done_t) if done_t else time.perf_counter()
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    steps_total = sum(p[5] for p in plan)
    return {
        "device_concurrency": {"max_requests": st["max_concurrent"], "mean_requests_while_busy": st["mean_concurrent"],
                               "busy_s": st["busy_s"], "sum_request_s": st["request_s_sum"],
                               "overlap": st["request_s_sum"] / st["busy_s"] if st["busy_s"] > 0 else None,
                               "what": "requests admitted and not finished at once (time-weighted over the time "
                                       "at least one was); overlap = summed admission-to-completion time / busy "
                                       "time (1: one at a time)"},
        "steps_per_request_mean": steps_total / max(n, 1),
        "requests": n,
        "completed": ok,
        "offered_rate_per_s": rate,
        "solves_per_s": ok / (t1 - t0),
        "arrival_window_s": t_sub - t0,
        "p50_ms": float(np.percentile(lat, 50) * 1e3) if ok else None,
        "p99_ms": float(np.percentile(lat, 99) * 1e3) if ok else None,
        "mean_ms": float(lat.mean() * 1e3) if ok else None,
        "hbm_budget_gb": budget / 1e9,
        "hbm_high_water_gb": st["hbm_high_water"] / 1e9,
        "rejected": st["rejected"],
        "work": ("ceil(t_end / h) steps, h ~ U[0.01, 0.1], per request" if multistep else
                 "one exponential step of size t_end per request (Sec. 2.5)") +
                ", load + solve + read through pinned host buffers; grids 32^3..192^3, FP32/FP64 50/50, t_end ~ U[1,50]",
    }


def cufft_comparison(torch, grid, steps=20, warmup=3):
    """Timing comparison only (not part of the product): cuFFT through torch.fft, forward R2C and
    inverse C2R of six FP32 fields of grid^3 per step, with no update or invariants."""
    x = torch.randn(6, grid, grid, grid, device="cuda", dtype=torch.float32)
    dims = (1, 2, 3)
    for _ in range(warmup):
        y = torch.fft.rfftn(x, dim=dims)
        x = torch.fft.irfftn(y, s=(grid,) * 3, dim=dims)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        y = torch.fft.rfftn(x, dim=dims)
        x = torch.fft.irfftn(y, s=(grid,) * 3, dim=dims)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del x, y
    torch.cuda.empty_cache()
    return {"what": "cuFFT via torch.fft: rfftn + irfftn of six FP32 fields per step (transforms only, no update, "
                    "no invariants); a timing comparison, not used by the library",
            "ms_per_step": ms, "steps": steps}


def _oracle_worker(task):
    """One host core: oracle solves (Alg. 1 + Alg. 2, one step each) at grid^3 for about budget_s."""
    grid, budget_s = task
    import synth
    from oracle import scheme

    g = synth.Grid((grid,) * 3)
    E0, H0 = synth.random_divfree_fields(g, seed=SEED, sigma=min(SIGMA, grid / 4))
    n = 0
    t0 = time.perf_counter()
    while True:
        scheme.solve(E0, H0, g.lo, g.hi, 1.0, 1.0, H * (n + 1), check_imag=False)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return g.npoints * n, n


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.processor() or platform.machine()


def cpu_baseline_all_cores(budget_s=12.0, grid=64):
    """The same oracle on every host core at once: one process per core (spawned, one numpy thread
    each), each solving its own copy of a 64^3 sample; throughput = all points solved / wall time."""
    import multiprocessing as mp

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [(16, 0.0)] * cores)  # start-up and imports outside the timed region
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(grid, budget_s)] * cores)
        el = time.perf_counter() - t0
    pts = sum(r[0] for r in res)
    solves = sum(r[1] for r in res)
    return {
        "value": pts / el,
        "unit": UNIT,
        "cores": cores,
        "kind": "oracle",
        "cpu": cpu_model(),
        "sample": f"{solves} oracle solves (Alg. 1 + Alg. 2, one step each, numpy FP64) at {grid}^3 spread over "
                  f"{cores} spawned processes (one per core, one numpy thread each), {el:.1f} s wall",
    }


def dft_gemm_eval(torch, mx, tiles=None, reps=64):
    """Tensor-core DFT-as-GEMM against the FMA radix-8 stage (mx_dft8_stage_eval): `reps` stages of
    tiles of 128 8-point vectors held on chip (time = the stage's arithmetic and data movement).
    Error: relative L2 against the same stages in FP64 on the first tile."""
    import ctypes as C

    tiles = tiles or 8 * torch.cuda.get_device_properties(0).multi_processor_count
    rng = np.random.default_rng(8)
    x = (rng.standard_normal((tiles * 128, 8)) + 1j * rng.standard_normal((tiles * 128, 8))).astype(np.complex64)
    xin = torch.tensor(x, device="cuda")
    out = torch.empty_like(xin)
    k = np.arange(8)
    a = -2.0 * np.pi * (k + 1) / 64.0
    w = ((np.cos(a) / np.sqrt(8)).astype(np.float32).astype(np.float64) +
         1j * (np.sin(a) / np.sqrt(8)).astype(np.float32).astype(np.float64))
    F = np.exp(-2j * np.pi * np.outer(k, k) / 8)
    ref = x[:128].astype(np.complex128)
    for _ in range(reps):
        ref = (ref * w) @ F.T
    res = {}
    names = {0: "fma-butterfly", 1: "tcgen05-tf32x1", 3: "tcgen05-tf32x3", 6: "tcgen05-tf32x6"}
    for v in (0, 1, 3, 6):
        best = None
        for _ in range(3):
            ms = C.c_double(0)
            mx.check(mx.mx_dft8_stage_eval(v, xin.data_ptr(), out.data_ptr(), tiles, reps, C.byref(ms)),
                     "mx_dft8_stage_eval")
            best = ms.value if best is None else min(best, ms.value)
        y = out[:128].cpu().numpy().astype(np.complex128)
        dft8s = tiles * 128 * reps
        res[names[v]] = {"ms": best, "ns_per_dft8_stage": best * 1e6 / dft8s,
                         "rel_l2_vs_fp64": float(np.linalg.norm(y - ref) / np.linalg.norm(ref)),
                         "mma_tflops": (2.0 * 16 * 16 * v * dft8s / (best * 1e-3) / 1e12) if v else None}
    res["what"] = (f"{reps} radix-8 stages (twiddle + 8-point DFT) of {tiles} tiles x 128 vectors; tensor-core "
                   "variants: 128x16x16 kind::tf32 MMAs with 1/3/6 products of TF32-split operands, result in "
                   "tensor memory")
    return res


def cpu_baseline_sample(budget_s=15.0):
    """The FP64 oracle (numpy, as it stands) on the host cores: Alg. 1 + Alg. 2 at 128^3."""
    import synth
    from oracle import scheme

    g = synth.Grid((128, 128, 128))
    E0, H0 = synth.random_divfree_fields(g, seed=SEED, sigma=SIGMA)
    n = 0
    t0 = time.perf_counter()
    while True:
        scheme.solve(E0, H0, g.lo, g.hi, 1.0, 1.0, H * (n + 1), check_imag=False)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 50:
            break
    return {
        "value": g.npoints * n / el,
        "unit": UNIT,
        "cores": 1,
        "kind": "oracle",
        "cpu": cpu_model(),
        "sample": f"{n} oracle solves (Alg. 1 + Alg. 2, one step each, numpy FP64, single-threaded) "
                  f"at 128^3 with the same spectrum type, {el:.1f} s",
    }


def e2e_run(torch, mx, grid, steps, stream):
    """Public API with host buffers: load (H2D + forward transform), K steps, read (inverse + D2H)."""
    n = (grid, grid, grid)
    lo, hi = (0.0, 0.0, 0.0), (2 * np.pi,) * 3
    gen = mx.Solver(n, lo, hi, 1.0, 1.0, mx.MX_FP32, mx.MX_FORM_SPECTRAL, stream=stream)
    gen.load_random(SEED, SIGMA)
    shape = (3, grid, grid, grid)
    E = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    Hh = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    gen.read(E, Hh)
    gen.close()
    Eo = torch.empty_like(E).pin_memory()
    Ho = torch.empty_like(Hh).pin_memory()
    s = mx.Solver(n, lo, hi, 1.0, 1.0, mx.MX_FP32, mx.MX_FORM_LITERAL, stream=stream)
    s.autotune()
    # one untimed pass so allocations and module loading are out of the timed region
    s.load(E, Hh)
    s.step(H, 3, 1)
    s.read(Eo, Ho)
    s.invariants()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.load(E, Hh)
    s.step(H, steps, 1)
    s.read(Eo, Ho)
    inv = s.invariants()
    el = time.perf_counter() - t0
    s.close()
    nbytes = E.numel() * 4 * 2
    return {
        "value": grid ** 3 * steps / el,
        "unit": UNIT,
        "h2d_bytes_per_step": nbytes / steps,
        "d2h_bytes_per_step": (nbytes + len(inv) * 200) / steps,
        "seconds": el,
        "what": f"literal FP32 form: mx_load_fields(pinned host E0,H0) + mx_step(h, {steps}, invariants every "
                "step) + mx_read_fields(pinned host) + mx_read_invariants; host wall clock",
    }


def _oracle_solve(task):
    """One oracle solve (Alg. 1 + Alg. 2, one step of size t) at grid^3; returns its seconds."""
    grid, t = task
    import synth
    from oracle import scheme

    g = synth.Grid((grid,) * 3)
    E0, H0 = synth.random_divfree_fields(g, seed=SEED, sigma=min(SIGMA, grid / 4))
    t0 = time.perf_counter()
    scheme.solve(E0, H0, g.lo, g.hi, 1.0, 1.0, t, check_imag=False)
    return time.perf_counter() - t0


def reference_arm(args, rank, world):
    """The oracle as the reference arm, on every host core: each step is one oracle solve per core
    (spawned processes, one numpy thread each) of a sample of the 512^3 workload scaled down so that
    the whole run stays within a few minutes; value = points solved per second of wall time."""
    if rank != 0:
        return
    import multiprocessing as mp

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    total = args.steps + args.warmup
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        grid = 16
        for cand in (128, 96, 64, 48, 32, 16):
            dt = max(pool.map(_oracle_solve, [(cand, H)] * cores))
            if dt * total < 150.0:
                grid = cand
                break
        for i in range(args.warmup):
            pool.map(_oracle_solve, [(grid, H * (i + 1))] * cores)
        t0 = time.perf_counter()
        for i in range(args.steps):
            pool.map(_oracle_solve, [(grid, H * (i + 1))] * cores)
        el = time.perf_counter() - t0
    value = cores * grid ** 3 * args.steps / el
    sample = (f"oracle (numpy FP64) Alg. 1 + Alg. 2 solve at {grid}^3 on each of {cores} host cores per step "
              f"(spawned processes, one numpy thread each; the 512^3 workload's per-step work scaled down to fit "
              f"the time limit)")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded random divergence-free fields (host generator)",
        "config": {"workload": f"oracle sample at {grid}^3 per core of the 512^3 precision-form workload",
                   "grid": [grid] * 3},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def tile_stream_ceiling(torch, mx, n):
    """GB/s that HBM delivers for the fused z pass's access pattern without its arithmetic: tensor-copy
    tiles of 4 columns x n x 6 components of the n^3 spectrum (rows of 32 bytes at a stride of one z
    plane), and of 8 and 16 columns (64- and 128-byte rows) for comparison (mx_tile_stream, best of 5)."""
    m = n // 2
    buf = torch.zeros(6 * n * n * m * 2, dtype=torch.float32, device="cuda")
    try:
        return {str(8 * c): mx.tile_stream(buf.data_ptr(), m, n, n, c) for c in (4, 8, 16)}
    finally:
        del buf
        torch.cuda.empty_cache()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch

    from paper_2210_06232_gb300 import maxexp as mx

    torch.cuda.set_device(local)
    if args.only == "dft8":
        print(json.dumps({"dft_as_gemm_stage": dft_gemm_eval(torch, mx, tiles=2 * 152, reps=64)}), flush=True)
        return
    if args.only == "batch":
        st = torch.cuda.Stream()
        print(json.dumps({"batched": batch_run(torch, mx, peaks()[0], args.steps, args.warmup, st)}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as td

        td.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = td
    stream = torch.cuda.Stream()
    peak, peak_src = peaks()
    grid = tuple(args.shape) if args.shape else args.grid
    if args.shape:
        args.no_secondary = True
    clocks = ClockSampler(gpu_smi_id(torch, local))

    # headline: FP32 precision form, the whole step (R2C -> update + invariants -> C2R) every step
    sched_s, ms, prof, ck, inv = run_form(torch, mx, grid, mx.MX_FP32, mx.MX_FORM_LITERAL, args.steps, args.warmup,
                                          stream, dist, clocks, keep=True)
    schedule = sched_s.schedule()
    sched_s.close()
    ms = max_over_ranks(torch, dist, ms)
    ns = npoints(grid)
    value = whole_job_value(world, ns * args.steps, ms)
    # dominant kernel of the step: every pass reads and writes six components' worth of the
    # packed half spectrum (x passes: six real fields on the other side, the same bytes)
    dom = max((k for k in prof if k not in ("table", "gen") and prof[k][1]), key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    bytes_per_launch = pass_bytes(dom, grid, 4)
    achieved = bytes_per_launch / (dom_ms / dom_n / 1e3) / 1e9
    launches = int(sum(v[1] for v in prof.values()))
    # every pass of the step against the same peak (algorithmic bytes / mean launch time)
    per_pass = {}
    for k, (k_ms, k_n) in prof.items():
        if k in ("table", "gen") or not k_n:
            continue
        a_gbs = pass_bytes(k, grid, 4) / (k_ms / k_n / 1e3) / 1e9
        per_pass[k] = {"kernel": KERNEL_NAMES.get(k, k), "ms_per_launch": k_ms / k_n,
                       "launches_per_step": k_n / args.steps, "achieved_gbs": a_gbs, "frac": a_gbs / peak,
                       "traffic": traffic_for(f"{k}_fp32_{grid}") if not args.shape else None}
    forms = {}
    name, e = form_entry("precision_fp32_literal", grid, mx.MX_FP32, mx.MX_FORM_LITERAL, ms, args.steps, prof, peak,
                         inv, world)
    forms[name] = e

    alu = None
    if not args.no_secondary:
        alu = {"fp64_fma_flops": mx.fma_peak(mx.MX_FP64), "fp32_fma_flops": mx.fma_peak(mx.MX_FP32)}
        plan = [("fp64_literal", mx.MX_FP64, mx.MX_FORM_LITERAL, min(args.steps, 10)),
                ("spectral_resident_fp32", mx.MX_FP32, mx.MX_FORM_SPECTRAL, args.steps),
                ("xy_resident_fp32", mx.MX_FP32, mx.MX_FORM_XY, args.steps),
                ("spectral_resident_fp64", mx.MX_FP64, mx.MX_FORM_SPECTRAL, min(args.steps, 50)),
                ("xy_resident_fp64", mx.MX_FP64, mx.MX_FORM_XY, min(args.steps, 20))]
        for nm, p, f, k in plan:
            _, ms2, prof2, _, inv2 = run_form(torch, mx, grid, p, f, k, 3, stream, dist)
            ms2 = max_over_ranks(torch, dist, ms2)
            forms[nm] = form_entry(nm, grid, p, f, ms2, k, prof2, peak, inv2, world,
                                   alu_peak=alu["fp64_fma_flops"] if p == mx.MX_FP64 else None)[1]

    e2e = e2e_run(torch, mx, grid, args.steps, stream) if not args.shape else None
    rows = tile_stream_ceiling(torch, mx, grid) if not args.shape and grid <= 512 else None
    batched = None
    if not args.no_secondary:
        batched = batch_run(torch, mx, peak, min(args.steps, 100), args.warmup, stream)
        batched["literal_form"] = batch_run(torch, mx, peak, min(args.steps, 20), args.warmup, stream,
                                            form=mx.MX_FORM_LITERAL)
    comparison = None if args.no_secondary else {"cufft_transforms": cufft_comparison(torch, grid),
                                                 "dft_as_gemm_stage": dft_gemm_eval(torch, mx)}
    serve = None
    if not args.no_secondary and rank == 0:
        serve = serve_run(torch, mx)
        serve["multistep"] = serve_run(torch, mx, duration=5.0, rate=SERVE_MULTISTEP_RATE, multistep=True)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_sample()
        cpu["all_cores"] = cpu_baseline_all_cores()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic: seeded random divergence-free fields, Gaussian spectrum sigma=16 (device generator)",
        "config": {
            "workload": f"{'x'.join(map(str, grid)) if args.shape else str(grid) + '^3'} precision form: FFTs and update "
                        "in FP32, phase c|k|h and invariant sums in "
                        "FP64, eps=mu=1, h=0.02, invariants every step",
            "grid": list(grid) if args.shape else [grid] * 3,
            "form": "literal: forward 3D R2C, exponential update + invariants, inverse 3D C2R every step",
            "l2": "state 3.2 GB per pass > 129 MB L2: inputs larger than L2, no flush",
            "parallelism": f"replicas x{world}",
        },
        "roofline": {
            "kernel": KERNEL_NAMES[dom],
            "bound": "hbm",
            "achieved": achieved,
            "peak": peak,
            "peak_source": peak_src,
            "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": traffic_for(f"{dom}_fp32_{grid}") if not args.shape else None,
            "algorithmic_bytes_per_launch": bytes_per_launch,
            # the same bytes moved in the fused pass's tiles with no arithmetic: the ceiling of its
            # access pattern (rows of 32 bytes), measured in this run
            "pattern_ceiling": None if rows is None or dom != "z_fused" else {
                "gbs": rows["32"], "rows_bytes": 32, "frac": achieved / rows["32"],
                "source": "mx_tile_stream: tensor-copy tiles of 4 columns x 512 z x 6 components, read and "
                          "written back, no arithmetic"},
        },
        "tile_stream_gbs_by_row_bytes": rows,
        "step_hbm_roofline_frac": forms["precision_fp32_literal"]["step_hbm_roofline_frac"],
        "roofline_per_pass": per_pass,
        "schedule": schedule,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": ck,
        "forms": forms,
        "batched": batched,
        "serve": serve,
        "comparison": comparison,
        "alu_peaks": alu,
    }
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
