"""Benchmark: 32^4 SU(3) Landau gauge fixing by checkerboard overrelaxation on GB300.

One step = one pass of the whole hot path over the lattice: the even and the odd
half-sweep of Algorithm 1 (K(x), the three SU(2)-subgroup maximisers with omega = 1.7,
g(x) applied to the 8 links; links reunitarised after every 20th sweep inside the odd
half-sweep) and the stop check of Eqs. (1)-(3) after every sweep (F and the odd-site
theta fused into the odd half-sweep, the finishing reduction, and the even-site theta
pass wherever the odd part alone cannot decide the stop: on the last sweep of the
budget here), on FP32 links stored as 12 reals, timed through gf_fix (CUDA-graph
replay).  Metric: effective link bandwidth, the algorithmic link bytes of the run
(16 V b per sweep, b = 48 B, plus 4 V b once for the exact check) over its time.

Also reported: the roofline of the half-sweep kernel (8 V b per launch over its
CUDA-event duration, against the measured HBM copy bandwidth, with ncu's DRAM bytes per
launch when the profiled source is unchanged), the same metric end to end through the
C ABI with pinned host buffers, time to theta < 1e-15 for pure FP64 and for mixed
FP32 -> FP64 and FP32 -> double-float -> FP64 fixing, the double-float polish sweep,
Fourier-accelerated steepest descent, the differentiable F/theta, the batched
Coulomb-slice and ensemble workloads (throughput, and time until every unit is below
theta = 1e-15), SM clocks over the whole GPU arm, and the CPU oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--skip-units]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "32^4 SU(3) OR sweep link GB/s vs HBM peak; time to θ<1e-15, mixed vs FP64"
DIMS = (32, 32, 32, 32)
EPS_FIELD, SEED = 0.5, 3
OMEGA = 1.7
LINK_B = 48                    # FP32, 12 reals
V = DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]
# One step = one sweep and its stop check.  Algorithmic bytes: the sweep reads and writes
# every link twice (16 V b); the check adds nothing where it is fused (F and the odd-site
# theta in the odd half-sweep) and 4 V b on the sweeps whose odd part alone cannot decide.
STEP_BYTES = 16 * V * LINK_B
CHECK_BYTES = 4 * V * LINK_B
HALF_SWEEP_BYTES = 8 * V * LINK_B
# FP32 flops of one FP32-12 site update (an FMA counts 2): K from 8 links with their third
# rows rebuilt, 480; three subgroup maximisers with first-order overrelaxation, 102; two
# rotations of K and two of G (the first subgroup is written into G), 336; G applied to
# the 8 links, 1224 (4 third rows + 6 x 3 complex MACs per forward link, 6 x 3 per
# backward link)
FLOP_PER_SITE = 2142
WORKLOAD = "landau-32^4-fp32-12: OR sweep (even+odd, omega 1.7, reunit every 20) + F/theta stop check"


def profiled_value(profile: str, sources, key: str) -> int | None:
    """A counter recorded in a committed ncu summary (`key: value`), if the kernel's sources
    still hash to the value recorded there (otherwise it describes another kernel)."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    m_val = re.search(re.escape(key) + r":\s*(\d+)", text)
    if not m_hash or not m_val:
        return None
    h = hashlib.sha256()
    for src in sources:
        h.update(open(os.path.join(ROOT, "paper_1412_1498_gb300", "csrc", src), "rb").read())
    return int(m_val.group(1)) if h.hexdigest() == m_hash.group(1) else None


def profiled_traffic(profile: str, sources) -> int | None:
    """DRAM bytes per launch from a committed ncu summary (see profiled_value)."""
    return profiled_value(profile, sources, "dram_bytes_per_launch")


AD_SOURCES = ("gf_device.cuh", "gf_kernels.cuh", "gf_autograd.cuh", "gf_inst_autograd.cu")


def reduce_over_ranks(ms_total: float, steps: int, world: int, bytes_per_step: int, dist=None, device=None):
    """Whole-job throughput of a weak-scaling run: every rank processed its own lattice;
    the slowest rank's time counts.  Returns (max ms over ranks, GB/s of all ranks)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms_total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    return ms_total, world * bytes_per_step * steps / (ms_total * 1e-3) / 1e9


def timed_fix_launches(steps: int) -> int:
    """Kernels a one-lattice gf_fix(eps, steps) launches when every sweep runs: the opening
    check (the odd-site F/theta pass and its finish, then the even-site pass and a reset,
    which find nothing to do when the odd part decides), then per replayed graph three per
    captured sweep (even and odd half-sweep, the odd-part finish) and the even-site pass
    with the loop finish that close the graph (they work on the budget's last sweep only:
    every other sweep is decided by its odd part here).  The library picks the graph
    lengths (16, 8, 4, 2 or 1 sweeps) from the sweeps left as below."""
    captured, replays, left = 0, 0, steps
    while left > 0:
        k = 0
        while k < 4 and (16 >> (k + 1)) >= left:
            k += 1
        if (16 >> k) - left > 2 and k < 4:
            k += 1
        captured += 16 >> k
        replays += 1
        left -= 16 >> k
    return 4 + captured * 3 + 2 * replays


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def nvsmi_id(device) -> str:
    """nvidia-smi's name for the CUDA device `device` of this process.  nvidia-smi ignores
    CUDA_VISIBLE_DEVICES, so a CUDA ordinal may name another GPU there: the device's UUID
    (or, failing that, its PCI bus id) names the same physical GPU in both."""
    import torch
    props = torch.cuda.get_device_properties(device)
    uuid = getattr(props, "uuid", None)
    if uuid is not None:
        u = str(uuid)
        return u if u.startswith(("GPU-", "MIG-")) else "GPU-" + u
    bus = getattr(props, "pci_bus_id", None)
    if bus is not None:
        dom = getattr(props, "pci_domain_id", 0)
        dev = getattr(props, "pci_device_id", 0)
        return f"{dom:08x}:{bus:02x}:{dev:02x}.0"
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    idx = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    parts = [p for p in vis.split(",") if p.strip()]
    return parts[idx].strip() if idx < len(parts) else str(idx)


class ClockSampler:
    """nvidia-smi samples (every 100 ms) of SM clock and throttle reasons, with the time
    each arrived, from before the warm-up to the end of the GPU arm."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id, self.proc, self.lines = gpu_id, None, []
        self.windows = {}

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, name: str, t0: float, t1: float):
        """Remember a wall-clock window (perf_counter seconds) to summarise on its own."""
        self.windows[name] = (t0, t1)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self, window: str | None = None):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        lo, hi = self.windows.get(window, (-1e300, 1e300)) if window else (-1e300, 1e300)
        for when, line in self.lines:
            if not (lo <= when <= hi):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_field(dims=DIMS, eps=EPS_FIELD, seed=SEED):
    from paper_1412_1498_gb300 import fields
    return fields.random_gauge_config(dims, eps, seed)


# ------------------------------------------------------------------------------ CPU oracle
def oracle_steps(U, budget_s: float | None = None, max_steps: int | None = None, first: int = 0):
    """Oracle steps (sweep + F/theta) on U until budget_s seconds or max_steps; (steps, s)."""
    import oracle
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.sweep(U, OMEGA, oracle.LANDAU, reunit=((first + n + 1) % 20 == 0))
        oracle.measure(U, oracle.LANDAU)
        n += 1
        el = time.perf_counter() - t0
        if (budget_s is not None and el >= budget_s) or (max_steps is not None and n >= max_steps):
            return n, el


def run_reference(args):
    """The oracle on the host cores, same workload / metric / unit (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = oracle.num_threads()
    # One step = one sweep + F/theta.  The sample is the full 32^4 lattice unless K + W
    # steps of it would take more than about two minutes; then a 32^3 x Lt slab (Lt even)
    # of the same field recipe, and the metric counts that slab's bytes.
    dims = DIMS
    probe = make_field((32, 32, 32, 4))
    _, t4 = oracle_steps(probe, max_steps=1)
    per_slice = t4 / 4
    total = args.steps + args.warmup
    if total * per_slice * 32 > 120.0:
        lt = max(2, int(120.0 / (total * per_slice)) // 2 * 2)
        dims = (32, 32, 32, min(32, lt))
    U = make_field(dims)
    if args.warmup:
        oracle_steps(U, max_steps=args.warmup)
    t0 = time.perf_counter()
    oracle_steps(U, max_steps=args.steps, first=args.warmup)
    el = time.perf_counter() - t0
    vol = dims[0] * dims[1] * dims[2] * dims[3]
    value = 16 * vol * LINK_B * args.steps / el / 1e9
    sample = (f"{args.steps} steps on a {'x'.join(map(str, dims))} lattice of the 32^4 workload's "
              "field recipe (FP64 oracle, 18 reals per link, OpenMP over one parity)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "lattice": list(DIMS)},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


UNITS_SWITCH = 1e-11   # FP32 -> double-float switch of the batched runs (FP32 floor ~1e-13)
UNITS_BUDGET = 200000  # loop sweeps allowed to the batched runs


def units_leg(gf, dev, stream, peak: float, n_coulomb: int = 400, n_ensemble: int = 200):
    """The batched-unit workloads: the Coulomb 32^3 x 64 field (eps 0.5, seed 4) with its 64
    time slices as convergence units, and the 48-lattice ensemble (16 x 16^4, 16 x 24^4,
    16 x 16^3 x 32; eps ~ U[0.3, 0.6], seeds 100-147) in one batch.

    Throughput: FP32-12 sweeps with the stop check after every sweep (eps = 1e-300, so every
    unit stays active; autotuned launch shape); link bytes counted as 16 V b per sweep,
    against the measured HBM copy bandwidth.  Time to theta < 1e-15 on every unit: mixed
    FP32-12 -> double-float -> FP64 (each lattice changes precision when its own units
    reach the switch), wall time of gf_fix from the uploaded field, every unit checked."""
    import torch
    from paper_1412_1498_gb300 import fields

    def timed(h, n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gf.gf_fix(h, 1e-300, n)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / n

    def throughput(dims_list, gauge, Us, n):
        fx = gf.GaugeFixer(dims_list, gauge, gf.GF_FP32_12, device=dev)
        up = lambda: [fx.upload(Ui, i) for i, Ui in enumerate(Us)]  # noqa: E731
        up()
        t, v = gf.gf_autotune(fx.h)
        up()
        gf.gf_fix(fx.h, 1e-300, 5)                 # graph capture
        up()
        ms = timed(fx.h, n)
        fx.close()
        return ms, t, v

    def to_theta(dims_list, gauge, Us, threads, variant):
        fx = gf.GaugeFixer(dims_list, gauge, gf.GF_FP32_12, mixed=True, device=dev)
        gf.gf_set_polish(fx.h, gf.GF_POLISH_SPLIT)
        gf.gf_set_mixed_switch(fx.h, UNITS_SWITCH)
        gf.gf_set_block_size(fx.h, threads)
        gf.gf_set_sweep_variant(fx.h, variant)
        for i, Ui in enumerate(Us):
            fx.upload(Ui, i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fx.fix(1e-15, UNITS_BUDGET)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        _, _, _, uT = fx.functional_theta()
        fx.close()
        its = r["iters"]
        return {"seconds": el, "converged_units": int((uT < 1e-15).sum()), "units": int(len(uT)),
                "rc": int(r["rc"]), "loop_sweeps": int(its.max()), "unit_sweeps": int(its.sum()),
                "unit_sweeps_min_median_max": [int(its.min()), int(np.median(its)), int(its.max())],
                "sweeps_with_fp32_units": int(r["phase_sweeps"][0]),
                "sweeps_with_polish_units": int(r["phase_sweeps"][1]),
                "theta_max": float(uT.max()), "switch": UNITS_SWITCH, "budget": UNITS_BUDGET}

    out = {}
    dims = (32, 32, 32, 64)
    Uc = [make_field(dims, EPS_FIELD, 4)]
    ms, t, v = throughput([dims], gf.GF_COULOMB, Uc, n_coulomb)
    vol = 32 * 32 * 32 * 64
    gbps = 16 * vol * LINK_B / (ms * 1e-3) / 1e9
    out["coulomb_32x32x32x64"] = {
        "sweeps": n_coulomb, "ms_per_sweep": ms, "slice_sweeps_per_s": 64e3 / ms, "link_GBps": gbps,
        "roofline_frac": gbps / peak, "block_threads": t, "sweep_kernel": {1: "register", 2: "pipelined"}.get(v, v),
        "time_to_theta_1e-15": to_theta([dims], gf.GF_COULOMB, Uc, t, v)}
    del Uc
    dims_list = [(16, 16, 16, 16)] * 16 + [(24, 24, 24, 24)] * 16 + [(16, 16, 16, 32)] * 16
    Us = fields.ensemble(dims_list, list(range(100, 148)), workers=min(16, os.cpu_count() or 1))
    ms, t, v = throughput(dims_list, gf.GF_LANDAU, Us, n_ensemble)
    vtot = sum(d[0] * d[1] * d[2] * d[3] for d in dims_list)
    gbps = 16 * vtot * LINK_B / (ms * 1e-3) / 1e9
    tt = to_theta(dims_list, gf.GF_LANDAU, Us, t, v)
    tt["unit_sweeps_per_s"] = tt["unit_sweeps"] / tt["seconds"]
    out["ensemble_48"] = {
        "sweeps": n_ensemble, "ms_per_sweep": ms, "unit_sweeps_per_s": 48e3 / ms,
        "site_updates_per_s": vtot * 1e3 / ms, "link_GBps": gbps, "roofline_frac": gbps / peak,
        "block_threads": t, "sweep_kernel": {1: "register", 2: "pipelined"}.get(v, v),
        "time_to_theta_1e-15": tt}
    return out


# ------------------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1412_1498_gb300 import gf

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    U = make_field()        # each rank: its own independent 32^4 lattice (weak scaling)
    stream = torch.cuda.current_stream(dev)
    fx = gf.GaugeFixer(DIMS, gf.GF_LANDAU, gf.GF_FP32_12, device=dev)
    gf.gf_set_check_interval(fx.h, 1)
    gf.gf_set_reunit_interval(fx.h, 20)
    fx.upload(U)

    # ---- launch shape: the library's autotuner times every block size / kernel variant,
    # unless a shape is given (profiling runs: timings under a profiler mislead the tuner)
    if args.launch:
        t, v = args.launch.split(":")
        best = (int(t), {"register": gf.GF_SWEEP_REGISTER, "pipelined": gf.GF_SWEEP_PIPELINED}[v])
        gf.gf_set_block_size(fx.h, best[0])
        gf.gf_set_sweep_variant(fx.h, best[1])
    else:
        best = gf.gf_autotune(fx.h)
    fx.upload(U)

    # ---- clock samples from here to the end of the GPU arm (the timed region of a short
    # run is shorter than one sampling period; its own window is summarised too)
    clocks = ClockSampler(nvsmi_id(dev)).__enter__()

    # ---- warm-up steps (untimed)
    if args.warmup:
        gf.gf_fix(fx.h, 1e-300, args.warmup)
    fx.upload(U)
    barrier()

    # ---- timed region: K steps through gf_fix (device-driven loop, CUDA graphs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    w0 = time.perf_counter()
    e0.record(stream)
    rc, iters, F, th = gf.gf_fix(fx.h, 1e-300, args.steps)
    e1.record(stream)
    barrier()
    clocks.mark("timed", w0, time.perf_counter())
    ms_total = e0.elapsed_time(e1)
    # roofline: the half-sweep kernel alone, back to back on the same stream
    n_half = 2 * max(20, args.steps // 2)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.perf_counter()
    k0.record(stream)
    for _ in range(n_half // 2):
        fx.or_sweep(2, OMEGA)
    k1.record(stream)
    k1.synchronize()
    clocks.mark("roofline", w0, time.perf_counter())
    half_ms = k0.elapsed_time(k1) / n_half
    assert int(iters[0]) == args.steps, (iters, args.steps)
    # the last sweep of the budget always takes the exact (even-site) check
    bytes_per_step = STEP_BYTES + CHECK_BYTES / args.steps
    ms_total, value = reduce_over_ranks(ms_total, args.steps, world, bytes_per_step, dist, dev)
    ms_step = ms_total / args.steps
    launches = timed_fix_launches(args.steps)

    # ---- end to end through the C ABI with pinned host buffers: upload, one step, download
    Uh = torch.from_numpy(U).pin_memory()
    out = torch.empty_like(Uh).pin_memory()
    e2e_steps = max(3, min(10, args.steps))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        fx.upload(Uh)
        gf.gf_fix(fx.h, 1e-300, 1)
        fx.download(out=out)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0) / e2e_steps
    e2e_value = world * (STEP_BYTES + CHECK_BYTES) / e2e_s / 1e9  # a 1-sweep fix checks exactly
    canon_bytes = 4 * V * 144

    # ---- time to theta < 1e-15: mixed FP32-12 -> FP64-18 vs pure FP64-18
    ttt = None
    if not args.skip_time_to_theta:
        ttt = {}
        for name, storage, mixed, polish in (("mixed", gf.GF_FP32_12, True, gf.GF_POLISH_FP64),
                                             ("mixed_split", gf.GF_FP32_12, True, gf.GF_POLISH_SPLIT),
                                             ("fp64", gf.GF_FP64_18, False, gf.GF_POLISH_FP64)):
            f2 = gf.GaugeFixer(DIMS, gf.GF_LANDAU, storage, mixed=mixed, device=dev)
            gf.gf_set_polish(f2.h, polish)
            f2.upload(U)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = f2.fix(1e-15, args.max_sweeps)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            ttt[name] = dict(seconds=el, sweeps=int(r["iters"][0]), phase_sweeps=list(r["phase_sweeps"]),
                             converged=r["rc"] == gf.GF_OK, F=float(r["F"][0]), theta=float(r["theta"][0]))
            f2.close()
            del f2
            torch.cuda.empty_cache()
        for m in ("mixed", "mixed_split"):
            ttt[f"F_err_{m}_vs_fp64"] = abs(ttt[m]["F"] - ttt["fp64"]["F"])
            ttt[f"speedup_{m}_over_fp64"] = ttt["fp64"]["seconds"] / ttt[m]["seconds"]

    # ---- double-float polish sweeps on the same field (the polish phase's kernel)
    split_probe = None
    if args.split_probe > 0:
        f3 = gf.GaugeFixer(DIMS, gf.GF_LANDAU, gf.GF_FP32_12, mixed=True, device=dev)
        gf.gf_set_polish(f3.h, gf.GF_POLISH_SPLIT)
        gf.gf_set_mixed_switch(f3.h, 1e9)        # no FP32 sweeps: straight to the polish
        f3.upload(U)
        gf.gf_fix(f3.h, 1e-300, 2)               # warm-up (graph capture)
        f3.upload(U)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        gf.gf_fix(f3.h, 1e-300, args.split_probe)
        p1.record(stream)
        p1.synchronize()
        split_probe = {"sweeps": args.split_probe, "ms_per_sweep_incl_conversions": p0.elapsed_time(p1) / args.split_probe,
                       "link_bytes_per_sweep": 16 * V * 144}
        f3.close()
        del f3

    # ---- Fourier-accelerated steepest descent (Algorithm 2), 32^4 FP32, seed 5, alpha 0.08
    fasd = None
    if args.fasd_iters > 0:
        U5 = make_field(DIMS, EPS_FIELD, 5)
        f4 = gf.GaugeFixer(DIMS, gf.GF_LANDAU, gf.GF_FP32_12, fasd=True, device=dev)
        gf.gf_set_method(f4.h, gf.GF_METHOD_FASD)
        f4.upload(U5)
        th0 = f4.functional_theta()[1][0]
        gf.gf_fix(f4.h, 1e-300, 2)                 # warm-up (graph capture)
        f4.upload(U5)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        _, _, Ff, thf = gf.gf_fix(f4.h, 1e-300, args.fasd_iters)
        q1.record(stream)
        q1.synchronize()
        ms_it = q0.elapsed_time(q1) / args.fasd_iters
        # bytes an iteration moves: links read for Delta (4 V b) and read and written in
        # the update (8 V b), k-space (4 complex FP32 fields, 32 V B) written by the Delta
        # pass and read back once, g (rows 0, 1: 48 V B) written by the inverse transform
        # and read once by the update; the z/t transform works on L2-resident k-space
        fasd_bytes = 12 * V * LINK_B + 2 * 48 * V + 2 * 32 * V
        fasd = {"iterations": args.fasd_iters, "ms_per_iteration": ms_it,
                "algorithmic_GBps": fasd_bytes / (ms_it * 1e-3) / 1e9, "bytes_per_iteration": fasd_bytes,
                "theta_start": float(th0), "theta_end": float(thf[0]), "F_end": float(Ff[0]),
                "workload": "32^4 Landau, FP32-12 links, FP32 FFTs, FP64 reductions, eps 0.5 seed 5, alpha 0.08"}
        f4.close()
        del f4, U5

    # ---- differentiable F(c), theta(c): forward and backward on the FP64 field (32^4;
    # --autograd-lattice L takes L^4, e.g. for a profiler run)
    autograd = None
    if args.autograd:
        from paper_1412_1498_gb300.autograd import functional_theta
        ad_dims = (args.autograd_lattice,) * 4
        ad_V = args.autograd_lattice ** 4
        f5 = gf.GaugeFixer(ad_dims, gf.GF_LANDAU, gf.GF_FP64_18, autograd=True, device=dev)
        f5.upload(make_field(ad_dims, EPS_FIELD, 5))
        c = torch.zeros((ad_V, 8), dtype=torch.float64, device=dev, requires_grad=True)
        for _ in range(2):
            Fa, _t = functional_theta(c, f5)
            Fa.backward()
        r0, r1, r2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        r0.record(stream)
        Fa, _t = functional_theta(c, f5)
        r1.record(stream)
        Fa.backward()
        r2.record(stream)
        r2.synchronize()
        fwd_ms, bwd_ms = r0.elapsed_time(r1), r1.elapsed_time(r2)
        autograd = {"lattice": list(ad_dims), "forward_ms": fwd_ms, "backward_ms": bwd_ms}
        # FP64-ALU roofline: FP64 flops per site of each pass (dadd + dmul + 2 dfma thread
        # instructions, counted by ncu at c = 0 and scaled by the sites) over the event time,
        # against the FP64 pipe's peak: 2 DFMA per clock per SM (152 SMs at 2070 MHz: 1.26
        # TFLOP/s, the nominal FP64 rate), at the SM clock sampled during the run
        fl_f = profiled_value("k_ad_landau_32x4_fp64.md", AD_SOURCES, "fp64_flops_forward_per_site")
        fl_b = profiled_value("k_ad_landau_32x4_fp64.md", AD_SOURCES, "fp64_flops_backward_per_site")
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clocks.summary()["sm_mhz"] or 2070.0
        ad_peak = sms * 4 * mhz * 1e6 / 1e12
        if fl_f and fl_b:
            af = fl_f * ad_V / (fwd_ms * 1e-3) / 1e12
            ab = fl_b * ad_V / (bwd_ms * 1e-3) / 1e12
            autograd["roofline"] = {
                "bound": "alu", "unit": "TFLOP/s", "peak": ad_peak,
                "peak_kind": f"FP64 pipe: 2 DFMA / clock / SM x {sms} SMs at {mhz:.0f} MHz",
                "forward": {"achieved": af, "frac": af / ad_peak, "fp64_flops_per_site": fl_f},
                "backward": {"achieved": ab, "frac": ab / ad_peak, "fp64_flops_per_site": fl_b}}
        f5.close()
        del f5

    peak, peak_kind = measured_peaks()

    # ---- batched units: Coulomb time slices, the 48-lattice ensemble
    units = None if args.skip_units else units_leg(gf, dev, stream, peak)
    clocks.__exit__(None, None, None)
    achieved = HALF_SWEEP_BYTES / (half_ms * 1e-3) / 1e9
    traffic = None
    if best[1] == gf.GF_SWEEP_PIPELINED:
        traffic = profiled_traffic("k_or_sweep_pipe_fp32_12_landau_32x4.md",
                                   ("gf_device.cuh", "gf_kernels.cuh", "gf_sweep_pipe.cuh"))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_or_sweep_pipe<Landau> (FP32-12)" if best[1] == gf.GF_SWEEP_PIPELINED
                else "k_or_sweep<FP32_12, Landau>",
                "bytes_per_launch": HALF_SWEEP_BYTES, "ms_per_launch": half_ms,
                "peak_kind": f"{peak_kind} HBM copy bandwidth",
                "fp32_tflops": FLOP_PER_SITE * (V // 2) / (half_ms * 1e-3) / 1e12,
                "flop_per_site_update": FLOP_PER_SITE}

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        import oracle
        oracle.build()
        Uc = U.copy()
        n, el = oracle_steps(Uc, budget_s=args.cpu_seconds)
        cpu = {"value": STEP_BYTES * n / el / 1e9, "unit": "GB/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"{n} steps of the full 32^4 workload in {el:.1f} s "
                                            "(FP64 oracle, 18 reals per link, OpenMP over one parity)"}

    clock_line = clocks.summary()
    timed = clocks.summary("timed")
    clock_line["gpu"] = clocks.gpu_id
    clock_line["scope"] = "whole GPU arm: warm-up, timed steps, roofline and every extra leg"
    clock_line["timed_region"] = {"samples": timed["samples"], "sm_mhz": timed["sm_mhz"],
                                  "reasons": timed["reasons"], "ms": ms_total}
    if clock_line["sm_mhz"]:
        # clock-normalised step cost: SM cycles per step at the arm's median clock
        clock_line["mcycles_per_step"] = ms_step * 1e-3 * clock_line["sm_mhz"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": list(DIMS), "storage": "fp32-12", "omega": OMEGA,
                       "check_interval": 1, "reunit_interval": 20, "block_threads": best[0],
                       "sweep_kernel": {1: "register", 2: "pipelined"}.get(best[1], str(best[1])),
                       "field": f"smooth eps={EPS_FIELD} seed={SEED} + Haar gauge",
                       "l2": "inputs larger than L2: 201 MB of links vs 129 MB L2",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GB/s", "h2d_bytes_per_step": canon_bytes,
                    "d2h_bytes_per_step": canon_bytes},
            "gpu_launches": launches,
            "sweeps_per_s": world * args.steps / (ms_total * 1e-3),
            "clocks": clock_line,
            "time_to_theta_1e-15": ttt,
            "split_polish_probe": split_probe,
            "fa_sd": fasd,
            "autograd": autograd,
            "units": units,
        }
        print(json.dumps(line))
    fx.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gf", choices=["gf", "reference"])
    ap.add_argument("--max-sweeps", type=int, default=20000)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--skip-time-to-theta", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--split-probe", type=int, default=100)
    # 63 iterations and the final measurement fill four 16-iteration graph replays exactly
    ap.add_argument("--fasd-iters", type=int, default=63)
    ap.add_argument("--autograd", type=int, default=1)
    ap.add_argument("--autograd-lattice", type=int, default=32, help="L of the L^4 autograd leg")
    ap.add_argument("--skip-units", action="store_true",
                    help="skip the Coulomb 32^3x64 slice and 48-lattice ensemble leg")
    ap.add_argument("--launch", default="", help="fixed launch shape THREADS:register|pipelined "
                    "instead of the autotuner (for profiler runs)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gf":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
