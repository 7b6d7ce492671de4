"""Benchmark of the GPU Douglas ADI pricing path.

Default workload (--workload headline): the 256-caplet batch (seed 1108003):
expiries U{1..10}y into 6m, strikes ATM +/- 200 bp, each caplet with its own
Nelson-Siegel curve and (epsilon, rho), on uneven grids n_r x n_r/2 x n_r/2
with n_r in {64, 96, ..., 256} and 2 n_r Douglas steps, FP32 march with FP64
set-up and read-out. One step of this benchmark = one hjm_price_batch call
over all 256 caplets (every shape group's set-up, terminal field, march and
read-out; the groups run as branches of one CUDA graph). Measured the same way
beside it, under "secondary": the 100-caplet batch of 5y-into-6m ATM caplets
on 128 x 64 x 64 with 400 steps (seed 1108002) and the bandwidth-stress
caplet, 10y-into-6m ATM on 512 x 256 x 256 with 1000 steps. Every working set
is larger than L2 (no flush needed between steps).

Metric: grid-point-steps/s (caplets/s reported beside it). `value` is timed
with CUDA events on the launching stream with the outputs in device memory
(the parameter structs are uploaded inside each call); `e2e` is the same call
with host outputs, wall-clocked. `roofline` is the dominant kernel's
algorithmic bytes (the pass's words per grid-point-step x the call's
grid-point-steps) over its device time per call (trace mode); `step_hbm` the
same for the whole step (7 words per grid-point-step). Under torchrun every
rank runs its own replica of the batch on its own GPU (weak scaling); value =
all ranks' grid-point-steps / the slowest rank's time.

--precision fp64 marches in FP64; --precision mixed marches in FP32 and
re-prices the instruments whose rounding bound misses --mixed-tol (default
1e-4; 0 re-prices every instrument) by FP32 increments on an FP64 state, in
FP64 where even that misses (the count is reported in config.mixed).

cpu_baseline and --impl reference time the CPU FP64 oracle (the plain C
reference written from the paper; its OpenMP build shares the lines of each
pass among all host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ADI grid-point-steps/s and caplet prices/s at 1e-4 rel vs FP64 oracle"
UNIT = "grid-point-steps/s"
KERNEL_KINDS = ("setup", "terminal", "pass1", "pass2", "pass3", "readout")
# Algorithmic words moved per grid point by each pass (Section 5.1 Douglas
# step as three line passes): pass 1 reads U^n and writes dU1, pass 2 reads
# dU1 and writes dU2, pass 3 reads dU2 and U^n and writes U^{n+1}.
WORDS_PER_POINT = {"pass1": 2, "pass2": 2, "pass3": 3}
# Craig-Sneyd family (--scheme cs|mcs|hv): a Douglas stage into Y3 (the same
# words) and a correction stage whose pass 1 also reads Y3 (3 words), so the
# pass-1 launches average 2.5 words per point.
WORDS_PER_POINT_CS = {"pass1": 2.5, "pass2": 2, "pass3": 3}
SCHEMES = {"douglas": (0, 0.5), "cs": (1, 0.5), "mcs": (2, 1.0 / 3.0), "hv": (3, 0.5 + 3 ** 0.5 / 6.0)}


def workload_items(name, instruments=None, march_steps=None, scheme="douglas"):
    """Items of a workload. instruments / march_steps shrink config2 for
    profiling captures (they change the workload named in the JSON line);
    scheme other than douglas switches every item to that ADI scheme."""
    items, desc = _workload_items(name, instruments, march_steps)
    sch, theta = SCHEMES[scheme]
    if sch:
        for x in items:
            x["grid"].update(scheme=sch, theta_adi=theta)
        desc += ", %s scheme (theta %.4g)" % (scheme.upper(), theta)
    return items, desc


def _workload_items(name, instruments=None, march_steps=None):
    from paper_1108_1688_gb300 import workloads as W
    if name == "headline":
        name = "config3"
    if name == "config2":
        n = instruments or 100
        ns = march_steps or 400
        return (W.config2_draws(n, n_steps=ns),
                "%d caplets 5y-into-6m ATM, NS curves, 128x64x64, %d steps" % (n, ns))
    if name == "config4":
        ns = march_steps or 1000
        return ([W.with_grid(W.config4(), n_steps=ns)],
                "1 caplet 10y-into-6m ATM, flat 3%%, 512x256x256, %d steps" % ns)
    if name == "config3":
        return W.config3_batch(), "256 caplets, expiries 1..10y, uneven grids 64..256 x n/2 x n/2, 2n steps"
    if name == "config1":
        return [W.config1()], "5y zero-coupon bond, flat 3%, 40x20x20, 100 steps"
    if name == "paper63":
        return (W.paper_timing_set(),
                "the 3 caplets of the paper's timing table (1y, 10y, 19y into 1y, ATM), 100x50x50, 12 steps/yr")
    raise SystemExit("unknown workload %s" % name)


def point_steps(items):
    from paper_1108_1688_gb300 import workloads as W
    return sum(W.point_steps(x) for x in items)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].replace(".", "").isdigit():
                    rows.append(f)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": float(rows[0][2]),
                "samples": len(rows), "reasons": sorted(reasons)}


# ------------------------------------------------------------ distributed

def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def reduce_max(value, world, device=None):
    """Max over ranks of a float (identity at world 1)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- helpers

MARCH_SOURCES = ("hjm_kernels.cuh", "hjm_march.cu", "hjm_pass1.cu", "hjm_pass1t.cu", "hjm_lines_t.cu",
                 "hjm_tma.cuh")
LINES_TMA = 15  # p2_warps / p3_warps code of the TMA-fed strided passes (HJM_LINES_TMA)


# The files each kernel with recorded DRAM counters is built from (its
# translation unit and the headers it includes): its counters in
# profiles/traffic.json are reported only while these files are unchanged.
KERNEL_SOURCES = {
    "k_pass1t": ("hjm_pass1t.cu", "hjm_kernels.cuh", "hjm_curve.cuh", "hjm_tma.cuh"),
    "k_lines_t": ("hjm_lines_t.cu", "hjm_kernels.cuh", "hjm_curve.cuh", "hjm_tma.cuh"),
    "k_pass1": ("hjm_pass1.cu", "hjm_kernels.cuh", "hjm_curve.cuh"),
    "k_pass2": ("hjm_march.cu", "hjm_kernels.cuh", "hjm_curve.cuh"),
    "k_pass3": ("hjm_march.cu", "hjm_kernels.cuh", "hjm_curve.cuh"),
    "k_split_lines": ("hjm_march.cu", "hjm_kernels.cuh", "hjm_curve.cuh"),
}


def source_digest(kernel=None):
    """Digest of one kernel's sources (KERNEL_SOURCES; stored with its ncu
    counters, so a stale counter is detected and reported as null), or with
    no kernel of all the Douglas pass kernels' sources."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1108_1688_gb300", "csrc")
    for name in (MARCH_SOURCES if kernel is None else KERNEL_SOURCES[kernel]):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_name(kind, tile, prec="fp32", scheme=0):
    """The kernel that runs a pass under a launch shape (7-tuple as from
    hjm_tile_get), for the roofline line."""
    if tile is None:
        return "k_" + kind
    if kind == "pass1":
        if tile[5] in (2, 3):
            return "k_pass1t" + (" + k_pass1" if scheme else "")
        if tile[5] == 1:
            return "k_pass1s_r96" if prec == "fp32" and tile[1] <= 8 else "k_pass1s"
        return "k_pass1_r96" if prec == "fp32" and tile[1] == 8 and not scheme else "k_pass1"
    if kind == "pass3" and tile[3] == 0:
        return "k_pass23"
    if kind in ("pass2", "pass3"):
        p = tile[3] if kind == "pass2" else tile[4]
        if p == LINES_TMA:
            return "k_lines_t"
        return "k_" + kind if p == 1 else "k_split_lines"
    return "k_" + kind


# FP64 arithmetic peak: the nominal 1.25 TFLOP/s of the part, i.e. 152 SMs x
# 2 FP64 fused multiply-adds per SM per clock x 2 flops at the 2.07 GHz
# maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def pass1_flops_per_point(S, M):
    """FP64 operations per grid point that pass 1 performs, counted from its
    arithmetic (a fused multiply-add counts 2, a division 1; face rows,
    a few per line, left out), for S lanes of M nodes per r line:
    the explicit operator's first sweep (v and y parts, mixed-term row
    difference: 15) and second sweep (r part from one first difference per
    node, reaction, mixed term, scaling by dt: 19), the rows of
    I - theta dt A_r (13), and the partition solve,
    per lane: local forward elimination 8 + 9 (M - 2), backward elimination
    5 (M - 3), the chunk's first row 9, the interface row divided by its
    diagonal 14, 14 per parallel-cyclic-reduction level (log2 S levels),
    back-substitution 4 + 4 (M - 2)."""
    levels = int(round(math.log2(S))) if S > 1 else 0
    lane = (8 + 9 * max(M - 2, 0) + 5 * max(M - 3, 0) + (9 if M >= 3 else 0) + 14 + 14 * levels
            + 4 + 4 * max(M - 2, 0))
    return 15 + 19 + 13 + lane / M


def recorded_traffic(kernel, workload, points_per_launch, tile=None):
    """DRAM bytes per launch of pass `kernel` from the committed ncu summary
    of this workload, if it was taken with the launch shape in use on the
    current sources of the kernel that ran it; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    w = d.get("workloads", {}).get(workload)
    if not w or tile is None:
        return None
    rec = w.get("tiles", {}).get(tile, {}).get("kernels", {}).get(kernel)
    if not rec or rec.get("kernel") not in KERNEL_SOURCES:
        return None
    if rec.get("source_digest") != source_digest(rec["kernel"]):
        return None
    return rec["dram_bytes_per_point"] * points_per_launch


def _oracle_rate(it, omp, budget_s, max_steps):
    """Grid-point-steps/s of the oracle on the set-up and the first Douglas
    steps of one instrument, within a time budget."""
    import oracle
    g = it["grid"]
    pts = g["n_r"] * g["n_v"] * g["n_y"]
    with oracle.Ctx(it, omp=omp) as X:
        t0 = time.perf_counter()
        U = X.terminal()
        n = 0
        while n < min(max_steps, g["n_steps"]) and time.perf_counter() - t0 < budget_s:
            U = X.step(n, U)
            n += 1
        dt = time.perf_counter() - t0
    return n * pts / dt, n, dt


def cpu_baseline(items, budget_s=12.0, max_steps=200):
    """The oracle, as it stands, on a bounded sample of the workload (the
    set-up and the first Douglas steps of its first instrument): the OpenMP
    build on every host core (the reported value) and the serial build."""
    it = items[0]
    g = it["grid"]
    cores = os.cpu_count() or 1
    v_omp, n_omp, s_omp = _oracle_rate(it, True, budget_s, max_steps)
    v_ser, n_ser, s_ser = _oracle_rate(it, False, budget_s, max_steps)
    return {"value": v_omp, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "instrument 0 of the workload: set-up and the first %d of %d ADI steps on %dx%dx%d "
                      "(FP64 C oracle, OpenMP over the lines of each pass, %d threads)"
                      % (n_omp, g["n_steps"], g["n_r"], g["n_y"], g["n_v"], cores),
            "seconds": s_omp,
            "serial": {"value": v_ser, "cores": 1, "steps": n_ser, "seconds": s_ser}}


# ------------------------------------------------------------------- arms

def run_reference(args):
    world, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    import oracle
    oracle.build(omp=True)
    items, desc = workload_items(args.workload, args.instruments, args.march_steps, args.scheme)
    it = items[0]
    g = it["grid"]
    pts = g["n_r"] * g["n_v"] * g["n_y"]
    per_step = max(1, args.ref_steps_per_step)
    cores = os.cpu_count() or 1
    with oracle.Ctx(it, omp=True) as X:
        U = X.terminal()
        n = 0
        for _ in range(args.warmup):
            for _ in range(per_step):
                U = X.step(n % g["n_steps"], U)
                n += 1
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for _ in range(per_step):
                U = X.step(n % g["n_steps"], U)
                n += 1
        dt = time.perf_counter() - t0
    value = args.steps * per_step * pts / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "sample": "%d ADI step(s) of instrument 0 per step" % per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d ADI step(s) of instrument 0 (%dx%dx%d) per step, FP64 C, OpenMP over "
                                   "the lines of each pass, %d threads" % (per_step, g["n_r"], g["n_y"], g["n_v"],
                                                                          cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_surrogate(args):
    """--workload config5: the pricing surrogate. Trains on PDE labels (FP32
    march on the label grid, untimed), then times hjm_surrogate_infer on a
    batch of 65,536 fresh rows with 5% out of the training box (network
    answers gated by the held-out error table, every other row priced by the
    march); value = caplet forward premia per second end to end. The
    answered rows are then judged against the march (untimed)."""
    import numpy as np
    import torch
    from paper_1108_1688_gb300 import _build
    _build.build()
    from paper_1108_1688_gb300 import hjm
    from paper_1108_1688_gb300 import workloads as W
    lg = [int(v) for v in args.label_grid.split("x")]
    label = W.surrogate_label_grid(*lg)
    n_rows = 65536
    cfg = hjm.surrogate_cfg(args.labels, args.epochs, 1024, 3e-3, W.SEED_BASE + 5, W.SURROGATE_BOX_LO,
                            W.SURROGATE_BOX_HI, label, None)
    t0 = time.perf_counter()
    h = hjm.hjm_surrogate_train(cfg)
    train_s = time.perf_counter() - t0
    table = hjm.hjm_surrogate_error_table(h)
    x = W.surrogate_draws(n_rows, seed=W.SEED_BASE + 51, out_of_box=0.05)
    stream = torch.cuda.current_stream()
    xd = torch.tensor(x).cuda()
    out = torch.empty(n_rows, dtype=torch.float64, device="cuda")
    used = torch.zeros(n_rows, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        hjm.hjm_surrogate_infer(h, xd, out, used, stream=stream)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            hjm.hjm_surrogate_infer(h, xd, out, used, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    # end to end: rows from pinned host memory, prices back to the host
    xh = torch.tensor(x).pin_memory()
    outh = torch.empty(n_rows, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xd.copy_(xh, non_blocking=True)
        hjm.hjm_surrogate_infer(h, xd, out, used, stream=stream)
        outh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # the network alone
    y = torch.empty(n_rows, dtype=torch.float32, device="cuda")
    hjm.hjm_surrogate_forward(h, xd, y, stream=stream)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(20):
        hjm.hjm_surrogate_forward(h, xd, y, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    net_ms = ev0.elapsed_time(ev1) / 20
    # judge every row with the march on the label grid
    got = out.cpu().numpy()
    u = used.cpu().numpy().astype(bool)
    items = [W.surrogate_item(r, label) for r in x]
    C = np.empty(n_rows)
    for a in range(0, n_rows, 4096):
        C[a:a + 4096] = hjm.hjm_price_batch(items[a:a + 4096], "fp32")
    want = np.array([c * math.exp(math.log1p(float(r[8]) * float(r[6])) / float(r[6]) * float(r[5]))
                     for c, r in zip(C, x)])
    err = np.abs(got - want)
    ans = ~u
    # discretisation error of the label grid: a sample of in-box rows priced
    # on the label grid and on 128 x 64 x 64 with 256 steps (FP32; forward
    # premia, the units of the errors above)
    fine = W.surrogate_label_grid(128, 64, 64, 256)
    xs = W.surrogate_draws(args.label_check, seed=W.SEED_BASE + 52)
    fwd = np.array([math.exp(math.log1p(float(r[8]) * float(r[6])) / float(r[6]) * float(r[5])) for r in xs])
    lab = np.concatenate([hjm.hjm_price_batch([W.surrogate_item(r, label) for r in xs[a:a + 1024]], "fp32")
                          for a in range(0, len(xs), 1024)]) * fwd
    ref = np.concatenate([hjm.hjm_price_batch([W.surrogate_item(r, fine) for r in xs[a:a + 1024]], "fp32")
                          for a in range(0, len(xs), 1024)]) * fwd
    gap = np.abs(lab - ref)
    line = {
        "metric": METRIC, "value": n_rows * args.steps / (ms * 1e-3), "unit": "caplet prices/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32",
        "data": "synthetic",
        "config": {"workload": "surrogate 9->4x256 SiLU->1, %d PDE labels on %s (%d epochs), inference batch "
                               "%d rows with 5%% out of the box, PDE fallback" % (args.labels, args.label_grid,
                                                                                args.epochs, n_rows),
                   "l2": "batch of %d rows (2.4 MB) is L2-resident; no flush (the fallback march dominates)"
                         % n_rows},
        "e2e": {"value": n_rows * args.steps / e2e_s, "unit": "caplet prices/s",
                "h2d_bytes_per_step": n_rows * 9 * 4, "d2h_bytes_per_step": n_rows * 8},
        "gpu_launches": None,
        "clocks": clk.summary(),
        "surrogate": {"train_s": round(train_s, 1), "coverage": round(float(ans.mean()), 4),
                      "max_err_answered": float(err[ans].max()) if ans.any() else None,
                      "median_err_answered": float(np.median(err[ans])) if ans.any() else None,
                      "max_err_fallback": float(err[u].max()) if u.any() else None,
                      "bins_under_gate": int((table <= 5e-5).sum()), "bins": int(table.size),
                      "network_ms_per_batch": round(net_ms, 4),
                      "network_rows_per_s": n_rows / (net_ms * 1e-3),
                      "error_table": [[float(v) if np.isfinite(v) else None for v in row]
                                      for row in np.asarray(table).reshape(9, 8)],
                      "label_grid_vs_128x64x64x256": {
                          "rows": int(len(xs)), "max": float(gap.max()), "median": float(np.median(gap)),
                          "p99": float(np.quantile(gap, 0.99)),
                          "rows_over_1e-4": int((gap > 1e-4).sum())}},
    }
    hjm.hjm_surrogate_destroy(h)
    print(json.dumps(line))


def _tiles_for_workload(hjm, items, prec, arr, stream, args):
    """Launch shapes: fixed (--tile), from a file (--tiles), or picked by the
    library's autotuner on the workload's grid shapes (untimed)."""
    if args.tile:
        t = [int(v) for v in args.tile.split(",")]
        for x in items:
            g = x["grid"]
            hjm.hjm_tile_set(g["n_r"], g["n_v"], g["n_y"], prec, t)
    elif args.tiles and os.path.exists(args.tiles):
        for key, t in json.load(open(args.tiles)).items():
            nr_, ny_, nv_ = (int(v) for v in key.split("x"))
            hjm.hjm_tile_set(nr_, nv_, ny_, prec, t)
    elif not args.no_autotune:
        hjm.hjm_autotune(arr, prec, steps=8, stream=stream)
    tiles = {}
    for x in items:
        g = x["grid"]
        key = "%dx%dx%d" % (g["n_r"], g["n_y"], g["n_v"])
        tiles[key] = list(hjm.hjm_tile_get(g["n_r"], g["n_v"], g["n_y"], prec))
    if args.tiles and not os.path.exists(args.tiles):
        json.dump(tiles, open(args.tiles, "w"))
    return tiles


def measure(wname, args, world, local, hjm):
    """One workload: autotune (untimed), W warm-up calls, K device-timed
    hjm_price_batch calls (value), K end-to-end calls with host outputs (e2e),
    a few traced calls for the per-kernel roofline. Returns the JSON line."""
    import numpy as np
    import torch

    items, desc = workload_items(wname, args.instruments, args.march_steps, args.scheme)
    scheme = SCHEMES[args.scheme][0]
    prec = args.precision
    # MIXED marches with the FP32 kernels and launch shapes, re-running in
    # FP64 the instruments whose rounding bound misses the tolerance
    kprec = "fp32" if prec == "mixed" else prec
    arr = hjm.make_items(items)
    import ctypes
    item_bytes = ctypes.sizeof(hjm.hjm_batch_item)
    n = len(items)
    ps = point_steps(items)
    stream = torch.cuda.current_stream()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    host_out = np.empty(n, dtype=np.float64)

    def step_dev():
        hjm.hjm_price_batch(arr, prec, tol_rel=args.mixed_tol, out=out, stream=stream)

    tiles = _tiles_for_workload(hjm, items, prec, arr, stream, args)
    for _ in range(args.warmup):
        step_dev()
    torch.cuda.synchronize()

    # ---- device-timed region (value)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step_dev()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    ms = ev0.elapsed_time(ev1)
    ms_max = reduce_max(ms, world, device="cuda")
    clocks = clk.summary()

    # ---- end to end through the public API with host buffers (e2e)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        hjm.hjm_price_batch(arr, prec, tol_rel=args.mixed_tol, out=host_out, stream=stream)  # syncs for the D2H read
    e2e_s = time.perf_counter() - t0
    e2e_max = reduce_max(e2e_s, world, device="cuda")

    # ---- per-kernel device times (trace mode: kernel by kernel, event pairs)
    calls = max(1, min(args.steps, 3))
    hjm.hjm_trace_enable(True)
    hjm.hjm_trace_read(reset=True)
    for _ in range(calls):
        step_dev()
    torch.cuda.synchronize()
    trace = hjm.hjm_trace_read(reset=True)
    hjm.hjm_trace_enable(False)
    hjm.hjm_wait_status()

    total_points = sum(x["grid"]["n_r"] * x["grid"]["n_v"] * x["grid"]["n_y"] for x in items)
    elem = 4 if kprec == "fp32" else 8
    dom = max(KERNEL_KINDS, key=lambda k: trace[k][1])
    shape_tiles = {tuple(t) for t in tiles.values()}
    tile_used = list(shape_tiles)[0] if len(shape_tiles) == 1 else None
    launches, tot_ms = trace[dom]
    avg_ms = tot_ms / max(launches, 1)
    roof = None
    if dom in WORDS_PER_POINT:
        # every pass of every step touches every point of every instrument
        # once, so one call moves words x elem x (grid-point-steps) bytes in
        # this pass; achieved = that / the pass's device time per call (for a
        # batch of one grid shape this is the per-launch figure)
        alg_call = (WORDS_PER_POINT_CS if scheme else WORDS_PER_POINT)[dom] * elem * ps
        ms_call = tot_ms / calls
        peak, peak_kind = measured_peaks()
        achieved = alg_call / (ms_call * 1e-3) / 1e9
        names = sorted({kernel_name(dom, tuple(t), kprec, scheme) for t in tiles.values()})
        shapes = {(x["grid"]["n_r"], x["grid"]["n_v"], x["grid"]["n_y"], x["grid"]["n_steps"]) for x in items}
        pts_launch = total_points / len(shapes)
        roof = {"bound": "hbm", "kernel": " / ".join(names), "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "algorithmic_bytes_per_launch": alg_call * calls / max(launches, 1), "avg_launch_ms": avg_ms,
                "launches_per_call": launches / calls,
                "traffic": recorded_traffic(dom, "%s-%s%s" % (wname, kprec, "-" + args.scheme if scheme else ""),
                                            pts_launch,
                                            ",".join(map(str, tile_used)) if tile_used else None)}
        if prec == "fp64" and dom == "pass1" and not scheme and tile_used is not None:
            # FP64 pass 1 is bound by FP64 arithmetic, not by HBM: report it
            # against the FP64 peak, the byte figures kept beside it
            fpp = pass1_flops_per_point(tile_used[0], tile_used[1])
            flops = fpp * ps / (tot_ms / calls * 1e-3)
            tf = flops / 1e12
            roof = {"bound": "alu", "kernel": roof["kernel"], "achieved": tf, "peak": FP64_PEAK_TFLOPS,
                    "peak_kind": "nominal (152 SMs x 2 FP64 FMA/clock x 2 flops x 2.07 GHz)", "unit": "TFLOP/s",
                    "frac": tf / FP64_PEAK_TFLOPS, "flops_per_point": fpp, "avg_launch_ms": avg_ms,
                    "hbm_achieved_gbs": achieved, "hbm_frac": achieved / peak, "traffic": roof["traffic"]}
    shares = {k: round(trace[k][1] / max(sum(v[1] for v in trace.values()), 1e-12), 4) for k in KERNEL_KINDS}
    # whole step against the HBM roofline: the three passes' algorithmic bytes
    # (7 words per grid-point-step, 15 for the Craig-Sneyd family) per call
    step_words = 15 if scheme else 7
    step_gbs = step_words * elem * ps / (ms_max / args.steps * 1e-3) / 1e9

    # step launches: set-up, terminal, per ADI step 3 per stage (2 with the
    # strided passes fused) and 2 stages for the Craig-Sneyd family, read-out
    # per shape group, plus the scatter of prices
    groups = {}
    for x in items:
        g = x["grid"]
        key = (g["n_r"], g["n_v"], g["n_y"], g["n_steps"])
        t = tiles["%dx%dx%d" % (g["n_r"], g["n_y"], g["n_v"])]
        per_stage = 2 if t[3] == 0 and x["model"]["gamma"] == 0.0 else 3
        groups[key] = g["n_steps"] * per_stage * (2 if scheme else 1)
    launches_per_step = sum(3 + s for s in groups.values()) + 1
    mixed = None
    if prec == "mixed":
        # how many instruments one call re-prices in FP64, and their launches
        # (the FP64 batch of those instruments, FP64 launch shapes)
        _, infos = hjm.hjm_price_batch(arr, prec, tol_rel=args.mixed_tol, out=host_out, infos=True, stream=stream)
        redo = [x for x, inf in zip(items, infos) if inf.escalated]
        rg = {}
        for x in redo:
            g = x["grid"]
            t = hjm.hjm_tile_get(g["n_r"], g["n_v"], g["n_y"], "fp64")
            per_stage = 2 if t[3] == 0 and x["model"]["gamma"] == 0.0 else 3
            rg[(g["n_r"], g["n_v"], g["n_y"], g["n_steps"])] = g["n_steps"] * per_stage * (2 if scheme else 1)
        if rg:
            launches_per_step += sum(3 + s for s in rg.values()) + 1
        mixed = {"tol_rel": args.mixed_tol, "escalated_per_step": len(redo),
                 "max_err_estimate": max(float(inf.err_estimate) for inf in infos)}

    line = {
        "metric": METRIC,
        "value": world * ps * args.steps / (ms_max * 1e-3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "mixed" if prec == "mixed" else ("f32" if kprec == "fp32" else "f64"),
        "data": "synthetic",
        "config": {"workload": desc, "name": wname, "instruments": n, "grid_point_steps_per_step": ps,
                   "caplets_per_s": world * n * args.steps / (ms_max * 1e-3),
                   "precision": prec, "l2": "working set %.0f MB > L2 (no flush)" % (2 * total_points * elem / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "param_upload_bytes_per_step": n * item_bytes,
                   "step_hbm": {"algorithmic_gbs": step_gbs, "frac": step_gbs / measured_peaks()[0],
                                "words_per_point_step": step_words},
                   "tiles": {"autotuned": not (args.no_autotune or args.tile or args.tiles),
                             "from_file": bool(args.tiles), "fixed": bool(args.tile),
                             "r_x_y_x_v": tiles}},
        "e2e": {"value": world * ps * args.steps / e2e_max, "unit": UNIT,
                "h2d_bytes_per_step": n * item_bytes, "d2h_bytes_per_step": n * 8},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "roofline": roof,
        "kernel_shares": shares,
        "source_digest": source_digest(),
    }
    if mixed is not None:
        line["config"]["mixed"] = mixed
    return line, items


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_1108_1688_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    barrier(world)
    from paper_1108_1688_gb300 import hjm

    # The headline: the 256-caplet uneven batch (the batched workload of the
    # paper-shaped configurations and the largest single-GPU one), with the
    # 100-caplet batch and the 512x256x256 bandwidth-stress caplet measured
    # separately beside it.
    if args.workload == "headline":
        main_w, secondary = "config3", ["config2", "config4"]
    else:
        main_w, secondary = args.workload, []
    line, items = measure(main_w, args, world, local, hjm)
    if secondary:
        line["secondary"] = []
        for w in secondary:
            sub, _ = measure(w, args, world, local, hjm)
            line["secondary"].append({k: sub[k] for k in ("value", "unit", "ms_per_step", "dtype", "config",
                                                          "e2e", "gpu_launches", "clocks", "roofline",
                                                          "kernel_shares")})
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            oracle.build(omp=True)
            line["cpu_baseline"] = cpu_baseline(items)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "config1", "config2", "config3", "config4", "config5", "paper63"],
                    help="headline (default): the 256-caplet uneven batch, with the 100-caplet batch and the "
                         "512x256x256 caplet measured beside it")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--mixed-tol", type=float, default=1e-4,
                    help="MIXED: relative tolerance of the rounding bound (a small one forces FP64 re-pricing)")
    ap.add_argument("--scheme", default="douglas", choices=list(SCHEMES),
                    help="ADI scheme: the paper's Douglas, or Craig-Sneyd / modified CS / Hundsdorfer-Verwer")
    ap.add_argument("--ref-steps-per-step", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="use the default launch shapes")
    ap.add_argument("--tile", default=None,
                    help="launch shape for every grid shape of the workload: 7 integers "
                         "p1_lanes,p1_nodes,p1_lines,p2_warps,p3_warps,p1_staged,p1_planes")
    ap.add_argument("--tiles", default=None,
                    help="JSON file of launch shapes: read if it exists (no autotuning), else written "
                         "after autotuning (profiling runs replay the same shapes)")
    ap.add_argument("--instruments", type=int, default=None, help="config2 only: fewer caplets (profiling)")
    ap.add_argument("--march-steps", type=int, default=None, help="config2/4: fewer Douglas steps (profiling)")
    ap.add_argument("--labels", type=int, default=1 << 20, help="config5: PDE labels")
    ap.add_argument("--epochs", type=int, default=120, help="config5: training epochs")
    ap.add_argument("--label-grid", default="96x48x48x192", help="config5: label march n_r x n_y x n_v x steps")
    ap.add_argument("--label-check", type=int, default=4096,
                    help="config5: in-box rows priced on the label grid and on 128x64x64x256")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "config5":
        run_surrogate(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
