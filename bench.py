#!/usr/bin/env python3
"""Throughput of the Kadir-Brady saliency hot path on B300.

One step = the whole hot path over one synthetic PET-shaped volume
(128x128x64 float32, 32 bins, radii 4..20, seed stride 8): binning, the
dense sweep at every voxel, octant hill-climbing from every grid seed and
mean shift for every (seed, radius) item.  The metric is window-entropies
per second: one window-entropy is one (centre, window) histogram whose
entropy is evaluated (dense: voxels x scales; octant: 8 x scales per
iteration run plus the final scales, where a search whose centres repeat
stops running iterations; mean shift: one per iteration).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ks|reference]

Prints one JSON line.  --impl reference times the CPU oracle instead, on a
bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "window-entropies/s"
WORKLOAD = "pet128"


# dram__bytes_read.sum and dram__bytes_write.sum of one k_dense launch on the
# pet128 workload, captured with ncu (launch path 4 with its unrolled entry
# loop, 4 warps in 4x1 rows, the autotuner's shape; profiles/k_dense_pet128.md):
# the padded bin volume is read once; the Y
# and s_best outputs (9 bytes per voxel) stay in L2 at the end of the launch,
# so the capture shows almost no writes.  They leave L2 later, so the line's
# traffic counts them as written.
DENSE_DRAM_READ = 3_784_448
DENSE_DRAM_WRITE = 512


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.seek(0)
        rows = [l.split(",") for l in self.f.read().strip().splitlines() if l.strip()]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if len(r) > 5 + k and r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def octant_run(res, traj):
    """Iterations and window passes the octant kernel runs per seed.  A
    converged search runs its iterations (the last pass serves the final
    evaluation).  A search whose centre after iteration t repeats the one
    after t - p (2 <= p <= 8) stops after t iterations and needs a final
    pass unless its centre at max_iter is the last pass's centre.  Any
    other search runs max_iter iterations and a final pass."""
    it = res["iters"].astype(np.int64)
    conv = res["converged"] != 0
    M = traj.shape[1] - 1
    stop = np.full(len(it), M, np.int64)
    final_at = np.zeros(len(it), bool)        # the final centre is the last pass's
    open_ = ~conv
    for t in range(2, M + 1):
        hit = np.zeros(len(it), bool)
        for p in range(2, min(t, 8) + 1):
            hit |= (traj[:, t] == traj[:, t - p]).all(1)
        new = open_ & hit
        stop[new] = t
        final_at[new] = (traj[new, M] == traj[new, t - 1]).all(1)
        open_ &= ~hit
    run_it = np.where(conv, it, stop)
    passes = np.where(conv, it, stop + (~final_at).astype(np.int64))
    return run_it, passes


def window_entropies(n_vox, S, oct_res, ms_res, oct_run_iters):
    """Histograms whose entropy the step evaluated (see module docstring)."""
    dense = n_vox * S
    octant = int(oct_run_iters.sum()) * 8 * S + len(oct_res) * S
    ms = int(ms_res["iters"].sum()) + int((ms_res["converged"] == 0).sum())
    return dense + octant + ms, {"dense": dense, "octant": octant, "meanshift": ms}


# --------------------------------------------------------------- CPU oracle
def oracle_sample(w, budget_s=12.0, nthreads=0):
    """Time the oracle on a bounded sample of the workload: a random subset of
    dense centres, of octant seeds and of mean-shift seeds, sized so the
    whole sample takes about budget_s seconds.  Returns (window-entropies/s,
    threads, description)."""
    import oracle
    b = oracle.bin_volume(w.volume, w.binning)
    B, S = w.binning["bins"], w.r_max - w.r_min + 1
    nz, ny, nx = w.volume.shape
    rng = np.random.default_rng(0)
    seeds = oracle.seed_grid(w.dims, w.stride)
    oracle.tables(oracle.ball_size(w.r_max))
    threads = nthreads or oracle.max_threads()
    # calibrate: a small sample of each part
    parts = []
    n_c, n_o, n_m = 4096, 32, 16
    t0 = time.perf_counter()
    cen = np.stack([rng.integers(0, nx, n_c), rng.integers(0, ny, n_c),
                    rng.integers(0, nz, n_c)], 1).astype(np.int32)
    oracle.dense(b, B, w.r_min, w.r_max, centres=cen, nthreads=threads)
    t1 = time.perf_counter()
    so = seeds[rng.choice(len(seeds), n_o, replace=False)]
    o = oracle.octant_climb(b, B, w.r_min, w.r_max, so, w.max_iter, nthreads=threads)
    t2 = time.perf_counter()
    sm = seeds[rng.choice(len(seeds), n_m, replace=False)]
    m = oracle.meanshift(b, B, w.r_min, w.r_max, sm, w.max_iter, nthreads=threads)
    t3 = time.perf_counter()
    # scale each part to ~budget/3 seconds (the seed parts are capped at the
    # whole grid; the dense sample takes up what they leave), then rescale
    # once if the sample ran well short of the budget
    per_c = max(t1 - t0, 1e-3) / n_c
    k_o = max(1.0, budget_s / 3 / max(t2 - t1, 1e-3))
    k_m = max(1.0, budget_s / 3 / max(t3 - t2, 1e-3))
    n_o, n_m = min(len(seeds), int(n_o * k_o)), min(len(seeds), int(n_m * k_m))
    t_seeds = (t2 - t1) * n_o / 32 + (t3 - t2) * n_m / 16
    n_c = max(n_c, int(max(budget_s / 3, budget_s - t_seeds) / per_c))
    for attempt in range(2):
        cen = np.stack([rng.integers(0, nx, n_c), rng.integers(0, ny, n_c),
                        rng.integers(0, nz, n_c)], 1).astype(np.int32)
        so = seeds[rng.choice(len(seeds), n_o, replace=False)]
        sm = seeds[rng.choice(len(seeds), n_m, replace=False)]
        t0 = time.perf_counter()
        oracle.dense(b, B, w.r_min, w.r_max, centres=cen, nthreads=threads)
        t_d = time.perf_counter() - t0
        o = oracle.octant_climb(b, B, w.r_min, w.r_max, so, w.max_iter, nthreads=threads)
        m = oracle.meanshift(b, B, w.r_min, w.r_max, sm, w.max_iter, nthreads=threads)
        dt = time.perf_counter() - t0
        if dt >= 0.6 * budget_s or attempt == 1:
            break
        n_c = int(n_c * max(1.0, (budget_s - (dt - t_d)) / max(t_d, 1e-3)))
    we = n_c * S + int(o["iters"].sum()) * 8 * S + len(so) * S + int(m["iters"].sum()) + \
        int((m["converged"] == 0).sum())
    desc = (f"{n_c} random dense centres, {n_o} octant seeds and {n_m} mean-shift seeds "
            f"(x{S} radii) of the {WORKLOAD} workload, {dt:.1f} s")
    return we / dt, threads, desc, dt


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1310_6736_b300 import synth
    w = synth.workload(WORKLOAD)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_sample(w, budget_s=2.0)
    vals = []
    # keep the whole run to about two minutes of oracle work
    budget = max(0.5, min(args.ref_budget, 120.0 / max(1, args.steps)))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, threads, desc, dt = oracle_sample(w, budget_s=budget)
        vals.append(v)
    total = time.perf_counter() - t0
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "window-entropies/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "pet128: 128x128x64 float32, 32 bins, r=4..20, stride 8, "
                                   "dense + octant + mean shift", "sample": desc},
            "cpu_baseline": {"value": value, "unit": "window-entropies/s", "cores": threads,
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "window-entropies/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm
def run_ks(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1310_6736_b300 import build, ks, synth
    build.build()
    w = synth.workload(WORKLOAD, seed=1 + rank)        # each rank: its own volume (weak scaling)
    nz, ny, nx = w.volume.shape
    n_vox = nx * ny * nz
    S = w.r_max - w.r_min + 1
    params = ks.make_params(w.r_min, w.r_max, w.stride, w.max_iter)
    if args.dense_config:                               # pin the dense launch shape
        ks.force_dense_config(*[int(x) for x in args.dense_config.split(",")])
    ctx = ks.Context()
    stream = torch.cuda.current_stream()
    raw_dev = torch.from_numpy(w.volume).cuda()
    Y = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    sb = torch.empty((nz, ny, nx), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 126 MB L2

    dev_out = {}

    def step(host=False):
        """One step (binning, then the dense sweep and both seed searches in
        one ks_saliency call); every output stays on the device unless
        host=True."""
        v = ctx.create_volume(raw_dev, w.binning)
        if host:
            _, _, o, m = ctx.saliency(v, params, (nz, ny, nx))
        else:
            o, m = ctx.saliency(v, params, (nz, ny, nx), out=(Y, sb, dev_out["oct"], dev_out["ms"]))
        ctx.release_volume(v)
        return o, m

    flush.zero_()
    o, m = step(host=True)                 # host records: the window-entropy count
    v = ctx.create_volume(raw_dev, w.binning)
    o_t, traj = ctx.seed_climb(v, params, want_traj=True)
    ctx.release_volume(v)
    assert np.array_equal(o_t, o)
    oct_iters_run, _ = octant_run(o, traj)
    dev_out["oct"] = torch.empty(len(o) * ks.SEED_RESULT.itemsize, dtype=torch.uint8, device="cuda")
    dev_out["ms"] = torch.empty(len(m) * ks.MS_RESULT.itemsize, dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    n_we, parts = window_entropies(n_vox, S, o, m, oct_iters_run)

    # ---- timed region: device time per step with CUDA events on the stream
    ctx.set_profiling(True)
    launches0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    launches = ctx.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    dense_ms, dense_n = ctx.kernel_time("ks_dense")
    seeds_ms, seeds_n = ctx.kernel_time("ks_seeds")
    bin_ms, bin_n = ctx.kernel_time("ks_bin")
    ctx.set_profiling(False)
    if dist:
        t = torch.tensor([tot_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    ms_step = tot_ms / args.steps
    value = ws * n_we / (ms_step * 1e-3)
    # the device-resident records of the last timed step equal the host ones
    dev_same = (np.array_equal(dev_out["oct"].cpu().numpy().view(ks.SEED_RESULT), o) and
                np.array_equal(dev_out["ms"].cpu().numpy().view(ks.MS_RESULT), m))

    # ---- end to end through the C ABI with host buffers: the raw volume in
    # pinned host memory, every result copied back into pinned host arrays
    e2e_times = []
    h2d = w.volume.nbytes
    d2h = n_vox * 9 + len(o) * ks.SEED_RESULT.itemsize + len(m) * ks.MS_RESULT.itemsize

    def pinned(nbytes):
        return torch.empty(nbytes, dtype=torch.uint8, pin_memory=True).numpy()

    vol_h = pinned(w.volume.nbytes).view(w.volume.dtype).reshape(w.volume.shape)
    vol_h[...] = w.volume
    Yh = pinned(n_vox * 8).view(np.float64).reshape(nz, ny, nx)
    sh = pinned(n_vox).reshape(nz, ny, nx)
    oh = pinned(len(o) * ks.SEED_RESULT.itemsize).view(ks.SEED_RESULT)
    mh = pinned(len(m) * ks.MS_RESULT.itemsize).view(ks.MS_RESULT)
    n_e2e = max(3, min(args.steps, 10))
    for i in range(2 + n_e2e):          # 2 untimed: the host path's first calls size its buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v = ctx.create_volume(vol_h, w.binning)                       # host -> device inside
        ctx.saliency(v, params, (nz, ny, nx), host_out=(Yh, sh, oh, mh))  # device -> host inside
        ctx.release_volume(v)
        torch.cuda.synchronize()
        if i >= 2:
            e2e_times.append(time.perf_counter() - t0)
    e2e_value = ws * n_we / statistics.median(e2e_times)
    e2e_same = bool(np.array_equal(oh, o) and np.array_equal(mh, m))

    # ---- the dense sweep alone (no seed blocks beside it), for its own rate
    v = ctx.create_volume(raw_dev, w.binning)
    ctx.set_profiling(True)
    for _ in range(5):
        flush.zero_()
        ctx.dense_saliency(v, params, (nz, ny, nx), out=(Y, sb))
    alone_ms, alone_n = ctx.kernel_time("ks_dense")
    ctx.set_profiling(False)
    ctx.release_volume(v)

    # ---- roofline of the dominant kernel (dense sweep: shared-memory bound)
    smem_peak = ctx.measure_smem_peak()
    red_peak = ctx.measure_smem_red_rate()             # reductions alone: the strict ceiling
    fp64_rate = ctx.measure_fp64_rate()                # the FP64 sums' pipe, for context
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    upd_per_launch = n_vox * ks_ball_size(w.r_max)     # window-voxel updates per launch
    dense_avg_s = dense_ms / max(1, dense_n) * 1e-3
    achieved = upd_per_launch / dense_avg_s
    peaks, peak_kind = _peaks()
    line = None
    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": "window-entropies/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "pet128: 128x128x64 float32 PET-shaped volume, 32 bins, "
                                   "radii 4..20, seed stride 8; dense + octant + mean shift",
                       "l2": "flushed between steps (256 MB write)",
                       "step": "create_volume (binning), then one ks_saliency call: the dense sweep "
                               "on the highest-priority stream, octant climb and mean shift on the "
                               "lowest-priority stream beside it",
                       "window_entropies_per_step": n_we, "parts": parts,
                       "volumes_per_s": ws / (ms_step * 1e-3),
                       "step_ms_p50": statistics.median(step_ms),
                       "step_ms_p99": float(np.percentile(step_ms, 99)),
                       "parallelism": f"{ws} independent volume(s), one per GPU",
                       "outputs": "device-resident (Y, s_best, seed and mean-shift records); "
                                  "equal to the host-output run: " + str(bool(dev_same)),
                       "dense_launch": dict(zip(("path", "warps", "tile_y", "tile_z"),
                                                ([int(x) for x in args.dense_config.split(",")]
                                                 if args.dense_config else
                                                 ctx.dense_config(w.binning["bins"], w.r_max))
                                                or (None,) * 4))},
            "roofline": {"bound": "smem", "achieved": achieved / 1e9,
                         "peak": smem_peak / 1e9, "unit": "Gupdates/s",
                         "frac": achieved / smem_peak,
                         "traffic": DENSE_DRAM_READ + max(DENSE_DRAM_WRITE, n_vox * 9),
                         "traffic_unit": "bytes per launch: dram__bytes_read.sum of one ncu "
                                         "capture plus the outputs' 9 bytes per voxel, which "
                                         "the capture shows still in L2 and which are written "
                                         "back to DRAM after the launch",
                         "traffic_measured": {"dram_read": DENSE_DRAM_READ,
                                              "dram_write": DENSE_DRAM_WRITE,
                                              "deferred_output_bytes": n_vox * 9},
                         "kernel": "k_dense", "peak_source":
                             "shared-memory histogram-increment micro-kernel, measured live",
                         "kernel_ms": dense_ms / max(1, dense_n),
                         "kernel_share_of_step": dense_ms / max(1e-9, tot_ms),
                         "in_step": "the seed searches run beside the dense sweep's last wave, "
                                    "so its event time in the step includes sharing the SMs",
                         "frac_of_reduction_only_rate": achieved / red_peak,
                         "alone": {"kernel_ms": alone_ms / max(1, alone_n),
                                   "achieved": upd_per_launch / (alone_ms / max(1, alone_n) * 1e-3)
                                   / 1e9,
                                   "frac": upd_per_launch / (alone_ms / max(1, alone_n) * 1e-3)
                                   / smem_peak,
                                   "launches": alone_n}},
            "micro_peaks": {"smem_increments_per_s": smem_peak,
                            "smem_reductions_only_per_s": red_peak,
                            "fp64_dadd_per_s": fp64_rate,
                            "fp64_dadd_per_sm_clock": fp64_rate / (n_sms * 1e6 *
                                                                   (clocks.get("sm_mhz") or 2032.0)),
                            "how": "ks_measure_smem_peak / ks_measure_fp64_rate micro-kernels"},
            "kernels_note": "event times per launch on its own stream: the seed launches "
                            "start beside the dense sweep and include the wait for free SMs",
            "kernels": {"ks_dense": {"ms": dense_ms, "launches": dense_n},
                        "ks_seeds": {"ms": seeds_ms, "launches": seeds_n},
                        "ks_bin": {"ms": bin_ms, "launches": bin_n}},
            "e2e": {"value": e2e_value, "unit": "window-entropies/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "host_memory": "pinned",
                    "records_equal_device_run": e2e_same},
            "gpu_launches": launches,
            "clocks": clocks,
            "peaks_source": peak_kind,
        }
    if rank == 0 and not args.no_extras:
        # per-part rates and rooflines of the two seed kernels (each alone)
        line["seed_rooflines"] = seed_rooflines(ctx, ks, w, params, smem_peak, flush)
        line["config"]["parts_per_s"] = {
            "dense": parts["dense"] / (alone_ms / max(1, alone_n) * 1e-3),
            "octant": line["seed_rooflines"]["octant"]["window_entropies_per_s"],
            "meanshift": line["seed_rooflines"]["meanshift"]["window_entropies_per_s"],
            "note": "window-entropies/s of each part run alone on the same volume"}
        line["config"]["selection"] = run_selection(ctx, ks, w, params)
        line["config"]["abmsod"] = abmsod_summary(ctx, ks, w, params)
        # the metric's other configurations at their stated sizes
        line["config"]["mr256_seeds"] = run_mr256_seeds(ctx, ks, synth)
        line["config"]["mr256_dense"] = run_mr256_dense(ctx, ks, synth, smem_peak)
        rows, what, hbm, kind = binning_rows(ctx, ks)
        line["config"]["binning"] = {"workload": what, "peak_hbm_gbs": hbm, "rows": rows,
                                     "min_frac_of_hbm": min(r["frac_of_hbm"] for r in rows)}
        line["config"]["batched"] = run_batched(ctx, ks, synth, count=64, max_dim=None, reps=2)
        line["config"]["serving"] = run_serving(ks.Context, ks, synth, rate=50.0, count=2000,
                                                pool=32)
    if rank == 0 and not args.no_cpu_baseline:
        v_cpu, threads, desc, dt = oracle_sample(w, budget_s=args.ref_budget)
        line["cpu_baseline"] = {"value": v_cpu, "unit": "window-entropies/s", "cores": threads,
                                "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _grid_subset(w, step):
    """Every step-th seed of the workload's grid (x fastest, as the library
    lays the grid out): a smaller case of the same launch for profilers."""
    nz, ny, nx = w.volume.shape
    h = w.stride // 2
    zz, yy, xx = np.meshgrid(np.arange(h, nz, w.stride), np.arange(h, ny, w.stride),
                             np.arange(h, nx, w.stride), indexing="ij")
    grid = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(np.int32)
    return grid[::step].copy()


def run_case(args):
    """Run one part of the step (for profilers): --case dense|octant|meanshift|bin.
    --seed-step n: every n-th grid seed only (seed cases); --workload: the
    synthetic workload (default pet128); --max-dim m: its corner crop of at
    most m voxels per axis."""
    import torch
    from paper_1310_6736_b300 import build, ks, synth
    build.build()
    if args.dense_config:
        ks.force_dense_config(*[int(x) for x in args.dense_config.split(",")])
    w = synth.workload(args.workload)
    vol = w.volume
    if args.max_dim:                      # a corner crop (smaller profiler captures)
        vol = np.ascontiguousarray(vol[:args.max_dim, :args.max_dim, :args.max_dim])
    nz, ny, nx = vol.shape
    params = ks.make_params(w.r_min, w.r_max, w.stride, w.max_iter)
    ctx = ks.Context()
    raw_dev = torch.from_numpy(vol).cuda()
    Y = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    sb = torch.empty((nz, ny, nx), dtype=torch.uint8, device="cuda")
    v = ctx.create_volume(raw_dev, w.binning)
    seeds = _grid_subset(w, args.seed_step) if args.seed_step > 1 else None
    t = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if args.case == "dense":
            ctx.dense_saliency(v, params, (nz, ny, nx), out=(Y, sb))
        elif args.case == "octant":
            ctx.seed_climb(v, params, seeds=seeds)
        elif args.case == "quadrant":
            ctx.seed_climb(v, params, seeds=seeds, planar=True)
        elif args.case == "meanshift":
            ctx.meanshift(v, params, seeds=seeds)
        elif args.case == "bin":
            ctx.release_volume(v)
            v = ctx.create_volume(raw_dev, w.binning)
        torch.cuda.synchronize()
        if i >= args.warmup:
            t.append(time.perf_counter() - t0)
    print(json.dumps({"case": args.case, "workload": args.workload, "shape": [nz, ny, nx],
                      "ms": [1e3 * x for x in t],
                      "dense_config": ctx.dense_config(w.binning["bins"], w.r_max)}), flush=True)
    ctx.close()
    return 0


def run_selection(ctx, ks, w, params, reps=5):
    """Selection of salient regions after the seed searches (threshold,
    merge of equal regions, order by W, top 20) on the step's workload:
    candidate building for both schemes (mean shift: Kadir-Brady at every
    item's final centre) and the selection itself, host wall time of the
    synchronous calls, median of `reps`."""
    v = ctx.create_volume(w.volume, w.binning)
    o, m = ctx.seed_climb(v, params), ctx.meanshift(v, params)
    t = {"octant_candidates": [], "meanshift_candidates": [], "select_octant": [],
         "select_meanshift": []}
    for _ in range(reps + 1):
        t0 = time.perf_counter()
        oc = ctx.octant_candidates(o)
        t1 = time.perf_counter()
        mc = ctx.meanshift_candidates(v, params, m)
        t2 = time.perf_counter()
        so = ctx.select_salient(oc, h_min=0.0, top_k=20)
        t3 = time.perf_counter()
        sm = ctx.select_salient(mc, h_min=0.0, top_k=20)
        t4 = time.perf_counter()
        for k, dt in zip(t, (t1 - t0, t2 - t1, t3 - t2, t4 - t3)):
            t[k].append(dt)
    ctx.release_volume(v)
    out = {k + "_ms": 1e3 * statistics.median(x[1:]) for k, x in t.items()}
    out.update({"octant_candidates": len(oc), "meanshift_candidates": len(mc),
                "selected_octant": len(so), "selected_meanshift": len(sm),
                "top_W_octant": float(so["W"][0]) if len(so) else None,
                "top_W_meanshift": float(sm["W"][0]) if len(sm) else None})
    return out


def run_window(ctx, ks, synth, name, top_k=20):
    """Window-level constrained entropy (Sec. 3.2): both seed searches and
    the top-20 selection on the MR workload, over the full intensity range
    (mr256) or the tumour window (mr256w).  Reports the time of each part,
    how much of the window the exclusion leaves counted (N / |Ball(r)| over
    the mean-shift candidates) and how many of the top 20 lie in a tumour."""
    import torch
    w = synth.workload(name)
    p = ks.make_params(w.r_min, w.r_max, w.stride, w.max_iter)
    v = ctx.create_volume(w.volume, w.binning)
    t = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    o = ctx.seed_climb(v, p)
    t["octant_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    m = ctx.meanshift(v, p)
    t["meanshift_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    oc = ctx.octant_candidates(o)
    mc = ctx.meanshift_candidates(v, p, m)
    so = ctx.select_salient(oc, h_min=0.0, top_k=top_k)
    sm = ctx.select_salient(mc, h_min=0.0, top_k=top_k)
    t["selection_s"] = time.perf_counter() - t0
    # the entropy threshold (Sec. 2.3, end) drops near-empty windows
    by_h = {}
    for h_min in (0.0, 1.0, 2.0):
        a_, b_ = (ctx.select_salient(oc, h_min=h_min, top_k=top_k),
                  ctx.select_salient(mc, h_min=h_min, top_k=top_k))
        by_h[str(h_min)] = {"octant": [len(a_), None], "meanshift": [len(b_), None],
                            "_sel": (a_, b_)}
    # counted fraction of each mean-shift window: N = sum of the bin counts
    # at the final centre = |Ball(r)| minus the not-counted voxels
    xyz = np.stack([m["x"], m["y"], m["z"]], 1)
    bins = ctx.volume_bins(v, w.volume.shape)
    ctx.release_volume(v)
    frac = []
    for i in range(0, len(m), max(1, len(m) // 400)):      # a sample of items
        x, y, z, r = int(m["x"][i]), int(m["y"][i]), int(m["z"][i]), int(m["r"][i])
        zz, yy, xx = np.ogrid[-r:r + 1, -r:r + 1, -r:r + 1]
        ball = zz * zz + yy * yy + xx * xx <= r * r
        sub = np.zeros((2 * r + 1,) * 3, np.uint8)
        nz, ny, nx = bins.shape
        z0, y0, x0 = max(0, z - r), max(0, y - r), max(0, x - r)
        z1, y1, x1 = min(nz, z + r + 1), min(ny, y + r + 1), min(nx, x + r + 1)
        sub[z0 - (z - r):z1 - (z - r), y0 - (y - r):y1 - (y - r), x0 - (x - r):x1 - (x - r)] = \
            bins[z0:z1, y0:y1, x0:x1]
        frac.append(float(((sub > 0) & ball).sum()) / float(ball.sum()))
    def hits(sel):
        return int(synth.in_tumour(w.meta, np.stack([sel["x"], sel["y"], sel["z"]], 1)).sum())
    for row in by_h.values():
        a_, b_ = row.pop("_sel")
        row["octant"][1], row["meanshift"][1] = hits(a_), hits(b_)
    return {"workload": name, "binning": w.binning, "seeds": len(o), "items": len(m),
            "selected_and_in_tumour_by_h_min": by_h,
            **{k: round(v_, 4) for k, v_ in t.items()},
            "counted_fraction_mean": float(np.mean(frac)) if frac else None,
            "tumours": len(w.meta.get("tumours", [])),
            "top20_in_tumour_octant": hits(so), "top20_in_tumour_meanshift": hits(sm),
            "octant_converged": int(o["converged"].sum()),
            "meanshift_converged": int(m["converged"].sum())}


def _closed_octant_updates(r):
    """Shared-memory updates of one octant pass over Ball(r): each offset
    counts once per closed octant it belongs to, 2^(zero components)."""
    g = np.arange(-r, r + 1)
    o = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    o = o[(o ** 2).sum(1) <= r * r]
    return int((2 ** (o == 0).sum(1)).sum())


def _passes(res):
    """Window passes of seed searches: one per iteration, plus the final
    pass at the centre where the last iteration moved (no convergence)."""
    return res["iters"].astype(np.int64) + (res["converged"] == 0)


def seed_rooflines(ctx, ks, w, params, smem_peak, flush, reps=5):
    """The two seed kernels alone on workload w (device outputs, L2 flushed
    between launches), against the measured shared-memory update rate:
    octant climb = closed-octant updates of Ball(r_max) per pass; mean
    shift = |Ball(r)| window voxels per pass of each (seed, r) item."""
    import torch
    v = ctx.create_volume(w.volume, w.binning)
    o, traj = ctx.seed_climb(v, params, want_traj=True)
    m = ctx.meanshift(v, params)
    od = torch.empty(len(o) * ks.SEED_RESULT.itemsize, dtype=torch.uint8, device="cuda")
    md = torch.empty(len(m) * ks.MS_RESULT.itemsize, dtype=torch.uint8, device="cuda")
    out = {}
    o_it, o_passes = octant_run(o, traj)
    oct_upd = int(o_passes.sum()) * _closed_octant_updates(w.r_max)
    ms_upd = int((_passes(m) * np.array([ks_ball_size(int(r)) for r in m["r"]])).sum())
    S = w.r_max - w.r_min + 1
    oct_we = int(o_it.sum()) * 8 * S + len(o) * S
    ms_we = int(m["iters"].sum()) + int((m["converged"] == 0).sum())
    for name, fn, upd, we, prefix in (
            ("octant", lambda: ctx.seed_climb(v, params, out=od), oct_upd, oct_we, "ks_seeds"),
            ("meanshift", lambda: ctx.meanshift(v, params, out=md), ms_upd, ms_we,
             "ks_seeds_persistent")):
        fn()
        ctx.set_profiling(True)
        for _ in range(reps):
            flush.zero_()
            fn()
        ms, n = ctx.kernel_time(prefix)
        ctx.set_profiling(False)
        t = ms / max(1, n) * 1e-3
        out[name] = {"kernel": "k_seeds<" + name + ">", "kernel_ms": t * 1e3,
                     "updates_per_launch": upd, "achieved_gupdates_s": upd / t / 1e9,
                     "frac_of_smem_peak": upd / t / smem_peak,
                     "window_entropies_per_launch": we,
                     "window_entropies_per_s": we / t, "launches": n}
    ctx.release_volume(v)
    out["unit"] = ("shared-memory histogram updates (octant: one per voxel and closed octant of "
                   "each pass the kernel runs; mean shift: one per window voxel of each pass)")
    out["octant"]["passes_run"] = int(o_passes.sum())
    out["octant"]["passes_of_every_iteration"] = int(_passes(o).sum())
    return out


def run_mr256_seeds(ctx, ks, synth, reps=3):
    """The MR-shaped workload's seed searches at full size (256x256x160
    int16, 64 bins, r = 4..32, stride 12: 5733 seeds, 166 257 mean-shift
    items): octant climb and mean shift, results on the device, CUDA events
    around the two calls."""
    import torch
    w = synth.workload("mr256")
    params = ks.make_params(w.r_min, w.r_max, w.stride, w.max_iter)
    v = ctx.create_volume(w.volume, w.binning)
    o, traj = ctx.seed_climb(v, params, want_traj=True)
    m = ctx.meanshift(v, params)
    od = torch.empty(len(o) * ks.SEED_RESULT.itemsize, dtype=torch.uint8, device="cuda")
    md = torch.empty(len(m) * ks.MS_RESULT.itemsize, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    times = {"octant": [], "meanshift": []}
    for _ in range(reps):
        for name, fn in (("octant", lambda: ctx.seed_climb(v, params, out=od)),
                         ("meanshift", lambda: ctx.meanshift(v, params, out=md))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            torch.cuda.synchronize()
            times[name].append(a.elapsed_time(b))
    same = (np.array_equal(od.cpu().numpy().view(ks.SEED_RESULT), o) and
            np.array_equal(md.cpu().numpy().view(ks.MS_RESULT), m))
    ctx.release_volume(v)
    S = w.r_max - w.r_min + 1
    oct_we = int(octant_run(o, traj)[0].sum()) * 8 * S + len(o) * S
    ms_we = int(m["iters"].sum()) + int((m["converged"] == 0).sum())
    t_o, t_m = min(times["octant"]), min(times["meanshift"])
    return {"workload": "mr256: 256x256x160 int16 MR-shaped, 64 bins, r = 4..32, stride 12",
            "seeds": len(o), "meanshift_items": len(m),
            "octant_ms": t_o, "meanshift_ms": t_m,
            "window_entropies": oct_we + ms_we,
            "window_entropies_per_s": (oct_we + ms_we) / ((t_o + t_m) * 1e-3),
            "volumes_per_s": 1e3 / (t_o + t_m), "device_records_equal_host": bool(same)}


def run_mr256_dense(ctx, ks, synth, smem_peak, reps=2):
    """The dense sweep of the MR-shaped volume (256x256x160 int16, 64 bins,
    r = 4..32), whose counts pass 16 bits: the wide launch paths.  The first
    call autotunes; then `reps` calls with the L2 flushed before each, the
    dense kernel's CUDA-event time.  Updates = centres x |Ball(r_max)|."""
    import torch
    w = synth.workload("mr256")
    params = ks.make_params(w.r_min, w.r_max, w.stride, w.max_iter)
    nz, ny, nx = w.volume.shape
    v = ctx.create_volume(w.volume, w.binning)
    Y = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    sb = torch.empty((nz, ny, nx), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ctx.dense_saliency(v, params, (nz, ny, nx), out=(Y, sb))
    ctx.set_profiling(True)
    for _ in range(reps):
        flush.zero_()
        ctx.dense_saliency(v, params, (nz, ny, nx), out=(Y, sb))
    k_ms, k_n = ctx.kernel_time("ks_dense")
    ctx.set_profiling(False)
    ctx.release_volume(v)
    ms = k_ms / max(k_n, 1)
    centres = nx * ny * nz
    upd = centres * ks_ball_size(w.r_max)
    S = w.r_max - w.r_min + 1
    return {"workload": "mr256: 256x256x160 int16 MR-shaped, 64 bins, r = 4..32, every voxel",
            "launch": ctx.dense_config(w.binning["bins"], w.r_max), "kernel_ms": ms,
            "updates_per_launch": upd, "achieved_gupdates_s": upd / (ms * 1e-3) / 1e9,
            "frac_of_smem_peak": upd / (ms * 1e-3) / smem_peak,
            "window_entropies_per_s": centres * S / (ms * 1e-3)}


def binning_rows(ctx, ks, steps=10, warmup=3):
    """Binning alone, an HBM-bound kernel: three raw types on a 1024x1024x256
    volume (every raw input at least twice the 126 MB L2, which is not
    flushed between the calls).  Per type, the ks_bin kernels'
    CUDA-event time over `steps` calls of ks_create_volume from device
    memory; the algorithmic bytes are the raw read (float32 also its min/max
    pass) plus one byte written per voxel.  A fourth row times the float32
    binning through ks_bin_f32_noalloc on the same volume: CUDA events on
    the stream around `steps` back-to-back calls (its two kernels per call,
    launch gaps included)."""
    import torch
    nz, ny, nx = 256, 1024, 1024
    n = nx * ny * nz
    peaks, kind = _peaks()
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    cases = [
        ("uint8, v >> 3 (32 bins)", lambda: torch.randint(0, 256, (nz, ny, nx), generator=g,
                                                          device="cuda", dtype=torch.uint8),
         {"kind": 0, "bins": 32, "shift": 3, "lo": 0, "hi": 255}, 2),
        ("int16, clamp to [0, 2047] >> 5 (64 bins)",
         lambda: torch.randint(-100, 2200, (nz, ny, nx), generator=g, device="cuda",
                               dtype=torch.int16),
         {"kind": 0, "bins": 64, "shift": 5, "lo": 0, "hi": 2047}, 3),
        ("float32, affine over [vmin, vmax] (32 bins; min/max pass)",
         lambda: torch.rand((nz, ny, nx), generator=g, device="cuda", dtype=torch.float32) * 100.0,
         {"kind": 1, "bins": 32, "shift": 0, "lo": 0, "hi": 0}, 9),
    ]
    rows = []
    for name, make, binning, bpv in cases:
        raw = make()
        for _ in range(warmup):
            ctx.release_volume(ctx.create_volume(raw, binning))
        ctx.set_profiling(True)
        for _ in range(steps):
            ctx.release_volume(ctx.create_volume(raw, binning))
        ms, launches = ctx.kernel_time("ks_bin")
        ctx.set_profiling(False)
        del raw
        t = ms / max(1, launches) * 1e-3
        gbs = n * bpv / t / 1e9
        rows.append({"raw": name, "voxels": n, "bytes_per_voxel": bpv, "ms": t * 1e3,
                     "achieved_gbs": gbs, "frac_of_hbm": gbs / peaks["hbm_gbs"],
                     "entry": "ks_create_volume"})
        if binning["kind"] == 1:
            import ctypes as C
            raw = make()
            out = torch.empty(n, dtype=torch.uint8, device="cuda")
            s = torch.cuda.current_stream()
            lib = ks.lib()

            def call():
                return lib.ks_bin_f32_noalloc(C.c_void_p(raw.data_ptr()), nx, ny, nz, 32,
                                              C.c_void_p(out.data_ptr()),
                                              C.c_void_p(s.cuda_stream))
            for _ in range(warmup):
                assert call() == 0
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            for _ in range(steps):
                assert call() == 0
            b.record(s)
            b.synchronize()
            t = a.elapsed_time(b) / steps * 1e-3
            gbs = n * bpv / t / 1e9
            rows.append({"raw": name, "voxels": n, "bytes_per_voxel": bpv, "ms": t * 1e3,
                         "achieved_gbs": gbs, "frac_of_hbm": gbs / peaks["hbm_gbs"],
                         "entry": "ks_bin_f32_noalloc (no device allocation; event time "
                                  "of back-to-back calls)"})
            del raw, out
    return rows, f"{nx}x{ny}x{nz} random volumes", peaks["hbm_gbs"], kind


def run_batched(ctx, ks, synth, count=64, max_dim=None, reps=3):
    """Batched form: `count` uneven volumes (uint8 spheres / int16 MR-like),
    octant climb + mean shift for every grid seed of every volume, as one
    persistent graph-captured launch vs one plain launch pair per volume.
    Both produce host results.  Returns a dict of volumes/s and timings."""
    import torch
    ws = synth.batch_volumes(seed=3, count=count, max_dim=max_dim)
    vols = [ctx.create_volume(w.volume, w.binning) for w in ws]
    ps = [ks.make_params(w.r_min, w.r_max, w.stride, w.max_iter) for w in ws]
    ctx.batch_seeds(vols, ps, kinds=3, use_graph=True)          # capture + warm
    for v, p in zip(vols, ps):
        ctx.seed_climb(v, p)
        ctx.meanshift(v, p)
    plain, batched = [], []
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        outs = [(ctx.seed_climb(v, p), ctx.meanshift(v, p)) for v, p in zip(vols, ps)]
        torch.cuda.synchronize()
        plain.append(time.perf_counter() - t)
        t = time.perf_counter()
        octs, mss = ctx.batch_seeds(vols, ps, kinds=3, use_graph=True)
        torch.cuda.synchronize()
        batched.append(time.perf_counter() - t)
    same = all(np.array_equal(o[0], a) and np.array_equal(o[1], b)
               for o, a, b in zip(outs, octs, mss))
    we = 0
    for (o, m), p in zip(outs, ps):
        S = p.r_max - p.r_min + 1
        we += int(o["iters"].sum()) * 8 * S + len(o) * S + int(m["iters"].sum()) + \
            int((m["converged"] == 0).sum())
    for v in vols:
        ctx.release_volume(v)
    tp, tb = min(plain), min(batched)
    return {"volumes": count, "max_dim": max_dim or 256, "seeds": int(sum(len(o[0]) for o in outs)),
            "window_entropies": we, "plain_s": tp, "batched_s": tb,
            "volumes_per_s_plain": count / tp, "volumes_per_s_batched": count / tb,
            "window_entropies_per_s_batched": we / tb, "speedup": tp / tb,
            "identical_results": bool(same)}


def run_serving(ctx_factory, ks, synth, rate=50.0, count=2000, pool=32, max_dim=None,
                dense_frac=0.3, seed=4, wave_iters=None):
    """Serving form: a Poisson stream of `count` requests at `rate`/s, each a
    volume from a pool drawn like the batched form (dims log-uniform in
    [48, 256], z <= 160; uint8 spheres / int16 MR-like), asking for both
    seed schemes (70%) or the dense sweep (30%).  Two arms replay the same
    stream in real time:
      - serving: the continuous-batching loop (ks_submit from a client
        thread at the arrival times, ks_poll for every result);
      - sequential: the plain path, one request at a time in arrival order
        (a request that arrives while another runs waits): create_volume
        from pinned host memory, the synchronous calls, results to host.
    Latency is completion minus arrival; volumes/s is requests over the
    span from the first arrival to the last completion."""
    import threading
    import torch
    reqs = synth.request_stream(seed=seed, count=count, rate=rate, dense_frac=dense_frac)
    ws = synth.batch_volumes(seed=seed + 100, count=pool, max_dim=max_dim)
    kinds = [ks.KS_REQ_DENSE if r["kind"] == "dense" else ks.KS_REQ_SEEDS for r in reqs]
    picks = [r["vol_seed"] % pool for r in reqs]
    params = [ks.make_params(w.r_min, w.r_max, w.stride, w.max_iter) for w in ws]
    # warm-up: every pool volume once as a seed request and once as a dense
    # sweep, so the dense autotuner has timed every class it will meet
    # (its measurements are shared by every context of the process, so
    # both arms below run with the same tuned shapes) and every kernel
    # variant is loaded
    ctx = ctx_factory()
    if wave_iters is not None:
        ctx.set_serve_wave_iters(wave_iters)
    for i in range(pool):
        for k in (ks.KS_REQ_SEEDS, ks.KS_REQ_DENSE):
            rid = ctx.submit(ws[i].volume, ws[i].binning, params[i], kind=k)
            ctx.poll(rid, -1)
            ctx.release_result(rid)
    ctx.set_profiling(True)
    ids = [None] * count
    t0 = time.perf_counter()
    t0_us = None

    def submitter():
        for i, r in enumerate(reqs):
            now = time.perf_counter() - t0
            if r["t"] > now:
                time.sleep(r["t"] - now)
            ids[i] = ctx.submit(ws[picks[i]].volume, ws[picks[i]].binning, params[picks[i]],
                                kind=kinds[i])

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat = []
    t_first, t_last = None, 0.0
    for i in range(count):
        st, res = ctx.poll(ids[i], -1)
        assert st == ks.KS_OK, st
        lat.append((res["t_done_us"] - res["t_submit_us"]) * 1e-3)
        t_first = res["t_submit_us"] if t_first is None else min(t_first, res["t_submit_us"])
        t_last = max(t_last, res["t_done_us"])
        ctx.release_result(ids[i])
    span = (t_last - t_first) * 1e-6
    seeds_ms, seeds_n = ctx.kernel_time("ks_seeds")
    dense_ms, dense_n = ctx.kernel_time("ks_dense")
    ctx.close()

    # sequential arm, measured: one worker, arrival order, real time
    ctx = ctx_factory()
    pinned = []
    for w in ws:
        h = torch.empty(w.volume.nbytes, dtype=torch.uint8, pin_memory=True).numpy()
        h = h.view(w.volume.dtype).reshape(w.volume.shape)
        h[...] = w.volume
        pinned.append(h)

    def plain(i):
        k = picks[i]
        v = ctx.create_volume(pinned[k], ws[k].binning)
        if kinds[i] == ks.KS_REQ_DENSE:
            ctx.dense_saliency(v, params[k], ws[k].volume.shape)
        else:
            ctx.seed_climb(v, params[k])
            ctx.meanshift(v, params[k])
        ctx.release_volume(v)

    for i in range(min(pool, 8)):                 # warm-up
        plain(picks.index(i) if i in picks else 0)
    torch.cuda.synchronize()
    seq_lat = []
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        now = time.perf_counter() - t0
        if r["t"] > now:
            time.sleep(r["t"] - now)
        plain(i)
        seq_lat.append((time.perf_counter() - t0 - r["t"]) * 1e3)
    seq_span = time.perf_counter() - t0 - reqs[0]["t"]
    ctx.close()
    return {"rate_per_s": rate, "requests": count, "pool_volumes": pool,
            "max_dim": max_dim or 256, "dense_fraction": dense_frac,
            "wave_iters": 0 if wave_iters is None else wave_iters,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "volumes_per_s": count / span, "span_s": span,
            "device_busy": {"seed_waves_ms": seeds_ms, "seed_launches": seeds_n,
                            "dense_ms": dense_ms, "dense_launches": dense_n,
                            "note": "CUDA-event time of the serving streams' launches; waves "
                                    "and dense sweeps overlap, so the sum can exceed the span"},
            "sequential_p50_ms": float(np.percentile(seq_lat, 50)),
            "sequential_p99_ms": float(np.percentile(seq_lat, 99)),
            "sequential_volumes_per_s": count / seq_span, "sequential_span_s": seq_span,
            "sequential": "measured: the plain calls, one request at a time in arrival order"}


# FP32 and INT32 lane operations the ABMSOD definition takes per window
# voxel of a kernel histogram, with the sums pass that reuses the window:
# histogram 16 (offset 1, d 2, kernel 10, rounding 2, sum 1), position sums
# 29, bandwidth sums 36; the two halves of an iteration give 45 and 52.
AB_OPS_PER_VOXEL = 48.5

# dram__bytes_read.sum + dram__bytes_write.sum of one k_abmsod launch on the
# pet128 workload (profiles/k_abmsod_pet128.md, medians over 17 launches):
# the touched part of the bin volume is read about once, the 34,816 records
# are written.
AB_DRAM_BYTES = 4_410_000


def abmsod_summary(ctx, ks, w, params, reps=3):
    """ABMSOD (Alg. 2) for every (grid seed, r) of the step's volume: device
    time of one ks_abmsod call (median of reps, CUDA events)."""
    import torch
    v = ctx.create_volume(w.volume, w.binning)
    n = ctx.seed_count(v, params) * (w.r_max - w.r_min + 1)
    out = torch.empty(n * ks.AB_RESULT.itemsize, dtype=torch.uint8, device="cuda")
    ctx.abmsod(v, params, out=out)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.abmsod(v, params, out=out)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    rec = out.cpu().numpy().view(ks.AB_RESULT)
    ctx.release_volume(v)
    ms = statistics.median(ts)
    return {"candidates": n, "iterations": int(rec["iters"].sum()),
            "window_voxels": int(rec["voxels"].sum()), "ms": ms,
            "candidate_iterations_per_s": int(rec["iters"].sum()) / (ms * 1e-3),
            "full_measurement": "python bench.py --mode abmsod"}


def run_abmsod(args):
    """Adaptive-bandwidth mean shift (Alg. 2, Eq. 7) for every (grid seed, r)
    of the PET-shaped workload, device-resident inputs and outputs; one
    step = one ks_abmsod call over all 2048 x 17 candidates."""
    import torch
    from paper_1310_6736_b300 import build, ks, synth
    build.build()
    torch.cuda.set_device(0)
    w = synth.workload(WORKLOAD)
    params = ks.make_params(w.r_min, w.r_max, w.stride, w.max_iter)
    ks.set_abmsod_team_radius(args.team_radius)
    ctx = ks.Context()
    stream = torch.cuda.current_stream()
    raw_dev = torch.from_numpy(w.volume).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    v = ctx.create_volume(raw_dev, w.binning)
    grid = None
    if args.seed_step > 1:        # a smaller case of the same launch (profiling)
        grid = _grid_subset(w, args.seed_step)
    n_seeds = len(grid) if grid is not None else ctx.seed_count(v, params)
    n_items = n_seeds * (w.r_max - w.r_min + 1)
    out = torch.empty(n_items * ks.AB_RESULT.itemsize, dtype=torch.uint8, device="cuda")
    host = ctx.abmsod(v, params, seeds=grid)
    iters, voxels = int(host["iters"].sum()), int(host["voxels"].sum())
    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        ctx.abmsod(v, params, seeds=grid, out=out)
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    launches0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(0) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            ctx.abmsod(v, params, seeds=grid, out=out)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    k_ms, k_n = ctx.kernel_time("ks_abmsod")
    ctx.set_profiling(False)
    same = np.array_equal(out.cpu().numpy().view(ks.AB_RESULT), host)
    # the paper's LV-detection shape (Sec. 3.1): 400 candidate positions
    # scattered at random over the volume, here each at every radius
    rng = np.random.default_rng(11)
    nz, ny, nx = w.volume.shape
    scatter = np.stack([rng.integers(0, nx, 400), rng.integers(0, ny, 400),
                        rng.integers(0, nz, 400)], 1).astype(np.int32)
    sc_out = torch.empty(400 * (w.r_max - w.r_min + 1) * ks.AB_RESULT.itemsize,
                         dtype=torch.uint8, device="cuda")
    ctx.abmsod(v, params, seeds=scatter, out=sc_out)
    sc_ms = []
    for _ in range(5):
        a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.abmsod(v, params, seeds=scatter, out=sc_out)
        b_.record(stream)
        torch.cuda.synchronize()
        sc_ms.append(a.elapsed_time(b_))
    sc_rec = sc_out.cpu().numpy().view(ks.AB_RESULT)
    ctx.release_volume(v)
    ms = statistics.median(step_ms)
    # end to end through the C ABI: host volume in, host records out
    e2e = []
    for i in range(2 + max(3, min(args.steps, 10))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vh = ctx.create_volume(w.volume, w.binning)
        ctx.abmsod(vh, params, seeds=grid)
        ctx.release_volume(vh)
        torch.cuda.synchronize()
        if i >= 2:
            e2e.append(time.perf_counter() - t0)
    clocks = clk.summary()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 128 * (clocks["sm_max_mhz"] or 2032.0) * 1e6
    kernel_s = k_ms / max(1, k_n) * 1e-3
    achieved = AB_OPS_PER_VOXEL * voxels / kernel_s
    line = {
        "metric": "ABMSOD candidate-iterations/s", "value": iters / (ms * 1e-3),
        "unit": "candidate-iterations/s", "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 voxel terms, i64 sums, f64 per item",
        "data": "synthetic",
        "config": {"workload": "pet128: 128x128x64 float32 PET-shaped volume, 32 bins; ABMSOD "
                               "for every (grid seed, r), stride 8 (2048 seeds), r = 4..20, "
                               f"max {w.max_iter} iterations",
                   "candidates": n_items, "iterations": iters, "window_voxels": voxels,
                   "window_voxels_per_s": voxels / (ms * 1e-3),
                   "candidates_per_s": n_items / (ms * 1e-3),
                   "step_ms_p50": ms, "step_ms_max": max(step_ms),
                   "l2": "flushed between steps (256 MB write)",
                   "outputs": "device-resident records; equal to the host-output run: " +
                              str(bool(same)),
                   "scattered_400": {"candidates": len(sc_rec),
                                     "iterations": int(sc_rec["iters"].sum()),
                                     "ms": statistics.median(sc_ms),
                                     "paper": "4.1 s per PET volume on a Tesla C2050 for about "
                                              "400 candidates x 10 iterations (context only)"}},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                     "unit": "T lane-ops/s", "frac": achieved / peak, "traffic": AB_DRAM_BYTES,
                     "traffic_unit": "bytes per launch (dram read + write, ncu)",
                     "kernel": "k_abmsod", "kernel_ms": k_ms / max(1, k_n),
                     "ops_per_window_voxel": AB_OPS_PER_VOXEL,
                     "peak_source": f"{sms} SMs x 128 FP32/INT32 lanes x max SM clock"},
        "e2e": {"value": iters / statistics.median(e2e), "unit": "candidate-iterations/s",
                "h2d_bytes_per_step": int(w.volume.nbytes),
                "d2h_bytes_per_step": n_items * ks.AB_RESULT.itemsize},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        import oracle
        b = oracle.bin_volume(w.volume, w.binning)
        seeds = oracle.seed_grid(w.dims, w.stride)
        rng = np.random.default_rng(0)
        threads = oracle.max_threads()
        n = 4 * threads
        for attempt in range(3):      # calibrate, then about ref_budget seconds
            pick = seeds[rng.choice(len(seeds), n, replace=False)]
            t0 = time.perf_counter()
            r = oracle.abmsod(b, w.binning["bins"], w.r_min, w.r_max, pick, w.max_iter,
                              nthreads=threads)
            dt = time.perf_counter() - t0
            if attempt > 0 and (dt >= 0.6 * args.ref_budget or n == len(seeds)):
                break
            n = int(min(len(seeds), max(n, n * args.ref_budget / max(dt, 1e-3))))
        line["cpu_baseline"] = {"value": int(r["iters"].sum()) / dt,
                                "unit": "candidate-iterations/s", "cores": threads,
                                "kind": "oracle",
                                "sample": f"{n} random grid seeds x {w.r_max - w.r_min + 1} radii "
                                          f"of the {WORKLOAD} workload, {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_bin(args):
    """Binning alone (binning_rows) as its own line."""
    from paper_1310_6736_b300 import ks
    ctx = ks.Context()
    rows, what, hbm, kind = binning_rows(ctx, ks, steps=args.steps, warmup=max(args.warmup, 3))
    ctx.close()
    line = {"metric": "binning bandwidth (algorithmic bytes / kernel time)",
            "value": min(r["frac_of_hbm"] for r in rows), "unit": "fraction of measured HBM copy",
            "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": what, "peak_hbm_gbs": hbm, "peaks_source": kind,
                       "rows": rows}}
    print(json.dumps(line), flush=True)
    return 0


def run_mode(args):
    import torch
    from paper_1310_6736_b300 import build, ks, synth
    build.build()
    torch.cuda.set_device(0)
    if args.mode == "abmsod":
        return run_abmsod(args)
    if args.mode == "bin":
        return run_bin(args)
    if args.mode == "window":
        ctx = ks.Context()
        rows = [run_window(ctx, ks, synth, name) for name in ("mr256", "mr256w")]
        ctx.close()
        line = {"metric": "tumour detections among the top 20 (full range vs window level)",
                "value": rows[1]["top20_in_tumour_meanshift"], "unit": "detections",
                "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
                "config": {"workload": "256x256x160 int16 MR-like volume with 1-4 tumours, "
                                       "r = 4..32, stride 12", "rows": rows}}
    elif args.mode == "batch":
        ctx = ks.Context()
        r = run_batched(ctx, ks, synth, count=args.count, max_dim=args.max_dim or None)
        ctx.close()
        line = {"metric": "volumes/s (batched vs plain)", "value": r["volumes_per_s_batched"],
                "unit": "volumes/s", "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
                "config": {"workload": "batch of uneven uint8/int16 volumes", **r}}
    else:
        rows = [run_serving(ks.Context, ks, synth, rate=rate, count=args.count,
                            max_dim=args.max_dim or None, pool=args.pool,
                            wave_iters=None if args.wave_iters < 0 else args.wave_iters)
                for rate in args.rates]
        line = {"metric": "p50/p99 latency and volumes/s (continuous batching vs sequential)",
                "value": rows[0]["p50_ms"], "unit": "ms (p50)", "higher_is_better": False,
                "n_gpus": 1, "data": "synthetic", "config": {"serving": rows}}
    print(json.dumps(line), flush=True)
    return 0


def ks_ball_size(r):
    d = np.arange(-r, r + 1)
    return int(((d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2)
                <= r * r).sum())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ks", choices=["ks", "reference"])
    ap.add_argument("--ref-budget", type=float, default=15.0,
                    help="seconds of oracle work per reference sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=["pet128", "mr256", "spheres48"],
                    help="--case: the synthetic workload")
    ap.add_argument("--case", choices=["dense", "octant", "quadrant", "meanshift", "bin"],
                    help="run one part of the step only (profiling)")
    ap.add_argument("--dense-config", default="",
                    help="force the dense launch shape: path,warps,tile_y,tile_z")
    ap.add_argument("--mode", choices=["step", "batch", "serve", "window", "abmsod", "bin"],
                    default="step",
                    help="batch: batched vs plain launches; serve: request-stream latency; "
                         "window: full range vs tumour window level on the MR workload; "
                         "abmsod: adaptive-bandwidth mean shift on the PET-shaped workload")
    ap.add_argument("--count", type=int, default=64, help="volumes (batch) or requests (serve)")
    ap.add_argument("--seed-step", type=int, default=1,
                    help="abmsod mode and seed cases: every n-th grid seed only (a smaller case "
                         "for profilers)")
    ap.add_argument("--team-radius", type=int, default=0,
                    help="abmsod mode: ks_set_abmsod_team_radius (0: the library's per-launch "
                         "choice; 33: every item on one warp)")
    ap.add_argument("--max-dim", type=int, default=0, help="cap on each volume dimension")
    ap.add_argument("--rates", type=float, nargs="+", default=[20.0, 50.0, 100.0])
    ap.add_argument("--pool", type=int, default=32, help="serving: distinct volumes in the pool")
    ap.add_argument("--wave-iters", type=int, default=-1,
                    help="serving: iterations per seed item and wave (-1: the library default)")
    ap.add_argument("--no-extras", action="store_true",
                    help="step mode: skip the short batched and serving measurements")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)
    if args.mode != "step":
        return run_mode(args)
    return run_ks(args)


if __name__ == "__main__":
    sys.exit(main())
