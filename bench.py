"""Benchmark of the implicit r-z PIC/MCC step on GB300.

One step = the whole hot path: bin layout, fused particle kernel (gather, D1
push, null-collision MCC, re-bin, deposit), circuit, assembly, field solve,
E field, diagnostics.  Workload (default): the 512x256 GEC-like cell with
32 M electrons + 32 M Ar+ (30 mTorr, 150 V through the L-network), the largest
single-GPU configuration; c2 is the 256x128 cell with 4 M + 4 M.  Synthetic
seeded inputs.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c2|c3|c1] [--solver plain|mixed] [--precision fp32|fp64]

N > 1 (launched under torch.distributed.run): each rank runs an independent
replica of the discharge (different seed); value = all ranks' particle-steps
over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (push+MCC+deposit); field-solve ms to 1e-10 residual, vs plain"
# Algorithmic bytes per particle-step of the particle kernel: the state read once
# and written once.  The roofline uses the hot-path scope's figure, 2 x 44 B in FP32
# (eight FP32 state words, a 64-bit id and a 32-bit cell index); this store keeps the
# cell implicit in the particle's bin, so the kernel itself moves 2 x 40 B.
BYTES_PER_PARTICLE_STEP = {"fp32": 88, "fp64": 152}
STORED_BYTES_PER_PARTICLE_STEP = {"fp32": 80, "fp64": 144}
KERNELS_PER_STEP = 10  # layout x3, particles, circuit, assemble x2, solve, efield, diag
# (plus one per pic_step call: the step counter set on the device)
KERNELS_PER_WINDOW = 6  # diag window, C_eq refresh (edges, dirichlet, solve, energy), circuit propagator


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c4", "selfbias"])
    ap.add_argument("--periods", type=int, default=50, help="RF periods per amplitude (--workload selfbias)")
    ap.add_argument("--solver", default="mg", choices=["plain", "mixed", "mg"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tile", default="auto",
                    help="particle tile RxZ in cells, or auto: chosen by the tile autotuner before timing")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = ("push_kernels.cuh", "push.cu")


def kernel_traffic():
    """DRAM bytes per particle-kernel launch from the committed ncu summary, scaled to
    the bench's particle count, if the summary was taken on the current kernel source;
    else None."""
    p = os.path.join(ROOT, "profiles", "k_particles_gec256.md")
    csrc = os.path.join(ROOT, "paper_2310_04957_gb300", "csrc")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        line = line.strip()
        if ":" in line and line.split(":")[0] in ("traffic_bytes_per_launch", "particles_in_launch", "source_sha256"):
            k, v = line.split(":", 1)
            kv[k] = v.strip()
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:  # the particle kernel and its unweighted instance
        h.update(open(os.path.join(csrc, name), "rb").read())
    sha = h.hexdigest()
    if kv.get("source_sha256") != sha:
        return None
    return {"bytes": float(kv["traffic_bytes_per_launch"]), "particles": float(kv["particles_in_launch"])}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi takes a while to start: let its first sample arrive before
            # the timed region begins (at most 3 s)
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def across_ranks(ms, work, dist=None, device="cuda"):
    """Weak-scaling aggregate over the ranks of a replica run: the slowest rank's
    time and the sum of all ranks' work (one MAX and one SUM all-reduce; no
    data-path collective)."""
    if dist is None:
        return ms, work
    import torch

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([work], device=device, dtype=torch.float64)
    dist.all_reduce(w)
    return float(t.item()), float(w.item())


def make_workload(name, rank=0):
    from paper_2310_04957_gb300 import workloads as W

    wl = W.PRESETS[name]()
    if rank:
        import dataclasses

        wl = dataclasses.replace(wl, seed=(wl.seed + 1000 * rank) & 0xFFFFFFFF)
    return wl


# run length of each configuration (the end-to-end leg runs it whole): 400 steps
# of the small cylinder, 2000 steps of the 256x128 cell, 5 RF periods of the
# 512x256 cell
RUN_STEPS = {"c1": 400, "c2": 2000, "c3": 1000}


def make_workload_name(name):
    return {"c1": "cylinder-32x32-100k", "c2": "gec-256x128-8M", "c3": "gec-512x256-64M"}[name]


def cpu_baseline(wlname, seconds_target=12.0):
    """The FP64 oracle as it stands, single-threaded, on a bounded sample of the workload:
    the same grid, gas, circuit and field solve with 1/10 of the particles."""
    import dataclasses

    from oracle import orc
    from paper_2310_04957_gb300 import workloads as W

    frac = 10 if wlname != "c1" else 1
    full = W.PRESETS[wlname]
    n_full = {"c1": 50_000, "c2": 4_000_000, "c3": 32_000_000}[wlname]
    wl = full(n_per_species=n_full // frac)
    o = orc.Oracle(wl)
    o.init_fields()
    o.step(1)
    t0 = time.perf_counter()
    steps = 0
    ps = 0
    while True:
        n = o.count(0) + o.count(1)
        o.step(1)
        steps += 1
        ps += n
        if time.perf_counter() - t0 > seconds_target or steps >= 200:
            break
    dt = time.perf_counter() - t0
    return {"value": ps / dt, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{wl.name}: same grid/gas/circuit/field solve, {n_full // frac} particles per species "
                      f"(1/{frac} of the workload), {steps} full steps, FP64, single thread"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    base = cpu_baseline(args.workload, seconds_target=max(5.0, 2.0 * args.steps / 10))
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": make_workload_name(args.workload)}, "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def field_solve_comparison(wl, steps=5):
    """Field solve to 1e-10 relative residual from the same warm starts: plain FP64
    PCG, mixed PCG, multigrid-preconditioned mixed PCG, and the learned solves
    (network trained here, on this workload's own run, by the library's kernels:
    up to 3 network applications, then the mixed or the multigrid PCG finishes).
    Medians over `steps` consecutive steps of ms per pic_field_solve call
    (assembly + solve + E field + one scalar read)."""
    import statistics

    from paper_2310_04957_gb300 import learned as Lr
    from paper_2310_04957_gb300 import pic

    net, d, info = Lr.train_on_discharge(wl)
    d.keep_warm(True)
    modes = (pic.PIC_SOLVER_PLAIN, pic.PIC_SOLVER_MIXED, pic.PIC_SOLVER_MG)
    rows = {m: [] for m in modes}
    rows["learned_mixed"], rows["learned_mg"], rows["learned_mg_guess"] = [], [], []
    for _ in range(steps):
        d.step(1)
        r = Lr.compare_solvers(d, modes=modes, repeats=2)
        for m in modes:
            rows[m].append(r[m])
        # up to 3 network applications, or one (the learned initial guess alone)
        for key, fin, apps in (("learned_mixed", pic.PIC_SOLVER_MIXED, 3), ("learned_mg", pic.PIC_SOLVER_MG, 3),
                               ("learned_mg_guess", pic.PIC_SOLVER_MG, 1)):
            d.attach_unet(net, maxit=apps, finish=fin)
            rows[key].append(Lr.compare_solvers(d, modes=(pic.PIC_SOLVER_LEARNED,), repeats=2)[pic.PIC_SOLVER_LEARNED])
    med = lambda m, k: statistics.median(x[k] for x in rows[m])
    out = {"tol": wl.pcg_tol, "steps": steps,
           "plain": {"ms": med(0, 3), "iters": med(0, 1)},
           "mixed": {"ms": med(1, 3), "inner_iters": med(1, 1)},
           "mg": {"ms": med(3, 3), "inner_iters": med(3, 1)},
           "training": info}
    for key in ("learned_mixed", "learned_mg", "learned_mg_guess"):
        out[key] = {"ms": med(key, 3), "network_applications": statistics.median(x[4][0] for x in rows[key]),
                    "finisher_inner_iters": med(key, 1), "max_rel_residual": max(x[2] for x in rows[key])}
    out["learned_vs_plain"] = out["plain"]["ms"] / out["learned_mixed"]["ms"]
    out["learned_vs_mixed"] = out["mixed"]["ms"] / out["learned_mixed"]["ms"]
    out["mg_vs_plain"] = out["plain"]["ms"] / out["mg"]["ms"]
    out["learned_mg_vs_mg"] = out["mg"]["ms"] / out["learned_mg"]["ms"]
    out["learned_guess_vs_mg"] = out["mg"]["ms"] / out["learned_mg_guess"]["ms"]
    d.close()
    net.close()
    return out


def run_sweep(args):
    """64 discharges of the seeded Latin-hypercube sweep (uneven grids and
    particle counts): autotuned particle tiles, then each discharge stepped alone
    (the sum of their times) against all of them stepped by one batch graph per
    step.  Host-timed with the device synchronised on both sides.  Under
    torchrun the discharges are dealt to the ranks (balanced by particle count);
    each rank batches its share; value = all ranks' particle-steps over the
    slowest rank's time (no data-path collective)."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2310_04957_gb300 import build

    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    from paper_2310_04957_gb300 import pic, sweep

    t_setup = time.perf_counter()
    pts_all = sweep.design(64, seed=4)
    mine = sweep.shard([p["n_per_species"] for p in pts_all], rank, world)
    pts = [pts_all[k] for k in mine]
    wls = [sweep.workloads([pts_all[k]], seed_base=100 + k)[0] for k in mine]
    choice, timings = sweep.autotune_tiles(wls)
    # solved alone, each discharge uses the fastest single-discharge solver (multigrid)
    ds = [pic.Discharge(wl, solver=pic.PIC_SOLVER_MG, tile=choice[sweep.tile_class(wl)]) for wl in wls]
    for d in ds:
        d.start()
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    K, Wm = args.steps, args.warmup
    seq_s, ps = 0.0, 0.0
    flagged = []  # (phase, discharge, status bits) of every discharge that reported a failure
    for i, d in enumerate(ds):
        d.step(Wm)
        torch.cuda.synchronize()
        n = d.count(0) + d.count(1)
        t0 = time.perf_counter()
        d.step(K)
        torch.cuda.synchronize()
        seq_s += time.perf_counter() - t0
        ps += n * K
        f = d.status()
        if f:
            flagged.append(("alone", mine[i], f))
    b = pic.Batch(ds)
    b.step(Wm)
    b.sync()
    n = sum(d.count(0) + d.count(1) for d in ds)
    if dist is not None:
        dist.barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        b.step(K)
        b.sync()
        t_b = time.perf_counter() - t0
    flags = 0
    for i, d in enumerate(ds):
        f = d.status()
        if f:
            flagged.append(("batch", mine[i], f))
    for _, _, f in flagged:
        flags |= f
    t_b, n_all = across_ranks(t_b, float(n), dist)
    seq_s, ps = across_ranks(seq_s, ps, dist)
    value = n_all * K / t_b
    if rank != 0:
        dist.barrier()
        dist.destroy_process_group()
        return 0
    n = int(n_all)
    line = {"metric": "aggregate particle-steps/s, 64-discharge batch vs sequential", "value": value,
            "unit": "particle-steps/s", "n_gpus": world, "steps": K, "warmup": Wm, "ms_per_step": 1e3 * t_b / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sweep-64-gec-lhs", "discharges": len(pts_all), "particles": int(n),
                       "grids": sorted({f"{w.nr}x{w.nz}" for w in wls}), "solver": "multigrid-preconditioned mixed CG, one thread-block cluster per discharge",
                       "parallelism": f"discharges dealt to {world} ranks" if world > 1 else "single",
                       "l2": "inputs larger than L2"},
            "sequential": {"value": ps / seq_s, "ms_per_step": 1e3 * seq_s / K,
                           "solver": "multigrid-preconditioned mixed, one discharge at a time"},
            "speedup_vs_sequential": (n * K / t_b) / (ps / seq_s),
            "autotuned_tiles": {f"{c[0]}x{c[1]}": list(t) for c, t in choice.items()},
            "autotune_ms": {f"{c[0]}x{c[1]}": {f"{k[0]}x{k[1]}": round(v, 4) for k, v in tv.items()}
                            for c, tv in timings.items()},
            "setup_s": t_setup, "status_flags": flags, "flagged": flagged, "clocks": clk.summary(),
            "gpu_launches": None, "e2e": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_selfbias(args):
    """Circuit I (Eq. 9) self-bias study, the analogue of Sec. 3's Fig. 2 on synthetic
    cross sections: the GEC-like cell at 128x64 and 100 mTorr, 200 k + 200 k particles,
    the source coupled through R_b = 0.5 ohm, L_b = 0.01 uH and the 5 nF blocking capacitor;
    for each source amplitude the discharge runs `--periods` RF periods and the last window's
    mean electrode potential (the DC self-bias) and mean electron density are reported."""
    import dataclasses

    import torch

    from paper_2310_04957_gb300 import build

    build.build()
    from paper_2310_04957_gb300 import pic
    from paper_2310_04957_gb300 import workloads as W

    rows, t_all = [], 0.0
    for V in (50.0, 100.0, 150.0, 200.0, 250.0, 300.0):
        wl = W.gec_case(128, 64, 100.0, V, n_per_species=200_000, seed_index=31)
        # ionization grows the population over the run: room for 3x the initial count
        wl = dataclasses.replace(wl, circuit=W.CIRCUIT_RLC, circ=(0.5, 0.01e-6, 5e-9, 0, 0, 0, 0, 0),
                                 capacity=(600_000, 600_000))
        d = pic.Discharge(wl, solver=pic.PIC_SOLVER_MG)
        d.start()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d.step(args.periods * wl.steps_per_rf)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        t_all += t
        c = d.circuit_diag()
        ne = d.field("ne_avg")
        rows.append({"V": V, "self_bias_V": c["u_dc"], "u1_amplitude_V": abs(c["u1"]),
                     "ne_mean_m3": float(ne[ne > 0].mean()), "electrons": d.count(0), "seconds": t,
                     "status": d.status()})
        d.close()
    steps = args.periods * 200 * len(rows)
    line = {"metric": "DC self-bias vs source amplitude, circuit I", "value": rows[-1]["self_bias_V"], "unit": "V",
            "n_gpus": 1, "steps": steps, "warmup": 0, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "gec-128x64-100mT-circuitI", "periods": args.periods, "rows": rows},
            "ms_per_step": 1e3 * t_all / steps}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c4":
        return run_sweep(args)
    if args.workload == "selfbias":
        return run_selfbias(args)
    rank, world, local = dist_env()
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2310_04957_gb300 import build

    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    from paper_2310_04957_gb300 import pic
    from paper_2310_04957_gb300 import workloads as W

    prec = pic.PIC_FP32 if args.precision == "fp32" else pic.PIC_FP64
    solver = {"plain": pic.PIC_SOLVER_PLAIN, "mixed": pic.PIC_SOLVER_MIXED, "mg": pic.PIC_SOLVER_MG}[args.solver]
    wl = make_workload(args.workload, rank)
    # particle tile: the library's autotuner times the particle phase of this
    # workload with each candidate tile (untimed, before the warm-up)
    tune_ms = None
    if args.tile == "auto":
        from paper_2310_04957_gb300 import sweep

        choice, timings = sweep.autotune_tiles([wl], candidates=((2, 2), (4, 2), (4, 4), (8, 4)), precision=prec)
        tile = choice[sweep.tile_class(wl)]
        tune_ms = {"%dx%d" % t: round(v, 4) for t, v in timings[sweep.tile_class(wl)].items()}
    else:
        tile = tuple(int(x) for x in args.tile.split("x"))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d = pic.Discharge(wl, precision=prec, solver=solver, stream=stream.cuda_stream, tile=tile)
        d.start()
        d.step(args.warmup)
        torch.cuda.synchronize()
        n0 = d.count(0) + d.count(1)
        d.enable_timing(True)

        def barrier():
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()

        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        with ClockSampler(local) as clk:
            e0.record(stream)
            d.step(args.steps)
            e1.record(stream)
            barrier()
        ms_total = e0.elapsed_time(e1)
        phases = d.step_timing()  # layout, particles, circuit, assembly, solve, efield, diag (ms, summed)
        d.enable_timing(False)
        n1 = d.count(0) + d.count(1)
        flags = d.status()
    n_avg = 0.5 * (n0 + n1)
    particle_steps = n_avg * args.steps
    # slowest rank's time; all ranks' work
    t_max, tot_ps = across_ranks(ms_total, particle_steps, dist)
    value = tot_ps / (t_max * 1e-3)
    k_ms = phases[1] / args.steps
    bpp = BYTES_PER_PARTICLE_STEP[args.precision]
    achieved = bpp * n_avg / (k_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = kernel_traffic()
    windows = (args.warmup + args.steps) // wl.steps_per_rf - args.warmup // wl.steps_per_rf

    # end to end through the public API with host buffers, over the configuration's
    # whole run: upload the initial state from host arrays, then every step pic_step
    # and a device->host read of the step's scalars
    e2e = None
    if not args.no_e2e:
        n_run = RUN_STEPS.get(args.workload, args.steps)
        # the inputs, the initial particle state, in page-locked host memory (prepared
        # before the timed region, as a caller's data would be)
        import dataclasses

        def pinned(a, dtype):
            buf = torch.empty(a.shape, dtype=dtype, pin_memory=True).numpy()
            buf[...] = a
            return buf

        wl_host = dataclasses.replace(wl, particles=tuple(
            W.Particles(*(pinned(getattr(P, k), torch.float64) for k in ("r", "z", "vr", "vt", "vz", "ar", "at", "az")),
                        pinned(P.id.view(np.int64), torch.int64).view(np.uint64),
                        None if P.w is None else pinned(P.w, torch.float64))
            for P in wl.particles))
        with torch.cuda.stream(stream):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # every step's scalars are read into page-locked host memory without
            # waiting, so the host keeps enqueuing steps ahead of the device
            log = torch.empty((n_run, pic.NSCALARS), dtype=torch.float64, pin_memory=True).numpy()
            d2 = pic.Discharge(wl_host, precision=prec, solver=solver, stream=stream.cuda_stream, tile=tile)
            d2.start()
            c0 = d2.count(0) + d2.count(1)
            step0 = d2.scalars()["step"]
            t1 = time.perf_counter()
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            for k in range(n_run):
                d2.step(1)
                d2.scalars_async(log[k])
            eb.record(stream)
            t2 = time.perf_counter()
            d2.sync()
            c1 = d2.count(0) + d2.count(1)
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            t_e2e = t3 - t0
            # each read landed, in order: the logged step counters run step0 + 1 ... step0 + n_run
            reads_ok = bool(np.array_equal(log[:, 0], step0 + 1 + np.arange(n_run)))
            sc = dict(zip(pic.SCALARS, log[-1].tolist()))
            ps = 0.5 * (c0 + c1) * n_run
            h2d = sum(getattr(P, k).nbytes for P in wl.particles for k in ("r", "z", "vr", "vt", "vz", "ar", "at", "az", "id"))
            e2e = {"value": ps / t_e2e, "unit": "particle-steps/s", "steps": n_run, "seconds": t_e2e,
                   "h2d_bytes_per_step": int(h2d / n_run + 4), "d2h_bytes_per_step": 8 * pic.NSCALARS,
                   "reads_verified": reads_ok,
                   "split_s": {"setup": round(t1 - t0, 4), "enqueue": round(t2 - t1, 4), "drain": round(t3 - t2, 4)},
                   "device_ms_per_step": ea.elapsed_time(eb) / n_run,
                   "includes": "pic_init + pic_set_particles from page-locked host FP64 arrays + pic_start, then for each "
                               "of the configuration's %d steps pic_step(1) and pic_diag_async(scalars) into "
                               "page-locked host memory, one pic_sync at the end" % n_run}
            d2.close()
    learned_cmp = None
    if rank == 0 and not args.no_learned and args.workload in ("c2", "c3"):
        learned_cmp = field_solve_comparison(wl)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args.workload)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": wl.name, "grid": [wl.nr, wl.nz], "particles": int(n_avg),
                       "precision": args.precision, "solver": args.solver,
                       "tile": list(tile), "tile_autotune_ms": tune_ms,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (particle store %.0f MB per buffer)" % (n_avg * bpp / 2 / 1e6)},
            "roofline": {"bound": "hbm", "kernel": "k_particles", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic["bytes"] / traffic["particles"] * n_avg if traffic else None,
                         "bytes_per_particle_step": bpp,
                         "stored_bytes_per_particle_step": STORED_BYTES_PER_PARTICLE_STEP[args.precision]},
            "phases_ms": {"layout": phases[0] / args.steps, "particles": k_ms, "circuit": phases[2] / args.steps,
                          "assembly": phases[3] / args.steps, "field_solve": phases[4] / args.steps,
                          "efield": phases[5] / args.steps, "diag": phases[6] / args.steps},
            "particle_phase": {"value": n_avg / ((phases[0] + phases[1]) / args.steps * 1e-3),
                               "unit": "particle-steps/s"},
            "field_solve": {"ms": phases[4] / args.steps, "solver": args.solver, "iters": sc["pcg_iters"] if e2e else None,
                            "tol": wl.pcg_tol, "comparison": learned_cmp},
            "gpu_launches": 1 + KERNELS_PER_STEP * args.steps + KERNELS_PER_WINDOW * windows,
            "status_flags": flags,
            "clocks": clk.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
