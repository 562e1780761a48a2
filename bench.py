"""Benchmark of the radiation step on B300.

Workload (one bench "step" = one rt_step time step = predictor + corrector
stage over the whole grid): the flat 3D periodic opacity/coupling box,
128^3 cells x 162 directions (n = 4), lognormal density, T ~ U[0.5, 2],
alpha^a = 1e-2 rho T^-3.5, alpha^s = 0.4 rho; intensities stored in FP32 with
the per-cell coupling (Newton solve, energy ledger) in FP64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--precision fp32|fp64|bf16] [--n-cells 128]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload.  With N > 1 (under
torchrun) every rank runs an independent replica of the workload (the step
does not exchange data across GPUs in this build), so the job value is the sum
over ranks with the time of the slowest rank.
"""
import argparse
import hashlib
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

METRIC = "cell-angle updates/s per rt_step, % of HBM roofline, at stated error vs FP64 oracle"
UNIT = "cell-angle updates/s"
STORAGE_BYTES = {"fp64": 8, "fp32": 4, "bf16": 2}
# per-cell fluid traffic of one full step: read rho, u_g, u^mu, kappa, alpha_s, eta
# (72 B) and write u_g and G (40 B), for each of the two stages
FLUID_BYTES_PER_CELL_STEP = 224.0

# DRAM traffic of one stage-kernel launch from an ncu capture (bytes per
# cell-angle), valid only for the stage-kernel source it was measured on.
# DRAM bytes (read + write) per cell-angle per stage launch, averaged over the
# two launches of a step, from an ncu capture of a 64^3 box (kerr3d: 64^3 cells
# of the torus recipe); traffic scales with the cells (each cell is read once
# per source array and written once; the Kerr-Schild tables are per (r, theta)
# point and are mostly served from L1/L2)
NCU_TRAFFIC = {("9b4acff03f82", "fp32", "flat3d"): 9.92,
               ("9b4acff03f82", "fp32", "kerr3d"): 18.58}   # {(sha1 of the stage sources, precision, workload): B}
STAGE_SOURCES = ("stage_common.cuh", "stage.cu", "stage_flat.cu")


def stage_source_hash():
    h = hashlib.sha1()
    for name in STAGE_SOURCES:
        with open(os.path.join(ROOT, "paper_2508_15532_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.rows, self.proc, self.idx = [], None, gpu_index
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")] + [time.perf_counter()])

    def wait_first(self, timeout=5.0):
        """Block until the first sample has arrived (nvidia-smi takes a while
        to start), so that the timed region that follows is sampled."""
        end = time.perf_counter() + timeout
        while self.proc and not self.rows and time.perf_counter() < end:
            time.sleep(0.01)

    def region(self, t0, t1):
        self.t0, self.t1 = t0, t1

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = self.rows
        if self.t0 is not None:     # the samples taken while the timed region ran
            inside = [r for r in rows if self.t0 <= r[-1] <= self.t1 + 0.025]
            rows = inside or rows
        sm = [float(r[1]) for r in rows if len(r) >= 10 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 10 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) >= 10:
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "interval_ms": 20}


def cpu_oracle_rate(n_cells, n_geo, steps):
    """The FP64 oracle on a bounded periodic sample of the workload recipe."""
    import oracle
    from paper_2508_15532_b300 import workloads as W
    cfg, f = W.flat3d(N=n_cells, n_geo=n_geo)
    o = oracle.Oracle(cfg)
    o.set_fluid(f["rho"], f["ug"], f["ucon"], f["kappa"], f["alpha_s"], f["eta"])
    o.set_intensity(f["I"])
    dt = o.cfl_dt(0.4)
    t0 = time.perf_counter()
    o.step(dt, steps)
    el = time.perf_counter() - t0
    nd = 10 * n_geo * n_geo + 2
    return n_cells ** 3 * nd * steps / el, el


def oracle_windows(f, N, dt, nsteps, I_gpu, ug_gpu, win=24, core=8, nwin=2, seed=11):
    """The CPU baseline and the stated error in one leg: the FP64 oracle (warmed
    on a small box first) steps windows of the full box (outflow edges; a cell
    after nsteps depends only on cells 2 nsteps per stage away, so a window's
    central part is exact), timed, and the GPU state of the same steps is
    compared with it there.  Returns (oracle cell-angle updates/s, sample
    text, errors)."""
    import oracle
    from paper_2508_15532_b300 import workloads as W
    nd = I_gpu.shape[1]
    cw = W.base_config(4, (8, 8, 8), (0, 0, 0), (1.0 / N,) * 3, (("outflow", "outflow"),) * 3)
    ow = oracle.Oracle(cw)                       # warm-up: library load, page faults, OpenMP pool
    sub8 = {k: np.asarray(f[k])[: 8 ** 3] for k in ("rho", "ug", "ucon", "kappa", "alpha_s", "eta")}
    ow.set_fluid(sub8["rho"], sub8["ug"], sub8["ucon"], sub8["kappa"], sub8["alpha_s"], sub8["eta"])
    ow.set_intensity(np.asarray(f["I"][: 8 ** 3], dtype=np.float64))
    ow.step(dt, 1)
    rng = np.random.default_rng(seed)
    starts = [(N - win // 2,) * 3] + [tuple(int(x) for x in rng.integers(0, N, 3)) for _ in range(nwin - 1)]
    I3, u3 = I_gpu.reshape(N, N, N, nd), ug_gpu.reshape(N, N, N)
    w = None
    eI = eE = eU = 0.0
    el = 0.0
    c = slice(core, win - core)
    for st in starts:
        ii = [(st[a] + np.arange(win)) % N for a in range(3)]
        sel = np.ix_(ii[2], ii[1], ii[0])
        sub = lambda a: np.ascontiguousarray(np.asarray(a).reshape(N, N, N, *np.asarray(a).shape[1:])[sel]
                                             .reshape(win ** 3, *np.asarray(a).shape[1:]))
        cs = W.base_config(4, (win, win, win), (0, 0, 0), (1.0 / N,) * 3, (("outflow", "outflow"),) * 3)
        o = oracle.Oracle(cs)
        o.set_fluid(sub(f["rho"]), sub(f["ug"]), sub(f["ucon"]), sub(f["kappa"]), sub(f["alpha_s"]), sub(f["eta"]))
        o.set_intensity(sub(np.asarray(f["I"], dtype=np.float64)))
        t0 = time.perf_counter()
        o.step(dt, nsteps)
        el += time.perf_counter() - t0
        if w is None:
            w = o.grid()["w"]
        Ir = o.intensity().reshape(win, win, win, nd)[c, c, c]
        Ig = I3[sel][c, c, c].astype(np.float64)
        fl = 1e-3 * np.abs(Ir).max()
        eI = max(eI, float((np.abs(Ig - Ir) / np.maximum(np.abs(Ir), fl)).max()))
        Er, Eg = Ir @ w, Ig @ w
        eE = max(eE, float((np.abs(Eg - Er) / np.abs(Er)).max()))
        ur = o.ug().reshape(win, win, win)[c, c, c]
        eU = max(eU, float((np.abs(u3[sel][c, c, c] - ur) / np.abs(ur)).max()))
    rate = len(starts) * win ** 3 * nd * nsteps / el
    sample = ("%d windows of %d^3 cells (one across the periodic boundary) of the %d^3 box, 162 directions, "
              "%d steps each (%.1f s), after a warm-up step on 8^3" % (len(starts), win, N, nsteps, el))
    errs = {"intensity_max_rel": eI, "intensity_floor": "1e-3 of the window's largest", "Ebar_max_rel": eE,
            "ugas_max_rel": eU, "steps": nsteps,
            "cells_compared": "%d windows x %d^3 central cells x %d directions" % (len(starts), win - 2 * core, nd),
            "bars": {"intensity": 1e-4, "Ebar": 2e-5}}
    return rate, sample, errs


def step_leg(dev, grid, cfg, f, prec, warm=1, steps=3):
    """ms per rt_step and the stage kernel's mean launch time for one more
    workload or precision (CUDA events on the library stream)."""
    import torch
    import paper_2508_15532_b300 as rt
    stream = torch.cuda.Stream(device=dev)
    tdt = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}[prec]
    with torch.cuda.stream(stream):
        st = rt.RadiationStep(grid, cfg, precision=prec, stream=stream.cuda_stream)
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
        st.set_fluid(*[T(f[k]) for k in ("rho", "ug", "ucon", "kappa", "alpha_s", "eta")])
        st.set_intensity(torch.as_tensor(np.asarray(f["I"])).to(dev).to(tdt))
        dt = st.cfl_dt(0.4)
        for _ in range(warm):
            st.step(dt, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        st.set_timing(True)
        e0.record(stream)
        for _ in range(steps):
            st.step(dt, 1)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / steps
        stage_ms, launches = st.get_timing()
        st.set_timing(False)
    del st
    return ms, stage_ms / max(launches, 1)


def max_over_ranks(x, dist=None):
    """The slowest rank's time (replicas: the job ends when the last rank does)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, world, rank):
    if rank != 0:
        return
    N = args.ref_cells
    for _ in range(args.warmup):
        cpu_oracle_rate(N, 4, 1)
    rate, el = cpu_oracle_rate(N, 4, args.steps)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "flat3d-periodic-opacity-coupling", "cells": [128, 128, 128], "directions": 162,
                   "reference_sample_cells": [N, N, N], "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d^3 periodic box of the same recipe, 162 directions, %d steps per timed step"
                                   % (N, 1)},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def adjoint_leg(dev, stream, grid, prec="fp64", nsteps=64, ckpt=8, N=64):
    """Reverse mode on its workload: 64^3 cells, 162 directions, 64 steps,
    a checkpoint every 8, FP64 (or FP32 storage: the mixed reverse pass).
    Returns the forward time per step (rt_step), the backward time per step
    (recompute + reverse, rt_step_adjoint through the autograd rollout) and
    their ratio, all timed with CUDA events."""
    import torch
    import paper_2508_15532_b300 as rt
    from paper_2508_15532_b300 import workloads as W
    from paper_2508_15532_b300.rollout import rollout
    cfg, f = W.adjoint3d(N=N, n_geo=4)
    with torch.cuda.stream(stream):
        st = rt.RadiationStep(grid, cfg, precision=prec, stream=stream.cuda_stream)
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
        fluid = dict(rho=T(f["rho"]), ucon=T(f["ucon"]), alpha_s=T(f["alpha_s"]))
        I0, ug0 = T(f["I"]), T(f["ug"])
        if prec == "fp32":
            I0 = I0.float()
        kappa = T(f["kappa"]).requires_grad_()
        eta = T(f["eta"]).requires_grad_()
        w = T(grid.query()[1])
        st.set_fluid(fluid["rho"], ug0, fluid["ucon"], kappa.detach(), fluid["alpha_s"], eta.detach())
        st.set_intensity(I0)
        dt = st.cfl_dt(0.4)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        st.step(dt, 3)
        e0.record(stream)
        st.step(dt, nsteps)
        e1.record(stream)
        stream.synchronize()
        fwd_ms = e0.elapsed_time(e1) / nsteps
        # untimed warm-up segment: the first backward allocates the library's
        # adjoint arena and loads the reverse kernels
        IW, _ = rollout(st, fluid, I0, ug0, kappa, eta, ckpt, dt=dt, ckpt_every=ckpt)
        ((IW.double() @ w) ** 2).sum().backward()
        kappa.grad = None
        eta.grad = None
        del IW
        IN, _ = rollout(st, fluid, I0, ug0, kappa, eta, nsteps, dt=dt, ckpt_every=ckpt)
        L = ((IN.double() @ w) ** 2).sum()
        stream.synchronize()
        e1.record(stream)
        L.backward()
        e2.record(stream)
        stream.synchronize()
        bwd_ms = e1.elapsed_time(e2) / nsteps
        ok = bool(torch.isfinite(kappa.grad).all() and torch.isfinite(eta.grad).all())
    del st
    return {"workload": "adjoint3d: %d^3 cells x 162 directions, %d steps, checkpoint every %d, %s" % (N, nsteps, ckpt, prec),
            "forward_ms_per_step": fwd_ms, "backward_ms_per_step": bwd_ms, "ratio": bwd_ms / fwd_ms,
            "gradients_finite": ok}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16"])
    ap.add_argument("--n-cells", type=int, default=128)
    ap.add_argument("--workload", default="flat3d", choices=["flat3d", "kerr3d", "kerr2d"])
    ap.add_argument("--kerr-dims", type=int, nargs=3, default=None, metavar=("NR", "NTH", "NPH"),
                    help="Kerr grid other than the workload's (a smaller case for profiling)")
    ap.add_argument("--ref-cells", type=int, default=32)
    ap.add_argument("--e2e-steps", type=int, default=9)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-extra-legs", action="store_true",
                    help="skip the FP64-step and kerr3d legs (profiling runs)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the reverse mode (FP64 and mixed) and print its JSON line")
    ap.add_argument("--adjoint-cells", type=int, default=64)
    ap.add_argument("--adjoint-precision", default="both", choices=["both", "fp64", "fp32"],
                    help="with --adjoint-only: which reverse pass to time")
    ap.add_argument("--adjoint-steps", type=int, default=64)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("gloo")

    if args.impl == "reference":
        run_reference(args, world, rank)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch
    import paper_2508_15532_b300 as rt
    from paper_2508_15532_b300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    if args.adjoint_only:
        g4 = rt.Grid(4)
        ck = min(8, args.adjoint_steps)
        precs = ("fp64", "fp32") if args.adjoint_precision == "both" else (args.adjoint_precision,)
        legs = {p: adjoint_leg(dev, stream, g4, p, nsteps=args.adjoint_steps, ckpt=ck, N=args.adjoint_cells)
                for p in precs}
        if rank == 0:
            first = legs[precs[0]]
            print(json.dumps({"metric": "reverse-mode time per step / forward time per step", "unit": "ratio",
                              "value": first["ratio"], "higher_is_better": False, "adjoint": legs.get("fp64"),
                              "adjoint_mixed": legs.get("fp32")}), flush=True)
        return
    N = args.n_cells
    prec = args.precision
    tdt = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}[prec]
    np_dt = np.float32 if prec != "fp64" else np.float64
    if args.workload == "flat3d":
        cfg, f = W.flat3d(N=N, n_geo=4, intensity_dtype=np_dt)
        wname = "flat3d-periodic-opacity-coupling"
    else:
        if args.kerr_dims:
            nr, nth, nph = args.kerr_dims
            cfg, f = W.kerr(nr=nr, nth=nth, nph=nph, n_geo=4, index=3 if nph > 1 else 2)
        else:
            cfg, f = (W.kerr3d if args.workload == "kerr3d" else W.kerr2d)(n_geo=4)
        f["I"] = f["I"].astype(np_dt)
        wname = args.workload + "-kerr-schild-a0.9-torus"
    nd = f["I"].shape[1]
    ncell = int(np.prod(cfg["nx"]))
    grid = rt.Grid(4)
    with torch.cuda.stream(stream):
        st = rt.RadiationStep(grid, cfg, precision=prec, stream=stream.cuda_stream)
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
        fluid_dev = [T(f[k]) for k in ("rho", "ug", "ucon", "kappa", "alpha_s", "eta")]
        st.set_fluid(*fluid_dev)
        I_host = torch.from_numpy(f["I"]).to(tdt).pin_memory()
        ug_host = torch.from_numpy(np.ascontiguousarray(f["ug"])).pin_memory()
        st.set_intensity(I_host)
        dt = st.cfl_dt(0.4)
    stream.synchronize()

    def barrier():
        if dist:
            dist.barrier()

    # ---- device-resident timing (inputs already in HBM; larger than L2)
    for _ in range(args.warmup):
        st.step(dt, 1)
    stream.synchronize()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st.set_timing(True)
    with ClockSampler(local) as clk:
        clk.wait_first()
        torch.cuda.synchronize(dev)
        t_start = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            st.step(dt, 1)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        clk.region(t_start, time.perf_counter())
    ms = ev0.elapsed_time(ev1)
    stage_ms, launches = st.get_timing()
    st.set_timing(False)
    barrier()
    ms = max_over_ranks(ms, dist)
    ms_per_step = ms / args.steps
    cell_angles = ncell * nd
    value = world * cell_angles * args.steps / (ms * 1e-3)

    # roofline of the stage kernel: algorithmic bytes per launch (two stage
    # launches per step: 2 + 3 intensity passes plus the per-cell fluid I/O)
    S = STORAGE_BYTES[prec]
    alg_step = cell_angles * 5 * S + ncell * FLUID_BYTES_PER_CELL_STEP
    alg_per_launch = alg_step / 2.0
    avg_launch_s = stage_ms * 1e-3 / max(launches, 1)
    peak, peak_kind = measured_peaks()
    achieved = alg_per_launch / avg_launch_s / 1e9
    traffic = NCU_TRAFFIC.get((stage_source_hash(), prec, args.workload))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (traffic * cell_angles if traffic else None),
                "peak_source": peak_kind, "algorithmic_bytes_per_launch": alg_per_launch,
                "avg_launch_ms": avg_launch_s * 1e3,
                "kernel": ({"fp32": "k_stage_fp2", "bf16": "k_stage_fp2", "fp64": "k_stage_fs"}[prec]
                           if args.workload == "flat3d" else "k_stage") + " (transport + interaction, fused)"}

    # ---- end to end through the public API with pinned host buffers: every
    # step uploads its inputs (I, u_g), steps, and reads its results back.
    # NCTX contexts on NCTX streams take steps in turn (a serving loop with
    # NCTX batches in flight): while one context's results come back, the
    # next one's inputs go up and a third one computes, so host->device and
    # device->host copies and the kernels overlap.
    NCTX = 3
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(NCTX - 1)]
    sts = [st]
    for q in range(1, NCTX):
        with torch.cuda.stream(streams[q]):
            sq = rt.RadiationStep(grid, cfg, precision=prec, stream=streams[q].cuda_stream)
            sq.set_fluid(*fluid_dev)
        sts.append(sq)
    outs = [(torch.empty_like(I_host).pin_memory(), torch.empty_like(ug_host).pin_memory()) for _ in range(NCTX)]
    out_I, out_ug = outs[0]
    for q in range(NCTX):
        sts[q].set_intensity(I_host); sts[q].set_ugas(ug_host); sts[q].step(dt, 1)
        sts[q].get_intensity(outs[q][0]); sts[q].get_ugas(outs[q][1])
    torch.cuda.synchronize(dev)
    barrier()
    E = max(NCTX, args.e2e_steps)
    t0 = time.perf_counter()
    for k in range(E + NCTX - 1):
        if k < E:
            q = k % NCTX
            sts[q].set_intensity(I_host)
            sts[q].set_ugas(ug_host)
            sts[q].step(dt, 1)
        kr = k - (NCTX - 1)
        if kr >= 0:
            q = kr % NCTX
            sts[q].get_intensity(outs[q][0])   # host buffer: waits for that context's stream
            sts[q].get_ugas(outs[q][1])
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    del sts[1:]
    e2e_s = max_over_ranks(e2e_s, dist)
    e2e_value = world * cell_angles * E / e2e_s
    h2d = I_host.numel() * I_host.element_size() + ug_host.numel() * 8
    d2h = out_I.numel() * out_I.element_size() + out_ug.numel() * 8

    # ---- stated error against the FP64 oracle and the CPU baseline (one leg):
    # two steps of the bench's workload from its initial state, in the bench's
    # launch configuration, compared on oracle windows that are also timed
    cpu = err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "flat3d":
        NE = 2
        with torch.cuda.stream(stream):
            st.set_intensity(I_host)
            st.set_ugas(ug_host)
            st.step(dt, NE)
            st.get_intensity(out_I)
            st.get_ugas(out_ug)
        stream.synchronize()
        rate, sample, err = oracle_windows(f, N, dt, NE, out_I.float().numpy() if prec == "bf16" else out_I.numpy(),
                                           out_ug.numpy())
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample}
    del f

    # ---- the all-FP64 GPU step and the Kerr-Schild torus (kerr3d) on the same box
    fp64_leg = kerr_leg = None
    if rank == 0 and world == 1 and not args.no_extra_legs and args.workload == "flat3d":
        peak_gbs = measured_peaks()[0]
        cfg64, f64 = W.flat3d(N=N, n_geo=4, intensity_dtype=np.float64)
        ms64, lms64 = step_leg(dev, grid, cfg64, f64, "fp64")
        del f64
        ca = ncell * nd
        alg64 = (ca * 5 * 8 + ncell * FLUID_BYTES_PER_CELL_STEP) / 2.0
        fp64_leg = {"workload": wname + " %d^3, all FP64" % N, "ms_per_step": ms64, "value": ca / (ms64 * 1e-3),
                    "unit": UNIT, "kernel": "k_stage_fs<double> (transport + interaction, fused)",
                    "avg_launch_ms": lms64, "roofline_frac": alg64 / (lms64 * 1e-3) / 1e9 / peak_gbs,
                    "algorithmic_bytes_per_launch": alg64}
        cfgk, fk = W.kerr3d(n_geo=4)
        fk["I"] = fk["I"].astype(np.float32)
        msk, lmsk = step_leg(dev, grid, cfgk, fk, "fp32")
        nck = int(np.prod(cfgk["nx"]))
        del fk
        algk = (nck * nd * 5 * 4 + nck * FLUID_BYTES_PER_CELL_STEP) / 2.0
        kerr_leg = {"workload": "kerr3d-kerr-schild-a0.9-torus %dx%dx%d, FP32 storage" % tuple(cfgk["nx"]),
                    "ms_per_step": msk, "value": nck * nd / (msk * 1e-3), "unit": UNIT,
                    "kernel": "k_stage (general: Kerr-Schild, MAPR angular flux, boosted interaction)",
                    "avg_launch_ms": lmsk, "roofline_frac": algk / (lmsk * 1e-3) / 1e9 / peak_gbs,
                    "algorithmic_bytes_per_launch": algk}

    adj = adj_mixed = None
    if world == 1 and not args.no_adjoint:
        del st
        adj = adjoint_leg(dev, stream, grid, "fp64")
        adj_mixed = adjoint_leg(dev, stream, grid, "fp32")
        st = None


    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32 (f64 coupling)", "fp64": "f64", "bf16": "bf16 storage, f32 math, f64 coupling"}[prec],
            "data": "synthetic",
            "config": {"workload": wname, "cells": [int(x) for x in cfg["nx"]], "directions": nd,
                       "precision": prec, "dt": dt, "parallelism": "replicas" if world > 1 else "single-gpu",
                       "l2": "inputs larger than L2 (%.2f GB per intensity array)" % (cell_angles * S / 1e9)},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "error_vs_oracle": err,
            "fp64_step": fp64_leg,
            "kerr3d": kerr_leg,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "steps": E, "mode": "pinned host buffers; %d contexts on %d streams take steps in turn" % (NCTX, NCTX)},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        if adj:
            line["adjoint"] = adj
            line["adjoint_mixed"] = adj_mixed
        print(json.dumps(line), flush=True)
    if st is not None:
        del st
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
