"""Benchmark of the grand-potential step on GB300.

Workload (default): the 3-D 256^3 directional eutectic -- 3 phases (alpha,
beta, liquid), ternary alloy, four-fold anisotropy 0.02, frozen pulled
temperature gradient, seeded lamellae, no-flux z / periodic x,y, FP32 state
with FP64 diagnostics every 100 steps.  One bench step = one explicit time step
of the whole path (the launch variant the autotuner picks: one fused step
kernel, or the split step's streaming + interface kernels; the diagnostics
kernel every 100th).

Prints ONE JSON line (rank 0).  `value` is whole-job MLUPS (cell updates per
second / 1e6) with the state resident in HBM; `e2e` is the same metric through
the public API with host buffers, host<->device copies inside the timed region;
`roofline` relates the step's algorithmic bytes (read and write every field
once) to the measured HBM peak, with the DRAM traffic and per-kernel shares of
the committed ncu summary for the same sources and launch variant.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIAG_EVERY = 100
E2E_SEGMENT = 100          # time steps per e2e iteration (one output interval)
WORKLOAD = "3-D 256^3 directional eutectic: 3 phases, ternary (2 solutes), aniso 0.02, FP32"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256, help="grid edge (256 = the benchmark workload)")
    ap.add_argument("--pre-steps", type=int, default=1000,
                    help="untimed steps from the seeded state before the warm-up (1000 = the middle of "
                         "the 2000-step workload)")
    ap.add_argument("--no-alu-roof", action="store_true", help="skip the FP32 peak and flop count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched / adjoint lines")
    ap.add_argument("--launch", default=None,
                    help="force a launch variant tx,ty,split,zchunk instead of tuning (e.g. 128,6,1,16)")
    ap.add_argument("--anti-trapping", action="store_true",
                    help="run the workload with the anti-trapping current (for profiling its kernels)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def algorithmic_bytes_per_cell(prob, itemsize):
    # read phi (N) and mu (K-1) once, write them once
    return 2 * itemsize * (prob.n_phases + prob.n_components - 1)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ CPU oracle
def oracle_sample_rate(prob, target_s):
    """Time the FP64 oracle on a block of the same workload; returns (MLUPS, cores, sample)."""
    import oracle
    cores = oracle.num_threads()
    nz_probe = 4
    sub = crop(prob, prob.nx, prob.ny, nz_probe)
    t0 = time.perf_counter()
    oracle.run(sub, sub.phi0, sub.mu0, 1)
    probe = time.perf_counter() - t0
    per_cell = probe / sub.cells
    nz = int(max(1, min(prob.nz, target_s / (per_cell * prob.nx * prob.ny))))
    sub = crop(prob, prob.nx, prob.ny, nz)
    steps = max(1, int(target_s / (per_cell * sub.cells)))
    t0 = time.perf_counter()
    oracle.run(sub, sub.phi0, sub.mu0, steps)
    el = time.perf_counter() - t0
    sample = (f"{steps} FP64 oracle step(s) of the bottom {nz} z-planes ({prob.nx}x{prob.ny}x{nz}"
              f" = {sub.cells} cells, lamellae + interface) from the workload's initial state")
    return sub.cells * steps / el / 1e6, cores, sample, el


def crop(prob, nx, ny, nz):
    return prob.copy(nx=nx, ny=ny, nz=nz, phi0=prob.phi0[:, :nz, :ny, :nx].copy(),
                     mu0=prob.mu0[:, :nz, :ny, :nx].copy())


# ------------------------------------------------------------------- arms
def run_reference(args, rank, world):
    """The FP64 CPU oracle as it stands, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    import workloads
    prob = workloads.eutectic_3d(n=args.n)
    if world > 1:   # the launcher caps every rank at one thread; rank 0 alone computes here
        oracle.set_threads(os.cpu_count() or 1)
    cores = oracle.num_threads()
    # size one bench step so that warmup + steps stay within ~3 minutes
    budget = 150.0 / max(1, args.steps + args.warmup)
    probe = crop(prob, prob.nx, prob.ny, 2)
    t0 = time.perf_counter()
    oracle.run(probe, probe.phi0, probe.mu0, 1)
    per_cell = (time.perf_counter() - t0) / probe.cells
    plane = max(32, int(budget / per_cell) // 20)
    nx = int(min(prob.nx, max(8, int(plane ** 0.5))))
    ny = int(min(prob.ny, max(4, plane // nx)))
    sub = crop(prob, nx, ny, 20)
    for _ in range(args.warmup):
        oracle.run(sub, sub.phi0, sub.mu0, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(sub, sub.phi0, sub.mu0, 1)
    el = time.perf_counter() - t0
    mlups = sub.cells * args.steps / el / 1e6
    sample = (f"each step = 1 FP64 oracle step on a {nx}x{ny}x20 block (bottom planes) of the "
              f"{prob.nx}^3 workload")
    line = {"impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "oracle_block": [nx, ny, 20]},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import workloads
    from paper_2404_01035_gb300 import Simulation

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    prob = workloads.eutectic_3d(n=args.n)
    prob.anti_trapping = int(args.anti_trapping)
    cells = prob.cells
    stream = torch.cuda.Stream(device=dev)
    sim = Simulation(prob, dtype="f32", stream=stream)
    sim.set_fields(prob.phi0, prob.mu0)
    tuned_ms = None
    if args.launch:
        tx, ty, sp, zc = (int(v) for v in args.launch.split(","))
        sim.set_launch(sim.tiles().index((tx, ty, sp)), zc)
    elif not args.no_tune:
        tuned_ms = sim.tune(None, steps_per_trial=25)
        sim.set_fields(prob.phi0, prob.mu0)
    tiles = sim.tiles()
    cur_tile, cur_zchunk = sim.launch()
    tx, ty, split = tiles[cur_tile]
    step_launches = (2 if split else 1) + (2 if args.anti_trapping else 0)   # kernels per time step
    if args.pre_steps > 0:   # a representative state: interfaces developed, not the sharp seed
        sim.step(args.pre_steps)
    sim.set_diag_every(DIAG_EVERY)
    sim.step(args.warmup)
    sim.sync()

    # ---- timed region: K steps, events on the library's stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    chunk_ev = []
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev[0].record(stream)
    done = 0
    launches = 0
    # chunks aligned on the diagnostics interval: events around the pure
    # step-kernel part of each chunk give the step kernel's own duration
    while done < args.steps:
        s0 = sim.time()[0]
        n = min(DIAG_EVERY - s0 % DIAG_EVERY, args.steps - done)
        pure = n - 1 if (s0 + n) % DIAG_EVERY == 0 else n
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(pure)
        b.record(stream)
        chunk_ev.append((a, b, pure))
        if pure < n:
            sim.step(1)
            launches += 2   # diagnostics: partial + final reduction
        launches += n * step_launches
        done += n
    ev[1].record(stream)
    stream.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    el = ev[0].elapsed_time(ev[1]) / 1e3
    kern_ms = sum(a.elapsed_time(b) for a, b, _ in chunk_ev)
    kern_n = sum(p for _, _, p in chunk_ev)
    sim.sync()
    if world > 1:
        t = torch.tensor([el], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    value = world * cells * args.steps / el / 1e6

    # ---- roofline of the step (all of its kernels)
    peaks, src = measured_peaks()
    bpc = algorithmic_bytes_per_cell(prob, 4)
    per_step_s = kern_ms / max(1, kern_n) / 1e3
    achieved = bpc * cells / per_step_s / 1e9
    launch = {"tx": tx, "ty": ty, "split": split, "zchunk": cur_zchunk}
    prof = committed_profile(launch, args.n) if not args.anti_trapping else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"],
            "traffic": prof["dram_bytes_per_step"] if prof else None,
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)",
            "scope": "one time step: " + ("k_gp_stream + k_gp_iface" if split else "k_gp_step")
                     + (" + k_at_list + k_at_work" if args.anti_trapping else ""),
            "bytes_per_cell": bpc, "step_ms": per_step_s * 1e3,
            "kernel_shares": prof["kernel_shares"] if prof else None}

    if not args.no_alu_roof:
        phi_h, mu_h = sim.get_fields()
        roof["alu"] = alu_roof(prob, phi_h, mu_h, sim.time()[1], per_step_s, bpc * cells / (peaks["hbm_gbs"] * 1e9),
                               stream)
        del phi_h, mu_h

    # ---- e2e through the public API with host (pinned) buffers, continuing
    # from the evolved state of the timed run
    e2e = None
    if not args.no_e2e:
        hphi = torch.empty((prob.n_phases,) + sim.shape, dtype=torch.float32, pin_memory=True)
        hmu = torch.empty((prob.n_components - 1,) + sim.shape, dtype=torch.float32, pin_memory=True)
        sim.get_fields_into(hphi, hmu, on_device=False)
        sim.set_diag_every(0)
        iters = 3
        for it in range(iters + 1):
            if it == 1:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            sim.set_fields_from(hphi, hmu, on_device=False)
            sim.step(E2E_SEGMENT)
            sim.get_fields_into(hphi, hmu, on_device=False)   # synchronises
        e2e_el = time.perf_counter() - t0
        e2e_v = world * cells * E2E_SEGMENT * iters / e2e_el / 1e6
        nbytes = hphi.numel() * 4 + hmu.numel() * 4
        e2e = {"value": e2e_v, "unit": "MLUPS", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps_per_e2e_iteration": E2E_SEGMENT,
               "note": "one e2e iteration = H2D of the full state from pinned memory, "
                       f"{E2E_SEGMENT} steps, D2H of the full state"}
    launch_info = {"tiles_compiled": tiles, "launch": launch}
    sim.close()

    extra = {}
    if not args.no_extras:
        extra["batched"] = bench_batched(stream)
        extra["adjoint"] = bench_adjoint(stream)
        extra["multigrain"] = bench_multigrain(stream)
        extra["frame_noise"] = bench_frame_noise(stream)
        extra["anti_trapping"] = bench_anti_trapping(stream)
        extra["grain_growth"] = bench_grain_growth(stream)
        extra["sparse_grain_growth"] = bench_sparse_grain_growth(stream)
        extra["elasticity"] = bench_elasticity(stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, sample, secs = oracle_sample_rate(prob, target_s=15.0)
        cpu = {"value": rate, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": sample, "seconds": secs}
    if rank == 0:
        line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "cells_per_gpu": cells, "grid": [args.n] * 3,
                           "phases": prob.n_phases, "components": prob.n_components,
                           "diag_every": DIAG_EVERY,
                           "state": f"evolved {args.pre_steps} steps from the seeded initial state before "
                                    f"the {args.warmup} warm-up steps",
                           "l2": "inputs larger than L2 (state 671 MB per buffer)",
                           "tuned_ms_per_step": tuned_ms, **launch_info},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches, **extra}
        print(json.dumps(line), flush=True)


def pure_stencil_mask(phi, bc):
    """Cells whose 19-point stencil (the 3x3x3 block without its corners,
    after the boundary mapping) is one pure phase: phi_l = 1 on all of it."""
    N = phi.shape[0]
    out = np.zeros(phi.shape[1:], dtype=bool)
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if abs(dz) + abs(dy) + abs(dx) < 3]

    def shifted(a, dz, dy, dx):
        for axis, d, b in ((0, dz, bc[2]), (1, dy, bc[1]), (2, dx, bc[0])):
            if d == 0:
                continue
            if b == 3:
                a = np.roll(a, -d, axis=axis)
            else:   # no-flux: the ghost is the adjacent interior cell
                idx = np.clip(np.arange(a.shape[axis]) + d, 0, a.shape[axis] - 1)
                a = np.take(a, idx, axis=axis)
        return a

    for l in range(N):
        one = phi[l] == 1.0
        acc = one.copy()
        for o in offs:
            if o != (0, 0, 0):
                acc &= shifted(one, *o)
        out |= acc
    return out


def alu_roof(prob, phi, mu, t, step_s, hbm_s, stream, samples=256, seed=20240401):
    """FP32 roof of one step: the measured FMA peak of the device and the
    step's algorithmic flops.  A cell whose 19-point stencil is one pure phase
    keeps phi exactly and its mu update reduces to the constant-coefficient
    Laplacian update (NM (2 dim + 2 + 2 NM) flops, counted by hand); every
    other cell costs the full update, counted by the oracle's op-counting
    scalar on a window around each of `samples` random such cells (mean)."""
    import oracle
    from paper_2404_01035_gb300.simulation import peak_fp32

    def _axis_index(c, n, bc, r):   # window indices with the boundary mapping
        idx = np.arange(c - r, c + r + 1)
        return idx % n if bc == 3 else np.clip(idx, 0, n - 1)
    peak_s = peak_fp32(False, stream)
    peak_p = peak_fp32(True, stream)
    phi = np.asarray(phi, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    pure = pure_stencil_mask(phi, prob.bc)
    n_iface = int((~pure).sum())
    n_bulk = int(pure.sum())
    NM, dim = prob.n_components - 1, prob.dim
    f_bulk = NM * (2 * dim + 2 + 2 * NM)
    rng = np.random.default_rng(seed)
    cand = np.argwhere(~pure)
    f_cells = []
    r = 2
    for k in rng.choice(len(cand), size=min(samples, len(cand)), replace=False):
        z, y, x = (int(v) for v in cand[k])
        ix, iy, iz = (_axis_index(x, prob.nx, prob.bc[0], r), _axis_index(y, prob.ny, prob.bc[1], r),
                      _axis_index(z, prob.nz, prob.bc[2], r))
        wp = phi[:, iz][:, :, iy][:, :, :, ix]
        wm = mu[:, iz][:, :, iy][:, :, :, ix]
        w = 2 * r + 1
        wprob = prob.copy(nx=w, ny=w, nz=w, bc=[3, 3, 3], z0=prob.z0 - (z - r) * prob.dx)
        a, b = oracle.count_flops(wprob, wp, wm, t0=t)
        f_cells.append(a[r, r, r] + b[r, r, r])
    f_iface = float(np.mean(f_cells)) if f_cells else 0.0
    flops = n_iface * f_iface + n_bulk * f_bulk
    peak = max(peak_s, peak_p)
    alu_s = flops / (peak * 1e12)
    roof_s = max(alu_s, hbm_s)
    return {"fp32_peak_tflops": peak, "fp32_peak_scalar_tflops": peak_s, "fp32_peak_paired_tflops": peak_p,
            "peak_source": "measured on this device (ms_peak_fp32: FMA chains, 64 warps per SM)",
            "flops_per_step": flops, "flops_per_interface_cell": f_iface, "flops_per_bulk_cell": f_bulk,
            "interface_cells": n_iface, "bulk_cells": n_bulk, "sampled_cells": len(f_cells),
            "alu_ms": alu_s * 1e3, "hbm_ms": hbm_s * 1e3, "roof_ms": roof_s * 1e3,
            "binding": "alu" if alu_s > hbm_s else "hbm", "frac_of_roof": roof_s / step_s,
            "achieved_tflops": flops / step_s / 1e12}


def _events_ms(stream, fn):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b)


def bench_batched(stream):
    """512 independent 2-D dendrites, 500 steps in one persistent launch, against
    the plain single-simulation step on the largest of them (512^2)."""
    import workloads
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300.batch import Batch
    probs = workloads.batched_dendrites_2d()
    b = Batch(probs, stream=stream)
    for i, p in enumerate(probs):
        b.set_fields(i, p.phi0, p.mu0)
    b.step(20)            # warm-up launch (graph capture for n = 20)
    b.sync()
    tuned = b.tune(steps_per_trial=50)   # tile height on the evolved states (restored)
    steps = 500
    b.step(steps)         # capture for n = 500, then time a replay
    b.sync()
    for i, p in enumerate(probs):
        b.set_fields(i, p.phi0, p.mu0)
    ms = _events_ms(stream, lambda: b.step(steps))
    b.sync()
    cells = b.cells
    tile = b.tile_height()
    b.close()
    batched = cells * steps / (ms / 1e3) / 1e6
    # the same 512 simulations stepped one after another through ms_step
    sims = []
    for p in probs:
        sim = Simulation(p, dtype="f32", stream=stream)
        sim.set_fields(p.phi0, p.mu0)
        sims.append(sim)
    for sim in sims:
        sim.step(2)

    def seq():
        for sim in sims:
            sim.step(steps)

    sms = _events_ms(stream, seq)
    for sim in sims:
        sim.close()
    seq_mlups = cells * steps / (sms / 1e3) / 1e6
    # one plain grid with the same number of cells (a 2-D dendrite, the
    # largest simulation's parameters)
    big = max(probs, key=lambda q: q.cells)
    ny = int(round(cells / 7488))
    one = workloads.binary_problem("batched_equiv", 7488, ny=ny, delta=big.delta[0, 1],
                                   Delta=big.meta.get("Delta", 0.2), R=6.0, dt=big.dt)
    sim = Simulation(one, dtype="f32", stream=stream)
    sim.set_fields(one.phi0, one.mu0)
    sim.step(5)
    pms = _events_ms(stream, lambda: sim.step(steps))
    sim.close()
    plain = one.cells * steps / (pms / 1e3) / 1e6
    return {"workload": "512 independent 2-D N=2 K=2 FP32 sims, edges 64..512, 500 steps, one "
                        "graph-captured persistent launch", "cells": int(cells), "tile_height": tile,
            "tuned_ms_per_step": tuned,
            "mlups": batched, "ms_per_step": ms / steps,
            "sequential_mlups": seq_mlups,
            "sequential": "the same 512 simulations, each stepped 500 steps by ms_step, one after another",
            "vs_sequential": batched / seq_mlups,
            "plain_step_mlups": plain,
            "plain_step": f"one {one.nx}x{one.ny} simulation ({one.cells} cells, about the batch's total), "
                          "one launch per step",
            "vs_plain_step": batched / plain,
            "hbm_frac": batched * 1e6 * 24 / (measured_peaks()[0]["hbm_gbs"] * 1e9)}


def bench_multigrain(stream, pre_steps=1000, steps=1000):
    """3-D 512^3 multigrain (8 phases: 7 rotated grains + liquid, binary, FP32,
    periodic): the launch the tuner picks, `steps` steps (the workload's 1000)
    timed after `pre_steps` untimed ones from the seeded state."""
    import workloads
    from paper_2404_01035_gb300 import Simulation
    p = workloads.multigrain_3d()
    sim = Simulation(p, dtype="f32", stream=stream)
    sim.set_fields(p.phi0, p.mu0)
    sim.step(pre_steps)
    sim.tune(None, steps_per_trial=10)   # trials on the evolved state, which is kept
    sim.step(10)
    ms = _events_ms(stream, lambda: sim.step(steps))
    tiles = sim.tiles()
    t, zc = sim.launch()
    phi, _ = sim.get_fields()
    sim.close()
    bulk = float(pure_stencil_mask(phi, p.bc).mean())
    mlups = p.cells * steps / (ms / 1e3) / 1e6
    bpc = algorithmic_bytes_per_cell(p, 4)
    return {"workload": f"3-D 512^3 multigrain: 8 phases (7 rotated grains + liquid), binary, FP32, "
                        f"periodic, {steps} steps timed after {pre_steps} untimed from the seeded state",
            "cells": int(p.cells), "mlups": mlups, "ms_per_step": ms / steps,
            "launch": {"tx": tiles[t][0], "ty": tiles[t][1], "split": tiles[t][2], "zchunk": zc},
            "bytes_per_cell": bpc, "pure_stencil_fraction": bulk,
            "algorithmic_hbm_frac": mlups * 1e6 * bpc / (measured_peaks()[0]["hbm_gbs"] * 1e9),
            "note": "cells whose stencil is one pure phase keep phi and move mu only, so the "
                    "algorithmic fraction (every field read and written once) can exceed 1"}


def bench_frame_noise(stream):
    """The 256^3 eutectic with phi noise on (amplitude 0.01) for 200 steps, and
    the cost of one moving-frame check (ms_front) and one 8-plane shift."""
    import workloads
    from paper_2404_01035_gb300 import Simulation
    p = workloads.eutectic_3d()
    p.noise_amp, p.noise_seed = 0.01, 20240401
    sim = Simulation(p, dtype="f32", stream=stream)
    sim.set_fields(p.phi0, p.mu0)
    sim.tune(None, steps_per_trial=10)
    sim.set_fields(p.phi0, p.mu0)
    sim.step(20)
    steps = 200
    ms = _events_ms(stream, lambda: sim.step(steps))
    stream.synchronize()
    t0 = time.perf_counter()
    front = sim.front()
    front_ms = (time.perf_counter() - t0) * 1e3
    shift_ms = _events_ms(stream, lambda: sim.shift(8, p.mu0[:, -1, 0, 0]))
    sim.close()
    return {"workload": "3-D 256^3 eutectic with phi noise (amplitude 0.01), 200 steps; moving-frame check "
                        "and an 8-plane shift", "mlups": p.cells * steps / (ms / 1e3) / 1e6,
            "ms_per_step": ms / steps, "front_plane": front, "front_ms_host": front_ms,
            "shift_8_planes_ms": shift_ms}


def bench_anti_trapping(stream):
    """The 256^3 eutectic with the anti-trapping current on, 200 steps from the
    seeded state after 20 warm-up steps, against the same run without it (the
    correction kernel's cost is the difference)."""
    import workloads
    from paper_2404_01035_gb300 import Simulation
    out = {"workload": "3-D 256^3 eutectic with the anti-trapping current (obstacle form), 200 steps"}
    steps = 200
    for at in (1, 0):
        p = workloads.eutectic_3d()
        p.anti_trapping = at
        sim = Simulation(p, dtype="f32", stream=stream)
        sim.set_fields(p.phi0, p.mu0)
        sim.tune(None, steps_per_trial=10)
        sim.set_fields(p.phi0, p.mu0)
        sim.step(20)
        ms = _events_ms(stream, lambda: sim.step(steps))
        key = "with" if at else "without"
        out[key] = {"mlups": p.cells * steps / (ms / 1e3) / 1e6, "ms_per_step": ms / steps}
        sim.close()
    out["correction_ms_per_step"] = out["with"]["ms_per_step"] - out["without"]["ms_per_step"]
    return out


def bench_grain_growth(stream):
    """Isotropic grain growth of 8 Voronoi grains in a periodic 256^3 box,
    FP32, 200 steps after 20 warm-up steps, tuned launch."""
    import workloads
    from paper_2404_01035_gb300 import Simulation
    p = workloads.grain_growth(n=256, dim=3, grains=8)
    sim = Simulation(p, dtype="f32", stream=stream)
    sim.set_fields(p.phi0, p.mu0)
    sim.tune(None, steps_per_trial=10)
    sim.set_fields(p.phi0, p.mu0)
    sim.step(20)
    steps = 200
    ms = _events_ms(stream, lambda: sim.step(steps))
    tile, zc = sim.launch()
    tx, ty, split = sim.tiles()[tile]
    sim.close()
    return {"workload": "3-D 256^3 isotropic grain growth, 8 Voronoi grains, periodic, FP32, 200 steps",
            "mlups": p.cells * steps / (ms / 1e3) / 1e6, "ms_per_step": ms / steps,
            "launch": {"tx": tx, "ty": ty, "split": split, "zchunk": zc}}


def bench_sparse_grain_growth(stream):
    """Sparse grain growth (few grains stored per cell, the projection over the
    locally active grains, Gamma_abc = 15 gamma) of 8 and of 32 Voronoi grains
    in a periodic 256^3 box, FP32: 200 steps timed after 100 untimed ones."""
    import workloads
    from paper_2404_01035_gb300.sparse_gg import SparseGrainGrowth
    out = {"workload": "3-D 256^3 isotropic grain growth, Voronoi grains, periodic, FP32, sparse storage "
                       "(at most 8 grains per cell), diffuse Voronoi start, Gamma_abc = 15 gamma, 200 steps after 100"}
    for grains in (8, 32):
        p = workloads.sparse_grain_growth(n=256, dim=3, grains=grains)
        s = SparseGrainGrowth(p, dtype="f32", stream=stream)
        try:
            s.set_fields(p.phi0)
            s.step(100)
            steps = 200
            ms = _events_ms(stream, lambda: s.step(steps))
            s.sync()
            listed, _ = s.stats()
            out[f"grains_{grains}"] = {"mlups": p.cells * steps / (ms / 1e3) / 1e6, "ms_per_step": ms / steps,
                                       "listed_cells_last_step": listed}
        except Exception as e:   # a cell needing more than 8 grains is reported, not hidden
            out[f"grains_{grains}"] = {"error": str(e)}
        s.close()
    return out


def bench_elasticity(stream):
    """The multigrain grid (7 grains + liquid, 8 phases) at 256^3 with a cubic
    stiffness and a dilatational eigenstrain of 1% in every grain: the FFT
    equilibrium before every step, against the same run without it."""
    import numpy as np
    import workloads
    from paper_2404_01035_gb300 import Simulation
    out = {"workload": "3-D 256^3 multigrain (8 phases), FP32, cubic stiffness, 1% dilatational eigenstrain "
                       "in the grains, 100 steps"}
    steps = 100
    for el in (1, 0):
        p = workloads.multigrain_3d(n=256)
        if el:
            C = np.zeros((6, 6))
            C[:3, :3] = 60.0
            np.fill_diagonal(C[:3, :3], 150.0)
            C[3, 3] = C[4, 4] = C[5, 5] = 75.0
            eig = np.zeros((p.n_phases, 3, 3))
            for g in range(p.n_phases - 1):
                eig[g] = np.eye(3) * 0.01
            p.elastic_C, p.eigenstrain = C, eig
        sim = Simulation(p, dtype="f32", stream=stream)
        sim.set_fields(p.phi0, p.mu0)
        sim.tune(None, steps_per_trial=5)
        sim.set_fields(p.phi0, p.mu0)
        sim.step(10)
        ms = _events_ms(stream, lambda: sim.step(steps))
        out["with" if el else "without"] = {"mlups": p.cells * steps / (ms / 1e3) / 1e6, "ms_per_step": ms / steps}
        sim.close()
    out["equilibrium_ms_per_step"] = out["with"]["ms_per_step"] - out["without"]["ms_per_step"]
    return out


def bench_adjoint(stream):
    """2-D 256^2 well-potential adjoint: 2000 steps forward with checkpoints every
    100, then the reverse pass, FP32 and FP64, against the plain forward step."""
    import torch
    import workloads
    from paper_2404_01035_gb300 import Simulation
    out = {"workload": "2-D 256^2, N=2 K=2, well potential, 2000 steps, checkpoint every 100"}
    for dtype in ("f32", "f64"):
        p = workloads.adjoint_well_2d(n=256, steps=2000, delta=0.02, mob=0.8)
        sim = Simulation(p, dtype=dtype, stream=stream)
        sim.set_fields(p.phi0, p.mu0)
        sim.step(50)
        sim.set_fields(p.phi0, p.mu0)
        fwd = _events_ms(stream, lambda: sim.step(2000))
        sim.set_fields(p.phi0, p.mu0)
        sim.enable_checkpoints(100)
        sim.step(2000)
        tdt = torch.float64 if dtype == "f64" else torch.float32
        seed = torch.ones((2, 1, 256, 256), dtype=tdt, device="cuda") * 1e-3
        stream.synchronize()
        t0 = time.perf_counter()
        sim.grad(seed)
        rev = (time.perf_counter() - t0) * 1e3
        sim.close()
        out[dtype] = {"forward_ms_per_step": fwd / 2000, "reverse_ms_per_step": rev / 2000,
                      "reverse_vs_forward": rev / fwd,
                      "forward_mlups": 65536 * 2000 / (fwd / 1e3) / 1e6,
                      "reverse_mlups": 65536 * 2000 / (rev / 1e3) / 1e6}
    return out


def committed_profile(launch, n):
    """The ncu figures committed for this source version, launch variant and grid
    (profiles/traffic_eutectic_3d_step.json), or None."""
    path = os.path.join(ROOT, "profiles", "traffic_eutectic_3d_step.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        entries = json.load(fh)
    digest = kernel_digest()
    for e in entries:
        if e.get("kernel_digest") == digest and e.get("launch") == launch and e.get("grid") == n:
            return e
    return None


def kernel_digest():
    """Digest of the sources of the benchmark's step kernels: the translation
    unit that instantiates the 3-phase, 2-solute kernels and every header it
    includes (recursively).  Ties a committed ncu traffic figure to the
    kernel version it was measured on."""
    import hashlib
    import re
    d = os.path.join(ROOT, "paper_2404_01035_gb300", "csrc")
    seen, todo = [], ["ms_inst_3d_n3.cu"]
    while todo:
        f = todo.pop(0)
        if f in seen or not os.path.exists(os.path.join(d, f)):
            continue
        seen.append(f)
        with open(os.path.join(d, f)) as fh:
            todo += re.findall(r'#include "([A-Za-z0-9_.]+)"', fh.read())
    h = hashlib.sha256()
    for f in sorted(seen):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def main():
    args = parse()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
