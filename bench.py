#!/usr/bin/env python
"""Throughput of the staggered-mesh EB advance (flux + WSRD on four grids).

One step = one forward-Euler pass of the whole path (Eq. basic_fv_srd) over
the same seeded input state:
flux divergence and provisional update on the c, u, v, w grids, then
weighted state redistribution of all five fields.  Workload: the 3D
Gaussian hill, 256 x 256 x 128 cells, synthetic seeded state.  The headline
``value`` is the mixed (FP32 state, FP64 tiny-cell geometry and weights)
path; the FP64 path is reported beside it under ``fp64``.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank advances its own
replica of the workload; value = all ranks' cell-updates / max time.
"""
from __future__ import annotations

import argparse
import contextlib
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EB cell-updates/s (flux+WSRD, 4 grids) mixed vs FP64 path, % of HBM roofline"
UNIT = "cell-updates/s"
FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--terrains", type=int, default=250,
                    help="warmstart: training terrains (8 samples each; 250 gives the 2000 training fields)")
    ap.add_argument("--epochs", type=int, default=12, help="warmstart: training epochs")
    ap.add_argument("--workload", choices=("hill256", "grf512", "ensemble", "anelastic", "warmstart", "slabs",
                                           "network"),
                    default="hill256",
                    help="ensemble: 64 uneven Gaussian-hill instances advanced together (mixed path); "
                         "anelastic: 192x192x96 random terrain, anelastic steps with the projection; "
                         "slabs: the 256x256x128 hill cut into one x-slab per rank (halo exchange each step)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--precision", choices=("both", "mixed", "f64"), default="both",
                    help="arms to run (profiling runs pick one)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--ensemble-schedule", choices=("tuned", "persistent", "branches"), default="tuned",
                    help="ensemble: the autotuner's schedule, or one forced after tuning the slab heights")
    ap.add_argument("--tile-rows", type=int, choices=(16, 14), default=None,
                    help="bulk kernel tile rows (with --slab-levels); default: chosen by the autotuner")
    ap.add_argument("--slab-levels", type=int, default=None,
                    help="bulk kernel slab height (0 = automatic); default: chosen by the autotuner")
    return ap.parse_args()


def workload(name):
    from paper_2604_11959_gb300 import inputs
    return {"hill256": inputs.HILL_256, "grf512": inputs.GRF_512, "anelastic": inputs.GRF_192}.get(name,
                                                                                                 inputs.HILL_256)


def run_warmstart(eb, terrains, epochs):
    """Trains the projection's warm-start network on 96x96x48-cell random
    terrains with the cell size of the 192x192x96 anelastic case, then
    compares cold (zero) and warm (network) starts of the same projection to
    a relative residual of 1e-10 on held-out terrains and on that case."""
    import torch
    from paper_2604_11959_gb300 import inputs, warmstart as ws
    r = ws.Recipe(terrains=terrains, epochs=epochs)
    logs = []
    t0 = time.perf_counter()
    scale = ws.target_scale(r)
    data, cold_train = ws.make_dataset(r, scale)
    t_data = time.perf_counter() - t0
    t1 = time.perf_counter()
    net = ws.train(r, data, log=logs.append)
    t_train = time.perf_counter() - t1
    params = net.get_params()
    # time one training step and count its arithmetic
    x, t, m = data[0]
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(5):
        net.train_step(x, t, m, 1e-12)
    b.record()
    torch.cuda.synchronize()
    ms_step = a.elapsed_time(b) / 5
    net.close()
    vox = r.nx * r.ny * r.nz
    fwd = sum(2 * ci * co * k ** 3 * vox / 8 ** lv for (ci, co, k), lv in
              zip(ws.LAYERS, (0, 0, 1, 1, 2, 2, 1, 1, 0, 0, 0)))
    flop_step = 3 * fwd   # forward, input gradient, weight gradient
    held, loose = [], []
    for q in range(4):
        w = ws.workload(r, 5000 + q)
        g, refs = ws.geometry(w)
        held.append(ws.compare(g, params, w, refs, 77 + q, scale))
        loose.append(ws.compare(g, params, w, refs, 77 + q, scale, rtol=1e-4))
        g.close()
    # the guess's relative error on held-out samples, all modes and smooth modes
    test_data, _ = ws.make_dataset(r, scale, first_terrain=5000, terrains=4)
    net = eb.UNet(r.nx, r.ny, r.nz)
    net.set_params(params)
    delta_all, delta_smooth = ws.guess_error(net, test_data)
    net.close()
    w = inputs.GRF_192
    refs = inputs.cell_reference(w.nz, w.Lz)
    g = eb.Geometry(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, torch.from_numpy(w.heights()).cuda(), precision="mixed",
                    ref_rho=torch.from_numpy(refs[0]).cuda(), ref_rhotheta=torch.from_numpy(refs[1]).cuda())
    big = ws.compare(g, params, w, refs, 1, scale)
    seq_jacobi = ws.sequence(g, params, w, refs, 1, scale)
    eb.set_preconditioner(g, "mg")
    big_mg = ws.compare(g, params, w, refs, 1, scale)
    seq_mg = ws.sequence(g, params, w, refs, 1, scale)
    g.close()
    return {"scale": scale, "samples": len(data), "mean_cold_iters_train": float(np.mean(cold_train)),
            "data_s": t_data, "train_s": t_train, "train_step_ms": ms_step,
            "train_tflops": flop_step / (ms_step * 1e-3) / 1e12, "log": logs,
            "held_out": [{"cold": c, "warm": h, "relres_cold": rc, "relres_warm": rw, "momentum_diff": d}
                         for c, h, rc, rw, d in held],
            "held_out_rtol_1e-4": [{"cold": c, "warm": h} for c, h, _, _, _ in loose],
            "grf192": {"cold": big[0], "warm": big[1], "relres_cold": big[2], "relres_warm": big[3],
                       "momentum_diff": big[4], "ratio": big[0] / max(1, big[1])},
            "grf192_multigrid": {"cold": big_mg[0], "warm": big_mg[1], "relres_cold": big_mg[2],
                                 "relres_warm": big_mg[3], "momentum_diff": big_mg[4],
                                 "ratio": big_mg[0] / max(1, big_mg[1])},
            "guess_relative_error": {"all_modes": delta_all, "smooth_modes_8cubed": delta_smooth,
                                     "samples": len(test_data), "held_out_terrains": 4},
            "consecutive_steps_grf192": {
                "note": "iterations to 1e-10 per projection of consecutive forward-Euler anelastic steps: "
                        "zero start, previous step's solution, network guess",
                "jacobi": [{"zero": a, "previous_step": b, "network": c} for a, b, c in seq_jacobi],
                "multigrid": [{"zero": a, "previous_step": b, "network": c} for a, b, c in seq_mg]}}


def init_ranks(world):
    """One process per GPU under torchrun (RANK, LOCAL_RANK, WORLD_SIZE and
    MASTER_* from the environment): the rank's GPU and a process group, NCCL
    between GPUs and gloo where CUDA is absent (the CPU tests).  None for a
    single process."""
    if world <= 1:
        return None
    import torch
    import torch.distributed as tdist
    if torch.cuda.is_available():
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
    else:
        tdist.init_process_group("gloo")
    return tdist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(value, dist):
    """The largest of the ranks' values: the slowest replica sets the job's
    time.  The value itself for a single process."""
    if dist is None:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_anelastic(eb, steps, warmup, clk=None, dist=None):
    """Anelastic steps (Algorithm 2, two stages, projection to a relative
    residual of 1e-10 from a zero guess, multigrid-preconditioned) on the
    192x192x96 random terrain, mixed path; and one projection timed alone
    with each preconditioner.  Algorithmic traffic per PCG iteration: 136
    bytes per cell for the FP64 conjugate-gradient vectors (operator 48,
    update 64, direction 24), plus 231 for the FP32 V-cycle (212 on the
    finest level: six sweeps of about 28 bytes each, restriction and
    prolongation; 19 more on the coarse levels)."""
    import torch
    from paper_2604_11959_gb300 import inputs
    w = inputs.GRF_192
    h = w.heights()
    refs = inputs.cell_reference(w.nz, w.Lz)
    g = eb.Geometry(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, torch.from_numpy(h).cuda(), precision="mixed",
                    ref_rho=torch.from_numpy(refs[0]).cuda(), ref_rhotheta=torch.from_numpy(refs[1]).cuda())
    eb.set_preconditioner(g, "mg")
    U = eb.device_state(inputs.anelastic_state(w, seed=1), "mixed", refs)
    dt = w.dt()
    out, its = eb.anelastic_step(g, U, dt, max(1, warmup), rtol=1e-10)
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize()
    with clk or contextlib.nullcontext():
        a.record(stream)
        out, its = eb.anelastic_step(g, U, dt, steps, rtol=1e-10)
        b.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms_step = max_over_ranks(a.elapsed_time(b) / steps, dist)
    eb.sync_status(g)
    # one projection alone with each preconditioner: the divergent momenta of the initial state
    cells = w.cells()
    hbm, kind = peaks()
    proj = {}
    for pc, bpc in (("mg", 136 + 231), ("jacobi", 136)):
        eb.set_preconditioner(g, pc)
        eb.project(g, {f: U[f].clone() for f in U}, dt, rtol=1e-10)   # work space, warm-up
        W = {f: U[f].clone() for f in U}
        torch.cuda.synchronize()
        a.record(stream)
        it, res = eb.project(g, W, dt, rtol=1e-10)
        b.record(stream)
        torch.cuda.synchronize()
        ms_proj = a.elapsed_time(b)
        achieved = float(bpc) * cells * it / (ms_proj * 1e-3) / 1e9
        proj[pc] = {"iters": it, "relres": res, "ms": ms_proj, "ms_per_iter": ms_proj / max(1, it),
                    "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                                 "frac": achieved / hbm, "bytes_per_cell_per_iter": bpc, "peak_kind": kind}}
    g.close()
    return {"value": cells / (ms_step * 1e-3), "ms_per_step": ms_step, "cells": cells, "iters_per_solve": its,
            "projection": proj, "workload": w.name}


def run_ensemble(eb, steps, warmup, clk=None, dist=None, schedule="tuned"):
    """64 uneven Gaussian-hill instances (64x64x32 .. 256x256x64, 94,371,840
    cells), mixed path, advanced together: one CUDA-graph launch per step,
    slab heights chosen by the autotuner.  Like the single-domain line, every
    step is one pass over the same input states, reloaded (untimed) before
    it: forward Euler from an evolving state turns non-finite within about
    150 steps on these states (short-wave growth at CFL 0.5), and the reload
    (3.8 GB) also leaves no state in L2."""
    import torch
    from paper_2604_11959_gb300 import inputs
    geoms, states, dts, cells = [], [], [], 0
    for b, (n, _, nz, h0, sig) in enumerate(inputs.ensemble_members()):
        w = inputs.Workload(f"hill-{b}", n, n, nz, 100, terrain="gaussian", hmax=h0, sigma=sig)
        h = w.heights()
        refs = w.references("sheltered")
        g = make_geom(eb, w, h, "mixed", refs)
        geoms.append(g)
        states.append(eb.device_state(w.state("sheltered", seed=b), "mixed", refs))
        dts.append(w.dt())
        cells += w.cells()
    ens = eb.Ensemble(geoms)

    def reload():
        for q, U in enumerate(states):
            ens.set_state(q, U)

    reload()
    slab = ens.tune(dts, reps=2)
    if schedule != "tuned":
        ens.set_schedule(schedule)
    for _ in range(warmup):
        reload()
        ens.step(dts, 1)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier(dist)
    torch.cuda.synchronize()
    with clk or contextlib.nullcontext():
        for q in range(steps):
            reload()
            evs[q][0].record(stream)
            ens.step(dts, 1)
            evs[q][1].record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in evs])), dist)
    for g in geoms:
        eb.sync_status(g)
    kinfo = ens.info()
    # the other schedule, timed the same way (reported beside the tuned one)
    other = "branches" if kinfo["schedule"] == "persistent" else "persistent"
    ens.set_schedule(other)
    ot = []
    for q in range(steps + 2):
        reload()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ens.step(dts, 1)
        b.record(stream)
        torch.cuda.synchronize()
        if q >= 2:
            ot.append(a.elapsed_time(b))
    for g in geoms:
        eb.sync_status(g)
    ens.close()
    for g in geoms:
        g.close()
    hbm, kind = peaks()
    # the step is one kernel: its algorithmic traffic is the whole step's, 43
    # bytes per cell-update of the mixed path (5 fields read and written, the
    # near-EB geometry and redistribution tables)
    step_bytes = 43 * cells
    achieved = step_bytes / (ms * 1e-3) / 1e9
    per_step = 1 if kinfo["schedule"] == "persistent" else 7 * len(geoms)
    return {"value": cells / (ms * 1e-3), "ms_per_step": ms, "cells": cells, "members": len(geoms),
            "slab_levels": slab, "kernel_ctas": kinfo["ctas"], "bulk_units": kinfo["units"],
            "schedule": kinfo["schedule"], "other_schedule": {"schedule": other, "ms_per_step": float(np.mean(ot))},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": None, "kernel": "the whole ensemble step (%s schedule)" % kinfo["schedule"],
                         "algorithmic_bytes_per_launch": step_bytes, "peak_kind": kind},
            "gpu_launches": per_step * steps}   # persistent: one kernel per step; branches: ~7 per member


def run_slabs(eb, steps, warmup, world, rank, dist, clk=None):
    """The 256x256x128 hill (mixed path, forward Euler) cut into one x-slab
    per rank: each rank holds its owned columns plus a 12-column halo, and
    every step exchanges the halos (NCCL point-to-point) and advances the
    slab with eb_step.  Strong scaling: the whole job is the one domain."""
    import torch
    from paper_2604_11959_gb300 import inputs, slabs as S
    w = inputs.HILL_256
    h = w.heights()
    refs = w.references("sheltered")
    U = w.state("sheltered")
    sl = S.Slabs(w.nx, world, rank, S.HALO_EULER)
    ws = inputs.Workload("slab", sl.ext, w.ny, w.nz, 1, Lx=sl.ext * w.Lx / w.nx, Ly=w.Ly, Lz=w.Lz)
    geom = make_geom(eb, ws, sl.heights(h), "mixed", refs)
    held0 = eb.device_state({f: np.ascontiguousarray(sl.scatter(U[f])) for f in S.FIELDS}, "mixed", refs)
    dt = w.dt()
    slab_levels = eb.tune(geom, held0, dt, reps=3)   # the bulk kernel's split for the slab's columns

    def step_one(Uq):
        return eb.step(geom, Uq, dt, 1)

    A = {f: held0[f].clone() for f in S.FIELDS}
    S.advance(sl, A, warmup, step_one, dist)
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    A = {f: held0[f].clone() for f in S.FIELDS}
    barrier(dist)
    torch.cuda.synchronize()
    with clk or contextlib.nullcontext():
        a.record(stream)
        A = S.advance(sl, A, steps, step_one, dist)
        b.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = max_over_ranks(a.elapsed_time(b) / steps, dist)
    eb.sync_status(geom)
    geom.close()
    return {"value": w.cells() / (ms * 1e-3), "ms_per_step": ms, "cells": w.cells(), "halo": sl.halo,
            "held_columns": sl.ext, "owned_columns": sl.width, "tuned_slab_levels": slab_levels}


def compressible_cost(eb, world, dist, warmup, steps):
    """The hill's mixed step with the sources of the compressible system
    switched on (eb_geom_set_sources: pressure gradient and buoyancy), timed
    like the headline (L2 flushed before every step, per-step events), beside
    the same handle's advection-only step.  The sources run as their own
    pass after the flux update, and the redistribution then follows them
    instead of running beside the bulk kernel."""
    import torch
    w = workload("hill256")
    h = w.heights()
    refs = w.references("sheltered")
    geom = make_geom(eb, w, h, "mixed", refs)
    eb.tune(geom, eb.device_state(w.state("sheltered"), "mixed", refs), w.dt(), reps=3)
    A = eb.device_state(w.state("sheltered"), "mixed", refs)
    out = geom.empty_state()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for on in (False, True):
        geom.set_sources(on, on)
        for _ in range(warmup):
            eb.step(geom, A, w.dt(), 1, out=out)
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            eb.step(geom, A, w.dt(), 1, out=out)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        res["with_sources" if on else "advection_only"] = max_over_ranks(float(np.mean(ms)), dist)
    eb.sync_status(geom)
    geom.close()
    return {"workload": w.name, "cells": w.cells(), "value": world * w.cells() / (res["with_sources"] * 1e-3),
            "ms_per_step": res["with_sources"], "ms_per_step_advection_only": res["advection_only"],
            "steps": steps, "sources": "pressure gradient (equation of state) and buoyancy"}


def restriction_cost(eb, dist, warmup, steps):
    """Two-level refinement on the hill: the 128x128x64 coarse level built
    from the 256x256x128 handle by merging its cells (eb_geom_build_coarse,
    timed once on the host clock), and the restriction of a mixed state onto
    it (eb_restrict, per-call events with the L2 flushed before each).  The
    restriction's algorithmic traffic: the fine state (5 fields, 4 B) read
    once, the coarse state written once."""
    import torch
    w = workload("hill256")
    h = w.heights()
    refs = w.references("sheltered")
    fine = make_geom(eb, w, h, "mixed", refs)
    from paper_2604_11959_gb300 import inputs
    rc = inputs.cell_reference(w.nz // 2, w.Lz)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    coarse = fine.coarse(ref_rho=torch.from_numpy(rc[0]).cuda(), ref_rhotheta=torch.from_numpy(rc[1]).cuda())
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    Uf = eb.device_state(w.state("sheltered"), "mixed", refs)
    Uc = coarse.empty_state()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        eb.restrict(fine, coarse, Uf, Uc)
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        eb.restrict(fine, coarse, Uf, Uc)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = max_over_ranks(float(np.mean(ms)), dist)
    fine_bytes = sum(int(np.prod(fine.shape(f))) for f in eb.FIELDS) * 4
    coarse_bytes = sum(int(np.prod(coarse.shape(f))) for f in eb.FIELDS) * 4
    hbm, kind = peaks()
    gbs = (fine_bytes + coarse_bytes) / (t * 1e-3) / 1e9
    coarse.close()
    fine.close()
    return {"workload": f"{w.name} -> 128x128x64", "coarse_build_s": build_s, "restrict_ms": t,
            "restrict_gbs": gbs, "restrict_hbm_frac": gbs / hbm, "algorithmic_bytes": fine_bytes + coarse_bytes}


def unet_cost(eb, warmup, steps=10):
    """The warm-start network's kernels on the 96x96x48 grid of its training
    samples, with seeded random parameters, inputs and targets: one forward
    pass and one training step (forward, input and weight gradients, Adam),
    timed with CUDA events.  The arithmetic counts 2 cin cout 27 per voxel and
    convolution pass (three passes per step); the BF16 hi + lo split of the
    FP32 activations doubles the tensor-core products and is not counted.
    Against the measured BF16 tensor peak (burst: the kernels are timed
    alone)."""
    import torch
    from paper_2604_11959_gb300 import warmstart as ws
    nx, ny, nz = 96, 96, 48
    net = eb.UNet(nx, ny, nz)
    net.set_params(ws.init_params(11))
    rng = np.random.default_rng(12)
    x = torch.from_numpy(rng.standard_normal((2, nz, ny, nx)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((nz, ny, nx)).astype(np.float32)).cuda()
    m = torch.ones((nz, ny, nx), dtype=torch.float32, device="cuda")
    out = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")

    def timed(fn):
        for _ in range(max(3, warmup)):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    f_ms = timed(lambda: net.forward(x, out))
    s_ms = timed(lambda: net.train_step(x, t, m, 1e-6))
    net.sync_status()
    net.close()
    vox = nx * ny * nz
    fwd = sum(2 * ci * co * k ** 3 * vox / 8 ** lv for (ci, co, k), lv in
              zip(ws.LAYERS, (0, 0, 1, 1, 2, 2, 1, 1, 0, 0, 0)))
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, kind = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        peak, kind = 1900.0, "fallback"
    return {"workload": "warm-start network 96x96x48 (16/32/64 channels)", "forward_ms": f_ms,
            "forward_tflops": fwd / (f_ms * 1e-3) / 1e12, "train_step_ms": s_ms,
            "train_step_tflops": 3 * fwd / (s_ms * 1e-3) / 1e12,
            "bf16_peak_tflops": peak, "peak_kind": kind,
            "forward_frac": fwd / (f_ms * 1e-3) / 1e12 / peak,
            "train_step_frac": 3 * fwd / (s_ms * 1e-3) / 1e12 / peak,
            "kernels": "tcgen05.mma implicit GEMMs, FP32 activations as BF16 hi + lo, TMEM accumulators"}


def other_configs(eb, world, dist, warmup, steps=10):
    """The other timed configurations, measured in the default run beside
    the headline: the 512x512x256 random terrain (mixed path, tuned, per-step
    events with the L2 flushed, bulk kernel against HBM) and the 64-member
    ensemble (tuned schedule).  The warm-start training (about two minutes)
    runs only as its own workload."""
    import torch
    w = workload("grf512")
    h = w.heights()
    refs = w.references("sheltered")
    geom, r = run_precision(eb, w, h, w.state("sheltered"), refs, "mixed", steps, warmup, world, dist)
    geom.close()
    torch.cuda.empty_cache()
    out = {"grf512": {"workload": w.name, "cells": w.cells(), "value": r["value"], "ms_per_step": r["ms_per_step"],
                      "steps": r["steps"], "phases_ms": r["phases_ms"], "roofline_frac": r["roofline"]["frac"],
                      "tuned_slab_levels": r["tuned_slab_levels"], "bulk_high_priority": r["bulk_high_priority"]}}
    out["hill256_compressible"] = compressible_cost(eb, world, dist, warmup, steps)
    out["hill256_restriction"] = restriction_cost(eb, dist, warmup, steps)
    out["warmstart_network"] = unet_cost(eb, warmup, steps)
    torch.cuda.empty_cache()
    e = run_ensemble(eb, steps, warmup, None, dist)
    torch.cuda.empty_cache()
    out["ensemble"] = {"workload": "ensemble-64-gaussian-hills", "cells": e["cells"], "value": e["value"] * world,
                       "ms_per_step": e["ms_per_step"], "steps": steps, "schedule": e["schedule"],
                       "other_schedule": e["other_schedule"], "step_hbm_frac": e["roofline"]["frac"]}
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class _Nvml:
    """Read-only NVML queries through ctypes (SM clock, its maximum and the
    clock event reasons); None where the library is not there."""
    # reason bits of nvmlDeviceGetCurrentClocksEventReasons (public nvml.h)
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    @classmethod
    def open(cls, device_index):
        try:
            import ctypes
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            import torch
            p = torch.cuda.get_device_properties(device_index)
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(h)) != 0:
                return None
            self = cls()
            self.lib, self.h, self.ct = lib, h, ctypes
            get = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.reasons_fn = get
            return self
        except Exception:
            return None

    def sample(self):
        c, m, r = self.ct.c_uint(), self.ct.c_uint(), self.ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(c)) != 0:   # NVML_CLOCK_SM
            return None
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, self.ct.byref(m))
        self.reasons_fn(self.h, self.ct.byref(r))
        return float(c.value), float(m.value), [k for k, b in self.BITS.items() if r.value & b]


class ClockSampler:
    """SM clock and clock event reasons sampled DURING a timed region: NVML
    every 0.5 ms from a thread when the library is there (a timed loop of a
    few tens of milliseconds still gets dozens of samples), else
    nvidia-smi -lms 20.  Enter it around the timed loop only."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.sm, self.mx, self.reasons = [], None, set()
        self.proc = None
        self.dev = device_index
        self.nvml = _Nvml.open(device_index)
        self.source = "nvml" if self.nvml else "nvidia-smi"

    def __enter__(self):
        self.stop = threading.Event()
        if self.nvml:
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "20", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _poll(self):
        while not self.stop.is_set():
            r = self.nvml.sample()
            if r:
                self.sm.append(r[0])
                self.mx = r[1]
                self.reasons.update(r[2])
            time.sleep(0.0005)

    def _read(self):
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.proc.stdout:
            parts = [p.strip() for p in ln.strip().split(",")]
            if len(parts) < 9:
                continue
            try:
                sm, mx = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            self.sm.append(sm)
            self.mx = mx
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    self.reasons.add(nm)

    def __exit__(self, *a):
        self.stop.set()
        if self.nvml:
            self.t.join(timeout=5)
        elif self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "source": self.source}
        return {"sm_mhz": float(np.median(self.sm)), "sm_max_mhz": self.mx, "reasons": sorted(self.reasons),
                "samples": len(self.sm), "sm_mhz_min": float(np.min(self.sm)), "source": self.source,
                "window": "timed steps only"}


# ---------------------------------------------------------------------------
# the oracle as CPU baseline (and the reference arm)
# ---------------------------------------------------------------------------
def oracle_domain(w):
    """The FP64 oracle on the whole domain of workload w: (module, domain,
    geometry, tables); built with all of this host's cores."""
    from oracle import eb_oracle as O
    O.build()
    O.set_threads(os.cpu_count() or 1)
    dom = O.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, w.heights())
    G = O.geometry(dom)
    return O, dom, G, O.wsrd_setup(dom, G)


def cpu_baseline(w, steps=None, warmup=0, budget_s=15.0, orc=None):
    """The FP64 oracle as it stands, timed on this host's cores on the whole
    domain of the workload, forward-Euler steps from the benchmark's state;
    geometry and table set-up untimed.  With ``steps`` it runs exactly
    ``warmup`` untimed and ``steps`` timed steps (the reference arm);
    otherwise as many steps as fit in about ``budget_s`` seconds."""
    O, dom, G, T = orc or oracle_domain(w)
    cores = os.cpu_count() or 1
    U = w.state("sheltered")
    for _ in range(warmup):
        U = O.step(dom, G, T, U, w.dt(), 1)
    if steps is None:
        t0 = time.perf_counter()
        U = O.step(dom, G, T, U, w.dt(), 1)
        steps = int(max(1, min(50, budget_s / max(time.perf_counter() - t0, 1e-3))))
    t0 = time.perf_counter()
    O.step(dom, G, T, U, w.dt(), steps)
    el = time.perf_counter() - t0
    return {"value": w.cells() * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle", "steps": steps,
            "ms_per_step": el * 1e3 / steps,
            "sample": f"whole {w.name} domain ({w.cells()} cells), {steps} forward-Euler steps in {el:.1f} s "
                      f"after {warmup} untimed; geometry and table set-up untimed"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
BULK_SOURCES = ("eb_bulk.cuh", "eb_fast.cu", "eb_geom.cu")


def bulk_source_hash():
    """Hash of the bulk kernel's source and of the set-up that decides its
    work (the first fast level of every column)."""
    srcs = [os.path.join(ROOT, "paper_2604_11959_gb300", "csrc", f) for f in BULK_SOURCES]
    return hashlib.sha256(b"".join(open(f, "rb").read() for f in srcs)).hexdigest()[:16]


def profile_record(kernel, workload_name, precision, key, tile_rows=16):
    """A figure of a committed ncu summary (DRAM bytes per launch, FP64
    operations per cell), valid only while the sources it was taken on are
    unchanged (their hash is recorded with it) and for the tile height it was
    taken at; None otherwise."""
    rows = "" if int(tile_rows) == 16 else f"_rows{int(tile_rows)}"
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload_name}_{precision}{rows}.txt")
    try:
        rec = {}
        for line in open(path):
            if ":" in line:
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        if rec.get("source_sha256_16") != bulk_source_hash():
            return None
        if int(rec.get("tile_rows", "16")) != int(tile_rows):
            return None
        return float(rec[key])
    except Exception:
        return None


def traffic_record(kernel, workload_name, precision, tile_rows=16):
    return profile_record(kernel, workload_name, precision, "dram_bytes_per_launch_full_size", tile_rows)


def make_geom(eb, w, h, precision, refs):
    """Geometry handle of workload w with the per-level profiles refs =
    (rho0, rho0 theta0[, background rho*u, background rho*v])."""
    import torch
    kw = {}
    if len(refs) == 4:
        kw = dict(ref_rhou=torch.from_numpy(np.ascontiguousarray(refs[2])).cuda(),
                  ref_rhov=torch.from_numpy(np.ascontiguousarray(refs[3])).cuda())
    return eb.Geometry(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, torch.from_numpy(h).cuda(), precision=precision,
                       ref_rho=torch.from_numpy(refs[0]).cuda(), ref_rhotheta=torch.from_numpy(refs[1]).cuda(), **kw)


def run_precision(eb, w, h, U, refs, precision, steps, warmup, world, dist, clk=None, slab_levels=None,
                  tile_rows=None):
    import torch
    geom = make_geom(eb, w, h, precision, refs)
    info = geom.info()
    # every step is one pass of the whole path over the same input state U0
    # (evolving the state for hundreds of forward-Euler steps would measure a
    # different, eventually degenerate, flow); outputs alternate between two
    # buffers and the L2 is flushed before each timed step
    A = eb.device_state(U, precision, refs)
    if slab_levels is None:
        slab = eb.tune(geom, A, w.dt(), reps=5)   # autotuned slab height of the bulk kernel's tiles
    else:
        slab = slab_levels
        if tile_rows is not None and precision == "mixed":
            eb.set_tile_rows(geom, tile_rows)
        eb.set_slab_levels(geom, slab)
    outs = [geom.empty_state(), geom.empty_state()]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    dt = w.dt()
    for q in range(warmup):
        eb.step(geom, A, dt, 1, out=outs[q % 2])
    eb.sync_status(geom)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier(dist)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with clk or contextlib.nullcontext():
        for q in range(steps):
            flush.zero_()   # evict the state from L2 (untimed)
            evs[q][0].record(stream)
            eb.step(geom, A, dt, 1, out=outs[q % 2])
            evs[q][1].record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    wall = time.perf_counter() - wall0
    ms = [a.elapsed_time(b) for a, b in evs]
    eb.sync_status(geom)
    ms_step = max_over_ranks(float(np.mean(ms)), dist)
    # the dominant kernel alone, timed with events on its stream
    prof = []
    for q in range(max(5, min(steps, 20))):
        flush.zero_()
        prof.append(eb.step_profile(geom, A, outs[q % 2], dt))
    prof = np.median(np.array(prof), axis=0)
    es = 8 if precision == "f64" else 4
    fast_bytes = info["fast_cells"] * 10 * es
    hbm, kind = peaks()
    achieved = fast_bytes / (prof[0] * 1e-3) / 1e9
    rows_now = int(geom.info()["tile_rows"])
    hbm_roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic_record("k_fast_tiled", w.name, precision, rows_now),
                "kernel": "k_fast_tiled", "tile_rows": rows_now,
                "algorithmic_bytes_per_launch": fast_bytes, "peak_kind": kind,
                "warp_instructions_per_fast_cell": profile_record("k_fast_tiled", w.name, precision,
                                                                  "warp_instructions_per_fast_cell",
                                                                  rows_now)}
    roof = hbm_roof
    if precision == "mixed":
        # the other tile height, timed the same way: the bulk kernel alone and
        # the whole step (the tuner keeps the faster step)
        tuned_rows = rows_now
        other = 14 if tuned_rows == 16 else 16
        eb.set_tile_rows(geom, other)
        alt = []
        for q in range(max(5, min(steps, 20))):
            flush.zero_()
            alt.append(eb.step_profile(geom, A, outs[q % 2], dt))
        alt = np.median(np.array(alt), axis=0)
        st_ms = []
        for q in range(max(5, min(steps, 20))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            eb.step(geom, A, dt, 1, out=outs[q % 2])
            b.record(stream)
            torch.cuda.synchronize()
            st_ms.append(a.elapsed_time(b))
        eb.set_tile_rows(geom, tuned_rows)
        hbm_roof["other_tile_rows"] = {
            "tile_rows": other, "bulk_ms": float(alt[0]),
            "frac": fast_bytes / (float(alt[0]) * 1e-3) / 1e9 / hbm, "step_ms": float(np.mean(st_ms)),
            "note": "the tuner keeps the tile height of the faster whole step"}
    if precision == "f64":
        # GB300's FP64 rate is low: the FP64 bulk kernel is bound by its FP64
        # arithmetic, measured against the DFMA rate of this GPU
        fpeak = eb.fma_peak("f64")
        fpc = profile_record("k_fast_tiled", w.name, precision, "fp64_flops_per_fast_cell")
        roof = {"bound": "fp64", "achieved": None, "peak": fpeak, "unit": "GFLOP/s", "frac": None,
                "kernel": "k_fast_tiled", "peak_kind": "measured (eb_fma_peak, DFMA = 2 flops)",
                "flops_per_fast_cell": fpc, "hbm": hbm_roof}
        if fpc:
            roof["achieved"] = fpc * info["fast_cells"] / (prof[0] * 1e-3) / 1e9
            roof["frac"] = roof["achieved"] / fpeak
    # per step: static pass-through (a fresh output buffer every call), the
    # tiled bulk kernel, the two near-EB kernels (face fluxes; CVs with and
    # without a record in one launch) and the three fused redistribution passes
    launches_per_step = 2 + (2 if sum(info["band_cvs"]) else 0) + (2 if sum(info["small_cvs"]) else 0) + \
        (1 if sum(info["affected_cvs"]) else 0)
    # bytes the whole step must move: every non-covered CV read and written
    # once, plus the band geometry records read by the near-EB kernel
    step_bytes = sum(info["cvs"][g] * (2 if g else 4) for g in range(4)) * es + \
        sum(info["band_records"]) * 10 * 8
    res = {
        "value": world * info["cells"] / (ms_step * 1e-3),
        "ms_per_step": ms_step,
        "wall_s": wall,
        "geometry": info,
        "phases_ms": {"fast": float(prof[0]), "band": float(prof[1]), "wsrd": float(prof[2]),
                      "step": float(prof[3])},
        "roofline": roof,
        "step_gbs": step_bytes / (ms_step * 1e-3) / 1e9,
        "step_frac": step_bytes / (ms_step * 1e-3) / 1e9 / hbm,
        "gpu_launches": launches_per_step * steps,
        "steps": steps,
        "tuned_slab_levels": slab,
        "bulk_high_priority": int(geom.info()["bulk_high_priority"]),
        "tile_rows": int(geom.info()["tile_rows"]),
    }
    return geom, res


def accuracy(eb, w, h, U, refs, nsteps, orc=None, oracle_steps=10):
    """Error of the paths after nsteps steps from the benchmark's state, the
    momenta stored about the state's background wind, per field as the
    relative L-inf error max |a - b| / max |b| over the non-covered
    prognostic CVs (full values, profiles added back):
      vs_oracle: the mixed and FP64 paths against the FP64 CPU oracle after
        ``oracle_steps`` three-stage Runge-Kutta steps on the whole domain
        (the oracle takes about 3 s per step here, so the benchmark stops
        there; the GPU parity tests run the full 100 steps against it);
      rk3 / forward_euler: the mixed path against the FP64 path after nsteps
        steps (the FP64 path equals the oracle to 1e-12);
      conservation: the change of sum alpha U over nsteps three-stage steps,
        relative to sum alpha |U|, per field and path (zero in exact
        arithmetic for rho, rho*theta, rho*u and rho*v: periodic sides, no
        flux through the terrain and the walls; rho*w changes by the flux
        beside its non-prognostic wall levels, equal for both paths).
    Forward Euler with third-order upwind amplifies the shortest waves by
    about 9% per step at CFL 0.5, which magnifies the float rounding."""
    import torch
    res = {"steps": nsteps, "state": "momenta stored about the background wind (eb_geom_set_wind_reference)"}
    geoms = {p: make_geom(eb, w, h, p, refs) for p in ("mixed", "f64")}
    alpha = {g: geoms["f64"].export(g, "alpha").cpu().numpy() for g in range(4)}
    act = {}
    for g in range(4):
        m = alpha[g] > 0
        if g == 3:
            m[0] = m[w.nz] = False
        act[g] = m
    fg = {"rho": 0, "rhotheta": 0, "rhou": 1, "rhov": 2, "rhow": 3}

    def full(S):
        return {f: eb.full_values(S, refs)[f] for f in FIELDS}

    def rel(a, b, f):
        m = act[fg[f]]
        return float(np.abs(a[m] - b[m]).max() / np.abs(b[m]).max())

    out = {}
    for p in ("mixed", "f64"):
        A = eb.device_state(U, p, refs)
        first = eb.step(geoms[p], A, w.dt(), oracle_steps, stages=3)
        last = eb.step(geoms[p], first, w.dt(), nsteps - oracle_steps, stages=3)
        fe = eb.step(geoms[p], A, w.dt(), nsteps, stages=1)
        eb.sync_status(geoms[p])
        out[p] = {"first": full(first), "last": full(last), "fe": full(fe)}
    U0 = {f: np.asarray(U[f]) for f in FIELDS}
    res["rk3"] = {"rel_linf_vs_f64": {f: rel(out["mixed"]["last"][f], out["f64"]["last"][f], f) for f in FIELDS}}
    res["forward_euler"] = {"rel_linf_vs_f64": {f: rel(out["mixed"]["fe"][f], out["f64"]["fe"][f], f)
                                                for f in FIELDS}}
    cons = {}
    for p in ("mixed", "f64"):
        d = {}
        for f in FIELDS:
            a, m = alpha[fg[f]], act[fg[f]]
            s0 = float((a[m] * U0[f][m]).sum())
            s1 = float((a[m] * out[p]["last"][f][m]).sum())
            d[f] = (s1 - s0) / float((a[m] * np.abs(U0[f][m])).sum())
        cons[p] = d
    cons["mixed_minus_f64"] = {f: cons["mixed"][f] - cons["f64"][f] for f in FIELDS}
    res["conservation"] = {"steps": nsteps, "stages": 3, "relative_change_of_sum_alpha_U": cons}
    if orc is not None:
        O, dom, G, T = orc
        want = O.step(dom, G, T, U0, w.dt(), oracle_steps, 3)
        res["vs_oracle"] = {"steps": oracle_steps, "stages": 3, "reference": "FP64 CPU oracle, whole domain",
                            "rel_linf": {p: {f: rel(out[p]["first"][f], want[f], f) for f in FIELDS}
                                         for p in ("mixed", "f64")}}
    for g in geoms.values():
        g.close()
    return res


def e2e(eb, geom, w, U, refs, precision, steps):
    """Same metric through the public API with host buffers: every step
    copies its input state from pinned host memory to the device, advances
    it (``eb.step``) and copies the result back to pinned host memory.  The
    steps are pipelined as a server would run them: copy-in, compute and
    copy-out of consecutive steps run on three streams, the device input and
    output buffers alternating between two sets (events order the reuse).
    Each state is one allocation (``Geometry.packed_state``), so a whole state
    moves with one copy per direction."""
    import torch
    hostU = eb.host_state(U, precision, refs)
    h_in, h_views = geom.packed_state("cpu", pin=True)
    for f in FIELDS:
        h_views[f].copy_(hostU[f])
    dev = [geom.packed_state() for _ in range(2)]
    out = [geom.packed_state() for _ in range(2)]
    hout = [geom.packed_state("cpu", pin=True) for _ in range(2)]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    bi = sum(t.numel() * t.element_size() for t in hostU.values())
    dt = w.dt()

    def run(n):
        ev_in, ev_cmp, ev_out = {}, {}, {}
        for q in range(n):
            b = q % 2
            with torch.cuda.stream(s_in):
                if q >= 2:
                    s_in.wait_event(ev_cmp[q - 2])     # input set b free again
                dev[b][0].copy_(h_in, non_blocking=True)
                ev_in[q] = torch.cuda.Event()
                ev_in[q].record(s_in)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(ev_in[q])
                if q >= 2:
                    s_cmp.wait_event(ev_out[q - 2])    # output set b read out
                eb.step(geom, dev[b][1], dt, 1, out=out[b][1], stream=s_cmp)
                ev_cmp[q] = torch.cuda.Event()
                ev_cmp[q].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_cmp[q])
                hout[b][0].copy_(out[b][0], non_blocking=True)
                ev_out[q] = torch.cuda.Event()
                ev_out[q].record(s_out)

    run(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run(steps)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    # the copies move the padded blocks: count the bytes actually copied
    bcopy = h_in.numel() * h_in.element_size()
    return {"value": w.cells() / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": bcopy, "d2h_bytes_per_step": bcopy,
            "field_bytes_per_step": bi, "ms_per_step": ms,
            "pipelined": "copy-in, compute and copy-out of consecutive steps overlap; one copy per state"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    w = workload(args.workload)
    if args.impl == "reference":
        if rank != 0:
            return 0
        cb = cpu_baseline(w, steps=args.steps, warmup=args.warmup)
        print(json.dumps({"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
                          "steps": cb["steps"], "warmup": args.warmup, "ms_per_step": cb["ms_per_step"],
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "impl": "reference",
                          "config": {"workload": w.name, "cells": w.cells(), "precision": "f64", "stages": 1,
                                     "path": "FP64 CPU oracle, whole domain"},
                          "cpu_baseline": cb,
                          "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return 0
    import torch
    dist = init_ranks(world)
    try:
        return run_arm(args, rank, world, w, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


def run_arm(args, rank, world, w, dist):
    """Our arm, every workload: one JSON line from rank 0."""
    import torch
    if args.workload == "warmstart":
        from paper_2604_11959_gb300 import build as libbuild, eb
        libbuild.build()
        eb.load()
        r = run_warmstart(eb, args.terrains, args.epochs)
        if rank == 0:
            print(json.dumps({"workload": "warmstart", "metric": "PCG iterations to relative residual 1e-10, "
                              "zero start / network start", "value": r["grf192"]["ratio"], "unit": "x",
                              "higher_is_better": True, "data": "synthetic", **r}))
        return 0
    if args.workload == "network":
        from paper_2604_11959_gb300 import build as libbuild, eb
        libbuild.build()
        eb.load()
        r = unet_cost(eb, args.warmup, args.steps)
        if rank == 0:
            print(json.dumps({"metric": "warm-start network training step, useful TFLOP/s", "unit": "TFLOP/s",
                              "value": r["train_step_tflops"], "higher_is_better": True, "data": "synthetic",
                              "steps": args.steps, "warmup": max(3, args.warmup), **r}))
        return 0
    if args.workload == "anelastic":
        from paper_2604_11959_gb300 import build as libbuild, eb
        libbuild.build()
        eb.load()
        clk = ClockSampler(torch.cuda.current_device())
        r = run_anelastic(eb, args.steps, args.warmup, clk, dist)
        if rank == 0:
            print(json.dumps({
                "metric": METRIC, "value": r["value"] * world, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": r["workload"], "cells": r["cells"], "model": "anelastic", "stages": 2,
                           "projection": "FP64 PCG with an FP32 multigrid V-cycle preconditioner to relative "
                                         "residual 1e-10, zero initial guess",
                           "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
                "iters_per_solve": r["iters_per_solve"], "projection": r["projection"],
                "roofline": r["projection"]["mg"]["roofline"], "clocks": clk.summary(),
                "cpu_baseline": None, "e2e": None}))
        return 0
    if args.workload == "slabs":
        from paper_2604_11959_gb300 import build as libbuild, eb
        libbuild.build()
        eb.load()
        clk = ClockSampler(torch.cuda.current_device())
        r = run_slabs(eb, args.steps, max(3, args.warmup), world, rank, dist, clk)
        if rank == 0:
            print(json.dumps({
                "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "gaussian-hill-256x256x128 in x-slabs", "cells": r["cells"],
                           "precision": "mixed", "stages": 1, "halo": r["halo"],
                           "held_columns_per_rank": r["held_columns"], "owned_columns_per_rank": r["owned_columns"],
                           "tuned_slab_levels": r["tuned_slab_levels"],
                           "parallelism": f"{world} x-slabs, halo exchange every step"},
                "roofline": None, "clocks": clk.summary(), "cpu_baseline": None, "e2e": None,
                "gpu_launches": 7 * args.steps}))   # per step: pass-through, bulk, 2 near-EB, 3 redistribution
        return 0
    if args.workload == "ensemble":
        from paper_2604_11959_gb300 import build as libbuild, eb
        libbuild.build()
        eb.load()
        clk = ClockSampler(torch.cuda.current_device())
        r = run_ensemble(eb, args.steps, max(3, args.warmup), clk, dist, args.ensemble_schedule)
        if rank == 0:
            print(json.dumps({
                "metric": METRIC, "value": r["value"] * world, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "ensemble-64-gaussian-hills", "cells": r["cells"], "members": r["members"],
                           "precision": "mixed", "stages": 1, "tuned_slab_levels": r["slab_levels"],
                           "kernel_ctas": r["kernel_ctas"], "bulk_units": r["bulk_units"],
                           "schedule": r["schedule"],
                           "launch": "tuned schedule, one CUDA-graph launch per step: the persistent cooperative "
                                     "kernel, or every member's kernels side by side",
                           "l2": "the same input states (3.8 GB, larger than L2) reloaded untimed before every "
                                 "timed step; per-step CUDA events",
                           "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
                "other_schedule": r["other_schedule"],
                "roofline": r["roofline"], "gpu_launches": r["gpu_launches"], "clocks": clk.summary(),
                "cpu_baseline": None, "e2e": None}))
        return 0
    from paper_2604_11959_gb300 import build as libbuild, eb, inputs
    libbuild.build()
    eb.load()
    h = w.heights()
    refs = w.references("sheltered")   # momenta stored about the state's background wind
    U = w.state("sheltered")
    dev_index = torch.cuda.current_device()
    mixed = f64 = e2e_res = None
    clk = ClockSampler(dev_index)
    if args.precision in ("both", "mixed"):
        geom, mixed = run_precision(eb, w, h, U, refs, "mixed", args.steps, args.warmup, world, dist, clk,
                                    args.slab_levels, args.tile_rows)
        if rank == 0 and not args.no_e2e:
            e2e_res = e2e(eb, geom, w, U, refs, "mixed", min(args.steps, 20))
        geom.close()
    if args.precision in ("both", "f64"):
        geom64, f64 = run_precision(eb, w, h, U, refs, "f64", max(10, args.steps // 10), args.warmup, world, dist,
                                    None if mixed else clk, args.slab_levels)
        geom64.close()
    others = None
    if args.precision == "both" and args.workload == "hill256":
        others = other_configs(eb, world, dist, max(3, args.warmup))
    acc = cb = orc = None
    if rank == 0 and world == 1 and not args.no_cpu:
        orc = oracle_domain(w)   # after every timed region: the oracle loads all host cores
        cb = cpu_baseline(w, orc=orc)
    if rank == 0 and args.precision == "both":
        acc = accuracy(eb, w, h, U, refs, w.steps, orc)
    if rank != 0:
        return 0
    head = mixed or f64
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64", "data": "synthetic",
        "config": {"workload": w.name, "cells": w.cells(), "precision": "mixed" if mixed else "f64", "stages": 1,
                   "state": "stratified, wind u=1 above the terrain, smooth seeded perturbations",
                   "l2": "512 MiB buffer written before every timed step (untimed); per-step CUDA events",
                   "tuned_slab_levels": head.get("tuned_slab_levels"),
                   "tuned_bulk_high_priority": head.get("bulk_high_priority"),
                   "tuned_tile_rows": head.get("tile_rows"),
                   "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
        "roofline": head["roofline"],
        "step_hbm_frac": head["step_frac"],
        "phases_ms": head["phases_ms"],
        "cpu_baseline": cb,
        "e2e": e2e_res,
        "gpu_launches": head["gpu_launches"],
        "clocks": clk.summary(),
        "geometry": {k: head["geometry"][k] for k in ("cells", "fast_cells", "band_cvs", "small_cvs",
                                                      "affected_cvs", "tiny_cvs", "min_alpha")},
    }
    if acc:
        line["accuracy"] = acc
    if others:
        line["other_configs"] = others
    if mixed and f64:
        line["fp64"] = {"value": f64["value"], "ms_per_step": f64["ms_per_step"], "roofline": f64["roofline"],
                        "step_hbm_frac": f64["step_frac"], "phases_ms": f64["phases_ms"], "steps": f64["steps"]}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
