#!/usr/bin/env python
"""Throughput of the S2O4 gas-kinetic step with ALM + IBM forcing on GB300.

One step = one full two-stage fourth-order step of the high-order GKS on the
whole grid (ghost fill, reconstruction, flux and update of both stages, the
CFL time step) followed by the actuator-line and immersed-boundary forcing.
The default workload is the rotor plus IBM tower and nacelle on a
384 x 256 x 256 grid in FP32 with compensated state; FP64 is timed on the
same grid for a few steps. Metric: MLUPS = cells x steps / seconds.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

For N > 1 launch one process per GPU with torch.distributed.run; each rank
runs an independent replica (the method is not sharded here), value is the
sum over ranks (weak scaling). ``--impl reference`` times the CPU oracle on
a bounded window of the same workload on the host cores.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_11102_gb300 import workloads as WL  # noqa: E402

# Hand estimates of the FP32 operations per face of the face box each launch
# processes (adds, multiplies, FMA = 2): used only when no measured count of
# the current kernel source is committed (profiles/flops.txt, ncu counts of
# the FFMA, FADD and FMUL instructions executed).
FLOPS_ESTIMATE = {
    # WENO5 on 4 variables x 2 sides (40 each), half-space equilibrium (~40
    # plus 2 erf, 2 exp, 2 expm1), normal slope (4 x 5)
    "face_eq": 4 * 2 * 40 + 46 + 20,
    # t1 pass (4 x (25 + 17) per row), t2 pass (2 x 4 x 63), 4 fluxes, average
    "face_flux_stage1": 168 + 504 + 4 * 118 + 8,
    "face_flux_stage2": 168 + 504 + 4 * 100 + 4,
}
FLOPS_ESTIMATE["flux_update_stage1"] = FLOPS_ESTIMATE["face_flux_stage1"]
FLOPS_ESTIMATE["flux_update_stage2"] = FLOPS_ESTIMATE["face_flux_stage2"]
# the source section of gks_stencil.cu each kernel group is built from
SECTIONS = {"face_eq": ("face state", "face flux"), "face_flux": ("face flux", "z flux + stage update"),
            "flux_update": ("z flux + stage update", "prep, CFL, misc")}
BYTES_PER_CELL_STEP = {"fp32c": 160, "fp64": 192}


# The headline metric: MLUPS of full S2O4 steps with ALM + IBM forcing
# (value: FP32-compensated; the FP64 figure, the HBM and ALU roofline
# fractions and the adjoint / forward time ratio are fields of the same line).
METRIC = "GKS MLUPS (FP64 vs FP32-compensated, ALM+IBM) + % HBM roofline; adjoint/fwd time"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-i",
                 str(gpu_index), "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(name):
    if name == "alm-ibm":
        return WL.alm_ibm_rotor((384, 256, 256))
    if name == "alm":
        return WL.alm_rotor((512, 192, 192))
    if name == "channel":
        return WL.channel((128, 128, 128))
    if name == "tgv":
        return WL.taylor_green_3d(32)
    if name == "tgv192":
        return WL.taylor_green_3d(192)
    if name == "tgv96":
        return WL.taylor_green_3d(96)
    raise ValueError(name)


def window(w, lo, size):
    """Sub-grid of a workload at the same spacing (cells lo..lo+size per axis),
    same boundary kinds, rotor and bodies, initial state cut from state0."""
    faces = [w.faces[a][lo[a]:lo[a] + size[a] + 1].copy() for a in range(3)]
    Q = w.state0[:, lo[2]:lo[2] + size[2], lo[1]:lo[1] + size[1], lo[0]:lo[0] + size[0]].copy()
    sub = WL.Workload(w.name + "-window", tuple(size), faces, w.mach, w.u_ref, w.mu, list(w.bc), cfl=w.cfl,
                      dt_fixed=w.dt_fixed, inflow=w.inflow, body_force=w.body_force, rho_ref=w.rho_ref,
                      state0=Q, rotors=list(w.rotors), bodies=list(w.bodies), steps=w.steps)
    return sub


def oracle_sample(w):
    """Bounded sample of the workload for the CPU oracle: a window of the grid
    around the rotor at the full resolution."""
    n = w.n
    size = (min(16, n[0]), min(80, n[1]), min(80, n[2]))
    if w.rotors:
        hub = w.rotors[0].hub
        lo = [int((hub[a] - w.faces[a][0]) / (w.faces[a][1] - w.faces[a][0])) - size[a] // 2 for a in range(3)]
    else:
        lo = [(n[a] - size[a]) // 2 for a in range(3)]
    lo = [max(0, min(lo[a], n[a] - size[a])) for a in range(3)]
    return window(w, lo, size), lo


def oracle_grid(w):
    import oracle
    o = oracle.OracleGrid(w.n, w.faces, w.mach, w.u_ref, w.mu, w.bc, cfl=w.cfl, dt_fixed=w.dt_fixed)
    o.set_inflow(*w.inflow)
    o.set_body_force(*w.body_force)
    for r in w.rotors:
        o.add_rotor(r.n_blades, r.r, r.chord, r.twist, r.width, r.hub, r.omega, r.azimuth0, r.radius, r.eps,
                    r.rho_inf, r.u_inf_ref, r.correction, r.tip_correction)
    for b in w.bodies:
        o.add_body(b.xyz, b.dS, b.eps, vel=b.vel, niter=b.niter, tol=b.tol)
    o.set_state(w.state0)
    return o


def time_oracle(w, steps, warmup):
    import oracle
    sample, lo = oracle_sample(w)
    o = oracle_grid(sample)
    for _ in range(warmup):
        o.step(1)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    mlups = sample.cells * steps / dt / 1e6
    desc = ("window of %dx%dx%d cells (origin cell %s) of the %s grid at the same spacing, same "
            "boundary kinds, rotor and bodies; %d step(s) after %d warm-up, FP64 oracle"
            % (sample.n + (tuple(lo), w.name, steps, warmup)))
    return mlups, dt, oracle.get_threads(), desc


def source_hash(group="face_flux"):
    """Hash of the source a kernel group's measured figures depend on: the
    device header and the group's section of gks_stencil.cu."""
    csrc = os.path.join(ROOT, "paper_2603_11102_gb300", "csrc")
    h = hashlib.sha256()
    with open(os.path.join(csrc, "gks_device.cuh"), "rb") as fh:
        h.update(fh.read())
    with open(os.path.join(csrc, "gks_stencil.cu")) as fh:
        text = fh.read()
    first, last = SECTIONS[group]

    def marker(name):
        for line in text.splitlines():
            if line.startswith("// ---") and line.rstrip().endswith(" " + name + " --"):
                return text.index(line)
        raise ValueError(name)
    h.update(text[marker(first):marker(last)].encode())
    return h.hexdigest()[:16]


def read_traffic(kernel, precision):
    """DRAM bytes per launch of a kernel from a committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    cur = source_hash(kernel) if kernel in SECTIONS else None
    for line in open(p):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == precision and parts[3] == cur:
            return float(parts[2])
    return None


def read_flops(precision):
    """Measured operations per face of each kernel group and stage (ncu counts
    of FFMA x 2 + FADD + FMUL, or the FP64 ones) from profiles/flops.txt,
    where they were taken on the current kernel sources; else the hand
    estimates. Returns ({group_stage: flops}, {group: source})."""
    out, src = {}, {}
    p = os.path.join(ROOT, "profiles", "flops.txt")
    hashes = {g: source_hash(g) for g in SECTIONS}
    if os.path.exists(p):
        for line in open(p):
            parts = line.split("#", 1)[0].split()
            if len(parts) == 5 and parts[1] == precision and parts[0] in hashes and parts[4] == hashes[parts[0]]:
                key = parts[0] if parts[2] == "-" else "%s_stage%s" % (parts[0], parts[2])
                out[key] = float(parts[3])
                src[parts[0]] = "measured (profiles/flops.txt)"
    for k, v in FLOPS_ESTIMATE.items():
        if k not in out:
            out[k] = v
            src.setdefault(k.split("_stage")[0], "hand estimate")
    return out, src


def measure_alu_peak(dev, kind, seconds=1.0, repeats=3):
    """Arithmetic peak of this GPU from the library's FMA-loop probe (kind 0
    FP32, 1 FP64, 2 packed FP32 pairs), timed with CUDA events on one stream:
    (best, median) TFLOP/s over `repeats` launches of about `seconds` each."""
    import torch

    from paper_2603_11102_gb300 import gks
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(4 * sms, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)

    def once(iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        fl = gks.alu_peak_probe(kind, iters, sink, st)
        b.record(st)
        b.synchronize()
        return fl, a.elapsed_time(b)

    iters = 16
    while True:
        fl, ms = once(iters)
        if ms > 50.0:
            break
        iters *= 4
    iters = max(1, int(iters * seconds * 1e3 / ms))
    rates = []
    for _ in range(repeats):
        fl, ms = once(iters)
        rates.append(fl / (ms / 1e3) / 1e12)
    return max(rates), statistics.median(rates), sms


def face_counts(n):
    out = []
    for d in range(3):
        t1, t2 = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
        out.append({"eq": (n[d] + 1) * (n[t1] + 4) * (n[t2] + 4), "flux": (n[d] + 1) * n[t1] * n[t2]})
    return out


def adjoint_workload(n=(256, 128, 128)):
    """Rotor as the ALM workload on a 256x128x128 grid, FP64, fixed dt equal
    to the CFL-0.5 step of the initial uniform stream."""
    w = WL.alm_rotor(n=n)
    h = min((w.faces[a][-1] - w.faces[a][0]) / w.n[a] for a in range(3))
    w.dt_fixed = 0.5 * h / (1.0 + 1.0 / w.mach)
    w.cfl = 0.9
    return w


def time_adjoint(args, dev):
    """Forward and checkpointed adjoint of the wake-deficit plus power
    objective; ratio = backward time (segment recomputation included) over
    the forward time of the same steps. Main figure, on the adjoint
    configuration (256x128x128 rotor, 200 steps, checkpoint every 20):
    recorded steps (each segment run forward once with its step tapes, then
    reversed from them) with FP32 arithmetic in the local reverse maps (the
    FD-checked default of this benchmark). Beside it, on a shorter run (20
    steps, checkpoint every 10): per-step recomputation, and recorded steps
    with FP64 reverse arithmetic."""
    import torch

    from paper_2603_11102_gb300 import adjoint, gks
    w = adjoint_workload()
    g = gks.Grid.from_workload(w, precision="fp64", device=dev)
    iplane = int(round((5.0 - w.faces[0][0]) / (w.faces[0][1] - w.faces[0][0])))
    npts = w.rotors[0].n_blades * len(w.rotors[0].r)

    def run(steps, K, tape, grid=None):
        s = torch.ones(npts, dtype=torch.float64, requires_grad=True)
        u = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        J = adjoint.rotor_objective(grid or g, s, u, steps, K=K, iplane=iplane, beta=1.0, tape=tape)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        J.backward()
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1, float(u.grad)

    out, tape_gb = {}, {}
    Kv, Nv = 10, args.adjoint_variant_steps
    for rev, tape, N, K in (("fp32", "on", args.adjoint_steps, args.adjoint_k), ("fp32", "off", Nv, Kv),
                            ("fp64", "on", Nv, Kv)):
        if N <= 0:
            continue
        g.set_adjoint_precision(rev)
        tape_gb[rev] = g.adjoint_tape_bytes() / 1e9
        try:
            run(K, K, tape)   # untimed warm-up segment (first launches, the buffers)
            out[rev, tape] = run(N, K, tape)
        except torch.cuda.OutOfMemoryError:
            # K tapes do not fit next to what else holds device memory: the
            # per-step recomputation, reported as such
            torch.cuda.empty_cache()
            run(K, K, "off")
            out[rev, tape] = run(N, K, "off")
            tape_gb[rev] = 0.0
        torch.cuda.empty_cache()
    g.close()
    # the FP32C steps and their recorded reverse (FP32 arithmetic) on the same
    # configuration
    if args.adjoint_steps > 0:
        g32 = gks.Grid.from_workload(w, precision="fp32c", device=dev)
        run(args.adjoint_k, args.adjoint_k, "on", g32)
        out["fp32c"] = run(args.adjoint_steps, args.adjoint_k, "on", g32)
        tape_gb["fp32c"] = g32.adjoint_tape_bytes() / 1e9
        g32.close()
        torch.cuda.empty_cache()
    fwd, bwd, gu = out["fp32", "on"]
    res = {"workload": w.name + "-fp64", "steps": args.adjoint_steps, "checkpoint_every": args.adjoint_k,
           "warmup": "one untimed segment, forward and backward",
           "reverse_arithmetic": "fp32 (FP64 forward, state adjoints and sums; Gauss-point tape in FP32)",
           "recorded_steps": ("%d tapes of %.1f GB" % (args.adjoint_k, tape_gb["fp32"]) if tape_gb["fp32"] > 0
                              else "none: out of device memory, per-step recomputation"),
           "forward_s": fwd, "backward_s": bwd, "ratio": bwd / fwd,
           "forward_ms_per_step": 1e3 * fwd / args.adjoint_steps,
           "objective": "plane-mean deficit at x = 5D + rotor power; gradient w.r.t. %d force scales and U_inf"
                        % npts, "grad_uinf": gu}
    if "fp32c" in out:
        f4, b4, g4 = out["fp32c"]
        res["fp32c"] = {"forward_s": f4, "backward_s": b4, "ratio": b4 / f4,
                        "forward_ms_per_step": 1e3 * f4 / args.adjoint_steps,
                        "recorded_steps": "%d tapes of %.1f GB" % (args.adjoint_k, tape_gb["fp32c"]),
                        "grad_uinf": g4, "grad_uinf_rel_diff_vs_fp64": abs(g4 - gu) / abs(gu)}
    if ("fp32", "off") in out:
        f2, b2, g2 = out["fp32", "off"]
        f3, b3, g3 = out["fp64", "on"]
        res["variants"] = {"steps": Nv, "checkpoint_every": Kv,
                           "ratio_recompute_per_step": b2 / f2, "grad_uinf_recompute_per_step": g2,
                           "ratio_fp64_reverse": b3 / f3, "grad_uinf_fp64_reverse": g3,
                           "fp64_tape_gb": tape_gb["fp64"]}
    return res


def time_small_graphs(dev, steps=500):
    """A launch-bound case: the 32^3 Taylor-Green vortex in FP32C, plain
    steps against steps replayed from a CUDA graph (gks_set_graphs)."""
    import torch

    from paper_2603_11102_gb300 import gks
    w = WL.taylor_green_3d(32)
    out = {"workload": "taylor-green-32^3", "precision": "fp32-compensated", "steps": steps}
    for key, on in (("plain_mlups", False), ("graph_mlups", True)):
        g = gks.Grid.from_workload(w, precision="fp32c", device=dev)
        g.set_graphs(on)
        g.step(5)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(g.stream)
        g.step(steps, sync=False)
        b.record(g.stream)
        g.sync()
        out[key] = w.cells * steps / (a.elapsed_time(b) / 1e3) / 1e6
        g.close()
    return out


def run_ours(args, world, rank, local):
    import torch

    from paper_2603_11102_gb300 import build, gks
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = make_workload(args.workload)
    peaks, peak_kind = load_peaks()
    g = gks.Grid.from_workload(w, precision=args.precision, device=dev)
    if args.precision == "fp64" and args.fp64_arithmetic == "ds":
        g.set_fp64_arithmetic("ds")
    for _ in range(args.warmup):
        g.step(1)
    stream = g.stream
    sampler = ClockSampler(local) if rank == 0 else None
    g.profile_enable(timing=True)
    barrier(world)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    prof = g.profile_read()
    ms = max_over_ranks(ms, world, dev)
    cells = w.cells
    value = world * cells * args.steps / (ms / 1e3) / 1e6
    ms_step = ms / args.steps

    # roofline of the dominant kernel group (FP32 or FP64 ALU bound); the
    # x/y face-flux kernel, the z-face kernel fused with the stage update and
    # the face-state kernel are each reported against the same ALU peak: the
    # FMA-loop probe's median rate on this GPU (after the timed region), the
    # operations of each launch from the measured per-face counts
    kms = prof["ms"]
    fc = face_counts(w.n)
    fp64_run = args.precision == "fp64"
    probe = {}
    if not args.no_alu_probe:
        for name, kind in (("fp32", 0), ("fp32x2", 2), ("fp64", 1)):
            best, med, sms = measure_alu_peak(dev, kind)
            probe[name] = {"best_tflops": best, "median_tflops": med}
        probe["sms"] = sms
        probe["method"] = ("library FMA loop (gks_alu_peak_probe): 4 blocks of 256 threads per SM, 8 independent "
                           "chains per thread (fp32x2: 4 chains of packed pairs, FFMA2), 3 launches of ~1 s timed "
                           "with CUDA events")
    clock_mhz = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if probe:
        if fp64_run:
            alu_peak = probe["fp64"]["median_tflops"]
            peak_source = "measured: median of the FP64 FMA-loop probe on this GPU"
        else:
            # the stencil kernels issue scalar and packed FP32 operations on the
            # same FMA pipes: the larger of the two probes' medians
            alu_peak = max(probe["fp32"]["median_tflops"], probe["fp32x2"]["median_tflops"])
            peak_source = "measured: the larger median of the FP32 and packed-FP32 FMA-loop probes on this GPU"
    elif not fp64_run:
        alu_peak = sms * 128 * 2 * clock_mhz * 1e6 / 1e12
        peak_source = "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz" % (sms, clock_mhz)
    else:
        alu_peak, peak_source = 1.25, "nominal GB300 FP64 1.25 TFLOP/s"
    FL, fl_src = read_flops(args.precision)
    group_flops = {
        "face_flux": args.steps * sum(fc[d]["flux"] * (FL["face_flux_stage1"] + FL["face_flux_stage2"])
                                      for d in (0, 1)),
        "flux_update": args.steps * fc[2]["flux"] * (FL["flux_update_stage1"] + FL["flux_update_stage2"]),
        "face_eq": args.steps * 2 * sum(fc[d]["eq"] * FL["face_eq"] for d in range(3)),
    }
    alu = {}
    for k, fl in group_flops.items():
        if kms.get(k, 0.0) > 0:
            a = fl / (kms[k] / 1e3) / 1e12
            alu[k] = {"achieved": round(a, 3), "frac": round(a / alu_peak, 4),
                      "avg_launch_ms": round(kms[k] / max(1, prof["launches"][k]), 4),
                      "flops_source": fl_src.get(k)}
    top = max(kms, key=kms.get)
    flops = group_flops.get(top)
    achieved = flops / (kms[top] / 1e3) / 1e12 if flops else None
    traffic = read_traffic(top, args.precision)
    roofline = {"bound": "alu", "kernel": top, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": (achieved / alu_peak) if achieved else None, "traffic": traffic,
                "peak_source": peak_source, "flops_source": fl_src.get(top),
                "launches": prof["launches"][top], "avg_launch_ms": kms[top] / max(1, prof["launches"][top]),
                "groups": alu, "alu_probe": probe or None}
    hbm_ach = cells * BYTES_PER_CELL_STEP[args.precision] * args.steps / (ms / 1e3) / 1e9
    hbm = {"achieved": hbm_ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": hbm_ach / peaks["hbm_gbs"], "bytes_per_cell_step": BYTES_PER_CELL_STEP[args.precision],
           "peak_source": peak_kind}
    share = {k: round(v / sum(kms.values()), 4) for k, v in kms.items() if v > 0}

    # end to end through the C ABI with host buffers: per step, upload the
    # state from page-locked memory, step, read the rotor loads back
    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI with host buffers: every step uploads
        # its whole input state from page-locked memory and reads its rotor
        # loads back (thrust and torque per blade, power, C_P, C_T). Steps
        # are independent (each starts from its uploaded state), so the
        # upload of step k+1 runs on a copy stream into the other of two
        # device staging buffers while step k computes; the grid stream waits
        # for the upload, scatters it into the state and steps; the loads
        # come back by an asynchronous copy into one of two page-locked
        # records, read on the host one step later, so that no step waits
        # for the host.
        host = torch.from_numpy(np.ascontiguousarray(w.state0.reshape(-1))).pin_memory()
        ke = max(1, min(args.steps, args.e2e_steps))
        stage = [torch.empty(host.numel(), dtype=torch.float64, device=dev) for _ in range(2)]
        cs = torch.cuda.Stream(dev)
        up = [torch.cuda.Event() for _ in range(2)]
        used = [torch.cuda.Event() for _ in range(2)]
        rid = next((i for i, o in enumerate(g.objects) if o[0] == "rotor"), None)
        recs = [g.forces_record(rid) for _ in range(2)] if rid is not None else None
        done = [torch.cuda.Event() for _ in range(2)]
        power = []
        # the user's step: no per-launch events, one graph launch per step
        # (captured here, before the timed region)
        g.profile_enable(timing=False)
        g.set_graphs(True)
        g.step(2)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(cs):
            stage[0].copy_(host, non_blocking=True)
            up[0].record(cs)
        for k in range(ke):
            b = k & 1
            if k + 1 < ke:
                with torch.cuda.stream(cs):
                    if k >= 1:
                        cs.wait_event(used[b ^ 1])
                    stage[b ^ 1].copy_(host, non_blocking=True)
                    up[b ^ 1].record(cs)
            stream.wait_event(up[b])
            g.set_state_tensor(stage[b], sync=False)
            used[b].record(stream)
            g.step(1, sync=False)
            if recs is not None:
                if k >= 2:
                    done[b].synchronize()          # step k-2's record, long done
                    power.append(float(recs[b][-3]))
                g.forces_async(rid, recs[b])
                done[b].record(stream)
        g.sync()   # also reports any error the steps flagged on the device
        te = time.perf_counter() - t0
        if recs is not None:
            for k in range(max(0, ke - 2), ke):
                power.append(float(recs[k & 1][-3]))
        te = max_over_ranks(te, world, dev)
        out_bytes = int(recs[0].numel() * 8) if recs is not None else 0
        e2e = {"value": world * cells * ke / te / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": int(host.numel() * 8),
               "d2h_bytes_per_step": out_bytes, "steps": ke,
               "overlap": "upload of step k+1 on a copy stream during step k (two device staging buffers); "
                          "the loads of step k read back asynchronously and consumed on the host at step k+2; "
                          "steps replayed from a CUDA graph",
               "power_read": len(power)}
        del stage

    # the global reductions (mass, momentum, kinetic energy; FP64 sums in a
    # fixed order), taken on demand and read on the host: the device time of
    # their two kernels per call over the whole grid (CUDA events of the
    # library's profiler on the grid's stream), which read the state once
    # (32 B per cell), and the host time of the whole call with its read-back
    reductions = None
    try:
        g.profile_enable(timing=True)
        g.diagnostics()
        torch.cuda.synchronize(dev)
        g.profile_enable(timing=True)
        nd = 20
        t0 = time.perf_counter()
        for _ in range(nd):
            g.diagnostics()
        tr = (time.perf_counter() - t0) / nd
        pr = g.profile_read()
        kd = pr["ms"]["misc"] / max(1, pr["launches"]["misc"])
        reductions = {"device_ms_per_call": kd, "calls": nd, "state_gb": cells * 32 / 1e9,
                      "gbs": cells * 32 / (kd / 1e3) / 1e9, "host_ms_per_call": tr * 1e3,
                      "timing": "device: CUDA events around the two reduction kernels on the grid's stream; "
                                "host: clock around the call (includes its read-back and synchronisation)"}
    except Exception as exc:   # reported, not fatal: the step figures above stand
        reductions = {"error": str(exc)[:200]}
    g.close()
    del g
    torch.cuda.empty_cache()

    # optional: the same workload as a slab group (gks_slab_step: x-slabs on
    # this GPU with the halo exchange of every stage), cuts evenly spaced and
    # moved off the forcing supports
    slab_group = None
    if args.slabs > 1:
        nx = w.n[0]
        fx = np.asarray(w.faces[0])
        dx = fx[1] - fx[0]
        forced = [int((r.hub[0] - fx[0]) / dx) for r in w.rotors] + \
                 [int((np.mean(np.asarray(b.xyz).reshape(-1, 3)[:, 0]) - fx[0]) / dx) for b in w.bodies]
        cuts = []
        for k in range(1, args.slabs):
            c = k * nx // args.slabs
            while any(abs(c - f) < 24 for f in forced):
                c += 8
            cuts.append(c)
        sg = gks.SlabGroup(w, cuts, precision=args.precision, device=dev)
        sg.step(2)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(sg.slabs[0].stream)
        sg.step(args.steps)
        b.record(sg.slabs[0].stream)
        torch.cuda.synchronize(dev)
        mss = max_over_ranks(a.elapsed_time(b), world, dev) / args.steps
        slab_group = {"slabs": args.slabs, "cuts": cuts, "value": world * cells / (mss / 1e3) / 1e6, "unit": "MLUPS",
                      "ms_per_step": mss, "steps": args.steps,
                      "note": "one GPU: the slabs' kernels run one after another on one stream; the halo copies "
                              "and the per-slab launches are the overhead against the single grid"}
        sg.close()
        del sg
        torch.cuda.empty_cache()

    fp64 = None
    if args.precision == "fp32c" and not args.no_fp64:
        g64 = gks.Grid.from_workload(w, precision="fp64", device=dev)
        g64.step(1)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(g64.stream)
        g64.step(args.fp64_steps)
        b.record(g64.stream)
        torch.cuda.synchronize(dev)
        ms64 = max_over_ranks(a.elapsed_time(b), world, dev)
        fp64 = {"value": world * cells * args.fp64_steps / (ms64 / 1e3) / 1e6, "unit": "MLUPS",
                "steps": args.fp64_steps, "ms_per_step": ms64 / args.fp64_steps, "arithmetic": "fp64"}
        # the same FP64 grid with double-single reconstruction and flux
        # (gks_set_fp64_arithmetic): FP64 state, face buffers, update and sums
        g64.set_fp64_arithmetic("ds")
        g64.step(1)
        torch.cuda.synchronize(dev)
        a.record(g64.stream)
        g64.step(args.fp64_steps)
        b.record(g64.stream)
        torch.cuda.synchronize(dev)
        msds = max_over_ranks(a.elapsed_time(b), world, dev)
        fp64["double_single"] = {"value": world * cells * args.fp64_steps / (msds / 1e3) / 1e6, "unit": "MLUPS",
                                 "steps": args.fp64_steps, "ms_per_step": msds / args.fp64_steps,
                                 "arithmetic": "double-single reconstruction and flux, FP64 state and sums"}
        g64.close()

    graphs = time_small_graphs(dev) if rank == 0 and not args.no_graphs else None

    adj = None
    if args.adjoint_steps > 0 and rank == 0:
        adj = time_adjoint(args, dev)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        mlups, secs, cores, desc = time_oracle(w, args.cpu_steps, 0)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": secs}
        # the same window on one host thread (fewer steps: ~1/cores of the rate)
        oracle.set_threads(1)
        m1, s1, _, _ = time_oracle(w, args.cpu_steps_one_thread, 0)
        oracle.set_threads(cores)
        cpu["one_thread"] = {"value": m1, "unit": "MLUPS", "cores": 1, "steps": args.cpu_steps_one_thread,
                             "seconds": s1}

    line = {"metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32c" else "f64", "data": "synthetic",
            "config": {"workload": w.name, "cells": cells,
                       "precision": "fp32-compensated" if args.precision == "fp32c" else "fp64",
                       "rotor_points": sum(r.n_blades * len(r.r) for r in w.rotors),
                       "ib_points": sum(len(b.dS) for b in w.bodies),
                       "l2": "inputs larger than L2 (state %.0f MB per replica)" % (
                           cells * (32 if args.precision == "fp32c" else 32) / 1e6),
                       "parallelism": "replicas x%d" % world},
            "roofline": roofline, "hbm_step": hbm, "kernel_share": share, "cpu_baseline": cpu,
            "clocks": clocks, "e2e": e2e, "gpu_launches": prof["total_launches"], "fp64": fp64,
            "small_grid_graphs": graphs, "adjoint": adj, "reductions": reductions}
    if slab_group is not None:
        line["slab_group"] = slab_group
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args, world, rank):
    """The CPU oracle as it stands, on a bounded window of the workload; each
    timed step is one oracle step of the window."""
    if rank != 0:
        return
    w = make_workload(args.workload)
    mlups, secs, cores, desc = time_oracle(w, args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": mlups,
            "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "cells": w.cells, "precision": "fp64 (oracle)",
                       "rotor_points": sum(r.n_blades * len(r.r) for r in w.rotors),
                       "ib_points": sum(len(b.dS) for b in w.bodies), "parallelism": "host cores"},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="alm-ibm", choices=["alm-ibm", "alm", "channel", "tgv", "tgv96", "tgv192"])
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--fp64-arithmetic", default="fp64", choices=["fp64", "ds"],
                    help="with --precision fp64: FP64 or double-single reconstruction and flux")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--no-graphs", action="store_true", help="skip the small-grid CUDA graph timing")
    ap.add_argument("--cpu-steps", type=int, default=20)
    ap.add_argument("--cpu-steps-one-thread", type=int, default=2)
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--adjoint-k", type=int, default=20)
    ap.add_argument("--adjoint-variant-steps", type=int, default=20)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-alu-probe", action="store_true", help="skip the FMA-loop peak measurement")
    ap.add_argument("--slabs", type=int, default=0,
                    help="also time the workload as a group of this many x-slabs on this GPU (gks_slab_step)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
