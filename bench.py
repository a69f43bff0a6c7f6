#!/usr/bin/env python3
"""Benchmark of the PNCG solver on the 98,304-tet twisted bar (16x16x64 Kuhn-split cells, 0.1 x 0.1 x 0.4 m,
Neo-Hookean E = 1e5 Pa, nu = 0.45, both end caps turned in opposite directions at 2 rad/s, dt = 1/30 s,
dhat = 5e-4 m, kappa = 1e4, 50 NCG iterations per time step).

One benchmark step is one time step: prediction, candidate passes, 50 PNCG iterations (gradient + Jacobi
diagonal, beta reductions, direction, p^T H p, step, update), velocity update.  The headline value is NCG
iterations per second of the FP32-mixed form (whole job: summed over all ranks), with the plain FP64 form timed
beside it.  Inputs (the kinematic targets of every step) are resident on the device before the timed region; L2
is flushed (a 256 MiB write) between timed steps and the flush is not timed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 (torchrun, one process per GPU) every rank runs its own independent replica of the problem.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NCG iters/s and ms per time step at 98k tets; % HBM peak; vs FP64 plain"
UNIT = "iter/s"
WORKLOAD = ("twisted bar: 16x16x64 Kuhn grid (98,304 tets, 18,785 verts), 0.1x0.1x0.4 m, Neo-Hookean E=1e5 "
            "nu=0.45 rho=1000, caps +-2 rad/s, dt=1/30 s, dhat=5e-4 m, kappa=1e4, 50 NCG iterations per step")


def rank_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float) -> float:
    """The largest of every rank's value (the whole job's time is its slowest rank's); the value itself without a
    process group.  NCCL reduces a device tensor, gloo a host one."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws: int, K: int, iters: int, total_ms: float) -> float:
    """Whole-job NCG iterations per second: each of the ws ranks advances its own replica by K time steps of
    `iters` iterations, and the job takes total_ms (the slowest rank's time)."""
    return ws * K * iters / (total_ms / 1e3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while GPU work runs (200 ms period)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def method_bytes(prec: int, n_tets: int, n_verts: int, n_active: int, per_tet_youngs: bool = False) -> int:
    """Algorithmic bytes of one NCG iteration of the method (not of this implementation): every array of the
    iteration crossing DRAM once per pass.  Per tet, the two element passes (gradient + Jacobi diagonal, p^T H p)
    each read the 4 indices, D_m^-1 and the rest volume: 2 (16 + 10 r) B with r the element size, i.e. 112 B in FP32
    and 192 B in FP64, plus 2 r B for a per-tet Young's modulus.  Per vertex 196 B in FP32 and 392 B in FP64: the
    gradient pass (x, x~, m read; g, diag written), the beta pass (g, diag, g_old, p_old), the direction pass, the p
    gather and the x update.  Per active pair 34 B (the pair's index list written and read, and its type)."""
    r = 4 if prec == 1 else 8
    per_tet = 2 * (16 + 10 * r) + (2 * r if per_tet_youngs else 0)
    per_vert = 196 if prec == 1 else 392
    return n_tets * per_tet + n_verts * per_vert + 34 * n_active


def algorithmic_bytes(kernel: str, prec: int, sizes: dict, n_cand: int, n_active: int, persistent: bool = False):
    """Bytes a phase of this implementation moves at least once (every array read or written counted once): the
    implementation's own count, reported beside the method's (method_bytes).

    Vertex state: x (double4, 32 B) and, in the FP32 form, its float-float copy (2 x float4); accumulators g, diag
    and the directions are 4-vectors of the element type (16 B float, 32 B double).  Per tet: 4 indices (16 B),
    D_m^-1 (9 values), h^2 V (1 value) and, in the FP32 form, the float-float rest metric (12 floats).  Candidates:
    int4 (16 B); active pairs (64 B float form, 112 B double form) written by the gradient pass and read by p^T H p.
    The persistent step stores P g in the beta pass and forms the direction inside the p^T H p pass.  The FP32
    form's per-tet p^T H p record (64 B written by the gradient pass, read by the p^T H p pass) is an
    implementation choice for accuracy, not a quantity of the method, and is not counted."""
    T, V = sizes["n_tets"], sizes["n_verts"]
    r = 4 if prec == 1 else 8
    v4 = 4 * r
    tet = 16 + 10 * r
    act = 64 if prec == 1 else 112
    xpos = 32                                # gathered positions per vertex (ff pair, or double4)
    if kernel == "k_grad":
        return T * (tet + (48 if prec == 1 else 0)) + V * (xpos + 4 * v4) + n_cand * 16 + n_active * act
    if kernel == "k_dots":
        return V * (5 if persistent else 4) * v4
    if kernel == "k_dir":
        return V * 4 * v4
    if kernel == "k_pHp":
        return T * tet + V * (xpos + (5 if persistent else 1) * v4) + n_active * act
    if kernel == "k_update":
        disp = 32 if prec == 1 else 32      # FP32: float copy now + at the build; FP64: x at the build
        return V * (64 + 32 + (4 if persistent else 3) * v4 + (32 if prec == 1 else 0) + disp)
    return None


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2405_08001_gb300", "csrc", "*"))):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, prec_name: str, phases: bool = False, scene: str = "twisted_bar"):
    """DRAM bytes per launch from the committed ncu summary of that kernel and workload, if it was taken on the
    current kernel sources (the summary's dram_bytes_per_launch line, scaled to a full launch where it says so)."""
    form = "_phases" if phases else ""
    path = os.path.join(ROOT, "profiles", f"{kernel}{form}_{scene}_{prec_name}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for ln in f:
            if ln.startswith("- ") and ":" in ln:
                k, v = ln[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


SHAPES = {(256, 2): 0, (512, 1): 1, (256, 3): 2, (256, 1): 3, (384, 1): 4}   # sim_options.block_shape of (threads, blocks/SM)


def shape_of(st):
    """The block shape a handle runs (its stats), as sim_options.block_shape and as a report."""
    key = (st["block_threads"], st["blocks_per_sm"])
    return SHAPES.get(key, 0), {"threads_per_block": key[0], "blocks_per_sm": key[1],
                                "launch": "persistent" if st["launch_form"] == 1 else "one kernel per phase"}


def window(W, K, cfg_steps):
    """First step of the timed window: the window ends with the configured run's last step (where the twisted
    bar carries the most contact candidates), after at least W untimed warm-up steps."""
    return max(W, cfg_steps - K)


def time_steps(B, torch, sim, targets, first, K, flush, cfg_steps):
    """Times K time steps one by one with CUDA events on the solver's stream; returns per-step milliseconds.  The
    steps are first .. cfg_steps - 1; a longer K starts over at `first` from the state saved there (the restore is
    not timed), so every timed step is a step of the configured run."""
    stream = torch.cuda.current_stream()
    span = max(1, cfg_steps - first)
    saved = None
    if K > span:
        torch.cuda.synchronize()
        x0, v0, _ = B.sim_get_state(sim.h)
        saved = (x0, v0)
    times = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for s in range(K):
        if s > 0 and s % span == 0:
            B.sim_set_state(sim.h, *saved)
        flush.zero_()
        ev[s][0].record(stream)
        B.sim_step_async(sim.h, 1, targets[first + s % span])
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    for a, b in ev:
        times.append(a.elapsed_time(b))
    return times


def timed_window(B, torch, sim, stream, flush, first, K, targets=None):
    """K steps from the current state (step `first`), each bracketed by CUDA events on the solver's stream, L2
    flushed before each (not timed).  Returns per-step milliseconds."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    keep = []
    for s in range(K):
        flush.zero_()
        ev[s][0].record(stream)
        keep.append(B.sim_step_async(sim.h, 1, None if targets is None else targets[first + s]))
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def side_workload(B, torch, S, stream, flush, sc, name, desc, unit_scale, unit, K, peak, peak_kind, phases,
                  per_tet_youngs):
    """One of the workloads whose working set exceeds L2 (the large pile, the batch): the run's lead-in untimed, then
    the K last steps of its configured run timed, then one profiled step; the HBM roofline from the method's bytes."""
    sim = B.Sim(sc, precision=B.SIM_FP32_MIXED, cuda_stream=stream.cuda_stream, persistent=0 if phases else 1,
                block_shape=-1)
    first = max(12, sc.steps - K)
    try:
        for s in range(first):
            B.sim_step_async(sim.h, 1, None)
        torch.cuda.synchronize()
        B.sim_get_state(sim.h, want_x=False, want_v=False)
        times = timed_window(B, torch, sim, stream, flush, first, K)
        _, _, st = B.sim_get_state(sim.h, want_x=False, want_v=False)
        prof = B.sim_profile_step(sim.h, None)
    except B.SimError as e:
        sim.close()
        return {"workload": desc, "error": str(e)}
    sizes = sim.sizes()
    sim.close()
    ms = sum(times) / K
    mb = st["iters_done"] * method_bytes(1, sizes["n_tets"], sizes["n_verts"], st["n_active"], per_tet_youngs)
    ib = sum(algorithmic_bytes(k, 1, sizes, st["n_candidates"], st["n_active"], persistent=not phases) * prof[k][1]
             for k in ("k_grad", "k_pHp", "k_dots", "k_dir", "k_update") if prof.get(k, (0, 0))[1] > 0)
    ach = mb / (ms * 1e-3) / 1e9
    return {"workload": desc, "value": round(unit_scale * sc.iters / (ms * 1e-3), 2), "unit": unit,
            "ms_per_step": round(ms, 4), "time_steps_per_s": round(1e3 / ms, 2), "steps": K,
            "timed_steps": f"{first}..{first + K - 1} of the {sc.steps}-step run (its last steps), "
                           f"steps 0..{first - 1} untimed",
            "roofline": {"bound": "hbm", "kernel": "k_persistent" if not phases else "all iteration kernels",
                         "achieved": round(ach, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": round(ach / peak, 4), "traffic": recorded_traffic("k_persistent", "fp32", scene=name),
                         "algorithmic_bytes_per_launch": int(mb), "implementation_bytes_per_launch": int(ib),
                         "bytes_basis": "method bytes per iteration x iterations per step (candidate builds not "
                                        "counted)"},
            "phases_us_per_iteration": {k: round(1e3 * v[0] / v[1], 2) for k, v in prof.items()
                                        if v[1] > 0 and k.startswith("k_")},
            "block_shape": shape_of(st)[1],
            "stats_last_step": {k: st[k] for k in ("n_candidates", "n_active", "n_rebuilds", "n_capped")}}


def equal_accuracy(B, torch, sc, stream, state, targets, ks, kref, name, shapes, repeat=3):
    """FP32-mixed against plain FP64 at equal final-energy accuracy on one time step (the fair comparison of the two
    precision forms: equal iteration counts would credit the FP32 form with steps that reach less).

    From a saved state the step is taken once per form with max(ks) iterations through the persistent kernel, one
    iteration batch at a time (sim_iterate), and the energy after K iterations is read for every K in `ks`; the
    converged reference x* is the FP64 form after `kref` iterations.  Energies are evaluated by the library's FP64
    energy pass (sim_eval_energy on an FP64 handle per scene; the parity tests match it to the oracle's energy):
    err(K) = (E(x_K) - E(x*)) / (E(x_0) - E(x*)), x_0 the step's start (kinematic targets applied); with several
    scenes (a batch) err is taken per scene and the median over scenes is used.  The target is the plain FP64 form's
    error at the headline iteration count ks[1]; each form's iteration count to reach it is interpolated linearly
    in K between the bracketing points of its curve, and its cost is the step time interpolated the same way (each
    (form, K) timed `repeat` times from the saved state, the fastest kept)."""
    import numpy as np
    x0, v0 = state
    fixed = sc.fixed.astype(bool) if sc.fixed is not None else None
    ranges = sc.scene_ranges()
    evals = []

    def energies(x, xt):
        if not evals:
            evals.extend(B.Sim(sc.subscene(i) if len(ranges) > 1 else sc, precision=B.SIM_FP64,
                               cuda_stream=stream.cuda_stream) for i in range(len(ranges)))
        return np.array([B.sim_eval_energy(e.h, x[v0_:v1_], xt[v0_:v1_])[0]
                         for e, (v0_, v1_, _, _) in zip(evals, ranges)])

    def sim_of(prec, K):   # in the block shape each form's autotuner chose on the benchmark's run
        return B.Sim(sc, precision=prec, cuda_stream=stream.cuda_stream, iters=K, persistent=1,
                     block_shape=shapes[prec])

    def timed(prec, K):
        sim = sim_of(prec, K)
        ms = []
        try:
            for r in range(repeat):
                B.sim_set_state(sim.h, x0, v0)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                keep = B.sim_step_async(sim.h, 1, targets)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            B.sim_get_state(sim.h, want_x=False, want_v=False)
        finally:
            sim.close()
        return min(ms)

    def curve(prec, Ks):
        sim = sim_of(prec, max(Ks))
        out = []
        try:
            B.sim_set_state(sim.h, x0, v0)
            B.sim_begin_step(sim.h, targets)
            done = 0
            for K in Ks:
                B.sim_iterate(sim.h, K - done)
                done = K
                x, _, _, _, xt, _ = B.sim_get_iterate(sim.h)
                out.append((x, xt))
        finally:
            sim.close()
        return out

    try:
        return _equal_accuracy_rows(B, x0, fixed, targets, ks, kref, name, ranges, energies, curve, timed)
    finally:
        for e in evals:
            e.close()


def _equal_accuracy_rows(B, x0, fixed, targets, ks, kref, name, ranges, energies, curve, timed):
    """The error curves, the target and the interpolated costs of equal_accuracy (its handles closed by the caller)."""
    import numpy as np
    (xr, xt), = curve(B.SIM_FP64, (kref,))
    Eref = energies(xr, xt)
    xs = x0.copy()
    if fixed is not None and targets is not None:
        xs[fixed] = targets
    E0 = energies(xs, xt)
    res = {}
    for prec, pname in ((B.SIM_FP64, "fp64"), (B.SIM_FP32_MIXED, "fp32_mixed")):
        rows = []
        for K, (x, xt2) in zip(ks, curve(prec, ks)):
            err = (energies(x, xt2) - Eref) / np.where(E0 - Eref != 0.0, E0 - Eref, 1.0)
            rows.append({"iters": K, "ms": round(timed(prec, K), 4), "energy_err": float(np.median(err))})
        res[pname] = rows
    target = res["fp64"][1]["energy_err"]

    def cost(rows):
        """(iterations, ms) where the error curve first reaches the target, interpolated linearly in K."""
        prev = None
        for r in rows:
            if r["energy_err"] <= target * (1 + 1e-9):
                if prev is None or prev["energy_err"] == r["energy_err"]:
                    return float(r["iters"]), r["ms"]
                f = (prev["energy_err"] - target) / (prev["energy_err"] - r["energy_err"])
                return (prev["iters"] + f * (r["iters"] - prev["iters"]), prev["ms"] + f * (r["ms"] - prev["ms"]))
            prev = r
        return None
    c64, c32 = cost(res["fp64"]), cost(res["fp32_mixed"])
    return {"workload": name, "reference": f"FP64, {kref} iterations (x*); energies by the library's FP64 energy pass",
            "error": "(E(x_K) - E(x*)) / (E(x_0) - E(x*)) after K iterations of one trajectory per form"
                     + ("; median over the scenes" if len(ranges) > 1 else ""),
            "target_err": target, "fp64": res["fp64"], "fp32_mixed": res["fp32_mixed"],
            "fp64_iters_at_target": round(c64[0], 2) if c64 else None,
            "fp32_iters_at_target": round(c32[0], 2) if c32 else None,
            "fp64_ms_at_target": round(c64[1], 4) if c64 else None, "fp32_ms_at_target": round(c32[1], 4) if c32 else None,
            "speedup_fp32_over_fp64": round(c64[1] / c32[1], 3) if (c64 and c32) else None}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = rank_info()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2405_08001_gb300 import binding as B, build, scenes as S
    build.build()
    B.load()
    sc = S.twisted_bar()
    iters = sc.iters
    W, K = args.warmup, args.steps
    cfg_steps = sc.steps
    first = window(W, K, cfg_steps)
    n_total = max(first + K, cfg_steps) + 4
    # a dedicated stream: the solver, the events and the L2 flush all run on it (the legacy default stream could
    # not be captured into the solver's CUDA graph)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    torch.cuda.set_stream(stream)
    targets = torch.tensor(sc.all_targets(n_total), dtype=torch.float64, device="cuda").contiguous()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sampler = ClockSampler(local)
    sampler.start()
    peak, peak_kind = measured_peaks()

    def one_form(prec, K_, form=1):
        sim = B.Sim(sc, precision=prec, cuda_stream=stream.cuda_stream, persistent=0 if args.phases else form,
                    block_shape=-1)
        first_ = window(max(W, 12), K_, cfg_steps)   # the autotuner's steps (two per candidate) come first
        for s in range(first_):
            B.sim_step_async(sim.h, 1, targets[s])
        torch.cuda.synchronize()
        B.sim_get_state(sim.h, want_x=False, want_v=False)     # raises on a kernel error
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        times = time_steps(B, torch, sim, targets, first_, K_, flush, cfg_steps)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        _, _, st = B.sim_get_state(sim.h, want_x=False, want_v=False)
        return sim, times, st

    sim32, t32, st32 = one_form(B.SIM_FP32_MIXED, K)
    shape32, shape32_rep = shape_of(st32)
    total_ms = max_over_ranks(sum(t32))
    value = job_value(ws, K, iters, total_ms)

    # kernel-by-kernel GPU times of three more steps (after the timed region); they continue the run from the state
    # the timed window left
    after = first + (K - 1) % max(1, cfg_steps - first) + 1
    prof = {}
    for s in range(3):
        for k, (ms, n) in B.sim_profile_step(sim32.h, targets[after + s]).items():
            a, b = prof.get(k, (0.0, 0))
            prof[k] = (a + ms, b + n)
    _, _, stp = B.sim_get_state(sim32.h, want_x=False, want_v=False)
    sizes = sim32.sizes()
    dom = max((k for k in prof if prof[k][1] > 0), key=lambda k: prof[k][0])
    step_ms = sum(v[0] for v in prof.values()) / 3
    iter_kernels = ("k_grad", "k_pHp", "k_dots", "k_dir", "k_update")
    phase_bw = {}
    for k in iter_kernels:
        if prof.get(k, (0, 0))[1] > 0:
            b = algorithmic_bytes(k, 1, sizes, stp["n_candidates"], stp["n_active"], persistent=not args.phases)
            phase_bw[k] = round(b / (prof[k][0] / prof[k][1] * 1e-3) / 1e9, 1)
    n_act = st32["n_active"]
    if args.phases:
        # the dominant iteration kernel; its method bytes are the iteration's share that kernel moves
        dom_all = dom
        dom = max((k for k in iter_kernels if prof.get(k, (0, 0))[1] > 0), key=lambda k: prof[k][0])
        per_launch_ms = prof[dom][0] / prof[dom][1]
        ibytes = algorithmic_bytes(dom, 1, sizes, stp["n_candidates"], stp["n_active"])
        mbytes = method_bytes(1, sizes["n_tets"], sizes["n_verts"], n_act) * ibytes / sum(
            algorithmic_bytes(k, 1, sizes, stp["n_candidates"], stp["n_active"]) for k in iter_kernels)
        traffic = recorded_traffic(dom, "fp32", phases=True)
    else:
        # the persistent kernel: one launch per time step; the method's bytes of its iterations (the candidate
        # build not counted) over the timed step
        dom_all = dom
        dom = "k_persistent"
        per_launch_ms = total_ms / K
        mbytes = st32["iters_done"] * method_bytes(1, sizes["n_tets"], sizes["n_verts"], n_act)
        ibytes = sum(algorithmic_bytes(k, 1, sizes, stp["n_candidates"], stp["n_active"], persistent=True) * prof[k][1] / 3
                     for k in iter_kernels if prof.get(k, (0, 0))[1] > 0)
        traffic = recorded_traffic(dom, "fp32")
    achieved = mbytes / (per_launch_ms * 1e-3) / 1e9
    kernels = {k: {"ms_per_step": round(v[0] / 3, 4), "launches_per_step": v[1] // 3,
                   "us_per_launch": round(1e3 * v[0] / v[1], 3) if v[1] else None,
                   "share": round(v[0] / 3 / step_ms, 4) if step_ms > 0 else None,
                   **({"implementation_gbs": phase_bw[k]} if k in phase_bw else {})}
               for k, v in prof.items() if v[1] > 0}
    sim32.close()

    # plain FP64 form on the same steps
    K64 = min(K, 40)
    # the FP64 form's launch form is autotuned during the warm-up steps (the per-phase form wins for FP64)
    sim64, t64, st64 = one_form(B.SIM_FP64, K64, form=2)
    shape64, shape64_rep = shape_of(st64)
    sim64.close()
    ms64 = sum(t64) / K64
    v64 = K64 * iters / (sum(t64) / 1e3)

    # IterMax = 150 (the iteration cap of the twist scenes in Sec. 5), on steps 80..89 of the run: with 75 or more
    # iterations per step the twisted bar ends between steps 100 and 115 with an inverted tet next to a cap (the
    # cap layer is compressed to under 1 % of its rest volume by then, and moving the caps to their next targets
    # at the start of a step flips it before the first iteration; the FP64 oracle does the same)
    def iter_max_150(K150=min(K, 10), f150=80):
        sim150 = B.Sim(sc, precision=B.SIM_FP32_MIXED, cuda_stream=stream.cuda_stream,
                       persistent=0 if args.phases else 1, iters=150)
        try:
            for s in range(f150):
                B.sim_step_async(sim150.h, 1, targets[s])
            torch.cuda.synchronize()
            B.sim_get_state(sim150.h, want_x=False, want_v=False)
            t150 = time_steps(B, torch, sim150, targets, f150, K150, flush, f150 + K150)
            _, _, st150 = B.sim_get_state(sim150.h, want_x=False, want_v=False)
        except B.SimError as e:
            return {"iters_per_step": 150, "error": str(e)}
        finally:
            sim150.close()
        ms150 = sum(t150) / K150
        return {"iters_per_step": 150, "value": round(K150 * 150 / (sum(t150) / 1e3), 2), "unit": UNIT,
                "ms_per_step": round(ms150, 4), "time_steps_per_s": round(1e3 / ms150, 2), "steps": K150,
                "timed_steps": f"{f150}..{f150 + K150 - 1}",
                "dE_last_over_dE0_last_step": st150["dE_last"] / st150["dE0"] if st150["dE0"] else None}

    iter150 = None if args.no_extras else iter_max_150()

    # PR+ against DK (Sec. 4.1): the whole run step by step, untimed; per step the last iteration's energy
    # decrease relative to the first (the convergence measure of the stopping rule in Sec. 4.4); the FP64 form's
    # state at the start of step 100 is kept for the equal-accuracy comparison
    conv = None if args.no_extras else {}
    for name, beta in ((("pr_plus", B.SIM_BETA_PR_PLUS), ("dk", B.SIM_BETA_DK)) if not args.no_extras else ()):
        simc = B.Sim(sc, precision=B.SIM_FP32_MIXED, cuda_stream=stream.cuda_stream,
                     persistent=0 if args.phases else 1, beta=beta)
        ratios, err = [], None
        for s in range(cfg_steps):
            try:
                B.sim_step_async(simc.h, 1, targets[s])
                _, _, stc = B.sim_get_state(simc.h, want_x=False, want_v=False)
            except B.SimError as e:
                err = str(e)
                break
            if stc["dE0"] > 0:
                ratios.append(max(stc["dE_last"], 1e-300) / stc["dE0"])
        simc.close()
        lr = np.log10(np.asarray(ratios))
        conv[name] = {"median_dE_last_over_dE0": float(10 ** np.median(lr)),
                      "geomean_dE_last_over_dE0": float(10 ** lr.mean()),
                      "worst_dE_last_over_dE0": float(10 ** lr.max()), "steps": len(ratios),
                      **({"error": err} if err else {})}

    # FP32-mixed against plain FP64 at equal final-energy accuracy (twisted bar step 100 and the batch's step 30)
    eq = None
    if not args.no_extras and not args.phases and rank == 0:
        simr = B.Sim(sc, precision=B.SIM_FP64, cuda_stream=stream.cuda_stream, persistent=1)
        for s in range(100):
            B.sim_step_async(simr.h, 1, targets[s])
        xb, vb, _ = B.sim_get_state(simr.h)
        simr.close()
        shapes = {B.SIM_FP32_MIXED: shape32, B.SIM_FP64: shape64}
        eq = {"twisted_bar": equal_accuracy(B, torch, sc, stream, (xb, vb), sc.targets(100), (25, 50, 75, 100),
                                            1000, "twisted bar, time step 100 (from the FP64 form's state)", shapes)}
        if not args.no_pile:
            bsc = S.batched()
            simr = B.Sim(bsc, precision=B.SIM_FP64, cuda_stream=stream.cuda_stream, persistent=1)
            for s in range(30):
                B.sim_step_async(simr.h, 1, None)
            xb, vb, _ = B.sim_get_state(simr.h)
            simr.close()
            eq["batched"] = equal_accuracy(B, torch, bsc, stream, (xb, vb), None, (25, 50, 75, 100), 400,
                                           "batched, 256 scenes, time step 30 (from the FP64 form's state)",
                                           {B.SIM_FP32_MIXED: 0, B.SIM_FP64: 0}, repeat=2)

    # end to end through the C ABI with host buffers: pinned targets in, positions out, every step (the step is
    # enqueued with sim_step_async; sim_get_state copies the positions out, synchronises and reports any error of
    # the step: one synchronisation per step)
    sim = B.Sim(sc, precision=B.SIM_FP32_MIXED, persistent=0 if args.phases else 1, block_shape=shape32)
    tg_host = torch.tensor(sc.all_targets(n_total), dtype=torch.float64).pin_memory()
    x_host = torch.empty((sc.n_verts, 3), dtype=torch.float64).pin_memory()
    for s in range(first):
        B.sim_step_async(sim.h, 1, tg_host[s])
        B.sim_get_state(sim.h, x_out=x_host, want_v=False)
    span = max(1, cfg_steps - first)
    saved = B.sim_get_state(sim.h)[:2] if K > span else None
    te = 0.0
    for s in range(K):
        if s > 0 and s % span == 0:
            B.sim_set_state(sim.h, *saved)   # not timed, as in the device-timed window
        t0 = time.perf_counter()
        B.sim_step_async(sim.h, 1, tg_host[first + s % span])
        B.sim_get_state(sim.h, x_out=x_host, want_v=False)
        te += time.perf_counter() - t0
    sim.close()
    e2e = {"value": round(K * iters / te, 2), "unit": UNIT, "ms_per_step": round(1e3 * te / K, 4),
           "h2d_bytes_per_step": int(tg_host[0].numel() * 8), "d2h_bytes_per_step": int(x_host.numel() * 8)}

    # the large pile and the batch: the same kernels at sizes whose working set exceeds L2, timed on the last steps
    # of their configured runs
    pile = batched = stack = None
    if not args.no_pile:
        pile = side_workload(B, torch, S, stream, flush, S.pile(), "large_pile",
                             "large pile: ten 16x16x64-cell bars (983,040 tets, 187,850 verts) stacked criss-cross "
                             "on a plane, E=2e5 nu=0.4, dt=1/30, dhat=5e-4, 50 NCG iterations per step, FP32-mixed",
                             1, UNIT, 5, peak, peak_kind, args.phases, False)
        # the same stack with every crossing starting face to face within dhat (0.5 dhat gaps, no jitter): about
        # 2e5 active pairs, the contact-dominated regime of the paper's scenes (Table 1: 39K-87K contacts)
        stack = side_workload(B, torch, S, stream, flush, S.pile(gap=0.5, jitter=False, steps=20), "contact_stack",
                              "contact-dominated stack: the large pile's ten bars criss-cross with 0.5 dhat gaps and "
                              "no jitter (every crossing face to face within dhat from the start; 983,040 tets), "
                              "20-step run, 50 NCG iterations per step, FP32-mixed", 1, UNIT, 5, peak, peak_kind,
                              args.phases, False)
        if not args.phases:
            bsc = S.batched()
            batched = side_workload(B, torch, S, stream, flush, bsc, "batched",
                                    "batched: 256 independent cubes of n^3 cells, n ~ U{4..16} (2,184,876 tets, "
                                    "459,790 verts), random rotations, 0.01-0.05 m over a plane, E ~ U[5e4, 5e5], "
                                    "dt=1/60, dhat=1e-3, 50 NCG iterations per step, per-scene beta and alpha, "
                                    "FP32-mixed", bsc.n_scenes, "scene-iterations/s", 5, peak, peak_kind, False, True)

    clocks = sampler.stop()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc, budget_s=args.cpu_seconds, side=not args.no_pile)

    if rank == 0:
        # per-phase form: predict + per iteration five broad-phase kernels (they return at once without a
        # rebuild) and five iteration kernels + finish; persistent form: one cooperative kernel per step
        launches_per_step = (2 + iters * 10) if args.phases else 1
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": round(total_ms / K, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tets": sizes["n_tets"], "verts": sizes["n_verts"],
                       "iters_per_step": iters, "precision": "fp32-mixed: f32 element/barrier arithmetic on "
                       "float-float vertex differences, f64 reductions and vertex state",
                       "l2": "flushed between timed steps (256 MiB write, not timed)", "parallelism": "replicas",
                       "graph": "one CUDA graph replay per time step",
                       "timed_steps": f"steps {first}..{min(first + K, cfg_steps) - 1} of the {cfg_steps}-step run "
                                      f"(the run's last steps, the most contact candidates)"
                                      + (f", repeated from step {first} to make {K}" if first + K > cfg_steps else "")
                                      + f"; steps 0..{first - 1} untimed",
                       "launch": "one kernel per phase" if args.phases else "one persistent cooperative kernel per step",
                       "block_shape": shape32_rep},
            "time_steps_per_s": round(K / (total_ms / 1e3), 2),
            "step_ms": {"median": round(statistics.median(t32), 4), "min": round(min(t32), 4),
                        "max": round(max(t32), 4), "note": "this rank's timed steps, one CUDA-event pair each"},
            "fp64_plain": {"value": round(v64, 2), "unit": UNIT, "ms_per_step": round(ms64, 4), "steps": K64,
                           "launch": "persistent" if st64["launch_form"] == 1 else "one kernel per phase",
                           "block_shape": shape64_rep,
                           "launch_choice": "autotuned (options.persistent = 2, block_shape = -1)" if not args.phases
                           else "per phase",
                           "speedup_fp32_over_fp64_equal_iterations": round(value / ws / v64, 3)},
            "fp32_vs_fp64_equal_accuracy": eq,
            "iter_max_150": iter150,
            "beta_convergence": None if conv is None else
            {"note": "whole 120-step run, FP32-mixed, 50 iterations per step, untimed", **conv},
            "roofline": {"bound": "hbm", "kernel": dom, "largest_phase": dom_all, "achieved": round(achieved, 1),
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": traffic, "algorithmic_bytes_per_launch": int(mbytes),
                         "implementation_bytes_per_launch": int(ibytes),
                         "bytes_basis": "method bytes per NCG iteration (112 B/tet + 196 B/vertex + 34 B/active "
                                        "pair, FP32) x the iterations of one launch; candidate builds not counted",
                         "us_per_launch": round(per_launch_ms * 1e3, 3)},
            "kernels": kernels,
            "large_pile": pile,
            "contact_stack": stack,
            "batched": batched,
            "stats_last_step": {k: st32[k] for k in ("n_candidates", "n_active", "n_rebuilds", "n_capped",
                                                     "n_near_fp64")},
            "e2e": e2e, "gpu_launches": launches_per_step * K, "clocks": clocks, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


BAR_STATE = os.path.join(ROOT, "oracle", "data", "twisted_bar_step100.npz")


def _bar_start(sc):
    """The twisted bar's state at the start of time step 100 (the first step of the GPU's timed window), computed by
    the oracle alone (oracle/make_bar_state.py); the rest pose at step 0 if the file is missing."""
    import numpy as np
    if os.path.exists(BAR_STATE):
        z = np.load(BAR_STATE)
        return z["x"].copy(), z["v"].copy(), int(z["step"])
    return sc.x0.copy(), sc.v0.copy(), 0


def _oracle_iterations(budget_s, step_first=None):
    """Worker: NCG iterations of the FP64 oracle on the twisted bar from the step-100 state for budget_s seconds of
    wall time (at least one); returns (iterations, seconds).  Runs in a process of its own."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2405_08001_gb300 import scenes as S
    sc = S.twisted_bar()
    o = oracle.Oracle.from_scene(sc)
    x, v, step = _bar_start(sc)
    tg = sc.targets(step)
    xt = o.predict(x, v, tg)
    x[sc.fixed.astype(bool)] = tg
    g = np.zeros_like(x); P = np.zeros_like(x); p = np.zeros_like(x)
    t0 = time.perf_counter()
    n = 0
    while n < sc.iters and (n == 0 or time.perf_counter() - t0 < budget_s):
        o.iteration(x, xt, g, P, p, n)
        n += 1
    return n, time.perf_counter() - t0, step


def _oracle_side(name):
    """Oracle NCG iterations/s on one of the side workloads (large pile, batch) at its initial state: one untimed
    iteration, then one timed (each includes the oracle's contact search).  Single-threaded."""
    import numpy as np
    import oracle as O
    from paper_2405_08001_gb300 import scenes as S
    sc = S.pile() if name == "large_pile" else S.batched()
    o = O.Oracle.from_scene(sc)
    x, v = sc.x0.copy(), sc.v0.copy()
    xt = o.predict(x, v, None)
    g, P, p = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
    o.iteration(x, xt, g, P, p, 0)
    t0 = time.perf_counter()
    o.iteration(x, xt, g, P, p, 1)
    dt = time.perf_counter() - t0
    scale = sc.n_scenes if name == "batched" else 1
    what = "batch" if name == "batched" else "large pile"
    return {"value": round(scale / dt, 4), "unit": "scene-iterations/s" if name == "batched" else UNIT,
            "cores": 1, "kind": "oracle",
            "sample": f"the second NCG iteration of the {what}'s first time step ({sc.n_tets:,} tets; FP64 C oracle, "
                      f"1 thread, {dt:.1f} s)"}


def cpu_baseline(sc, budget_s=15.0, side=True):
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the same workload: NCG iterations of
    the twisted bar's time step 100 (the first step of the GPU's timed window, its contact search included), from
    the oracle's own step-100 state.  Single-threaded (the value), and as independent replicas on every host core
    at once (the oracle is serial; all cores busy), each in a spawned process."""
    import multiprocessing as mp
    n, dt, step = _oracle_iterations(budget_s)
    cores = os.cpu_count() or 1
    multi = None
    if cores > 1:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            outs = pool.starmap(_oracle_iterations, [(budget_s / 2,)] * cores)
        multi = {"value": round(sum(a for a, _, _ in outs) / max(b for _, b, _ in outs), 4), "unit": UNIT,
                 "cores": cores, "kind": "oracle, one independent replica per core"}
    out = {"value": round(n / dt, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{n} NCG iterations of time step {step} of the 98,304-tet twisted bar from the oracle's own "
                     f"step-{step} state (FP64 C oracle, 1 thread, {dt:.1f} s)",
           "all_cores": multi}
    if side:
        out["side_workloads"] = {w: _oracle_side(w) for w in ("large_pile", "batched")}
    return out


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle on the same workload and metric; each benchmark step is one NCG
    iteration (a bounded sample), iterations continuing through the time steps of the twist from the oracle's own
    state at the start of step 100, the first step of the GPU's timed window."""
    import numpy as np
    ws, rank, local = rank_info()
    if rank != 0:
        return
    import oracle
    from paper_2405_08001_gb300 import scenes as S
    sc = S.twisted_bar()
    o = oracle.Oracle.from_scene(sc)
    x, v, step0 = _bar_start(sc)
    fx = sc.fixed.astype(bool)
    state = {"step": step0 - 1, "k": sc.iters}

    def one_iteration():
        if state["k"] >= sc.iters:
            if state["step"] >= step0:
                v[:] = (x - state["xt0"]) / sc.dt
            state["step"] += 1
            tg = sc.targets(state["step"])
            state["xt0"] = x.copy()
            state["xtil"] = o.predict(x, v, tg)
            x[fx] = tg
            state["g"] = np.zeros_like(x); state["P"] = np.zeros_like(x); state["p"] = np.zeros_like(x)
            state["k"] = 0
        o.iteration(x, state["xtil"], state["g"], state["P"], state["p"], state["k"])
        state["k"] += 1

    for _ in range(args.warmup):
        one_iteration()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        one_iteration()
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps / tot
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * tot / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "step": "one NCG iteration of the FP64 CPU oracle (bounded sample)",
                       "timed_steps": f"iterations of time steps {step0}.. of the run, from the oracle's own "
                                      f"step-{step0} state"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": round(value, 4), "unit": UNIT,
                             "sample": f"{args.steps} consecutive NCG iterations of the twisted bar from time step "
                                       f"{step0}, 1 thread"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--phases", action="store_true", help="one kernel per phase instead of the persistent step")
    ap.add_argument("--no-pile", action="store_true", help="skip the large-pile and batched measurements")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the IterMax-150 run and the PR+ / DK convergence comparison")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
