#!/usr/bin/env python3
"""Throughput of the coupled D2Q9 + D2Q5 porous cascaded LB step on GB300.

Workload (N = 1): natural convection in a 4096 x 4096 porous cavity with the
seeded porosity eps(x) = 0.3 + 0.6 Phi(g(x)) (g a unit Gaussian random field,
correlation length 32 cells, seed 20211012), Da 1e-3, Ra 1e6, Pr 0.71,
sigma 1, FP64.  One bench step = one LB time step over the whole grid (all
nodes, both lattices, walls).  N > 1 runs one independent replica per GPU
(weak scaling, no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  `value` = cells x steps / time over all
ranks (MLUPS), timed with CUDA events on the library's stream, inputs
resident in HBM (the 3.8 GB state is far larger than the 129 MB L2).  `e2e`
is the same metric through the public C ABI from pinned host buffers:
clb_init (porosity upload) + K steps + clb_macros (four fields back) +
clb_nusselt, wall-clock.  `--impl reference` times the FP64 CPU oracle on
the host cores on a bounded sample of the same workload.

Secondary objects on the same line: `forms` (FP16-storage forms at 8192^2),
`accuracy` (FP16 forms against the FP64 path on the 8192^2 sigma 0.8 cavity
at a fixed step count), `batch` (512 seeded cavities, graph and persistent
launch modes), `mrt_cost` (the porous shift matrices against the unit-shift
MRT limit, Table 2's comparison), `cavity64` (the 64^2 Table 1 cavity to
steady state), `cpu_baseline` (all host cores and one), `steady_state` (time
to steady state of each form on the Table 1 case), `warm_start` (FP64 march
from rest vs from the learned warm start) and `surrogate_training`; the last
key, `summary`, repeats their headline figures compactly.
`--no-forms/--no-accuracy/--no-batch/--no-cpu/--no-steady/--no-warm/--no-mrt`
skip them; `--validate-batch` adds the per-case Nusselt number of a
stratified 64-case sample of the batch at steady state, FP16N against FP64.
`--gpus N` without a launcher starts N local ranks itself (torchrun).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX = NY = 4096          # --size changes this (smaller sizes are for profiler captures only)
CASE = dict(Ra=1e6, Da=1e-3, Pr=0.71, sigma=1.0)
PHI_SEED, PHI_ELL = 20211012, 32.0
METRIC = "coupled D2Q9+D2Q5 MLUPS"
UNIT = "MLUPS"
WORKLOAD = ("{n}x{n} porous cavity, seeded GRF porosity 0.3+0.6*Phi(g) (l=32, seed 20211012), "
            "Da 1e-3, Ra 1e6, Pr 0.71, sigma 1, FP64")

# Algorithmic bytes per coupled cell update of the FP64 form: 14 distribution
# values read and 14 written (8 B each) plus the porosity (8 B).
BYTES_PER_CCU_F64 = 28 * 8 + 8
# FP64 floating-point operations per coupled cell update executed by the FP64
# step kernel (dadd + dmul + 2 dfma per launch / nodes, ncu instruction
# counters of the current kernel), and its FP64 pipe instructions (dadd +
# dmul + dfma) per node.
FP64_FLOP_PER_CCU = 257.5
FP64_INST_PER_CCU = 175.4
# DRAM bytes (read + write) per node of one launch of the current FP64 step
# kernel, ncu on the 2048^2 case of the same workload, scaled by the node
# count (traffic grows with the nodes): 14 + 14 values and the 64-byte
# per-node constant table.
DRAM_BYTES_PER_CCU_MEASURED = 282.7
SMS, DFMA_PER_CLK_PER_SM = 152, 2   # GB300 FP64 pipe: 2 DFMA/clk/SM (1.25 TFLOP/s at 2.07 GHz)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": reasons}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(seconds: float, dist=None, device: str = "cuda") -> float:
    """The largest of the ranks' times, on every rank (the job ends with its
    slowest replica); `seconds` itself without a process group."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(cells: int, steps: int, world: int, seconds: float) -> float:
    """Node updates of all replicas (each advances `cells` nodes `steps`
    times) per second of the slowest one, in millions."""
    return cells * steps * world / seconds / 1e6


def _porosity():
    from paper_2110_05943_gb300.inputs import porosity_field
    return porosity_field(NX, NY, seed=PHI_SEED, ell=PHI_ELL)


def cpu_oracle_rate(phi, budget_s: float = 12.0, side: int = 512, nthreads=None):
    """FP64 oracle on the SW corner block (side x side) of the workload, with
    the full cavity's lattice parameters (L = n - 1); MLUPS on all host cores
    (nthreads None) or on the given number of threads."""
    side = min(side, NX)
    import oracle
    sub = phi[:side, :side].copy()
    p = oracle.Problem(nx=side, ny=side, L=float(NY - 1), **CASE)
    o = oracle.Oracle(p, phi=sub, nthreads=nthreads)
    t0 = time.perf_counter()
    o.step(2)
    dt = max(time.perf_counter() - t0, 1e-6) / 2
    steps = max(3, int(budget_s / dt))
    t0 = time.perf_counter()
    o.step(steps)
    t = time.perf_counter() - t0
    return {"value": side * side * steps / t / 1e6, "unit": UNIT, "cores": o.nthreads, "kind": "oracle",
            "sample": f"{side}x{side} corner block of the {NX}^2 workload (same porosity values and lattice "
                      f"parameters, walls on all four sides), {steps} FP64 steps, {t:.1f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    import oracle
    phi = _porosity()
    side = min(512, NX)
    sub = phi[:side, :side].copy()
    p = oracle.Problem(nx=side, ny=side, L=float(NY - 1), **CASE)
    o = oracle.Oracle(p, phi=sub)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    t = time.perf_counter() - t0
    v = side * side * args.steps / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(n=NX), "sample": f"{side}x{side} corner block per step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": o.nthreads, "kind": "oracle",
                             "sample": f"{side}x{side} corner block of the {NX}^2 workload, "
                                       f"{args.steps} FP64 steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def steady_state_forms(clb, torch, total=350_000, window=20, every=2500):
    """Time to steady state of each storage form on the paper's own grid for
    the Table 1 row Da 1e-2, Ra 1e4, phi 0.6, Pr 1 (128^2; paper: Nu 1.4873):
    steps and wall time until the hot-wall Nusselt number changes by at most
    1e-4 (relative) over 1000 steps, and the Nusselt number then.  Each run
    then continues to `total` steps; the mean Nusselt number over the last
    window x every steps is the converged value that the forms are compared
    by (at the stopping step they are still in the slow tail of the
    transient, so their difference there says little about storage
    precision)."""
    out = {}
    for name, prec in (("f64", 0), ("f16n", 2), ("f16s", 1)):
        p = clb.clb_params_default(nx=128, ny=128, Ra=1e4, Da=1e-2, Pr=1.0, precision=prec)
        sim = clb.Simulation.create(p, 0.6, clb.clb_bc_cavity(1.0, 0.0),
                                    stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prev = sim.nusselt(clb.W)
        done = None
        while sim.time < 400_000:
            sim.step(1000)
            nu = sim.nusselt(clb.W)
            if abs(nu - prev) <= 1e-4 * abs(nu):
                done = (sim.time, time.perf_counter() - t0, nu)
                break
            prev = nu
        sim.step(max(0, total - window * every - sim.time))
        vals = []
        for _ in range(window):
            sim.step(every)
            vals.append(sim.nusselt(clb.W))
        sim.close()
        out[name] = {"steps": done[0] if done else None, "seconds": done[1] if done else None,
                     "nu": done[2] if done else None, "nu_converged": float(np.mean(vals)),
                     "nu_converged_sd": float(np.std(vals))}
    ref = out["f64"]
    for name in ("f16n", "f16s"):
        o = out[name]
        o["rel_nu_converged_vs_f64"] = abs(o["nu_converged"] / ref["nu_converged"] - 1)
        if o["nu"] is not None and ref["nu"] is not None:
            o["rel_nu_vs_f64"] = abs(o["nu"] / ref["nu"] - 1)
            o["speedup_vs_f64"] = ref["seconds"] / o["seconds"]
    return {"workload": "128x128 cavity, phi 0.6, Da 1e-2, Ra 1e4, Pr 1 (Table 1 row; paper Nu 1.4873)",
            "criterion": "|dNu| <= 1e-4 Nu over 1000 steps (time to steady); converged Nu = mean over steps "
                         f"{total - window * every}..{total}",
            "forms": out}


FORMS = {  # storage form -> (precision code, algorithmic bytes per coupled cell update)
    "f16n": (2, 28 * 2 + 2 * 8 + 4),   # 14 FP16 deviations read+written, 8 B record read+written, FP32 1/phi
    "f16s": (1, 28 * 2 + 4),           # 14 FP16 deviations read+written, FP32 phi
}
# DRAM bytes (read + write) per node of one launch of the current FP16 step
# kernels, ncu on the 4096^2 case of the same workload; traffic grows with
# the node count.  None: not captured for the kernel as it stands.
FORMS_DRAM_PER_NODE = {"f16n": 76.3, "f16s": 60.3}
# DRAM bytes (read + write) per node of one launch of the current batch
# kernel (k_step_batch_mix, graph mode), ncu on the first 128 of the 512
# cases (10.08 M nodes), scaled by the node count; None: not captured for
# the kernel as it stands.
BATCH_DRAM_PER_NODE = 80.6


def reduced_precision_forms(clb, torch, args, hbm_peak, src):
    """Throughput of the FP16-storage forms on the 8192^2 seeded cavity
    (Da 1e-3, Ra 1e6, Pr 0.71, sigma 0.8), CUDA events over the timed steps."""
    from paper_2110_05943_gb300.inputs import porosity_field
    n = 8192
    phi = porosity_field(n, n, seed=PHI_SEED, ell=PHI_ELL)
    out = {}
    stream = torch.cuda.current_stream()
    for name, (prec, bpn) in FORMS.items():
        p = clb.clb_params_default(nx=n, ny=n, Ra=1e6, Da=1e-3, Pr=0.71, sigma=0.8, precision=prec)
        sim = clb.Simulation.create(p, phi, clb.clb_bc_cavity(1.0, 0.0), stream=stream.cuda_stream)
        sim.step(args.warmup)
        torch.cuda.synchronize()
        steps = max(args.steps, 64)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        sim.close()
        gbs = bpn * n * n / (t / steps) / 1e9
        out[name] = {"workload": f"{n}x{n} porous cavity, seeded GRF porosity, Da 1e-3, Ra 1e6, Pr 0.71, sigma 0.8",
                     "value": n * n * steps / t / 1e6, "unit": UNIT, "steps": steps, "ms_per_step": t / steps * 1e3,
                     "dtype": "f32 arithmetic, f16 storage",
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                  "frac": gbs / hbm_peak, "bytes_per_ccu": bpn,
                                  "traffic": (FORMS_DRAM_PER_NODE[name] * n * n if FORMS_DRAM_PER_NODE[name] else None),
                                  "traffic_source": "ncu dram bytes per node at 4096^2 x nodes per launch",
                                  "kernel": f"k_step2<StoreH16{'N' if name == 'f16n' else ''}>",
                                  "peak_source": f"{src} hbm_gbs"}}
    return out


def _batch_make(clb, torch, sel, prec):
    stream = torch.cuda.current_stream()
    params = [clb.clb_params_default(nx=c.nx, ny=c.ny, Ra=c.Ra, Da=c.Da, Pr=c.Pr, sigma=c.sigma, precision=prec)
              for c in sel]
    return clb.Batch(params, [c.phi for c in sel], [clb.clb_bc_cavity(1.0, 0.0) for _ in sel],
                     stream=stream.cuda_stream)


def _t_diff(c):
    """Thermal diffusion time max(nx, ny)^2 / alpha of a batch case (alpha =
    nu / Pr, nu from Eq. 46 with L = ny - 1): the time scale to steady state."""
    nu = 0.1 * (c.ny - 1) * math.sqrt(c.Pr / (3.0 * c.Ra))
    return max(c.nx, c.ny) ** 2 / (nu / c.Pr)


def batched_form(clb, torch, args, hbm_peak, src):
    """512 seeded cavities of uneven size (sides log-uniform in [64, 1024],
    aspect 1-4; log10 Ra in [3, 6], log10 Da in [-4, -1], eps in [0.4, 0.9],
    sigma in [0.5, 2], Pr 0.71), FP16N, with the tiling chosen by
    clb_batch_tune; aggregate MLUPS over the timed steps in both launch
    modes (one launch per step replayed from graphs; one persistent launch
    per 32 steps).  Accuracy: the 8 cases with the shortest diffusion time,
    as a batch in FP64 and in FP16N, converged (criteria below); relative
    difference of the hot-wall Nusselt number per case."""
    from paper_2110_05943_gb300.inputs import batch_cases
    cases = batch_cases(512, seed=7)[:args.batch_cases]
    stream = torch.cuda.current_stream()
    b = _batch_make(clb, torch, cases, 2)
    choice = b.tune(steps=3)
    steps = max(args.steps, 64)
    rates = {}
    for mode, name in ((clb.CLB_BATCH_GRAPH, "graph"), (clb.CLB_BATCH_PERSISTENT, "persistent")):
        b.set_mode(mode)
        b.step(max(args.warmup, 32))
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        b.sync()
        rates[name] = b.nodes * steps / (e0.elapsed_time(e1) / 1e3) / 1e6
    nodes = b.nodes
    nu = b.nusselt(0)
    b.close()
    best = max(rates, key=rates.get)
    bpn = FORMS["f16n"][1]
    gbs = bpn * rates[best] * 1e6 / 1e9
    out = {"workload": f"{len(cases)} seeded porous cavities (batch_cases seed 7), uneven grids, FP16N",
           "cases": len(cases),
           "value": rates[best], "unit": UNIT, "mode": best, "mlups_by_mode": rates, "steps": steps,
           "nodes_per_step": nodes, "ms_per_step": nodes / (rates[best] * 1e6) * 1e3, "tile_choice": choice,
           "finite_cases": int(np.isfinite(nu).sum()),
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                        "bytes_per_ccu": bpn,
                        "traffic": BATCH_DRAM_PER_NODE * nodes if BATCH_DRAM_PER_NODE else None,
                        "traffic_source": "ncu dram bytes per node of k_step_batch_mix on 128 of the cases x nodes "
                                          "per step",
                        "kernel": "k_step_batch_mix (graph) / k_step_batch_persist <StoreH16N>",
                        "peak_source": f"{src} hbm_gbs"}}
    if args.no_batch_check:
        return out

    # validation subset: the 8 cases with the shortest thermal diffusion time
    quick = sorted(range(len(cases)), key=lambda i: _t_diff(cases[i]))[:8]
    sel = [cases[i] for i in quick]
    # FP64: to |dNu| <= 1e-6 Nu per 4000 steps.  FP16N: its time to steady by
    # the metric's |dNu| <= 1e-4 Nu per 1000 steps (its stochastic rounding
    # leaves Nu fluctuations of ~1e-5, so a tighter rule never fires), then
    # on to the FP64 run's step count plus 20,000 and the mean Nu over the
    # last 20,000 steps; errors are taken between those converged values.
    v = _batch_make(clb, torch, sel, 0)
    prev = v.nusselt(0)
    t0 = time.perf_counter()
    while v.time < 240_000:
        v.step(4000)
        nu64 = v.nusselt(0)
        if np.all(np.abs(nu64 - prev) <= 1e-6 * np.abs(nu64)):
            break
        prev = nu64
    steps64, sec64 = v.time, time.perf_counter() - t0
    v.close()
    v = _batch_make(clb, torch, sel, 2)
    prev = v.nusselt(0)
    t0 = time.perf_counter()
    while v.time < 240_000:
        v.step(1000)
        cur = v.nusselt(0)
        if np.all(np.abs(cur - prev) <= 1e-4 * np.abs(cur)):
            break
        prev = cur
    steps16, sec16 = v.time, time.perf_counter() - t0
    v.step(max(0, steps64 + 20_000 - v.time))
    vals = []
    for _ in range(20):
        v.step(1000)
        vals.append(v.nusselt(0))
    nu16 = np.mean(vals, axis=0)
    v.close()
    err = np.abs(nu16 / nu64 - 1)
    out["validation"] = {"cases": [f"{c.nx}x{c.ny} Ra {c.Ra:.3g} Da {c.Da:.3g} eps {c.phi:.2f} sigma {c.sigma:.2f}"
                                     for c in sel],
                           "criterion": "FP64 |dNu| <= 1e-6 Nu / 4000 steps; FP16N time to |dNu| <= 1e-4 Nu / "
                                        "1000 steps, Nu = mean over the 20,000 steps after FP64's step count",
                           "nu_f64": [float(x) for x in nu64], "nu_f16n": [float(x) for x in nu16],
                           "max_rel_nu_error": float(np.nanmax(err)), "steps_f64": steps64,
                           "steps_f16n": steps16, "seconds_f64": sec64, "seconds_f16n": sec16}
    return out


def _batch_window_means(clb, torch, sel, prec, start, window=20, every=1000):
    """Mean hot-wall Nu of each case over `window` samples `every` steps
    apart, taken after step start[k] (cases with start None are retired);
    the batch retires each case once its window is complete."""
    n = len(sel)
    b = _batch_make(clb, torch, sel, prec)
    active = np.array([s is not None for s in start])
    b.set_active(active.astype(np.int32))
    sums, cnt = np.zeros(n), np.zeros(n, dtype=int)
    while active.any():
        b.step(every)
        cur = b.nusselt(0)
        for k in np.nonzero(active)[0]:
            if b.time > start[k]:
                sums[k] += cur[k]
                cnt[k] += 1
        done = active & (cnt >= window)
        if done.any():
            active &= ~done
            b.set_active(active.astype(np.int32))
    b.close()
    return np.where(cnt > 0, sums / np.maximum(cnt, 1), np.nan)


def batch_validation(clb, torch, n=64, cap=200_000):
    """Per-case hot-wall Nusselt number of a stratified sample of the
    512-case batch at steady state, FP16N against FP64: the cases sorted by
    thermal diffusion time, split into n strata of 512 / n, the fastest of
    each taken.  A case is steady at the first multiple of 2000 steps at
    which its FP64 Nu changed by at most 1e-6 Nu over the last 2000 steps
    (cap `cap` steps).  Each form's Nu is then the mean of 20 samples over
    the same 20,000 steps after that point (the stochastic rounding of the
    FP16 form leaves Nu fluctuations of ~1e-5, and a flow that still
    oscillates slowly is compared over the same window)."""
    from paper_2110_05943_gb300.inputs import batch_cases
    cases = batch_cases(512, seed=7)
    order = sorted(range(len(cases)), key=lambda i: _t_diff(cases[i]))
    per = len(cases) // n
    idx = [order[k * per] for k in range(n)]
    sel = [cases[i] for i in idx]
    t0 = time.perf_counter()
    b = _batch_make(clb, torch, sel, 0)
    active = np.ones(n, dtype=bool)
    at = [None] * n
    prev = b.nusselt(0)
    while active.any() and b.time < cap:
        b.step(2000)
        cur = b.nusselt(0)
        hit = active & (np.abs(cur - prev) <= 1e-6 * np.abs(cur))
        for k in np.nonzero(hit)[0]:
            at[k] = b.time
        if hit.any():
            active &= ~hit
            b.set_active(active.astype(np.int32))
        prev = cur
    b.close()
    nu64 = _batch_window_means(clb, torch, sel, 0, at)
    s64 = time.perf_counter() - t0
    t0 = time.perf_counter()
    nu16 = _batch_window_means(clb, torch, sel, 2, at)
    s16 = time.perf_counter() - t0
    ok = [k for k in range(n) if at[k] is not None]
    err = {k: abs(nu16[k] / nu64[k] - 1) for k in ok}
    return {"workload": f"{n} of the 512 batch cavities, stratified by thermal diffusion time "
                        f"(fastest of each stratum of {per})",
            "criterion": f"steady: FP64 |dNu| <= 1e-6 Nu over 2000 steps (cap {cap} steps); each form's Nu = "
                         "mean of 20 samples over the next 20,000 steps",
            "cases": [{"case": int(i), "grid": f"{cases[i].nx}x{cases[i].ny}", "Ra": round(cases[i].Ra, 1),
                       "Da": float(f"{cases[i].Da:.3g}"), "steady_at": at[k],
                       "nu_f64": None if at[k] is None else float(nu64[k]),
                       "nu_f16n": None if at[k] is None else float(nu16[k]), "rel_err": err.get(k)}
                      for k, i in enumerate(idx)],
            "converged": len(ok), "max_rel_nu_error": max(err.values()) if err else None,
            "median_rel_nu_error": float(np.median(list(err.values()))) if err else None,
            "within_1e-4": int(sum(e <= 1e-4 for e in err.values())), "seconds_f64": s64, "seconds_f16n": s16}


def accuracy_forms(clb, torch, n=8192, steps=1000):
    """The FP16-storage forms against the FP64 path (parity-tested against
    the oracle) on the n^2 seeded cavity with sigma 0.8 (Da 1e-3, Ra 1e6,
    Pr 0.71) after the same number of steps: max |a - b| of u_x, u_y over
    the grid, relative to max |u| of the FP64 field and to the velocity
    scale u_c = Ma c_s of Eq. 46; max |T_a - T_b| (the walls differ by dT =
    1); the relative difference of the hot-wall Nusselt number; and each
    form's time per step."""
    from paper_2110_05943_gb300.inputs import porosity_field
    phi = porosity_field(n, n, seed=PHI_SEED, ell=PHI_ELL)
    stream = torch.cuda.current_stream()
    uc = 0.1 / math.sqrt(3.0)
    ref = None
    out = {"workload": f"{n}x{n} porous cavity, seeded GRF porosity, Da 1e-3, Ra 1e6, Pr 0.71, sigma 0.8",
           "steps": steps, "u_c": uc}
    for name, prec in (("f64", 0), ("f16n", 2), ("f16s", 1)):
        p = clb.clb_params_default(nx=n, ny=n, Ra=1e6, Da=1e-3, Pr=0.71, sigma=0.8, precision=prec)
        sim = clb.Simulation.create(p, phi, clb.clb_bc_cavity(1.0, 0.0), stream=stream.cuda_stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        f = torch.empty((3, n, n), dtype=torch.float64, device="cuda")
        clb.clb_macros_device(sim.handle, None, f[0].data_ptr(), f[1].data_ptr(), f[2].data_ptr())
        nu = sim.nusselt(clb.W)
        sim.close()
        torch.cuda.synchronize()
        if ref is None:
            ref = (f, nu, float(f[:2].abs().max()))
            out[name] = {"ms_per_step": ms, "nu": nu, "max_abs_u": ref[2]}
            continue
        du = [float((f[k] - ref[0][k]).abs().max()) for k in range(2)]
        out[name] = {"ms_per_step": ms, "nu": nu, "max_abs_err_ux": du[0], "max_abs_err_uy": du[1],
                     "rel_err_u": max(du) / ref[2], "err_u_over_uc": max(du) / uc,
                     "max_abs_err_T": float((f[2] - ref[0][2]).abs().max()), "rel_err_nu": abs(nu / ref[1] - 1),
                     "speedup_vs_f64": out["f64"]["ms_per_step"] / ms}
        del f
    del ref
    torch.cuda.empty_cache()
    return out


def mrt_cost(clb, torch, steps=32):
    """Cost of the porous shift matrices: the FP64 step on the bench workload
    with the shift (N, N_T of Eqs. 14, 31) and in the unit-shift limit (N =
    N_T = I, the MRT scheme named at the end of Sec. 2), CUDA-event time per
    step; Table 2 of the paper reports the ratio on a CPU."""
    phi = _porosity()
    stream = torch.cuda.current_stream()
    ms = {}
    for name, shift in (("clb", 1), ("mrt", 0)):
        p = clb.clb_params_default(nx=NX, ny=NY, shift=shift, **CASE)
        sim = clb.Simulation.create(p, phi, clb.clb_bc_cavity(1.0, 0.0), stream=stream.cuda_stream)
        sim.step(4)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[name] = e0.elapsed_time(e1) / steps
        sim.close()
    return {"workload": WORKLOAD.format(n=NX), "ms_per_step_clb": ms["clb"], "ms_per_step_mrt": ms["mrt"],
            "ratio_clb_over_mrt": ms["clb"] / ms["mrt"],
            "paper_cpu_ratio": "2099.33 s / 1812.31 s = 1.158 (Table 2, i5-8400)"}


def cavity64(clb, torch, cap=20_000, every=100):
    """The 64^2 porous cavity (phi 0.6, Da 1e-2, Ra 1e4, Pr 1, sigma 1):
    20,000 steps or until max(r_u, r_T) over `every` steps drops below 1e-8;
    mean Nusselt number of both isothermal walls (Table 1 "Present" at 128^2:
    1.4873)."""
    p = clb.clb_params_default(nx=64, ny=64, Ra=1e4, Da=1e-2, Pr=1.0, sigma=1.0)
    sim = clb.Simulation.create(p, 0.6, clb.clb_bc_cavity(1.0, 0.0),
                                stream=torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    r = (1.0, 1.0)
    while sim.time < cap:
        sim.step(every)
        r = sim.residual()
        if max(r) < 1e-8:
            break
    sec = time.perf_counter() - t0
    out = {"workload": "64x64 cavity, phi 0.6, Da 1e-2, Ra 1e4, Pr 1, sigma 1, FP64",
           "criterion": "20,000 steps or max(r_u, r_T) < 1e-8 over 100 steps", "steps": sim.time,
           "residual": max(r), "seconds": sec, "nu_hot": sim.nusselt(clb.W), "nu_cold": sim.nusselt(clb.E)}
    sim.close()
    return out


def warm_start_form(clb, torch, ncase=4):
    """The learned warm start with the committed weights on the first `ncase`
    held-out 128^2 cavities (warmstart_cases seed 11, indices 2000...): FP64
    march from rest and from the network's prediction to max(r_u, r_T) <= 1e-8
    over 100-step intervals; steps, wall time (inference included), the step
    after which Nu stays within 1e-4 of the cold run's converged value, and
    the final Nusselt numbers."""
    from paper_2110_05943_gb300 import surrogate, warmstart
    from paper_2110_05943_gb300.inputs import warmstart_cases
    wpath = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2110_05943_gb300", "weights",
                         "warmstart_128.npz")
    net = surrogate.Net.create(torch, seed=0).load(wpath)
    stream = torch.cuda.current_stream().cuda_stream
    rows = []
    for c, phi in warmstart_cases(2000 + ncase, seed=11)[2000:]:
        t0 = time.perf_counter()
        init = surrogate.warm_fields(net, phi, c.Ra, c.Da, c.Pr, c.sigma)
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t0
        sc, tc, nc, okc, hc = warmstart.march(c, phi, None, stream, torch=torch)
        sw, tw, nw, okw, hw = warmstart.march(c, phi, init, stream, torch=torch)
        rows.append({"Ra": round(c.Ra, 1), "Da": float(f"{c.Da:.4g}"), "steps_cold": sc, "steps_warm": sw,
                     "sec_cold": round(tc, 3), "sec_warm": round(tw + t_inf, 3),
                     "steps_nu_1e-4_cold": warmstart.steps_to_nu(hc, nc),
                     "steps_nu_1e-4_warm": warmstart.steps_to_nu(hw, nc),
                     "nu_cold": nc, "nu_warm": nw, "rel_nu": abs(nw / nc - 1), "converged": bool(okc and okw)})
    ok = [r for r in rows if r["converged"]]
    return {"workload": f"first {ncase} held-out 128x128 warm-start cavities, FP64 march, committed weights",
            "criterion": "max(r_u, r_T) <= 1e-8 over 100-step intervals",
            "steps_ratio_total": (sum(r["steps_warm"] for r in ok) / sum(r["steps_cold"] for r in ok)) if ok else None,
            "wall_speedup_total": (sum(r["sec_cold"] for r in ok) / sum(r["sec_warm"] for r in ok)) if ok else None,
            "max_rel_nu": max((r["rel_nu"] for r in ok), default=None), "cases": rows}


def surrogate_training(torch, bf16_peak, src, batch=16, steps=20):
    """One Adam training step of the warm-start network (batch 16 at 128^2,
    seeded random inputs and targets): forward, channel-weighted MSE, input
    and weight gradients and Adam, all in the library's kernels (TMA-fed
    tcgen05 convolutions).  Tensor-core FLOPs per step / CUDA-event time per step,
    against the measured BF16 peak.  The working set (~0.1 GB of activations)
    stays in L2 between steps, as it does in training."""
    from paper_2110_05943_gb300 import surrogate
    net = surrogate.Net.create(torch, seed=0)
    rng = np.random.default_rng(0)
    n, h, w = batch, 128, 128
    X = surrogate.to_bf16(torch, rng.standard_normal((n, h, w, surrogate.N_IN)).astype(np.float32))
    Y = torch.from_numpy(rng.standard_normal((n, h, w, surrogate.N_OUT)).astype(np.float32)).to("cuda")
    wts = torch.tensor([1.0, 1.0, 2.0, 0.5], device="cuda")

    def one(t):
        out, A = net.forward(X, n, h, w)
        _, g = net.loss_and_grad(out, Y, wts)
        net.backward(g, A, n, h, w)
        net.adam(t, 1e-4)

    for t in range(1, 4):
        one(t)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for t in range(4, 4 + steps):
        one(t)
    e1.record(stream)
    torch.cuda.synchronize()
    if surrogate._lib().clb_nop_check(None) != 0:
        raise RuntimeError("surrogate kernels timed out")
    sec = e0.elapsed_time(e1) / 1e3 / steps
    fl = net.train_flops(n, h, w)
    tf = fl / sec / 1e12
    return {"workload": f"warm-start network ({net.nparams} parameters), one training step, batch {n} at {h}x{w}",
            "ms_per_step": sec * 1e3, "samples_per_s": n / sec,
            "roofline": {"bound": "tensor", "achieved": tf, "peak": bf16_peak, "unit": "TFLOP/s",
                         "frac": tf / bf16_peak, "flop_per_step": fl, "traffic": None,
                         "kernel": "k_conv_tma / k_wgrad_tma (TMA + tcgen05) + elementwise, whole step",
                         "peak_source": f"{src} bf16_tflops"}}


def _summary(line):
    """Headline figures of every section, compact (the last key of the line)."""
    r3 = lambda v: None if v is None else float(f"{v:.4g}")
    s = {f"f64_{line['config']['nx']}": {"mlups": r3(line["value"]), "frac": r3(line["roofline"]["frac"]),
                      "bound": line["roofline"]["bound"],
                      "fp64_pipe_frac": r3(line["roofline"].get("fp64_pipe_frac")),
                      "e2e_mlups": r3((line.get("e2e") or {}).get("value"))}}
    for name, f in (line.get("forms") or {}).items():
        s[f"{name}_8192"] = {"mlups": r3(f["value"]), "hbm_frac": r3(f["roofline"]["frac"])}
    for key, tag in (("accuracy", "acc_8192"), ("accuracy_2048", "acc_2048")):
        a = line.get(key)
        if a:
            s[tag] = {k: {"u_rel": r3(a[k]["rel_err_u"]), "u_uc": r3(a[k]["err_u_over_uc"]),
                          "T": r3(a[k]["max_abs_err_T"]), "nu": r3(a[k]["rel_err_nu"])} for k in ("f16n", "f16s")}
            s[tag]["steps"] = a["steps"]
    b = line.get("batch")
    if b:
        s[f"batch_{b['cases']}"] = {"mlups": r3(b["value"]), "mode": b["mode"], "hbm_frac": r3(b["roofline"]["frac"]),
                          "by_mode": {k: r3(v) for k, v in b["mlups_by_mode"].items()},
                          "max_rel_nu_err_8": r3((b.get("validation") or {}).get("max_rel_nu_error"))}
    v = line.get("batch_validation")
    if v:
        s["batch_validation"] = {"converged": v["converged"], "of": len(v["cases"]),
                                 "max_rel_nu_err": r3(v["max_rel_nu_error"]), "within_1e-4": v["within_1e-4"]}
    m = line.get("mrt_cost")
    if m:
        s["clb_over_mrt"] = r3(m["ratio_clb_over_mrt"])
    c = line.get("cavity64")
    if c:
        s["cavity64_nu"] = r3(c["nu_hot"])
    st = line.get("steady_state")
    if st:
        s["steady_128"] = {k: {"rel_nu": r3(f.get("rel_nu_converged_vs_f64")), "speedup": r3(f.get("speedup_vs_f64"))}
                           for k, f in st["forms"].items() if k != "f64"}
    cb = line.get("cpu_baseline")
    if cb:
        s["oracle_mlups"] = {"cores": cb["cores"], "all": r3(cb["value"]),
                             "one": r3((line.get("cpu_baseline_1core") or {}).get("value"))}
    w = line.get("warm_start")
    if w:
        s["warm_start"] = {"steps_ratio": r3(w["steps_ratio_total"]), "wall_speedup": r3(w["wall_speedup_total"]),
                           "max_rel_nu": r3(w["max_rel_nu"])}
    t = line.get("surrogate_training")
    if t:
        s["surrogate_tflops"] = r3(t["roofline"]["achieved"])
    return s


def run_ours(args):
    import torch

    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2110_05943_gb300 import clb
    clb.load()
    phi = _porosity()
    stream = torch.cuda.current_stream()
    prec = {"f64": 0, "f16s": 1, "f16n": 2}[args.precision]
    p = clb.clb_params_default(nx=NX, ny=NY, precision=prec, **CASE)
    sim = clb.Simulation.create(p, phi, clb.clb_bc_cavity(1.0, 0.0), stream=stream.cuda_stream)
    sim.step(args.warmup)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    sim.step(args.steps)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    t = t_start.elapsed_time(t_end) / 1e3
    nu = sim.nusselt(clb.W)
    sim.close()
    t = max_over_ranks(t, dist)
    cells = NX * NY
    value = whole_job_mlups(cells, args.steps, ws, t)
    per_launch = t / args.steps

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        phi_pin = torch.from_numpy(phi).pin_memory()
        outs = [torch.empty((NY, NX), dtype=torch.float64).pin_memory() for _ in range(4)]
        import ctypes
        L = clb.load()
        dp = lambda a: ctypes.cast(a.data_ptr(), ctypes.POINTER(ctypes.c_double))
        bc = clb.clb_bc_cavity(1.0, 0.0)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        h = ctypes.c_void_p()
        rc = L.clb_init(ctypes.byref(h), ctypes.byref(p), dp(phi_pin), None, ctypes.byref(bc),
                        ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.clb_last_error(None)
        assert L.clb_step(h, args.steps) == 0
        assert L.clb_macros(h, *[dp(o) for o in outs]) == 0
        nuv = ctypes.c_double()
        assert L.clb_nusselt(h, 0, ctypes.byref(nuv)) == 0
        L.clb_destroy(h)
        te = time.perf_counter() - t0
        barrier()
        te = max_over_ranks(te, dist)
        e2e = {"value": whole_job_mlups(cells, args.steps, ws, te), "unit": UNIT,
               "h2d_bytes_per_step": phi.nbytes / args.steps,
               "d2h_bytes_per_step": (4 * cells * 8 + 8) / args.steps,
               "includes": "clb_init (allocation + porosity upload) + steps + clb_macros + clb_nusselt"}

    if rank != 0:
        return
    peaks, src = _peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    gbs = BYTES_PER_CCU_F64 * cells / per_launch / 1e9
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    fp64_peak = SMS * DFMA_PER_CLK_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    if args.precision != "f64":
        bpn = FORMS[args.precision][1]
        gb = bpn * cells / per_launch / 1e9
        tr = FORMS_DRAM_PER_NODE[args.precision]
        roof = {"bound": "hbm", "achieved": gb, "peak": hbm_peak, "unit": "GB/s", "frac": gb / hbm_peak,
                "traffic": tr * cells if tr else None, "kernel": f"k_step2<{args.precision}>",
                "bytes_per_ccu": bpn, "peak_source": f"{src} hbm_gbs"}
    else:
        ach = FP64_FLOP_PER_CCU * cells / per_launch / 1e12
        inst_rate = FP64_INST_PER_CCU * cells / per_launch
        inst_peak = SMS * DFMA_PER_CLK_PER_SM * sm_mhz * 1e6
        roof = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                "traffic": DRAM_BYTES_PER_CCU_MEASURED * cells,
                "kernel": "k_step<StoreF64, shift, forchheimer>", "flop_per_ccu": FP64_FLOP_PER_CCU,
                "peak_source": f"FP64 pipe: {SMS} SMs x {DFMA_PER_CLK_PER_SM} DFMA/clk x 2 flop x {sm_mhz:.0f} MHz "
                               "(median SM clock, timed region)",
                "fp64_pipe_frac": inst_rate / inst_peak,
                "hbm": {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                        "bytes_per_ccu": BYTES_PER_CCU_F64, "peak_source": f"{src} hbm_gbs"}}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "f64" else "f32 arithmetic, f16 storage", "data": "synthetic",
            "config": {"workload": f"{NX}x{NY} porous cavity, seeded GRF porosity, Ra 1e6, Da 1e-3, Pr 0.71, "
                                   f"sigma 1, {args.precision.upper()}",
                       "porosity": "0.3+0.6*Phi(g), g Gaussian random field l=32, seed 20211012",
                       "nx": NX, "ny": NY, "cells": cells, "replicas": ws,
                       "l2": f"state {NX * NY * 14 * 16 / 1e9:.2f} GB per replica (two buffers) vs 0.13 GB L2: "
                             "no flush",
                       "parallelism": f"replicas x{ws}", "nu_hot_wall_after": nu},
            "roofline": roof, "clocks": clocks, "gpu_launches": args.steps,
            "e2e": e2e}
    if ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_rate(phi)
        line["cpu_baseline_1core"] = cpu_oracle_rate(phi, budget_s=8.0, side=256, nthreads=1)
    if not args.no_forms:
        line["forms"] = reduced_precision_forms(clb, torch, args, hbm_peak, src)
    if not args.no_accuracy:
        # the literal precision workload (at 1000 steps its flow has barely
        # started: max |u| ~ 1e-4), and a 2048^2 one run until the flow is
        # developed
        line["accuracy"] = accuracy_forms(clb, torch, n=8192, steps=1000)
        line["accuracy_2048"] = accuracy_forms(clb, torch, n=2048, steps=30_000)
    if not args.no_batch:
        line["batch"] = batched_form(clb, torch, args, hbm_peak, src)
    if args.validate_batch:
        line["batch_validation"] = batch_validation(clb, torch)
    if not args.no_mrt:
        line["mrt_cost"] = mrt_cost(clb, torch)
        line["cavity64"] = cavity64(clb, torch)
    if not args.no_steady:
        line["steady_state"] = steady_state_forms(clb, torch)
    if not args.no_warm and ws == 1:
        line["warm_start"] = warm_start_form(clb, torch)
        line["surrogate_training"] = surrogate_training(torch, float(peaks.get("bf16_tflops", 1900.0)), src)
    line["summary"] = _summary(line)
    print(json.dumps(line), flush=True)


def _free_port() -> int:
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch_ranks(gpus: int, argv) -> int:
    """Run this script on `gpus` local ranks under torch.distributed.run
    (one process per GPU, rendezvous on 127.0.0.1); returns its exit code."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.abspath(__file__)] + list(argv)
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-steady", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP16-storage forms at 8192^2")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the FP16-vs-FP64 accuracy run at 8192^2")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-case batch")
    ap.add_argument("--no-mrt", action="store_true", help="skip the MRT cost ratio and the 64^2 cavity")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm-start comparison")
    ap.add_argument("--batch-cases", type=int, default=512,
                    help="cavities in the batch section (default 512, the workload; fewer for profiling)")
    ap.add_argument("--no-batch-check", action="store_true", help="skip the 8-case Nusselt check of the batch")
    ap.add_argument("--validate-batch", action="store_true",
                    help="add the stratified 64-case steady-state Nusselt validation of the batch (minutes)")
    ap.add_argument("--size", type=int, default=4096, help="grid side (default 4096; smaller for profiling)")
    ap.add_argument("--precision", choices=("f64", "f16s", "f16n"), default="f64",
                    help="storage form of the main measurement (default f64, the reported workload)")
    args = ap.parse_args()
    global NX, NY
    NX = NY = args.size
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.gpus < 1:
        ap.error("--gpus must be >= 1")
    ws = os.environ.get("WORLD_SIZE")
    if ws is None:
        if args.gpus > 1:
            raise SystemExit(launch_ranks(args.gpus, sys.argv[1:]))
    elif int(ws) != args.gpus:
        raise SystemExit(f"bench.py: --gpus {args.gpus} but the launcher started WORLD_SIZE={ws} ranks")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
