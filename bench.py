#!/usr/bin/env python
"""Benchmark of the octree FMM gravity solve (Sec. 2.2) on GB300.

Headline workload: the 7-level AMR binary of two n = 3/2 polytropes (mass ratio 0.6, radii 0.1
and 0.085, separation 0.3, density floor 1e-10 of the peak, subgrids refined where the density
exceeds 1e-4 of the peak: 30,089 subgrids, 13,479,936 leaf cells), theta = 0.5, angular-momentum
correction on.  One step = one whole solve (multipoles up, multipole interactions and near field,
expansions down, net force and torque) on that step's density rho0 (1 + 1e-3 u_k), the per-step
re-solve of an evolving star with the tree held fixed.

Metric: directed cell-cell multipole interactions per second (direct near-field pairs are
reported separately), and ms per solve, for the FP64 path (`value`), the mixed FP32/FP64 path
(`mixed`) and the double-float path (`df64`), each with its error against the FP64 path on the same
input.  Beside it: the 0.9M-cell 5-level binary (`small`: the three paths, the mixed path's errors
and residual torque at theta 0.35 / 0.5 / 0.7, the time-derivative solve, the binary diagnostics),
the 64-tree forest (`batched`) and the 9-level merger binary at theta = 0.34 (`paper_binary`).
The rooflines divide by FMA rates measured on the same GPU in the same run
(fmm_measure_fma_rate).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own replica of the workload (independent trees, no
collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

THETA = 0.5
# the headline workload: the 7-level binary (the largest single-GPU configuration)
BIG = {"levels": 7, "q": 0.6, "a": 0.3}
WORKLOAD = ("AMR binary: two n=3/2 polytropes, q=0.6, R=0.1/0.085, a=0.3, floor 1e-10 (density "
            "contrast 1e10), refine where rho > 1e-4 rho_peak, 7 levels, theta=0.5, AMC on; each "
            "step solves rho0 (1 + 1e-3 u_k), u_k ~ U[-1, 1] per cell, seed 20210120 + k")
# the 0.9M-cell binary: FP64, mixed at three opening angles, the time derivative, diagnostics
SMALL = {"levels": 5, "q": 0.7, "a": 0.35}
SMALL_WORKLOAD = ("AMR binary: two n=3/2 polytropes, q=0.7, R=0.1/0.085, a=0.35, floor 1e-10, "
                  "refine where rho > 1e-4 rho_peak, 5 levels, theta=0.5, AMC on")
METRIC = "FMM cell-cell interactions/s (directed M2L pairs) and gravity-solve ms per solve"


def big_workload(synth):
    return synth.workload_binary(BIG["levels"], q=BIG["q"], a=BIG["a"])


def small_workload(synth):
    return synth.workload_binary(SMALL["levels"], q=SMALL["q"], a=SMALL["a"])


# Algorithmic flops per directed interaction, counted from the kernels' formulas (an FMA counts
# 2, a multiply or add 1, a reciprocal square root 1).  Same-level leaf pairs (multipole or
# direct) are two point masses at cell centres: 4 FMAs against tabulated 1/|d| and d/|d|^3.
# Direct pairs across a level jump evaluate the point-mass field from the separation.  A refined
# source adds its detraced 2nd and 3rd moments; a refined target adds the 12 independent
# components of the 2nd and 3rd derivatives of its expansion; the correction contracts the 4th
# derivative with detraced 3rd moments.
FLOPS = {"m2l_leaf_leaf": 8, "p2p_same": 8, "p2p_mixed": 26, "m2l_leaf_refined": 126,
         "m2l_refined_leaf": 142, "m2l_refined_refined": 231}
# which interaction kernel evaluates which pairs
KERNEL_PAIRS = {"k_m2l_ref": ("m2l_refined_leaf", "m2l_refined_refined", "m2l_leaf_refined",
                              "p2p_mixed"),
                "k_m2l_leaf": ("m2l_leaf_leaf", "p2p_same"),
                # mixed path: refined targets of levels >= 1 (the root level stays with the root
                # and boundary blocks, so its pairs are taken off this kernel's count)
                "k_m2l_stage": ("m2l_refined_leaf", "m2l_refined_refined")}
def root_pairs(theta):
    """Directed well-separated pairs among the 512 cells of a refined root: the root level's
    share of the refined-pair count."""
    d = np.arange(-7, 8)
    d2 = (d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2)
    mult = (8 - np.abs(d))[:, None, None] * (8 - np.abs(d))[None, :, None] * (8 - np.abs(d))[None, None, :]
    ws = (1.0 / np.sqrt(np.maximum(d2, 1)) < theta) & (d2 > 0)
    return int((mult * ws).sum())


# nominal rates (152 SMs, 2 FP64 or 128 FP32 FMA per clock per SM, 2.07 GHz), context only: the
# rooflines divide by the rates fmm_measure_fma_rate measures
SMS = 152
SM_MAX_GHZ = 2.07
NOMINAL_TFLOPS = {64: SMS * 2 * 2 * SM_MAX_GHZ / 1e3, 32: SMS * 128 * 2 * SM_MAX_GHZ / 1e3}


def measured_traffic(workload: str):
    """Per-launch DRAM bytes of the interaction kernels on one workload from the committed ncu
    summary, if the kernel sources are the ones it was captured from (else nothing: the counters
    are stale).  Lines: `workload kernel read_bytes write_bytes`."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(here, "paper_2101_08226_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("fmm.cu", "fmm_kernels.cuh", "dfloat.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    out, sha = {}, None
    try:
        with open(os.path.join(here, "profiles", "dram_traffic.txt")) as fh:
            for line in fh:
                parts = line.split()
                if not parts or parts[0].startswith("#"):
                    continue
                if parts[0] == "sha256":
                    sha = parts[1]
                elif parts[0] == workload and len(parts) == 4:
                    out[parts[1]] = int(parts[2]) + int(parts[3])
    except OSError:
        return {}
    return out if sha == h.hexdigest() else {}


def reduce_max(x: float, dist, world: int, device) -> float:
    """The maximum of x over all ranks (the job is as slow as its slowest replica)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank: int, step: int) -> int:
    """Seed of the density perturbation of one step of one rank's replica."""
    return rank * 1000 + step


def whole_job_rate(world: int, units_per_step: float, steps: int, max_total_ms: float) -> float:
    """Units processed by all ranks (independent replicas, equal work) per second of the slowest
    rank's timed region."""
    return world * units_per_step * steps / (max_total_ms * 1e-3)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    def __init__(self, dev_uuid):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", dev_uuid, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], None, set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_flops(counts):
    return sum(FLOPS[k] * v for k, v in counts.items())


def measure_paper_binary(tree_api, synth, torch, dev, stream, steps, flush, graded=False):
    """The merger binary in the paper's proportions (9 levels, theta = 0.34, 2.07M leaf cells):
    the same metric on the paper's deepest tree and smallest opening angle.  graded: the same
    binary refined by the mass-based reading of the density criterion (one level per factor 8 in
    density below rho_peak / 8; leaves on every level from 2 to 9)."""
    w = (synth.workload_paper_binary(graded=True, refine_frac=0.125) if graded
         else synth.workload_paper_binary())
    t = tree_api.Tree(w.max_level, w.flags)
    n_sub, n_leaf_sub, _ = t.info()
    rho0 = synth.leaf_density(w.field, t.leaves())
    floor = w.field.floor * w.field.rho_peak
    rhos = [torch.from_numpy(synth.perturbed_density(rho0, 500 + k, floor_value=floor)).to(dev)
            for k in range(steps + 2)]
    counts = t.counts_by_type(w.theta)
    n_m2l = sum(v for k, v in counts.items() if k.startswith("m2l"))
    rule = ("graded refinement: level 9 above rho_peak/8, one level less per factor 8 in density"
            if graded else "refine_frac 1e-4")
    out = {"workload": "merger binary in the paper's proportions: q=0.5, accretor 50 finest cells "
                       f"across, donor filling its Roche lobe, a=0.024 of the box, 9 levels, {rule}, "
                       "theta=0.34",
           "subgrids": n_sub, "leaf_cells": n_leaf_sub * 512, "m2l_pairs": n_m2l,
           "pair_types": counts, "l2": "flushed before every timed solve"}
    for precision in ("fp64", "mixed"):
        for k in range(2):
            t.solve(rhos[k], w.theta, precision, True, stream=stream, check_status=False)
        torch.cuda.synchronize()
        ms = []
        for k in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t.solve(rhos[2 + k], w.theta, precision, True, stream=stream, check_status=False)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        t.sync_status(stream)
        tm = float(np.mean(ms))
        out[precision] = {"value": n_m2l / (tm * 1e-3), "ms_per_solve": tm,
                          "gpu_launches": t.last_launches()}
    out["unit"] = "interactions/s"
    t.close()
    return out


def measure_binary6(tree_api, synth, torch, dev, stream, steps, flush):
    """The 5-level binary's field refined one level deeper (6 levels, about 2M leaf cells): the
    size between the 0.9M-cell and the 13.5M-cell binaries, FP64 and mixed (autotuned)."""
    w = synth.workload_binary(6, q=SMALL["q"], a=SMALL["a"])
    t = tree_api.Tree(w.max_level, w.flags)
    n_sub, n_leaf_sub, _ = t.info()
    rho0 = synth.leaf_density(w.field, t.leaves())
    floor = w.field.floor * w.field.rho_peak
    rhos = [torch.from_numpy(synth.perturbed_density(rho0, 600 + k, floor_value=floor)).to(dev)
            for k in range(steps + 2)]
    counts = t.counts_by_type(THETA)
    n_m2l = sum(v for k, v in counts.items() if k.startswith("m2l"))
    out = {"workload": SMALL_WORKLOAD.replace("5 levels", "6 levels"), "subgrids": n_sub,
           "leaf_cells": n_leaf_sub * 512, "m2l_pairs": n_m2l, "l2": "flushed before every timed solve"}
    v, _, _, _ = t.autotune(rhos[0], THETA, "mixed", reps=3, stream=stream)
    out["mixed_variant"] = int(v)
    for precision in ("fp64", "mixed"):
        for k in range(2):
            t.solve(rhos[k], THETA, precision, True, stream=stream, check_status=False)
        torch.cuda.synchronize()
        ms = []
        for k in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t.solve(rhos[2 + k], THETA, precision, True, stream=stream, check_status=False)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        t.sync_status(stream)
        tm = float(np.mean(ms))
        out[precision] = {"value": n_m2l / (tm * 1e-3), "ms_per_solve": tm,
                          "gpu_launches": t.last_launches()}
    out["unit"] = "interactions/s"
    t.close()
    return out


def measure_batched(tree_api, synth, torch, dev, stream, steps, timer):
    """The 64 seeded trees of uneven depth (levels 2..5, single stars or binaries) as one forest:
    every level of every tree in one set of launches, replayed as one CUDA graph, the mixed path's
    launch variant chosen by the autotuner.  Same metric as the headline."""
    ws = synth.batched_workloads(64)
    trees = [tree_api.Tree(w.max_level, w.flags) for w in ws]
    f = tree_api.Forest(trees)
    n_sub, n_leaf_sub, _ = f.info()
    rho = torch.from_numpy(np.concatenate([synth.leaf_density(w.field, t.leaves())
                                           for w, t in zip(ws, trees)])).to(dev)
    counts = f.counts(THETA)
    out = {"workload": "64 independent trees, levels 2-5, single n=3/2 polytropes or binaries "
                       "(q ~ U[0.3,1], a ~ U[0.25,0.5]), seeds 20210120+t, theta=0.5",
           "subgrids": n_sub, "leaf_cells": n_leaf_sub * 512, "m2l_pairs": counts["m2l"],
           "p2p_pairs": counts["p2p_same"] + counts["p2p_mixed"]}
    # the autotuner picks the forest's mixed launch variant (untimed)
    v, _, _, _ = f.autotune(rho, THETA, "mixed", reps=3, stream=stream)
    out["mixed_variant"] = int(v)
    for precision in ("fp64", "mixed"):
        for _ in range(2):
            f.solve(rho, THETA, precision, True, stream=stream, check_status=False)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f.solve(rho, THETA, precision, True, stream=stream, check_status=False)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        f.sync_status(stream)
        t = float(np.mean(ms))
        out[precision] = {"value": counts["m2l"] / (t * 1e-3), "ms_per_solve": t,
                          "gpu_launches": f.last_launches()}
    out["unit"] = "interactions/s"
    out["persistent_level_passes"] = persistent_vs_launches(timer, f, [rho], ("fp64", "mixed"), steps)
    f.close()
    for t in trees:
        t.close()
    return out


def cpu_model():
    """The host CPU's name as the OS reports it (x86: "model name"; Arm: implementer/part ids)."""
    try:
        fields = {}
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip(), v.strip())
        if "model name" in fields:
            return fields["model name"]
        if "CPU part" in fields:
            return f"Arm implementer {fields.get('CPU implementer', '?')} part {fields['CPU part']}"
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(seconds_target=20.0):
    """The oracle, as it stands, on a bounded sample of the headline workload: phi and g at
    randomly chosen leaf cells, each with its ancestors' expansions and its direct sums.  A call
    has a fixed cost (the oracle's moments of every cell, from their definition) and a cost per
    sampled cell; two probe calls size the timed sample to about `seconds_target`."""
    import oracle as O
    from paper_2101_08226_gb300 import synth
    w = big_workload(synth)
    t = O.Tree(w.max_level, w.flags)
    rho = synth.leaf_density(w.field, t.leaves())
    rng = np.random.default_rng(20210120)

    def run(ns):
        idx = rng.choice(rho.size, ns, replace=False)
        t0 = time.perf_counter()
        _, _, c = O.sample(t, rho, THETA, idx, with_counts=True)
        return time.perf_counter() - t0, c

    n0, n1 = 256, 4096
    d0, _ = run(n0)
    d1, c = run(n1)
    ns, dt = n1, d1
    per_cell = max((d1 - d0) / (n1 - n0), 1e-6)
    if d1 < 0.5 * seconds_target:
        ns = int(min(rho.size // 2, max(n1, (seconds_target - (d0 - n0 * per_cell)) / per_cell)))
        dt, c = run(ns)
    return {"value": c["m2l"] / dt, "unit": "interactions/s", "cores": O.max_threads(),
            "cpu": cpu_model(), "kind": "oracle",
            "sample": f"{ns} random leaf cells of the 13.5M-cell headline tree (their own and their "
                      f"ancestors' {c['m2l']} multipole interactions and "
                      f"{c['p2p_same'] + c['p2p_mixed']} direct pairs), {dt:.1f} s including the "
                      "oracle's moments of every cell"}


def run_reference(args):
    """The oracle on the headline workload: each step evaluates a bounded sample of leaf cells
    (a fresh random set of 16,384 per step, about 3 s on 16 cores, the oracle's moments of every
    cell included) on the host cores; value = multipole interactions / s."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle as O
    from paper_2101_08226_gb300 import synth
    w = big_workload(synth)
    t = O.Tree(w.max_level, w.flags)
    rho0 = synth.leaf_density(w.field, t.leaves())
    floor = w.field.floor * w.field.rho_peak
    rng = np.random.default_rng(7)
    ns = 16384
    times = []
    total_m2l = 0
    for step in range(args.warmup + args.steps):
        rho = synth.perturbed_density(rho0, replica_seed(0, step), floor_value=floor)
        idx = rng.choice(rho.size, ns, replace=False)
        t0 = time.perf_counter()
        _, _, c = O.sample(t, rho, THETA, idx, with_counts=True)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            total_m2l += c["m2l"]
    value = total_m2l / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "levels": BIG["levels"], "theta": THETA},
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": O.max_threads(),
                             "cpu": cpu_model(),
                             "kind": "oracle",
                             "sample": f"each step: {ns} random leaf cells of the 13.5M-cell tree, "
                                       "the step's perturbed density"},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_solve_only(args):
    """Profiling driver: one workload's tree, `--warmup` untimed solves then `--steps` more in the
    given precision (graph-replayed, as in the timed run), nothing else -- a small, fixed launch
    sequence to run under ncu."""
    import torch
    from paper_2101_08226_gb300 import api, build, synth
    build.build()
    theta = THETA
    if args.solve_workload == "paper9":
        w = synth.workload_paper_binary()
        theta = w.theta
    elif args.solve_workload == "binary7":
        w = big_workload(synth)
    elif args.solve_workload == "binary6":
        w = synth.workload_binary(6, q=SMALL["q"], a=SMALL["a"])
    elif args.solve_workload != "forest64":
        w = small_workload(synth)
    if args.solve_workload == "forest64":  # the 64 seeded trees of uneven depth as one forest
        ws = synth.batched_workloads(64)
        trees = [api.Tree(x.max_level, x.flags) for x in ws]
        tree = api.Forest(trees)
        rho = torch.from_numpy(np.concatenate([synth.leaf_density(x.field, t.leaves())
                                               for x, t in zip(ws, trees)])).cuda()
    else:
        tree = api.Tree(w.max_level, w.flags)
        rho = torch.from_numpy(synth.leaf_density(w.field, tree.leaves())).cuda()
    if args.variant is not None:
        tree.set_variant(theta, args.variant)
    for _ in range(args.warmup + args.steps):
        phi, g, net = tree.solve(rho, theta, args.solve_only, True)
    torch.cuda.synchronize()
    print(json.dumps({"solve_only": args.solve_only, "workload": args.solve_workload,
                      "solves": args.warmup + args.steps,
                      "launches_per_solve": tree.last_launches(), "net": net.cpu().tolist()}))


class Timer:
    """Times whole solves of one tree on one stream with CUDA events, after W untimed solves, an
    L2 flush (a 256 MiB write, larger than the 129 MB L2) before each timed one, and the library's
    per-phase events recorded inside the solve's graph."""

    def __init__(self, torch, dist, world, dev, stream):
        self.torch, self.dist, self.world, self.dev, self.stream = torch, dist, world, dev, stream
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def solves(self, tree, rhos, theta, precision, warmup, steps, out, call=None):
        torch = self.torch
        call = call or (lambda r: tree.solve(r, theta, precision, True, *out, self.stream,
                                             check_status=False))
        tree.set_profiling(True)
        for k in range(warmup):
            call(rhos[k % len(rhos)])
        torch.cuda.synchronize()
        tree.sync_status(self.stream)
        if self.world > 1:
            self.dist.barrier()
        torch.cuda.synchronize()
        step_ms, phases = [], []
        for k in range(warmup, warmup + steps):
            self.flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            call(rhos[k % len(rhos)])
            e1.record(self.stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            phases.append(tree.phase_times())
        torch.cuda.synchronize()
        tree.sync_status(self.stream)
        tree.set_profiling(False)
        total = reduce_max(float(np.sum(step_ms)), self.dist, self.world, self.dev)
        return {"total_ms": total, "step_ms": step_ms, "phases": np.mean(np.array(phases), axis=0),
                "launches": tree.last_launches() * steps}


def persistent_vs_launches(timer, tree, rhos, precisions, steps):
    """ms per solve with the level passes (upward octant phases, downward level phases) as one
    launch per phase and as one persistent, level-ordered launch per direction
    (fmm_set_persistent): the same inputs, flushes and events."""
    res = {}
    for precision in precisions:
        row = {}
        for name, on in (("per_phase_launches", False), ("persistent", True)):
            tree.set_persistent(on)
            r = timer.solves(tree, rhos, THETA, precision, 2, steps, None,
                             call=lambda x: tree.solve(x, THETA, precision, True, stream=timer.stream,
                                                       check_status=False))
            row[name] = {"ms_per_solve": r["total_ms"] / steps, "gpu_launches": tree.last_launches(),
                         "upward_ms": float(r["phases"][0]), "downward_ms": float(r["phases"][2])}
        res[precision] = row
    tree.set_persistent(False)
    return res


def kernel_flops_of(counts, depth):
    kf = {k: sum(FLOPS[c] * counts[c] for c in cs) for k, cs in KERNEL_PAIRS.items()}
    if depth > 0:
        kf["k_m2l_stage"] -= FLOPS["m2l_refined_refined"] * root_pairs(THETA)
    return kf


def roofline(ph, precision, kernel_flops, peaks, traffic, variant=0):
    """The dominant interaction kernel of this precision, timed with CUDA events on the stream it
    runs on, inside the timed region: FP64 / df64, the general kernel (refined and boundary
    targets, root) or the leaf kernel; mixed, the refined targets' staging kernel (that of the
    tree's launch variant: k_m2l_stage_pipe for r = 3)."""
    if precision == "mixed" and float(ph[6]) > 0:
        ms = {"k_m2l_stage": float(ph[6]), "k_m2l_leaf": float(ph[5])}
        k = "k_m2l_stage"
    else:
        ms = {"k_m2l_ref": float(ph[4]), "k_m2l_leaf": float(ph[5])}
        k = max(ms, key=ms.get)
    bits = 64 if precision == "fp64" else 32
    ach = kernel_flops[k] / (ms[k] * 1e-3) / 1e12
    tname = {"fp64": "double", "df64": "dfloat", "mixed": "float"}[precision]
    kname = k if k == "k_m2l_stage" else f"{k}<{tname}>"
    if k == "k_m2l_stage" and variant % 4 == 3:
        kname = "k_m2l_stage_pipe"
    if precision == "mixed" and k == "k_m2l_ref":
        kname = "k_m2l_ref<float> or k_m2l_split<float> + k_m2l_stage (one stream)"
    peak = peaks[bits]
    how = f"FP{bits} FMA rate"
    if bits == 32 and peaks.get(-32, 0.0) > peak:  # packed FP32 pairs retire FMAs faster
        peak, how = peaks[-32], "FP32 FMA rate in packed pairs (fma.rn.f32x2)"
    return {"bound": "alu", "kernel": kname, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": traffic.get(kname),
            "traffic_unit": "DRAM bytes per launch (ncu)",
            "kernel_ms": ms[k], "kernel_flops": kernel_flops[k],
            "other_kernel_ms": {kk: v for kk, v in ms.items() if kk != k},
            "peak_source": f"measured: {how}, fmm_measure_fma_rate on this GPU in this "
                           "run (2 flops per FMA)",
            "frac_of_nominal": ach / NOMINAL_TFLOPS[bits]}


def phases_of(ph, precision="fp64"):
    out = {"upward": float(ph[0]), "interactions": float(ph[1]), "downward": float(ph[2]),
           "reductions": float(ph[3])}
    # the leaf kernel runs on the tree's second stream from the end of the first upward step (it
    # overlaps "upward"); "after_leaf_kernel" runs from its end to the end of the interactions
    if precision == "mixed":
        out.update({"k_m2l_leaf": float(ph[5]), "after_leaf_kernel": float(ph[4]),
                    "k_m2l_stage": float(ph[6])})
    else:
        out.update({"k_m2l_ref": float(ph[4]), "k_m2l_leaf": float(ph[5])})
    return out


def field_errors(torch, phi, g, net, phi64, g64, net64, m):
    """Errors of a solve against the FP64 path's solve of the same input: infinity norms over the
    largest reference value, mass-weighted RMS of the per-cell relative error, the worst per-cell
    relative error with a floor of 1e-3 of the largest value, and net force and torque over the
    normalisation S."""
    gn = g64.norm(dim=1)
    wgt = m / m.sum()
    dg = (g - g64).norm(dim=1)
    dphi = (phi - phi64).abs()
    return {
        "g_inf_rel": float(((g - g64).abs().max() / g64.abs().max()).item()),
        "g_rms_mass_weighted": float(torch.sqrt((wgt * (dg / gn) ** 2).sum()).item()),
        "g_max_cell_rel_floor1e-3": float((dg / torch.clamp(gn, min=1e-3 * float(gn.max()))).max().item()),
        "phi_inf_rel": float((dphi.max() / phi64.abs().max()).item()),
        "phi_rms_mass_weighted": float(torch.sqrt((wgt * (dphi / phi64.abs()) ** 2).sum()).item()),
        "phi_max_cell_rel": float((dphi / phi64.abs()).max().item()),
        "force_over_norm": float((net[:3].abs().max() / net[6]).item()),
        "torque_over_norm": float((net[3:6].abs().max() / net[6]).item()),
        "force_over_norm_fp64": float((net64[:3].abs().max() / net64[6]).item()),
        "torque_over_norm_fp64": float((net64[3:6].abs().max() / net64[6]).item()),
    }


def leaf_mass(torch, tree, rho):
    dx3 = np.repeat(1.0 / (8 * 2.0 ** tree.leaves()[:, 0]) ** 3, 512)
    return rho * torch.from_numpy(dx3).to(rho.device)


def measure_scf(api, synth, torch, timer, dev, n_iter=10):
    """The self-consistent-field construction of the binary (Sec. 4.1) on the device: the
    5-level starting model (two equal-K n = 3/2 polytropes, q = 0.5, a = 0.45), fmm_scf_init and
    n_iter iterations (each: mass scaling, a gravity solve, L1, C1, C2, K, the new density), timed
    with CUDA events around the iterations, FP64 and mixed solves."""
    w = synth.workload_scf_binary(5)
    tree = api.Tree(w.max_level, w.flags)
    params, rho0, K0 = synth.scf_inputs(w, tree.leaves())
    out = {"workload": "SCF binary: n=3/2, q=0.5, accretor radius 0.1, donor 0.126 (equal K), "
                       "a0=0.45, f=0.8385, 5 levels, theta=0.5", "leaf_cells": int(rho0.size),
           "iterations": n_iter}
    for precision in ("fp64", "mixed"):
        p = dict(params, precision=precision)
        rho = torch.from_numpy(rho0.copy()).to(dev)
        tree.scf_init(p, rho, K0, stream=timer.stream)
        tree.scf_iterate(p, rho, 1, stream=timer.stream)  # captures the solve's graph
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(timer.stream)
        st, hist, _, _ = tree.scf_iterate(p, rho, n_iter, stream=timer.stream)
        e1.record(timer.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        dK = abs(hist[-1][0] / hist[-2][0] - 1.0) if n_iter > 1 else None
        out[precision] = {"ms_per_iteration": ms / n_iter, "K": st["K"], "Omega": st["Omega"],
                          "last_relative_change_of_K": dK,
                          "kepler_omega2_a3_over_M": st["Omega"] ** 2 * st["a"] ** 3 /
                          (params["M1"] + params["M2"])}
    tree.close()
    return out


def measure_small(api, synth, torch, timer, dev, steps, peaks, rank):
    """The 0.9M-cell 5-level binary: the three paths; the mixed path's errors and residual
    torque against the FP64 path at theta = 0.35, 0.5, 0.7; the time-derivative solve; the
    binary diagnostics."""
    stream = timer.stream
    w = small_workload(synth)
    tree = api.Tree(w.max_level, w.flags)
    n_sub, n_leaf_sub, depth = tree.info()
    n = n_leaf_sub * 512
    rho0 = synth.leaf_density(w.field, tree.leaves())
    floor = w.field.floor * w.field.rho_peak
    rhos = [torch.from_numpy(synth.perturbed_density(rho0, replica_seed(rank, k), floor_value=floor)).to(dev)
            for k in range(3 + steps)]
    counts = tree.counts_by_type(THETA)
    n_m2l = sum(v for k, v in counts.items() if k.startswith("m2l"))
    kflops = kernel_flops_of(counts, depth)
    traffic = measured_traffic("binary_q0.7_L5")
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    g = torch.empty((n, 3), dtype=torch.float64, device=dev)
    net = torch.empty(7, dtype=torch.float64, device=dev)
    out = {"workload": SMALL_WORKLOAD, "subgrids": n_sub, "leaf_cells": n, "m2l_pairs": n_m2l,
           "pair_types": counts, "unit": "interactions/s"}
    # tuned in the configuration the timer runs (per-phase events on), which moves kernels a little
    tree.set_profiling(True)
    variant, tuned_ms, _, _ = tree.autotune(rhos[0], THETA, "mixed", reps=3, stream=stream)
    tree.set_profiling(False)
    out["mixed_variant"] = int(variant)
    out["autotune_median_ms"] = {str(v): round(float(x), 4) for v, x in enumerate(tuned_ms) if x > 0}
    for precision in ("fp64", "mixed", "df64"):
        r = timer.solves(tree, rhos, THETA, precision, 3, steps, (phi, g, net))
        tm = r["total_ms"] / steps
        out[precision] = {"value": n_m2l / (tm * 1e-3), "ms_per_solve": tm,
                          "roofline": roofline(r["phases"], precision, kflops, peaks, traffic,
                                               variant),
                          "phases_ms": phases_of(r["phases"], precision),
                          "gpu_launches": tree.last_launches()}
    out["persistent_level_passes"] = persistent_vs_launches(timer, tree, rhos, ("fp64", "mixed"),
                                                            min(steps, 10))
    # the default launch variant, timed the same way, beside the tuner's choice (on every rank,
    # whatever each rank's tuner chose: the timer synchronises the ranks)
    tree.set_variant(THETA, 0)
    r = timer.solves(tree, rhos, THETA, "mixed", 3, steps, (phi, g, net))
    out["mixed"]["ms_per_solve_variant_0"] = r["total_ms"] / steps
    tree.set_variant(THETA, variant)
    # the mixed path against the FP64 path at the three opening angles (the same input)
    m = leaf_mass(torch, tree, rhos[0])
    sweep = {}
    for theta in (0.35, 0.5, 0.7):
        phi64, g64, net64 = tree.solve(rhos[0], theta, "fp64", True, stream=stream)
        phi32, g32, net32 = tree.solve(rhos[0], theta, "mixed", True, stream=stream)
        c = tree.counts(theta)
        sweep[str(theta)] = dict(field_errors(torch, phi32, g32, net32, phi64, g64, net64, m),
                                 m2l_pairs=c["m2l"])
    out["mixed_vs_fp64_by_theta"] = sweep
    # the time-derivative solve: rho and d rho / dt in one call (Sec. 2.1)
    rhodot = torch.from_numpy(rho0 * np.random.default_rng(31).uniform(-1.0, 1.0, rho0.size)).to(dev)
    phidot = torch.empty(n, dtype=torch.float64, device=dev)
    dt_out = {"what": "fmm_solve_dt: the rho solve plus dphi/dt (same operator, source with a "
                      "dipole); d rho/dt = rho u, u ~ U[-1, 1]"}
    for precision in ("fp64", "mixed"):
        r = timer.solves(tree, rhos, THETA, precision, 2, min(steps, 5), None,
                         call=lambda x: tree.solve_dt(x, rhodot, THETA, precision, True, phi, g,
                                                      phidot, net, stream, check_status=False))
        tm = r["total_ms"] / min(steps, 5)
        base = out[precision]["ms_per_solve"]
        dt_out[precision] = {"ms_per_solve": tm, "ms_rho_solve_alone": base,
                             "added_ms_for_dphi_dt": tm - base, "ratio_to_rho_solve": tm / base,
                             "gpu_launches": tree.last_launches()}
    out["dphi_dt"] = dt_out
    # binary diagnostics (Sec. 4): five passes of the fixed-point iteration on the device
    s1, s2 = w.field.stars
    sep = float(np.linalg.norm(np.subtract(s2.center, s1.center)))
    _, g, _ = tree.solve(rhos[-1], THETA, "fp64", True, stream=stream)
    diag_ms = []
    for k in range(2 + min(steps, 5)):
        timer.flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sums, _, _, _ = tree.binary_iterate(rhos[-1], g, (1.7 / sep ** 3) ** 0.5, s1.center,
                                            s2.center, 5, stream=stream)
        e1.record(stream)
        e1.synchronize()
        if k >= 2:
            diag_ms.append(e0.elapsed_time(e1))
    tdiag = float(np.mean(diag_ms))
    out["binary_diagnostics"] = {
        "what": "fmm_binary_iterate: 5 passes of star membership by the effective acceleration "
                "and per-star M, sum m x, F, T, each pass's centres and critical radii computed on "
                "the device from the previous pass",
        "ms_per_iteration_of_5_passes": tdiag, "leaf_cells": n,
        "input_gb_per_s": 5 * 32 * n / (tdiag * 1e-3) / 1e9,
        "stars": [{"M": float(r[0]), "cells": int(r[10])} for r in sums]}
    tree.close()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    from paper_2101_08226_gb300 import api, build, synth
    build.build()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    timer = Timer(torch, dist, world, dev, stream)

    # roofline denominators, measured on this GPU
    peaks, peak_ms = {}, {}
    for bits in (64, 32, -32):  # -32: FP32 in packed pairs
        peaks[bits], peak_ms[bits] = api.measure_fma_rate(bits, 5, stream=stream)

    w = big_workload(synth)
    tree = api.Tree(w.max_level, w.flags)
    n_sub, n_leaf_sub, depth = tree.info()
    n = n_leaf_sub * 512
    rho0 = synth.leaf_density(w.field, tree.leaves())
    counts = tree.counts_by_type(THETA)
    n_m2l = sum(v for k, v in counts.items() if k.startswith("m2l"))
    kflops = kernel_flops_of(counts, depth)
    floor = w.field.floor * w.field.rho_peak
    n_steps = args.warmup + args.steps
    rhos = [torch.from_numpy(synth.perturbed_density(rho0, replica_seed(rank, k), floor_value=floor)).to(dev)
            for k in range(n_steps)]
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    g = torch.empty((n, 3), dtype=torch.float64, device=dev)
    net = torch.empty(7, dtype=torch.float64, device=dev)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    traffic = measured_traffic("binary_q0.6_L7")

    # the library's autotuner picks the mixed path's launch variant for this tree (untimed)
    # (tuned with the per-phase events on, as the timed solves run)
    tree.set_profiling(True)
    tuned_variant, tuned_ms, _, _ = tree.autotune(rhos[0], THETA, "mixed", reps=3, stream=stream)
    tree.set_profiling(False)
    sampler = ClockSampler(uuid) if (uuid and rank == 0) else None
    r64 = timer.solves(tree, rhos, THETA, "fp64", args.warmup, args.steps, (phi, g, net))
    phi64, g64, net64 = phi.clone(), g.clone(), net.clone()
    r32 = timer.solves(tree, rhos, THETA, "mixed", args.warmup, args.steps, (phi, g, net))
    err32 = field_errors(torch, phi, g, net, phi64, g64, net64, leaf_mass(torch, tree, rhos[-1]))
    rdf = timer.solves(tree, rhos, THETA, "df64", args.warmup, args.steps, (phi, g, net))
    errdf = field_errors(torch, phi, g, net, phi64, g64, net64, leaf_mass(torch, tree, rhos[-1]))
    # the same mixed solve with its kernels launched one by one instead of one graph replay
    tree.set_graphs(False)
    r32d = timer.solves(tree, rhos, THETA, "mixed", 1, min(args.steps, 5), (phi, g, net))
    tree.set_graphs(True)
    pers = persistent_vs_launches(timer, tree, rhos, ("fp64", "mixed"), min(args.steps, 5))
    clocks = sampler.stop() if sampler else None

    # end to end through the C ABI with pinned host buffers, copies inside the timed region: every
    # step copies its density in and its phi, g and net sums out; the pipelined entry point
    # overlaps one step's copies with the neighbouring steps' solves
    rho_h = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
    for k in range(2):
        rho_h[k].copy_(rhos[-1 - k].cpu())
    phi_h = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(2)]
    g_h = [torch.empty((n, 3), dtype=torch.float64).pin_memory() for _ in range(2)]
    net_h = [torch.empty(7, dtype=torch.float64).pin_memory() for _ in range(2)]

    def host_steps(count):
        for k in range(count):
            tree.solve_host_async(rho_h[k % 2].numpy(), THETA, "fp64", phi_h[k % 2].numpy(),
                                  g_h[k % 2].numpy(), net_h[k % 2].numpy(), stream=stream)
        tree.sync_status(stream)

    host_steps(2)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    host_steps(args.steps)
    e2e_s = reduce_max(time.perf_counter() - t0, dist, world, dev)
    # the synchronous entry point (one step's copies, solve, copies back, then the next step)
    t0 = time.perf_counter()
    for k in range(min(args.steps, 5)):
        tree.solve_host(rho_h[k % 2].numpy(), THETA, "fp64", True, phi_h[0].numpy(), g_h[0].numpy(),
                        net_h[0].numpy(), stream)
    e2e_sync_s = (time.perf_counter() - t0) / min(args.steps, 5)
    tree.close()
    del rhos, rho_h, phi, g, net, phi64, g64, net64
    torch.cuda.empty_cache()

    small = measure_small(api, synth, torch, timer, dev, min(args.steps, 10), peaks, rank)
    six = measure_binary6(api, synth, torch, dev, stream, min(args.steps, 5), timer.flush)
    batched = measure_batched(api, synth, torch, dev, stream, min(args.steps, 3), timer)
    paper = measure_paper_binary(api, synth, torch, dev, stream, min(args.steps, 3), timer.flush)
    graded = measure_paper_binary(api, synth, torch, dev, stream, min(args.steps, 3), timer.flush,
                                  graded=True)
    scf = measure_scf(api, synth, torch, timer, dev)
    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    cpu = cpu_baseline() if world == 1 else None
    t64, t32, tdf = r64["total_ms"], r32["total_ms"], rdf["total_ms"]

    def med(r):
        return float(np.median(r["step_ms"]))

    line = {
        "metric": METRIC, "value": whole_job_rate(world, n_m2l, args.steps, t64),
        "unit": "interactions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t64 / args.steps,
        "ms_per_step_median": med(r64),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "levels": BIG["levels"], "theta": THETA,
                   "subgrids": n_sub, "leaf_cells": n, "m2l_pairs": n_m2l,
                   "p2p_pairs": counts["p2p_same"], "p2p_mixed_pairs": counts["p2p_mixed"],
                   "pair_types": counts,
                   "l2": "flushed (256 MiB write) before every timed step; inputs and workspace "
                         "(about 10 GB) far larger than L2",
                   "launch": "one CUDA graph replay per step, after one pointer-table kernel",
                   "parallelism": f"{world} independent replicas"},
        "roofline": roofline(r64["phases"], "fp64", kflops, peaks, traffic),
        "phases_ms": phases_of(r64["phases"]),
        "mixed": {"value": whole_job_rate(world, n_m2l, args.steps, t32),
                  "ms_per_step": t32 / args.steps, "ms_per_step_median": med(r32),
                  "dtype": "f32 pairs, f64 rest", "speedup_vs_fp64": t64 / t32,
                  "err_vs_fp64": err32,
                  "roofline": roofline(r32["phases"], "mixed", kflops, peaks, traffic,
                                       tuned_variant),
                  "phases_ms": phases_of(r32["phases"], "mixed"),
                  "ms_per_step_direct_launches": r32d["total_ms"] / min(args.steps, 5),
                  "autotune": {"variant": int(tuned_variant),
                               "median_ms_per_variant": [round(float(x), 4) for x in tuned_ms],
                               "variants": "r + 4 l + 12 p + 24 c; r: refined targets 0 staged "
                                           "on a second stream, 1 staged on one stream, 2 "
                                           "per-parity blocks from L2, 3 staged with a "
                                           "copy-issuing warp and full / empty barriers; l: leaf "
                                           "kernel 0 four targets per lane and 2 subgrids per "
                                           "block, 1 two targets per thread and 1 subgrid per "
                                           "block, 2 four targets per lane and 4 subgrids per "
                                           "block; p: leaf kernel 0 beside the upward pass, 1 "
                                           "after it; c: boundary lists split over four lanes "
                                           "above an estimated cost of 6000, 1500, 24000, never; "
                                           "-1: not timed (coordinate search)"},
                  "gpu_launches": r32["launches"]},
        "df64": {"value": whole_job_rate(world, n_m2l, args.steps, tdf),
                 "ms_per_step": tdf / args.steps, "ms_per_step_median": med(rdf),
                 "dtype": "double-float (2 x f32) pair arithmetic, f64 rest",
                 "speedup_vs_fp64": t64 / tdf, "err_vs_fp64": errdf,
                 "roofline": roofline(rdf["phases"], "df64", kflops, peaks, traffic),
                 "phases_ms": phases_of(rdf["phases"]), "gpu_launches": rdf["launches"]},
        "peaks": {"fp64_tflops": peaks[64], "fp32_tflops": peaks[32], "fp32x2_tflops": peaks[-32],
                  "ms_per_launch": {"fp64": peak_ms[64], "fp32": peak_ms[32], "fp32x2": peak_ms[-32]},
                  "nominal_tflops": {"fp64": NOMINAL_TFLOPS[64], "fp32": NOMINAL_TFLOPS[32]},
                  "how": "fmm_measure_fma_rate: 8 independent FMA chains per thread, 2048 threads "
                         "per SM, about 40 ms per launch, fastest of 5"},
        "e2e": {"value": world * n_m2l * args.steps / e2e_s, "unit": "interactions/s",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n + 24 * n + 56,
                "precision": "fp64",
                "api": "fmm_solve_host_async (pinned host buffers, steps pipelined), wall clock",
                "synchronous_fmm_solve_host_ms_per_step": 1e3 * e2e_sync_s},
        "gpu_launches": r64["launches"],
        "persistent_level_passes": pers,
        "small": small,
        "binary_6_levels": six,
        "batched": batched,
        "paper_binary": paper,
        "paper_binary_graded": graded,
        "scf": scf,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--solve-workload", choices=["binary5", "binary6", "binary7", "paper9", "forest64"],
                    default="binary5",
                    help="with --solve-only: the 5-level binary (default), the same at 6 levels, "
                         "the 7-level headline binary, the 9-level merger binary in the paper's "
                         "proportions, or the 64-tree forest")
    ap.add_argument("--variant", type=int, default=None,
                    help="with --solve-only mixed: the launch variant (fmm_set_variant)")
    ap.add_argument("--solve-only", choices=["fp64", "mixed", "df64"], default=None,
                    help="profiling driver: run warmup + steps solves of the benchmark tree, no timing")
    args = ap.parse_args()
    if args.solve_only:
        run_solve_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
