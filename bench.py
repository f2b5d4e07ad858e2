#!/usr/bin/env python
"""D3(BJ) E + F + virial throughput on GB300 (atom-steps/s).

Workload: the bilayer-graphene binding/sliding scan, 128 structures of 1,440
C atoms (184,320 atoms) in one batched call, mixed precision.  One step = one
full pass of the pipeline over the batch: neighbour build (cell lists,
periodic images, per-atom lists), coordination numbers (Eq. 4), reference
weights (Eq. 3), dispersion pass (Eq. 2), coordination-number chain rule and
per-structure sums -- nothing is reused between steps.  The FP64 form is
timed on the same batch.  Inputs are synthetic (seeded generator).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun: each rank evaluates its own scan of the same shape
(jitter seed 1 + rank; independent structures, no collective on the data
path) and the value is the atoms of all ranks divided by the slowest rank's
time.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload (the only reference that exists for this method here).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3(BJ) E+F+virial atom-steps/s, 1 GB300, mixed vs FP64 form; % of roofline"
UNIT = "atom-steps/s"
L2_BYTES = 129 * 1024 * 1024
# FP32 lane instructions per unique dispersion pair within R_pot, as the
# measurement contract counts them (FFMA = FMUL = FADD = 1; the C6 bilinear form
# evaluated directly): 45 + 2 Na Nb + 3 Nb with Na, Nb the numbers of reference
# CNs of the two elements (Eq. 3).  Over a mix of elements the pair average is
# 45 + 2 E[Na] E[Nb] + 3 E[Nb], E[N] the atom-fraction weighted reference count.
def contract_ops_per_pair(tables, types) -> float:
    nref = np.asarray(tables.nref, dtype=np.float64)
    frac = np.bincount(np.asarray(types), minlength=len(nref)) / max(1, len(types))
    en = float((frac * nref).sum())
    return 45.0 + 2.0 * en * en + 3.0 * en


# The factorised FP32 count the kernels implement (FMA = 2 FLOP), kept as a second
# figure: distance 3 + r^2 5 + powers 3 + denominators 2 + reciprocals 2 + C6 and its
# two CN derivatives 6*Nref (projections of Eq. 3 per atom) + damping sum 3 + energy 2
# + dE/dn (both atoms) 4 + force scalar 8 + force vector and both atoms' sums 9 +
# symmetric virial 12 = 53 + 6*Nref.
def disp_flops_per_pair(nref: int) -> int:
    return 53 + 6 * nref


# FP32 work of one evaluation of the optional three-body term per unique triangle
# (FMA = 2 FLOP): three side vectors and squared lengths 24 + the C6 of the third
# pair 2*Nref + P, P^(-1/2), P^(-3/2) 9 + the law-of-cosines factors and N 8 +
# angular factor 4 + damping q, f and x df/dx 16 + sqrt(C6 C6 C6) and s9 8 +
# energy 2 + dN/dx for three sides 14 + dE/d(side^2) for three sides 36 + dE/dn for
# three atoms 8 + forces on three atoms 18 + symmetric virial of three sides 36
# = 183 + 2*Nref.  (The kernel evaluates each triangle from all three vertices.)
def atm_flops_per_triangle(nref: int) -> int:
    return 183 + 2 * nref


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_batch(rank: int, **kw):
    """The workload of one rank: the bilayer scan with its own jitter seed, so
    every rank evaluates different structures of the same shapes (weak scaling:
    per-rank work fixed, no data exchanged between ranks)."""
    from paper_2310_05279_gb300 import workloads as wl
    return wl.bilayer_scan(seed=1 + rank, **kw)


def reduce_max(x: float, device) -> float:
    """Maximum of x over the ranks of the default process group (x itself at N = 1)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(atoms_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the atoms of all ranks over the slowest rank's time."""
    return world * atoms_per_rank / seconds


PAIR_HELPERS = "paper_2310_05279_gb300/csrc/d3gb_pair.cuh"  # device helpers inlined into the pair kernels


def kernel_source_sha(path: str, kernel: str, whole_file: bool = False):
    """SHA-256 of a kernel's definition in a CUDA source (from the line that
    declares the __global__ function to the first closing brace in column 0),
    or of the whole file when the kernel's code spans it, together with the
    shared pair helpers it inlines."""
    import hashlib
    import re
    with open(path) as f:
        text = f.read()
    with open(os.path.join(ROOT, PAIR_HELPERS)) as f:
        helpers = f.read()
    if whole_file:
        return hashlib.sha256((text + "\n" + helpers).encode()).hexdigest()
    lines = text.split("\n")
    pat = re.compile(r"__global__.*\b" + re.escape(kernel) + r"\(")
    for k, line in enumerate(lines):
        if pat.search(line):
            end = next((j for j in range(k, len(lines)) if lines[j] == "}"), None)
            if end is None:
                return None
            return hashlib.sha256(("\n".join(lines[k:end + 1]) + "\n" + helpers).encode()).hexdigest()
    return None


def recorded_counters(kernel: str):
    """The committed ncu record of `kernel` (profiles/traffic.json), or None when
    the kernel's code has changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f).get(kernel)
    if not rec:
        return None
    src = os.path.join(ROOT, rec["source"])
    whole = rec.get("hash_of", "").startswith("the whole file")
    if not os.path.exists(src) or kernel_source_sha(src, kernel, whole) != rec.get("kernel_sha256"):
        return None
    return rec


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or None."""
    rec = recorded_counters(kernel)
    return float(rec["dram_bytes_per_launch"]) if rec else None


def recorded_pipes(kernel: str):
    """Pipe utilisation of `kernel` from the committed ncu capture (percent of
    peak), or None: which unit the kernel is actually bound by."""
    rec = recorded_counters(kernel)
    return rec.get("pipes") if rec else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples (every 10 ms), each stamped
    on arrival; only samples between mark_start() and mark_stop() are kept."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        import threading
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "10"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
            return

        def reader():
            for line in self.p.stdout:
                self.lines.append((time.time(), line))
        self.th = threading.Thread(target=reader, daemon=True)
        self.th.start()
        time.sleep(0.3)  # let the sampler start before the timed region

    def mark_start(self):
        self.t0 = time.time()

    def mark_stop(self):
        self.t1 = time.time()

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.05)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, smax, reasons = [], [], set()
        for t, line in self.lines:
            if self.t0 is not None and not (self.t0 <= t <= self.t1 + 0.02):
                continue
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "sample_period_ms": 10}


def time_steps(torch, fn, steps, warmup, flush=None, stream=None):
    """Per-step CUDA-event times (ms) with an untimed L2 flush between steps."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return times


def count_pairs(torch, batch, rc, dev):
    """Unique pairs within rc over the whole batch (bookkeeping for the roofline
    denominator).  Minimum image is exact here: every cell edge exceeds 2 rc in
    the plane, and along z the vacuum keeps all periodic images beyond rc."""
    tot = 0
    for s in range(batch.nstruct):
        pos, _, cell, _ = batch.structure(s)
        L = torch.tensor(np.diag(cell), dtype=torch.float64, device=dev)
        assert np.allclose(cell, np.diag(np.diag(cell)))
        x = torch.tensor(pos, dtype=torch.float64, device=dev)
        d = x[:, None, :] - x[None, :, :]
        d = d - L * torch.round(d / L)
        r2 = (d * d).sum(-1)
        tot += int(((r2 < rc * rc) & (r2 > 0)).sum().item()) // 2
    return tot


def count_triangles(torch, batch, rc, dev):
    """Unique triangles with all three sides below rc over the batch: trace(A^3)/6 of
    each structure's adjacency matrix (minimum image is exact, as in count_pairs)."""
    tot = 0
    for s in range(batch.nstruct):
        pos, _, cell, _ = batch.structure(s)
        L = torch.tensor(np.diag(cell), dtype=torch.float64, device=dev)
        x = torch.tensor(pos, dtype=torch.float64, device=dev)
        d = x[:, None, :] - x[None, :, :]
        d = d - L * torch.round(d / L)
        r2 = (d * d).sum(-1)
        A = ((r2 < rc * rc) & (r2 > 0)).to(torch.float32)
        tot += int(round(float(((A @ A) * A).sum().item()))) // 6
    return tot


def md_leg(torch, dev, params, steps, warmup=3, skin=0.5, dt=0.5, T_K=300.0):
    """Velocity-Verlet NVE loop on the 1,048,576-atom box with Verlet-list reuse:
    the library rebuilds the lists (on the device) only when an atom moved more
    than skin/2.  One step = half kick, drift, D3 forces, half kick; the timed
    region holds `steps` whole steps (CUDA events on the launching stream).  The
    box's positions and lists (> 2 GB) are far larger than L2."""
    from paper_2310_05279_gb300 import D3, workloads as wl
    b = wl.mof_like_box()
    m = wl.atom_masses(b)
    x = torch.tensor(b.pos, dtype=torch.float64, device=dev)
    typ = torch.tensor(b.types, dtype=torch.int32, device=dev)
    v = torch.tensor(wl.maxwell_velocities(m, T_K, seed=2), dtype=torch.float64, device=dev)
    acc = torch.tensor(1.0 / (m * wl.EV_PER_AMU_A2_FS2), dtype=torch.float64, device=dev)[:, None]  # (A/fs^2) per (eV/A)
    d3 = D3(b.tables, params, precision="mixed", skin=skin)
    out = d3.compute_batch(x, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()

    def step():
        v.add_(out["F"] * acc, alpha=0.5 * dt)
        x.add_(v, alpha=dt)
        d3.compute_batch(x, typ, b.offsets, b.cells, b.pbc, out=out)
        v.add_(out["F"] * acc, alpha=0.5 * dt)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    n0 = d3.build_count()
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    e.record(stream)
    e.synchronize()
    ms = a.elapsed_time(e) / steps
    builds = d3.build_count() - n0
    d3.sync_status()
    return {"workload": f"mof_like_box: {b.natoms:,} atoms (H:C:N:O:Zn = 40:36:8:12:4), 262.45 A cube",
            "integrator": f"NVE velocity Verlet, dt {dt} fs, Maxwell-Boltzmann {T_K:.0f} K start; "
                          "kicks and drifts are torch elementwise updates",
            "skin_A": skin, "steps": steps, "ms_per_step": ms, "value": b.natoms / (ms * 1e-3),
            "unit": UNIT, "builds_in_timed_steps": int(builds), "l2": "inputs and lists larger than L2"}


def backward_leg(torch, dev, params, steps, warmup=3):
    """The hand-written backward (dL/d(s6, s8, a1, a2) and dL/dx) of a mixed
    handle on the damping-refit batch, beside the forward on the same batch."""
    from paper_2310_05279_gb300 import D3, workloads as wl
    b = wl.fit_batch()
    d3 = D3(b.tables, params, precision="mixed")
    pos = torch.tensor(b.pos, dtype=torch.float64, device=dev)
    typ = torch.tensor(b.types, dtype=torch.int32, device=dev)
    g = np.random.Generator(np.random.PCG64(4))
    dLdE = torch.tensor(g.normal(size=b.nstruct), dtype=torch.float64, device=dev)
    dLdF = torch.tensor(0.01 * g.normal(size=(b.natoms, 3)), dtype=torch.float64, device=dev)
    out = d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc)
    d3.sync_status()

    def fwd():
        d3.compute_batch(pos, typ, b.offsets, b.cells, b.pbc, out=out)

    def bwd():
        d3.backward(pos, typ, b.offsets, b.cells, b.pbc, dLdE, dLdF)
    tf = time_steps(torch, fwd, steps, warmup)
    tb = time_steps(torch, bwd, steps, warmup)
    d3.sync_status()
    mf, mb = sum(tf) / len(tf), sum(tb) / len(tb)
    return {"workload": f"fit_batch: {b.nstruct} structures of 200-2000 atoms ({b.natoms:,} atoms), mixed handle",
            "forward_ms": mf, "backward_ms": mb, "backward_over_forward": mb / mf,
            "value": b.natoms / (mb * 1e-3), "unit": UNIT,
            "what": "dL/d(s6, s8, a1, a2) and dL/dx for upstream dL/dE, dL/dF (forward-mode, neighbour build included)"}


def cpu_baseline(batch, params, budget_s=15.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload's structures."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.compute(*batch.structure(0), batch.tables, params)
    one = time.perf_counter() - t0
    if batch.nstruct == 1:  # one structure: the timed call above is the sample
        n0 = len(batch.structure(0)[0])
        return {"value": n0 / one, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                "sample": f"1 structure ({n0} atom-steps, {one:.1f} s), FP64 C/OpenMP"}
    nsamp = int(max(1, min(batch.nstruct - 1, budget_s / max(one, 1e-3))))
    idx = list(np.linspace(1, batch.nstruct - 1, nsamp).astype(int))
    t0 = time.perf_counter()
    atoms = 0
    for s in idx:
        r = oracle.compute(*batch.structure(s), batch.tables, params)
        atoms += len(batch.structure(s)[0])
    dt = time.perf_counter() - t0
    return {"value": atoms / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{len(idx)} of {batch.nstruct} structures ({atoms} atom-steps, {dt:.1f} s), FP64 C/OpenMP"}


def run_reference(args):
    rank, world, _ = dist_env()
    from paper_2310_05279_gb300 import workloads as wl
    if rank != 0:
        return 0
    batch = wl.bilayer_scan()
    params = dict(wl.PBE_BJ)
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.compute(*batch.structure(0), batch.tables, params)
    one = time.perf_counter() - t0
    budget = max(0.5, 120.0 / max(1, args.steps))  # seconds of oracle work per step
    per_step = max(1, min(batch.nstruct, int(budget / max(one, 1e-3))))
    idx = list(np.linspace(0, batch.nstruct - 1, per_step).astype(int))
    for _ in range(args.warmup):
        oracle.compute(*batch.structure(idx[0]), batch.tables, params)
    times, atoms = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        a = 0
        for s in idx:
            oracle.compute(*batch.structure(s), batch.tables, params)
            a += len(batch.structure(s)[0])
        times.append(time.perf_counter() - t0)
        atoms = a
    value = atoms / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "bilayer_scan 128 x 1440 C atoms (sampled per step)", "sample_structures": len(idx),
                       "atoms_per_step": atoms, "parallelism": "OpenMP host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{len(idx)} of {batch.nstruct} structures per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def profiled_stages(torch, d3, step, steps, flush, stream):
    """Per-stage times (ms per call) of `steps` calls with CUDA events between the
    stages on the launching stream (kernels enqueued directly, not replayed);
    'lists' is the list-builder kernel alone, inside 'build'."""
    d3.profile_reset()
    d3.profile(True)
    time_steps(torch, step, steps, 1, flush=flush, stream=stream)
    pr = d3.profile_read()
    lms, lcalls = d3.profile_stage(7)
    d3.profile(False)
    d3.sync_status()
    st = {k: pr["ms"][k] / max(1, pr["calls"][k]) for k in pr["ms"]}
    st["lists"] = lms / max(1, lcalls)
    return st


def alu_roofline(kernel, work, t_ms, peak, unit, what, extra=None):
    """Roofline of an arithmetic-bound kernel: `work` operations per launch over its
    event-timed duration against `peak` operations per second."""
    ach = work / (t_ms * 1e-3)
    d = {"bound": "alu", "kernel": kernel, "achieved": ach / 1e12, "peak": peak / 1e12, "unit": unit,
         "frac": ach / peak, "algorithmic": what}
    if extra:
        d.update(extra)
    return d


def list_roofline(stats, t_ms, hbm_gbs, kernel):
    """The list builder against the measured HBM copy bandwidth: bytes it must move
    per launch are the lists it writes (4 B per entry, plus a count per row) and one
    read of every atom's compact position record (16 B, real and image atoms)."""
    entries = stats["cluster_list_entries"] + stats["cn_list_entries"] + stats["disp_list_entries"]
    rows = stats["clusters"] + stats["real_atoms"] * (2 if stats["list_mode"] == 0 else 1)
    nbytes = 4 * entries + 4 * rows + 16 * (stats["real_atoms"] + stats["image_atoms"])
    ach = nbytes / (t_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": hbm_gbs, "unit": "GB/s",
            "frac": ach / hbm_gbs, "traffic": recorded_traffic(kernel), "bytes_per_launch": nbytes,
            "list_bytes_written": 4 * entries,
            "algorithmic": f"{entries:,} list entries x 4 B + {rows:,} row counts x 4 B + "
                           f"{stats['real_atoms'] + stats['image_atoms']:,} position records x 16 B"}


def run_forward_leg(torch, dev, batch, params, precision, steps, warmup, flush, stream, graphs=True):
    """Time one batched call per step (neighbour build included, L2 flushed between
    steps) and profile its stages; returns the step time, stages, list statistics,
    launch shapes and the autotuner's candidate times."""
    from paper_2310_05279_gb300 import D3
    pos = torch.tensor(batch.pos, dtype=torch.float64, device=dev)
    typ = torch.tensor(batch.types, dtype=torch.int32, device=dev)
    d3 = D3(batch.tables, params, precision=precision)
    if not graphs:
        d3.set_graphs(False)
    out = d3.compute_batch(pos, typ, batch.offsets, batch.cells, batch.pbc)
    d3.sync_status()

    def step():
        d3.compute_batch(pos, typ, batch.offsets, batch.cells, batch.pbc, out=out)
    t = time_steps(torch, step, steps, warmup, flush=flush, stream=stream)
    d3.sync_status()
    ms = statistics.mean(t)
    stages = profiled_stages(torch, d3, step, max(2, min(steps, 5)), flush, stream)
    stats = d3.list_stats()
    res = {"ms_per_step": ms, "value": batch.natoms / (ms * 1e-3), "unit": UNIT, "stage_ms": stages,
           "lists": stats, "launch_shapes": d3.launch_shapes(), "tune_ms": d3.tune_times()}
    del d3
    return res


def rooflines(fwd, fp64, batch, peaks, rates, sm_count, fmax, pairs):
    """Dispersion-pass rooflines on the contract count (FP32 and FP64 forms), the
    factorised count, the MUFU reciprocal, and the list builder."""
    nref = int(batch.tables.max_ref)
    ops = contract_ops_per_pair(batch.tables, batch.types)
    fp32_peak = sm_count * 128 * fmax
    mufu_peak = sm_count * 16 * fmax
    t = fwd["stage_ms"]["disp"]
    r = {"roofline": alu_roofline(
        "k_disp_cl (dispersion pass, Eq. 2; stage = image rows + pass + fixed-point finish)", ops * pairs, t,
        fp32_peak, "T FP32 lane-instructions/s",
        f"{ops:.1f} FP32 lane instructions per unique pair within R_pot (45 + 2 Na Nb + 3 Nb, FFMA = 1) x "
        f"{pairs:,} pairs",
        {"traffic": recorded_traffic("k_disp_cl"), "pipes": recorded_pipes("k_disp_cl"),
         "peak_source": f"{sm_count} SMs x 128 FP32 lanes x {fmax / 1e6:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)",
         "measured_ffma_rate": rates["fp32_lane_ops_per_s"] / 1e12,
         "timing": "dispersion stage events over the profiled steps (kernels enqueued directly)"})}
    fl = disp_flops_per_pair(nref)
    r["roofline_factorised"] = alu_roofline(
        "k_disp_cl", fl * pairs, t, 2 * fp32_peak, "TFLOP/s",
        f"{fl} FLOP (FMA = 2) per unique pair, the per-atom C6 projections of Eq. 3 counted once per pair")
    r["mufu"] = alu_roofline(
        "k_disp_cl", 1.0 * pairs, t, mufu_peak, "T MUFU ops/s",
        "one reciprocal (rcp) per unique pair: 1/((r^6 + R^6)(r^8 + R^8))",
        {"measured_mufu_rate": rates["mufu_ops_per_s"] / 1e12})
    r["build_roofline"] = list_roofline(fwd["lists"], fwd["stage_ms"]["lists"], float(peaks["hbm_gbs"]),
                                        "k_build_clist")
    if fp64 is not None:
        r["fp64_roofline"] = alu_roofline(
            "k_disp<FP64> (per-atom full lists: each pair evaluated from both atoms)", ops * pairs,
            fp64["stage_ms"]["disp"], rates["fp64_lane_ops_per_s"], "T FP64 lane-instructions/s",
            f"{ops:.1f} lane instructions per unique pair (DFMA = 1) x {pairs:,} pairs",
            {"peak_source": "measured DFMA lane rate (d3_peak_rates: independent FMA chains, 8 blocks of 256 "
                            "threads per SM, best of 3)"})
    return r


def box_leg(torch, dev, params, steps, flush, stream, peaks, rates, sm_count, fmax, md_steps, md_skin):
    """The 1,048,576-atom box as one call (build included), mixed and FP64, with its
    rooflines; the NVE loop with list reuse; the oracle on a 2,048-atom periodic box
    of the same generator as the CPU baseline."""
    from paper_2310_05279_gb300 import workloads as wl
    b = wl.mof_like_box()
    mixed = run_forward_leg(torch, dev, b, params, "mixed", steps, 2, flush, stream)
    fp64 = run_forward_leg(torch, dev, b, params, "fp64", 2, 1, flush, stream)
    pairs = int(mixed["lists"]["pairs_within_rpot"])
    res = {"workload": f"mof_like_box: {b.natoms:,} atoms (H:C:N:O:Zn = 40:36:8:12:4), 262.45 A cube, one call "
                       "per step with the neighbour build", "mixed": mixed,
           "fp64": {k: fp64[k] for k in ("ms_per_step", "value", "unit", "stage_ms")},
           "mixed_speedup": fp64["ms_per_step"] / mixed["ms_per_step"], "pairs_within_rpot": pairs}
    res.update(rooflines(mixed, fp64, b, peaks, rates, sm_count, fmax, pairs))
    if md_steps > 0:
        res["md_loop"] = md_leg(torch, dev, params, md_steps, skin=md_skin)
    small = wl.mof_like_box(ncell=8)
    res["cpu_baseline"] = cpu_baseline(small, params, budget_s=8.0)
    res["cpu_baseline"]["sample"] += " (2,048-atom periodic box of the same generator: same density and mix)"
    return res


def uneven_leg(torch, dev, params, steps, flush, stream):
    """The 512-structure uneven batch (config 3) in one call, mixed and FP64, and by
    size class (each class its own batched call and handle), with the launch shapes
    the autotuner chose and the times it measured for the candidates."""
    from paper_2310_05279_gb300 import workloads as wl
    b = wl.uneven_batch()
    sizes = np.diff(b.offsets)
    res = {"workload": f"uneven_batch: {b.nstruct} triclinic structures of 50-4000 atoms ({b.natoms:,} atoms)"}
    res["whole"] = run_forward_leg(torch, dev, b, params, "mixed", steps, 2, flush, stream)
    f64 = run_forward_leg(torch, dev, b, params, "fp64", 2, 1, flush, stream)
    res["whole_fp64"] = {k: f64[k] for k in ("ms_per_step", "value", "unit", "stage_ms")}
    res["mixed_speedup"] = f64["ms_per_step"] / res["whole"]["ms_per_step"]
    classes = []
    for lo, hi in ((50, 200), (200, 1000), (1000, 4001)):
        idx = [int(s) for s in np.nonzero((sizes >= lo) & (sizes < hi))[0]]
        if not idx:
            continue
        sub = b.subset(idx)
        m = run_forward_leg(torch, dev, sub, params, "mixed", steps, 2, flush, stream)
        f = run_forward_leg(torch, dev, sub, params, "fp64", 2, 1, flush, stream)
        tm = m["tune_ms"]
        spread = {k: (max(v) / min(v) - 1.0) if min(v) > 0 else None for k, v in tm.items()}
        classes.append({"sizes": f"{lo}-{hi - 1}", "structures": len(idx), "atoms": sub.natoms,
                        "mixed": m["value"], "mixed_ms": m["ms_per_step"], "fp64": f["value"],
                        "fp64_ms": f["ms_per_step"], "mixed_speedup": f["ms_per_step"] / m["ms_per_step"],
                        "unit": UNIT, "launch_shapes": m["launch_shapes"], "autotune_candidate_ms": tm,
                        "autotune_spread": spread})
    res["size_classes"] = classes
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-graphs", action="store_true", help="enqueue every kernel directly (no graph replay)")
    ap.add_argument("--md-steps", type=int, default=100,
                    help="NVE steps of the 1M-atom box leg with list reuse (0: skip)")
    ap.add_argument("--md-skin", type=float, default=0.5,
                    help="Verlet skin (A) of the NVE leg (0.5 A was fastest of 0.5 / 0.75 / 1.0 / 1.5)")
    ap.add_argument("--backward-steps", type=int, default=5, help="steps of the backward leg (0: skip)")
    ap.add_argument("--three-body-steps", type=int, default=5,
                    help="steps of the extra leg with the optional three-body term (0: skip)")
    ap.add_argument("--box-steps", type=int, default=5,
                    help="steps of the 1M-atom box leg, one call each (0: skip the box leg)")
    ap.add_argument("--uneven-steps", type=int, default=5, help="steps of the uneven-batch leg (0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_2310_05279_gb300 import D3, peak_rates, workloads as wl
    from paper_2310_05279_gb300 import build as libbuild
    libbuild.build()
    batch = rank_batch(rank)
    N = batch.natoms
    params = dict(wl.PBE_BJ)
    pos = torch.tensor(batch.pos, dtype=torch.float64, device=dev)
    typ = torch.tensor(batch.types, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def flush():
        flush_buf.fill_(1.0)

    d3 = D3(batch.tables, params, precision="mixed")
    if args.no_graphs:
        d3.set_graphs(False)
    out = d3.compute_batch(pos, typ, batch.offsets, batch.cells, batch.pbc)
    d3.sync_status()

    def step():
        d3.compute_batch(pos, typ, batch.offsets, batch.cells, batch.pbc, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    d3.profile_reset()  # launch counter only: the timed steps run without stage events (graph replay)
    clk = ClockSampler(dev.index)
    clk.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk.mark_start()
    times = time_steps(torch, step, args.steps, 0, flush=flush, stream=stream)
    torch.cuda.synchronize()
    clk.mark_stop()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    launches_per_step = d3.profile_read()["launches"] / max(1, args.steps)
    shapes = d3.launch_shapes()
    tune_ms = d3.tune_times()
    d3.sync_status()
    ms = reduce_max(sum(times) / len(times), dev)
    value = job_value(N, world, ms * 1e-3)

    # stage breakdown of the same steps with CUDA events between the stages on the
    # launching stream (the kernels are then enqueued directly instead of replayed)
    stage_ms = profiled_stages(torch, d3, step, args.steps, flush, stream)
    stats = d3.list_stats()
    dom = max((k for k in stage_ms if k != "lists"), key=lambda k: stage_ms[k])
    fwd = {"stage_ms": stage_ms, "lists": stats}

    # FP64 form on the same batch
    fp64 = None
    if args.fp64_steps > 0:
        f = run_forward_leg(torch, dev, batch, params, "fp64", args.fp64_steps, 1, flush, stream)
        msf = reduce_max(f["ms_per_step"], dev)
        fp64 = {"value": job_value(N, world, msf * 1e-3), "unit": UNIT, "ms_per_step": msf, "dtype": "f64",
                "stage_ms": f["stage_ms"], "mixed_speedup": msf / ms, "lists": f["lists"]}

    # measured arithmetic rates and the rooflines of the dispersion pass and the list build
    peaks, peak_kind = measured_peaks()
    rates = peak_rates()
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    fmax = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    pairs = int(stats["pairs_within_rpot"])
    pairs_host = count_pairs(torch, batch, params["rc_disp"], dev)
    roofs = rooflines(fwd, fp64, batch, peaks, rates, sm_count, fmax, pairs)
    roofs["roofline"]["pairs_check"] = {"counted_by_pass": pairs, "counted_on_host": pairs_host}
    roofs["roofline"]["peak_kind"] = peak_kind

    # the optional three-body term (not part of the paper's model) on the same batch:
    # the whole step with it on, and its own pass against the FP32 roofline
    three_body = None
    if args.three_body_steps > 0:
        atm = dict(s9=1.0, alpha9=16.0, rc3=params["rc_cn"])
        d3a = D3(batch.tables, dict(params, **atm), precision="mixed")
        outa = d3a.compute_batch(pos, typ, batch.offsets, batch.cells, batch.pbc)
        d3a.sync_status()

        def step_atm():
            d3a.compute_batch(pos, typ, batch.offsets, batch.cells, batch.pbc, out=outa)
        ta = time_steps(torch, step_atm, args.three_body_steps, 3, flush=flush, stream=stream)
        stage_a = profiled_stages(torch, d3a, step_atm, args.three_body_steps, flush, stream)
        del d3a
        msa = reduce_max(sum(ta) / len(ta), dev)
        tri = count_triangles(torch, batch, atm["rc3"], dev)
        nref = int(batch.tables.max_ref)
        fl = atm_flops_per_triangle(nref)
        tf = fl * tri / (stage_a["three_body"] * 1e-3) / 1e12
        fp32_flops = sm_count * 128 * 2 * fmax / 1e12
        three_body = {"value": job_value(N, world, msa * 1e-3), "unit": UNIT, "ms_per_step": msa,
                      "three_body_ms": stage_a["three_body"], "stage_ms": stage_a, "triangles": tri,
                      "params": atm, "note": "optional triple-dipole term; the paper's model leaves it out",
                      "flop_per_triangle": fl,
                      "roofline": {"bound": "alu", "kernel": "k_atm", "achieved": tf, "peak": fp32_flops,
                                   "unit": "TFLOP/s", "frac": tf / fp32_flops, "traffic": recorded_traffic("k_atm"),
                                   "pipes": recorded_pipes("k_atm"),
                                   "algorithmic": f"{fl} FLOP per unique triangle x {tri:.4g}"}}

    # the hand-written backward on the damping-refit batch
    backward = backward_leg(torch, dev, params, args.backward_steps) if args.backward_steps > 0 else None

    # the 1M-atom box (one call per step, and the NVE loop with list reuse)
    box = None
    if args.box_steps > 0 and rank == 0:
        box = box_leg(torch, dev, params, args.box_steps, flush, stream, peaks, rates, sm_count, fmax,
                      args.md_steps, args.md_skin)
    md = box.get("md_loop") if box else (md_leg(torch, dev, params, args.md_steps, skin=args.md_skin)
                                         if args.md_steps > 0 else None)

    # the uneven batch, whole and by size class
    uneven = uneven_leg(torch, dev, params, args.uneven_steps, flush, stream) \
        if args.uneven_steps > 0 and rank == 0 else None

    # end to end through the host-memory entry point (pinned buffers, copies inside)
    e2e = None
    if not args.no_e2e:
        pin_pos = torch.tensor(batch.pos, dtype=torch.float64).pin_memory()
        pin_typ = torch.tensor(batch.types, dtype=torch.int32).pin_memory()
        hout = dict(E=torch.empty(batch.nstruct, dtype=torch.float64).pin_memory(),
                    F=torch.empty((N, 3), dtype=torch.float64).pin_memory(),
                    W=torch.empty((batch.nstruct, 3, 3), dtype=torch.float64).pin_memory())
        for _ in range(2):
            d3.compute_batch_host(pin_pos, pin_typ, batch.offsets, batch.cells, batch.pbc, out=hout)
        e2e_t = []
        for _ in range(max(3, args.steps // 2)):
            flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d3.compute_batch_host(pin_pos, pin_typ, batch.offsets, batch.cells, batch.pbc, out=hout)
            e2e_t.append(time.perf_counter() - t0)
        e2e_s = reduce_max(statistics.mean(e2e_t), dev)
        e2e = {"value": job_value(N, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": N * 3 * 8 + N * 4,
               "d2h_bytes_per_step": batch.nstruct * 8 + N * 3 * 8 + batch.nstruct * 9 * 8,
               "entry_point": "d3_compute_batch_host (pinned host buffers)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "bilayer_scan: 128 AB-graphene bilayers x 1440 C atoms (184,320 atoms), "
                                   "d 2.8-8.0 A x 8 slides", "structures": batch.nstruct, "atoms": N,
                       "precision": "mixed (FP32 pair math; fixed-point, compensated and FP64 sums)",
                       "rc_disp_A": 12.0, "rc_cn_A": 6.0, "neighbour_build": "every step",
                       "l2": "flushed between timed steps",
                       "launch": "direct" if args.no_graphs else "graph replay of the steady-state call",
                       "launch_shapes": {**shapes, "how": "measured by the library's autotuner at plan time",
                                         "candidate_ms": tune_ms},
                       "parallelism": f"data-parallel x{world}: each rank its own 128-structure scan "
                                      "(jitter seed 1 + rank), no collective on the data path"},
            **roofs,
            "rates": {k: v / 1e12 for k, v in rates.items()}, "rates_unit": "T ops/s (measured on this GPU)",
            "stage_ms": stage_ms, "dominant_stage": dom, "lists": stats,
            "split": {"with_build": value,
                      "without_build": job_value(N, world, max(1e-9, ms - stage_ms["build"]) * 1e-3),
                      "unit": UNIT,
                      "how": "the timed step minus the neighbour-build stage of the profiled pass (the build "
                             "runs in every timed step; with a skin it is amortised over the steps between rebuilds)"},
            "fp64_form": fp64,
            "mof_like_box": box,
            "uneven_batch": uneven,
            "three_body": three_body,
            "md_loop": md,
            "backward": backward,
            "e2e": e2e,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "gpu_launches_per_step": launches_per_step,
            "clocks": clocks}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(batch, params)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
