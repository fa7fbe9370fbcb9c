"""Benchmark of the fused TLSPH step on B300: particle-steps/s at 1M particles and % of HBM roofline.

Workload: the 3D finite-strain J2 block, 128 x 128 x 64 = 1,048,576 particles on a
jittered lattice (dp = 1 mm, h = 1.5 dp, Wendland C2, E = 200 GPa, nu = 0.3,
sigma_y0 = 250 MPa, H = 1 GPa), bottom face fixed, top face pressed at 5 m/s,
FP32 fields with FP64 displacement accumulation.  A step is one pass of the whole
hot path (deformation gradient, J2 return map, momentum with viscosity, update,
next step size): 3 kernels (k_gradient, k_stress, k_pass2).

Beside the headline it measures the batched form (512 independent 2D specimens in one
autotuned launch) and the learned form (the J2 update served by a network trained on
return-map samples of this block, against the plain step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--no-batched] [--no-surrogate] [--no-cpu] [--paper-cases]

Prints ONE JSON line.  ``--impl reference`` times the FP64 CPU oracle (the
method as plainly written, test infrastructure) on a bounded sample of the
same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
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
sys.path.insert(0, ROOT)

from paper_2602_15149_b300 import workloads as W  # noqa: E402

METRIC = "TL-SPH particle-steps/sec at 1M particles, % HBM roofline; surrogate vs plain"
UNIT = "particle-steps/s"
SHAPE = (128, 128, 64)
FALLBACK_HBM_GBS = 6400.0
FALLBACK_BF16_TFLOPS = 1400.0
MLP_FLOP_PER_ROW = 2 * (16 * 128 + 128 * 128 + 128 * 128 + 128 * 16)  # 73,728
# FP32 operations per neighbour pair of the 3D J2 step with viscosity, counted from the pair bodies
# (an FMA counts 2; rsqrt, reciprocal 1): the deformation-gradient pass 39 for F - I plus 28 for the
# viscosity sum (3D computes it for every pair and keeps it for pairs in compression); the force pass
# 35.  Peak: 148 SMs x 128 FP32 lanes x 2 x 2.032 GHz.
FLOP_PER_PAIR = {"gradient": 39.0 + 28.0, "pass2": 35.0}
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12

# DRAM bytes per launch of each kernel (k_pass2 = "pass2", k_gradient, k_stress) from one ncu capture
# of the 1M-particle block at full size (dram__bytes_read.sum + dram__bytes_write.sum, one pass, the
# launches of step 6), keyed by the hash of the kernel sources it was taken on; reported as null once
# the kernels change.
NCU_TRAFFIC = {"sources": "de79c4696cfaf835", "pass2": 216817408.0, "gradient": 140381952.0, "stress": 154305536.0}


def source_hash() -> str:
    """Hash of the device code (every kernel is defined in the csrc/*.cuh headers)."""
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2602_15149_b300", "csrc", "*.cuh"))):
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def bf16_peak():
    """Dense bf16 tensor peak in TFLOP/s: the sustained figure (the MLP runs inside a long step)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured (sustained)"
    return FALLBACK_BF16_TFLOPS, "fallback"


def kernel_bytes(dim, nnz, n, ts=4, j2=True, frac=False, visc=True, fused=False):
    """Algorithmic HBM bytes per launch of each kernel of a step (every particle's own records
    read / written once, neighbour gathers served on chip, neighbour indices read once per
    neighbour pass: 4 B per pair, the CSR definition, also when the kernels walk the stencil or
    lattice layout) for the library's layout.  Mirrors algorithmic_bytes() in tlsph_capi.cu.
    fused: the stress runs in the tail of the deformation-gradient kernel, so F - I and the
    viscosity sum never go through memory ("gradient" then holds both passes, "stress" 0)."""
    v4, nsym, q = 4 * ts, (6 if dim == 3 else 3), dim * dim * ts
    vi, fr = (1 if visc else 0), (1 if frac else 0)
    grad = n * (4 + 8 / 32 + (2 + (1 if vi + fr else 0)) * v4 + nsym * ts + dim * dim * ts + vi * dim * ts
                + fr * ts) + 4 * nnz
    stress = n * (dim * dim * ts + nsym * ts + 2 + v4 + (3 * v4 if dim == 3 else v4) + vi * 2 * dim * ts)
    if j2:
        stress += n * 2 * 7 * ts
    if frac:
        stress += n * (v4 + 2 * ts)
    p2 = n * (4 + 8 / 32 + 3 * v4 + q + vi * dim * ts + 2 + 4 + 2 + 2 * 8 * dim + 2 * v4 + fr * 4 * ts) + 4 * nnz
    if fused:
        # G and the viscosity sum stay in registers; Ahat is read once
        grad, stress = grad + stress - n * (2 * (dim * dim + vi * dim) * ts + nsym * ts), 0.0
    return {"gradient": grad, "stress": stress, "pass2": p2}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running.  mark(t0, t1) sets the
    window the summary covers (host wall-clock seconds); ensure_sample() keeps the GPU busy with the
    same work until a sample lands in that window when the timed region was shorter than the
    sampling interval."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"tlsph_clocks_{os.getpid()}.csv")
        self.window = None
        self.extended_s = 0.0

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        # wait for nvidia-smi's first line, so that sampling runs before the timed region starts
        t0 = time.time()
        while self.proc and time.time() - t0 < 5.0 and not self._rows():
            time.sleep(0.02)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def _rows(self):
        """(host time, sm MHz, max MHz, reasons) of every sample written so far."""
        import datetime
        out = []
        if not os.path.exists(self.path):
            return out
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                sm, smax = float(f[2]), float(f[3])
            except ValueError:
                continue
            out.append((ts, sm, smax, {nm for k, nm in enumerate(names) if f[6 + k].lower().startswith("active")}))
        return out

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def ensure_sample(self, busy, limit_s=3.0):
        """If no sample lies in the window, call busy() (more of the same steps, untimed) until one lands."""
        if not self.proc or self.window is None:
            return
        t0, t1 = self.window
        start = time.time()
        while not [r for r in self._rows() if t0 <= r[0] <= t1 + self.extended_s] and time.time() - start < limit_s:
            busy()
            self.extended_s = time.time() - t1
        self.extended_s = max(self.extended_s, 0.0)

    def summary(self):
        rows = self._rows()
        if self.window is not None:
            t0, t1 = self.window
            rows = [r for r in rows if t0 <= r[0] <= t1 + self.extended_s]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        reasons = set()
        for r in rows:
            reasons |= r[3]
        return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "window": ("the timed region" if self.extended_s == 0.0 else
                           f"the timed region and {self.extended_s:.2f} s more of the same steps (the region was "
                           f"shorter than the 200 ms sampling interval)")}


def configure_layout(g, args):
    """The neighbour walk of the timed context (--layout, --rows-gradient, --rows-force, --fuse-stress,
    --patch, --zstream)."""
    from paper_2602_15149_b300 import tlsph
    g.set_option(tlsph.OPT_NEIGHBOUR_LAYOUT, {"auto": tlsph.LAYOUT_AUTO, "stencil": tlsph.LAYOUT_STENCIL,
                                              "csr": tlsph.LAYOUT_CSR}[args.layout])
    g.set_option(tlsph.OPT_LATTICE_ROWS_GRADIENT, args.rows_gradient)
    g.set_option(tlsph.OPT_LATTICE_ROWS_FORCE, args.rows_force)
    g.set_option(tlsph.OPT_FUSE_STRESS, 1 if args.fuse_stress else 0)
    g.set_option(tlsph.OPT_LATTICE_PATCH, args.patch)
    g.set_option(tlsph.OPT_LATTICE_ZSTREAM, args.zstream)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_specimens(nspec, rank, ws):
    """The specimens rank takes in an N-rank run of the batched form: every ws-th, from rank on
    (specimens are ordered by size, so the shares balance).  No data crosses ranks."""
    return list(range(rank, nspec, ws))


def max_over_ranks(x, device=None):
    """The largest x of all ranks (x itself when the run has one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, device=None):
    """The sum of x over all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def oracle_sample(seconds=15.0, shape=(32, 32, 16)):
    """The FP64 oracle as it stands on a bounded sample of the workload (same lattice recipe,
    material and loading, smaller block): particle-steps/s on the host cores."""
    from tests.oracle_cases import make_oracle
    case = W.block_3d(nx=shape[0], ny=shape[1], nz=shape[2])
    o = make_oracle(case)
    o.step(1)
    t0 = time.perf_counter()
    steps = 0
    while steps < 1 or (time.perf_counter() - t0 < seconds and steps < 10000):
        o.step(1)
        steps += 1
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": case.n * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"block_3d_j2 {shape[0]}x{shape[1]}x{shape[2]} = {case.n} particles, {steps} steps "
                      f"after 1 warm-up step ({el:.1f} s), FP64 OpenMP"}


def oracle_sample_one_thread(seconds=8.0, shape=(32, 32, 16)):
    """oracle_sample on one host thread (a child process with OMP_NUM_THREADS=1, since the OpenMP
    runtime of this process already holds its thread count); None if the child fails."""
    code = ("import json, bench; r = bench.oracle_sample(%r, %r); print(json.dumps(r))" % (seconds, tuple(shape)))
    env = {**os.environ, "OMP_NUM_THREADS": "1"}
    try:
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             timeout=seconds * 10 + 120)
        return json.loads(out.stdout.strip().splitlines()[-1]) if out.returncode == 0 else None
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (the method as plainly written) on the host cores.
    Its step is one time step of a bounded sample of the workload: the same lattice recipe,
    material and loading on a 32 x 32 x 16 block (16,384 particles), so that --steps 2000 ends
    within a few minutes."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from tests.oracle_cases import make_oracle
    shape = (32, 32, 16)
    case = W.block_3d(nx=shape[0], ny=shape[1], nz=shape[2], steps=args.steps)
    o = make_oracle(case)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    val = case.n * args.steps / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"block_3d_j2 {shape[0]}x{shape[1]}x{shape[2]} = {case.n} particles (same recipe as the "
              f"128x128x64 block), {args.steps} steps after {args.warmup} warm-up steps, FP64 OpenMP")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "block_3d_j2 128x128x64 J2 block, bounded sample 32x32x16 (FP64 CPU oracle)",
                       "particles": case.n},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def measure_batched(args, device, stream):
    """The batched form: 512 independent 2D specimens (log-uniform 500-50k particles, random
    materials and loading) stepped together; execution mode and block picked by the autotuner."""
    import torch
    from paper_2602_15149_b300 import tlsph

    ws, rank, _ = dist_env()
    full = W.batched(nspec=args.batch_specimens, steps=args.steps)
    case = W.subset(full, shard_specimens(args.batch_specimens, rank, ws)) if ws > 1 else full
    t0 = time.perf_counter()
    g = tlsph.from_case(case, device=device, stream=stream.cuda_stream)
    setup_s = time.perf_counter() - t0
    best, allt = g.autotune(trial_steps=5)
    g.step(args.warmup)
    steps = max(10, min(args.steps, 1000))
    dev = torch.device("cuda", device)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step_async(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    st = g.sync(check=False)
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    particles = int(sum_over_ranks(case.n, dev))
    info = g.get_info()
    g.close()
    # algorithmic bytes of one step of this rank's specimens (the library's model: own records once per
    # pass, 4 B per neighbour pair per neighbour pass), summed over ranks, against the measured copy peak
    step_bytes = sum_over_ranks(info["bytes_per_step"], dev)
    peak, peak_src = peaks()
    achieved = step_bytes / (ms / steps * 1e-3) / 1e9
    return {"workload": f"batched_2d {args.batch_specimens} specimens, {particles} particles, "
                        f"log-uniform 500-50k each, NH/J2, own clocks", "particles": particles,
            "specimens": args.batch_specimens, "steps": steps, "ms_per_step": ms / steps,
            "value": particles * steps / (ms * 1e-3), "unit": UNIT, "tuned": best, "candidates": allt,
            "sharding": f"specimens by rank ({ws} ranks, no collective on the data path)",
            "setup_s": setup_s, "status": int(st), "mean_neighbours": info["nnz"] / case.n,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_src, "algorithmic_bytes_per_step": step_bytes,
                         "bytes_per_particle_step": step_bytes / particles}}


def timed_steps(g, steps, stream, dev):
    import torch
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step_async(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    st = g.sync(check=False)
    return e0.elapsed_time(e1), int(st)


def measure_leapfrog(args, shape, device, stream, plain):
    """Algorithm 2 (leapfrog: predictor, forces at the half level, corrector) on the same block, against
    the plain Algorithm 1 step."""
    import torch
    from paper_2602_15149_b300 import tlsph

    dev = torch.device("cuda", device)
    case = W.block_3d(*shape, steps=args.steps)
    case.integrator = tlsph.INTEGRATOR_LEAPFROG
    g = tlsph.from_case(case, device=device, stream=stream.cuda_stream)
    g.step(args.warmup)
    ms, st = timed_steps(g, args.steps, stream, dev)
    g.close()
    value = case.n * args.steps / (ms * 1e-3)
    return {"workload": "block_3d_j2, Algorithm 2 (leapfrog)", "ms_per_step": ms / args.steps, "value": value,
            "unit": UNIT, "vs_algorithm_1": value / plain["value"], "status": st,
            "kernels_per_step": 4}


def measure_phase_field(args, device, stream):
    """Phase-field fracture on the full notched plate (500 x 200, FP32) with the two degraded
    hyperelastic laws: the neo-Hookean J-split and the St. Venant-Kirchhoff spectral split."""
    import torch
    from paper_2602_15149_b300 import tlsph

    dev = torch.device("cuda", device)
    out = {}
    for model in ("nh", "svk"):
        case = W.notched_plate(model=model, steps=args.steps)
        g = tlsph.from_case(case, device=device, stream=stream.cuda_stream)
        g.step(args.warmup)
        ms, st = timed_steps(g, args.steps, stream, dev)
        g.close()
        out[model] = {"ms_per_step": ms / args.steps, "value": case.n * args.steps / (ms * 1e-3), "status": st}
    out["workload"] = "notched_plate 500x200 phase field, FP32"
    out["unit"] = UNIT
    out["svk_vs_nh"] = out["svk"]["value"] / out["nh"]["value"]
    return out


def measure_crack_branching(args, device, stream):
    """The paper's crack-branching case at its published size (1600 x 640 = 1,024,000 particles, SVK,
    phase field) run to 80 us: throughput of the stepping (CUDA events around each 1 us chunk; the
    read-back of s between chunks is not timed) and the crack's milestones against the printed values."""
    import torch
    from paper_2602_15149_b300 import crack, tlsph

    dev = torch.device("cuda", device)
    case = W.crack_branching(t_end=80e-6)
    g = tlsph.from_case(case, device=device, stream=stream.cuda_stream)
    g.step(1)
    t, dt = g.time()
    per = max(1, int(round(1e-6 / dt)))
    split = crack.CrackTracker(case.X0, case.dp, 0.02, 0.05, threshold=0.25, branch_gap_rows=1)
    sustained = crack.CrackTracker(case.X0, case.dp, 0.02, 0.05, threshold=0.25, branch_gap_rows=4)
    ms, steps, st = 0.0, 1, 0
    while t < 80e-6:
        m, st1 = timed_steps(g, per, stream, dev)
        ms += m
        steps += per
        st |= st1
        t, dt = g.time()
        sv = g.read_state("S")
        split.add(t, sv)
        sustained.add(t, sv)
    g.close()
    geo = sustained.geometry()
    us = lambda x: None if x is None else x * 1e6
    return {"workload": "crack_branching 1600x640 SVK phase field (the paper's case), to 80 us, FP32",
            "particles": case.n, "steps": steps, "ms_per_step": ms / (steps - 1),
            "value": case.n * (steps - 1) / (ms * 1e-3), "unit": UNIT, "status": st,
            "t_initiation_us": us(split.t_init), "t_first_split_us": us(split.t_branch),
            "t_sustained_branches_us": us(sustained.t_branch),
            "branch_x_mm": None if geo["branch_x"] is None else geo["branch_x"] * 1e3,
            "divergence_angle_deg": geo["angle_deg"], "asymmetry": geo["asymmetry"],
            "paper": {"t_initiation_us": 14.0, "t_branching_us": 35.0, "divergence_angle_deg": 60.0}}


def measure_flyer_plate(args, device, stream):
    """The paper's flyer-plate impact (two 100 x 100 J2 plates, contact between the bodies) run to 300 us in
    FP32: throughput of the stepping (CUDA events around each chunk) and when plasticity starts."""
    import torch
    from paper_2602_15149_b300 import tlsph

    dev = torch.device("cuda", device)
    case = W.flyer_plate()
    g = tlsph.from_case(case, device=device, stream=stream.cuda_stream)
    g.set_option(tlsph.OPT_MODE, tlsph.MODE_GRAPH)
    g.step(args.warmup)
    ms, steps, st, t, t_plastic = 0.0, 0, 0, 0.0, None
    l0 = g.get_info()["kernel_launches"]
    while t < 300e-6:
        m, st1 = timed_steps(g, 200, stream, dev)
        ms += m
        steps += 200
        st |= st1
        t, _ = g.time()
        if t_plastic is None and g.read_state("EPSP").max() > 0.0:
            t_plastic = t
    launches = g.get_info()["kernel_launches"] - l0
    g.close()
    return {"workload": "flyer_plate 2 x 100x100 J2 plates at +-200 m/s, contact, to 300 us, FP32",
            "particles": case.n, "steps": steps, "ms_per_step": ms / steps, "value": case.n * steps / (ms * 1e-3),
            "unit": UNIT, "status": st, "kernels_per_step": launches / steps,
            "t_first_plastic_us": None if t_plastic is None else t_plastic * 1e6,
            "t_contact_expected_us": 125.0}


def measure_taylor_bar(args, device, stream):
    """The paper's 3D Taylor bar (J2, wall and start given by expressions) at dx = 0.4 mm to 80 us in FP32:
    stepping throughput (CUDA events) and the final energy split and shape."""
    import torch
    from paper_2602_15149_b300 import tlsph

    dev = torch.device("cuda", device)
    case = W.taylor_bar(dx=0.4e-3)
    g = tlsph.from_case(case, device=device, stream=stream.cuda_stream)
    g.set_option(tlsph.OPT_MODE, tlsph.MODE_GRAPH)
    KE0 = g.energies()["KE"]
    ms, steps, st, t = 0.0, 0, 0, 0.0
    while t < 80e-6:
        m, st1 = timed_steps(g, 1000, stream, dev)
        ms += m
        steps += 1000
        st |= st1
        t, _ = g.time()
    e = g.energies()
    x = case.X0 + g.read_state("U")
    base = x[case.X0[:, 2] < case.dp]
    g.close()
    return {"workload": "taylor_bar dx 0.4 mm J2 cylinder at -227 m/s onto a wall, to 80 us, FP32",
            "particles": case.n, "steps": steps, "ms_per_step": ms / steps, "value": case.n * steps / (ms * 1e-3),
            "unit": UNIT, "status": st, "KE_final": e["KE"] / KE0, "PW_final": e["PW"] / KE0,
            "energy_retained": (e["KE"] + e["SE"] + e["PW"]) / KE0, "length_mm": float(x[:, 2].max() + case.dp / 2) * 1e3,
            "base_radius_mm": float(np.sqrt(base[:, 0] ** 2 + base[:, 1] ** 2).max() + case.dp / 2) * 1e3}


def measure_model_variants(args, shape, device, stream):
    """The paper's performance study varies only the material law at 1M particles (SVK, NH, both with phase
    field, J2).  The same five variants of the block (same lattice, loading and step count), each timed on
    its own context, and the block at three sizes with SVK (the paper's size study)."""
    import torch
    from paper_2602_15149_b300 import tlsph

    dev = torch.device("cuda", device)
    steps = max(20, min(args.steps, 300))
    variants = {"A1_svk": (W.MODEL_SVK, 0), "A2_nh": (W.MODEL_NH, 0), "B1_svk_fracture": (W.MODEL_SVK, 1),
                "B2_nh_fracture": (W.MODEL_NH, 1), "C_j2": (W.MODEL_J2, 0)}
    out = {}
    for name, (model, frac) in variants.items():
        case = W.block_3d(*shape, steps=steps)
        m = case.materials[0]
        if model != W.MODEL_J2:
            case.materials = [W.Material(model=model, rho=m.rho, E=m.E, nu=m.nu, beta1=m.beta1, fracture=frac,
                                         Gc=2.0e4 if frac else 0.0, eps0=2.0 * case.dp if frac else 0.0)]
        g = tlsph.from_case(case, device=device, stream=stream.cuda_stream)
        g.step(args.warmup)
        ms, st = timed_steps(g, steps, stream, dev)
        g.close()
        out[name] = {"ms_per_step": ms / steps, "value": case.n * steps / (ms * 1e-3), "status": st}
    t = [v["ms_per_step"] for v in out.values()]
    sizes = {}
    for sh in ((48, 48, 32), (64, 64, 64), (128, 128, 64), (192, 192, 96), (256, 256, 128)):
        case = W.block_3d(*sh, steps=steps)
        m = case.materials[0]
        case.materials = [W.Material(model=W.MODEL_SVK, rho=m.rho, E=m.E, nu=m.nu, beta1=m.beta1)]
        g = tlsph.from_case(case, device=device, stream=stream.cuda_stream)
        g.step(args.warmup)
        ms, st = timed_steps(g, steps, stream, dev)
        g.close()
        sizes[case.n] = {"ms_per_step": ms / steps, "value": case.n * steps / (ms * 1e-3), "status": st}
    return {"workload": f"block_3d {'x'.join(map(str, shape))} with the five material variants, {steps} steps each",
            "unit": UNIT, "variants": out, "spread": (max(t) - min(t)) / min(t),
            "size_scaling_svk": sizes}


def measure_surrogate(args, shape, device, stream, plain):
    """The learned form on the same 1M J2 block: return-map samples from an exact run, training on
    the GPU, then the block stepped with the network in the J2 update (both scopes), against the
    plain step.  Stress error of held-out samples is judged by the exact return map."""
    import torch
    from paper_2602_15149_b300 import surrogate, tlsph

    dev = torch.device("cuda", device)
    steps = args.sur_steps  # the configuration's run length, whatever --steps the headline takes
    case = W.block_3d(*shape, steps=steps)
    n = case.n
    every = 20
    points = max(1, steps // every)
    t0 = time.perf_counter()
    x, y, pn = surrogate.generate_samples(case, n_target=args.sur_samples, steps=steps, every=every,
                                      stride_elastic=16, stride_plastic=8, device=device,
                                      stream=stream.cuda_stream, per_call=2 * args.sur_samples // points)
    gen_s = time.perf_counter() - t0
    m = x.shape[0]
    perm = torch.randperm(m, device=dev, generator=torch.Generator(device=dev).manual_seed(1))
    x, y, pn = x.index_select(0, perm), y.index_select(0, perm), pn.index_select(0, perm)
    ntr = int(0.95 * m)
    net, info = surrogate.train(x[:ntr], y[:ntr], epochs=args.sur_epochs, batch=2048, lr=2e-3, device=device,
                                time_budget_s=args.sur_train_s)
    err = surrogate.stress_error(net, x[ntr:], y[ntr:], pn[ntr:], case.materials[0].sigma_y0)
    del x, y, pn
    torch.cuda.empty_cache()

    # the plain (exact) step over the same steps: the reference of both accuracy and speed
    exact = tlsph.from_case(case, device=device, stream=stream.cuda_stream)
    exact.step(args.warmup)
    ms_exact, st_exact = timed_steps(exact, steps - args.warmup, stream, dev)
    ue, epe = exact.read_state("U"), exact.read_state("EPSP")
    exact.close()
    plain_value = n * (steps - args.warmup) / (ms_exact * 1e-3)
    out = {"workload": f"block_3d_j2 {'x'.join(map(str, shape))}, {steps} steps (the configuration's run), "
                       f"samples every {every} steps of the exact run", "steps": steps,
           "plain": {"ms_per_step": ms_exact / (steps - args.warmup), "value": plain_value, "status": st_exact},
           "samples": m, "train_samples": ntr, "sample_gen_s": gen_s, "training": info, "stress_error": err,
           "network": "16-128-128-128-16 SiLU, bf16 weights, fp32 accumulation (tcgen05.mma with TMEM "
                      "accumulators; mma.sync m16n8k16 for comparison)"}
    for name, scope, path in (("all", tlsph.SURROGATE_ALL, tlsph.TENSOR_TCGEN05),
                              ("plastic", tlsph.SURROGATE_PLASTIC, tlsph.TENSOR_TCGEN05),
                              ("all_mma_sync", tlsph.SURROGATE_ALL, tlsph.TENSOR_MMA_SYNC)):
        g = tlsph.from_case(case, device=device, stream=stream.cuda_stream)
        net.set_tensor_path(path)
        g.set_surrogate(net, scope)
        net.set_tensor_path(tlsph.TENSOR_TCGEN05)
        g.step(args.warmup)
        ms, st = timed_steps(g, steps - args.warmup, stream, dev)
        steps_t = steps - args.warmup
        used, outside, elastic = g.surrogate_counts()
        noconv = g.get_info()["noconverge"]
        us, eps = g.read_state("U"), g.read_state("EPSP")
        g.set_option(tlsph.OPT_KERNEL_TIMING, 1)
        g.step(100)
        kt = g.kernel_times()
        g.close()
        stress_ms = kt["stress_ms"] / max(kt["stress_launches"], 1)
        mlp_rows = used / max(steps, 1)  # network rows per launch (warm-up + timed steps)
        tflops = MLP_FLOP_PER_ROW * mlp_rows / (stress_ms * 1e-3) / 1e12
        peak, src = bf16_peak()
        out[name] = {"tensor_path": "tcgen05" if path == tlsph.TENSOR_TCGEN05 else "mma.sync",
                     "ms_per_step": ms / steps_t, "value": n * steps_t / (ms * 1e-3), "unit": UNIT,
                     "vs_plain": (n * steps_t / (ms * 1e-3)) / plain_value,
                     "status": st, "noconverge": noconv, "rows_network": used, "rows_outside_envelope": outside,
                     "rows_elastic_exact": elastic,
                     "network_fraction": used / max(used + outside + elastic, 1),
                     "stress_kernel_ms": stress_ms, "plain_stress_kernel_ms": plain["stress_ms"],
                     "stress_error_p99": err["p99"],
                     "rel_l2_u_vs_exact": float(np.linalg.norm(us - ue) / np.linalg.norm(ue)),
                     "max_abs_eps_p_diff": float(np.abs(eps - epe).max()),
                     "tensor": {"achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                                "peak_source": src, "flop_per_row": MLP_FLOP_PER_ROW,
                                "rows_per_launch": mlp_rows}}
    return out


def run_ours(args):
    import torch
    from paper_2602_15149_b300 import tlsph

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)

    shape = tuple(int(x) for x in args.shape.split(","))
    case = W.block_3d(*shape, steps=args.steps)
    n = case.n
    g = tlsph.from_case(case, device=local, stream=stream.cuda_stream)
    configure_layout(g, args)
    info = g.get_info()
    nnz = info["nnz"]

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # warm-up
    g.step(args.warmup)
    l0 = g.get_info()["kernel_launches"]
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t_a = time.time()
        e0.record(stream)
        g.step_async(args.steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clk.mark(t_a, time.time())
        st = g.sync(check=False)
        clk.ensure_sample(lambda: (g.step_async(200), torch.cuda.synchronize(dev)))
    barrier()
    ms = e0.elapsed_time(e1)
    launches = g.get_info()["kernel_launches"] - l0
    ms = max_over_ranks(ms, dev)
    value = ws * n * args.steps / (ms * 1e-3)

    # per-kernel durations (CUDA events around each launch on the same stream)
    g.set_option(tlsph.OPT_KERNEL_TIMING, 1)
    g.step(min(args.steps, 200))
    kt = g.kernel_times()
    g.set_option(tlsph.OPT_KERNEL_TIMING, 0)
    kb = kernel_bytes(3, nnz, n)
    kms = {k: kt[k + "_ms"] / max(kt[k + "_launches"], 1) for k in ("gradient", "stress", "pass2")}
    dom = max(kms, key=kms.get)
    dom_bytes, dom_ms = kb[dom], kms[dom]
    peak, peak_src = peaks()
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    traffic = NCU_TRAFFIC.get(dom) if NCU_TRAFFIC.get("sources") == source_hash() else None
    plain = {"value": n * args.steps / (ms * 1e-3), "stress_ms": kms["stress"]}
    step_bytes = sum(kb.values())
    g.close()
    torch.cuda.synchronize(dev)

    # end to end through the C-ABI with host buffers: setup from host arrays, every step with
    # its status read back, final displacement copied to the host
    barrier()
    t0 = time.perf_counter()
    g2 = tlsph.from_case(case, device=local, stream=stream.cuda_stream)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    for _ in range(args.steps):
        g2.step(1)
    u = g2.read_state("U")
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    e2e_steps_s = time.perf_counter() - t1
    g2.close()
    e2e_s = max_over_ranks(e2e_s, dev)
    e2e_steps_s = max_over_ranks(e2e_steps_s, dev)
    e2e_setup_s = e2e_s - e2e_steps_s
    h2d = n * (8 * 3 + 8 + 4 + 8 * 3) + sum(n for _ in case.bcs)
    d2h = u.nbytes + 8 * 4 * args.steps

    batched = measure_batched(args, local, stream) if not args.no_batched else None
    sur = measure_surrogate(args, shape, local, stream, plain) if not args.no_surrogate else None
    # the paper's reproductions and the other integrator / laws: opt-in (--paper-cases)
    paper = args.paper_cases
    leapfrog = measure_leapfrog(args, shape, local, stream, plain) if paper else None
    phase_field = measure_phase_field(args, local, stream) if paper else None
    crack_b = measure_crack_branching(args, local, stream) if paper else None
    flyer = measure_flyer_plate(args, local, stream) if paper else None
    taylor = measure_taylor_bar(args, local, stream) if paper else None
    variants = measure_model_variants(args, shape, local, stream) if paper else None
    if rank != 0:
        return 0
    cpu = oracle_sample() if not args.no_cpu else None
    if cpu is not None:  # the same sample on one host thread, beside the all-cores figure
        one = oracle_sample_one_thread()
        if one is not None:
            cpu["one_thread"] = {"value": one["value"], "unit": UNIT, "cores": 1, "sample": one["sample"]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"block_3d_j2 {'x'.join(map(str, shape))} jittered lattice, J2 plasticity, top "
                               "pressed at 5 m/s (FP32 fields, FP64 displacement)", "particles": n, "neighbour_pairs": nnz,
                   "mean_neighbours": nnz / n, "l2": "inputs larger than L2 (~1.3 GB of state), no flush",
                   "neighbour_layout": (f"lattice (ball of 122 entries, NX {info['lattice_nx']}, NXNY "
                                        f"{info['lattice_nxny']}, one mask word per layer)" if info["lattice_nx"] else
                                        f"stencil ({info['stencil']} differences, 16 B row masks)"
                                        if info["stencil"] else "SELL-32 CSR rows"),
                   "parallelism": f"replicas x{ws} (independent blocks)",
                   "walk": {"layout": args.layout, "rows_gradient": args.rows_gradient, "rows_force": args.rows_force,
                            "fuse_stress": bool(args.fuse_stress), "patch": args.patch,
                            "zstream": args.zstream}},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src, "traffic": traffic,
                     "algorithmic_bytes_per_launch": dom_bytes, "avg_launch_ms": dom_ms,
                     "kernel_ms": kms, "kernel_bytes": kb,
                     "step_frac": step_bytes / (ms / args.steps * 1e-3) / 1e9 / peak},
        "alu": {"bound": "alu", "unit": "TFLOP/s", "peak": FP32_PEAK_TFLOPS,
                "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 flop x 2.032 GHz",
                "flop_per_pair": FLOP_PER_PAIR,
                "kernel": {k: (FLOP_PER_PAIR[k] * nnz / (kms[k] * 1e-3) / 1e12) for k in FLOP_PER_PAIR},
                "kernel_frac": {k: (FLOP_PER_PAIR[k] * nnz / (kms[k] * 1e-3) / 1e12) / FP32_PEAK_TFLOPS
                                for k in FLOP_PER_PAIR},
                "step": sum(FLOP_PER_PAIR.values()) * nnz / (ms / args.steps * 1e-3) / 1e12},
        "clocks": clk.summary(),
        "e2e": {"value": ws * n * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps, "setup_s": e2e_setup_s,
                "steps_value": ws * n * args.steps / e2e_steps_s,
                "note": "value includes the reference setup (sort, neighbour rows, masks) from host arrays; "
                        "steps_value is the stepping alone, a status read back after every step"},
        "gpu_launches": launches,
        "batched": batched,
        "surrogate": sur,
        "surrogate_vs_plain": sur["all"]["vs_plain"] if sur else None,
        "surrogate_status": sur["all"]["status"] if sur else None,
        "surrogate_noconverge": sur["all"]["noconverge"] if sur else None,
        "surrogate_stress_err_p99": sur["stress_error"]["p99"] if sur else None,
        "surrogate_rel_l2_u": sur["all"]["rel_l2_u_vs_exact"] if sur else None,
        "leapfrog": leapfrog,
        "phase_field": phase_field,
        "crack_branching": crack_b,
        "flyer_plate": flyer,
        "taylor_bar": taylor,
        "model_variants": variants,
        "status": int(st),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-specimens measurement")
    ap.add_argument("--batch-specimens", type=int, default=512)
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-surrogate measurement")
    ap.add_argument("--paper-cases", action="store_true",
                    help="also run the paper's reproductions (crack branching, flyer plate, Taylor bar, the five "
                         "material variants and the size study), Algorithm 2 and the phase-field plate")
    ap.add_argument("--sur-steps", type=int, default=2000,
                    help="run length of the surrogate leg: samples, exact run and network run (the "
                         "configuration's 2000 steps, whatever --steps is)")
    ap.add_argument("--sur-samples", type=int, default=10_000_000, help="return-map samples for training")
    ap.add_argument("--sur-epochs", type=int, default=10)
    ap.add_argument("--sur-train-s", type=float, default=90.0, help="training time limit (s)")
    ap.add_argument("--layout", default="auto", choices=["auto", "stencil", "csr"],
                    help="neighbour walk of the headline step: auto (the lattice walk on this block), the stencil "
                         "table walk, or SELL-32 rows (for comparing the walks; the metric uses auto)")
    ap.add_argument("--rows-gradient", type=int, default=1, choices=[1, 2],
                    help="lattice walk: rows per thread of the deformation-gradient kernel")
    ap.add_argument("--rows-force", type=int, default=2, choices=[1, 2, 4],
                    help="lattice walk: rows per thread of the force kernel")
    ap.add_argument("--fuse-stress", action="store_true",
                    help="lattice walk: the stress in the tail of the deformation-gradient kernel")
    ap.add_argument("--patch", type=int, default=0, choices=[0, 32, 64, 128],
                    help="lattice walk: x width of a block's patch of rows (0: whole x lines)")
    ap.add_argument("--zstream", type=int, default=0,
                    help="lattice walk: planes per thread of the force pass streaming along z (0: off)")
    ap.add_argument("--shape", default=",".join(map(str, SHAPE)),
                    help="lattice of the J2 block (the metric's workload is 128,128,64; smaller shapes for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
