"""Throughput of the moving-grid split-operator propagator on one GB300.

Headline workload: the 8D Henon-Heiles model of Sec. III.C on a 12^8 moving
grid in FP64 (complex128, 4.3e8 points, 6.9 GB), fourth-order Suzuki
composition (5 TVT stages per step), dt = 0.01.  One timed iteration is one
mg_propagate call of one time step (one persistent kernel launch); value =
grid points x time steps / second.  The state is larger than L2, so no flush
is needed between iterations.  The FP64 path is bound by the FP64 units: its
roofline is stated against the FP64 FMA rate measured in the same run.

Secondary lines (other keys of the same JSON line): the 256 x 256 atom-diatom
workload, 3D harmonic 32^3, 16^8 FP32, mixed precision, batch, adjoint,
convergence orders, an ensemble.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica on its own GPU
(the single-grid path has no data to exchange); value is the sum over ranks
divided by the slowest rank's time.
"""
import argparse
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

METRIC = "grid-point·steps/s on 1 GB300 at stated error vs FP64 oracle; % HBM roofline"
UNIT = "grid-point·steps/s"
AMU = 1822.888486
N_GRID = (256, 256)
DQ = (0.08, 0.04)
MINV = (1 / (2.67 * AMU), 1 / (0.5 * AMU))
POT = [0.17, 1.0, 1.4, 5.0, 1.8]  # Dm, a, re, A, beta
SCHEME, STAGES, DT = "yoshida4", 3, 1.0
STEPS_PER_CALL = 100
CPU_SAMPLE_STEPS = 30
# headline: 8D Henon-Heiles, 12^8 FP64
HH_N, HH_D, HH_LAM = 12, 8, 0.111803
HH_SCHEME, HH_STAGES, HH_DT = "suzuki4", 5, 0.01
HH_STEPS_PER_CALL = 3  # time steps per timed call: 3 x 5 stages, 16 kinetic units after merging
HH_E2E_ITERS = 5
HH_CPU_D = 5   # oracle sample: the same model on 12^5, one time step
HH_REF_D = 4   # reference arm: one time step on 12^4 per timed step
ADJ_STEPS = 2000  # the full length of the gradient workload
FLUSH_BYTES = 512 << 20  # > 129 MB L2

# DRAM bytes (read + write) of one headline propagate launch (HH_STEPS_PER_CALL
# time steps on 12^8), from an ncu capture of the same launch shape on 12^7
# scaled by 12 (both plans make three group passes per transform, so the
# traffic grows with the points streamed); valid only for the kernel sources
# it was taken on (sha256 of the files below, concatenated).
TRAFFIC_RECORD = {"kernel_sha256": "b75ca5663633c7aabe3b4aad4a7d4f24fdef045a54cefd26460f78a74f4367c1",
                  "bytes_per_launch": 1.338555108e12}  # (55.30 + 56.24) GB on 12^7 x 12
KERNEL_SOURCES = ("mg_short.cu", "mg_short.h", "mg_device.cuh", "mg_plan.h")

# FP64 peak from unit counts and clocks (152 SMs x 2 FP64 FMA/clk x 2 flop x
# 2.07 GHz): used only where the measured rate is missing
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def algorithmic_flops_per_point_stage(N, D):
    """5 log2(N) per transform (radix-2 count, two transforms per stage),
    10 D for the diagonal phase factors, 2 (D + 2) for the reductions."""
    n = int(np.prod(N))
    return 2 * 5 * math.log2(n) + 10 * D + 2 * (D + 2)


def algorithmic_bytes_per_point_stage(elem=16):
    return 4 * elem  # read + write of psi for the forward and for the inverse transform


def initial(mgmod):
    rbar = mgmod.mg_morse_mean(POT[0], POT[1], POT[2], 0.5 * AMU)
    fac = [("gauss", 8.0, -10.0, 0.5), ("morse", POT[0], POT[1], POT[2], 0.5 * AMU)]
    return fac, [8.0, rbar], [-10.0, 0.0]


def traffic_per_launch():
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1909_06412_gb300", "csrc", f), "rb").read())
    h = h.hexdigest()
    return TRAFFIC_RECORD["bytes_per_launch"] if h == TRAFFIC_RECORD["kernel_sha256"] else None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d.get("hbm_gbs", 6800.0)), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus, backend="nccl"):
    """One process per GPU under torchrun (RANK/WORLD_SIZE/MASTER_* from the
    environment); (rank, world, local rank, torch.distributed or None)."""
    if n_gpus <= 1 and "RANK" not in os.environ:
        return 0, 1, 0, None
    import torch.distributed as dist

    dist.init_process_group(backend)
    return dist.get_rank(), dist.get_world_size(), int(os.environ.get("LOCAL_RANK", 0)), dist


def job_time_and_units(t_local, units_local, dist, device="cpu"):
    """Whole-job numbers of independent replicas: the slowest rank's time and
    the units all ranks processed (no data-path collective: only these two
    numbers cross ranks)."""
    if dist is None:
        return t_local, units_local
    import torch

    v = torch.tensor([t_local, float(units_local)], dtype=torch.float64, device=device)
    t = v[:1].clone()
    u = v[1:].clone()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def headline_config(world):
    """The workload of the headline line, shared by both arms."""
    return {
        "workload": f"8D Henon-Heiles (Sec. III.C), {HH_N}^{HH_D} moving grid, FP64 complex128 "
                    f"({HH_N ** HH_D:.3g} points, {16 * HH_N ** HH_D / 1e9:.2f} GB), {HH_SCHEME} "
                    f"({HH_STAGES} TVT stages per step), dt = {HH_DT}, lambda = {HH_LAM}",
        "grid": [HH_N] * HH_D, "scheme": HH_SCHEME, "stages_per_step": HH_STAGES, "dt": HH_DT,
        "time_steps_per_iteration": HH_STEPS_PER_CALL,
        "parallelism": "replicas" if world > 1 else "single GPU",
    }


def hh_oracle(oracle, D):
    """The headline model on a 12^D grid for the oracle (same n, lambda,
    spacing, initial Gaussians at q = 2)."""
    dq = math.sqrt(2 * math.pi / HH_N)
    o = oracle.Grid((HH_N,) * D, (dq,) * D)
    o.set_potential(oracle.POT_HENON_HEILES, [HH_LAM])
    o.set_separable([("gauss", 2.0, 0.0, 1.0)] * D, [2.0] * D, [0.0] * D)
    return o


def _oracle_sample_worker(D):
    """One oracle time step of the headline model on a 12^D grid (its own
    process); returns (points, seconds)."""
    import oracle

    o = hh_oracle(oracle, D)
    t0 = time.perf_counter()
    o.propagate(1, HH_DT, HH_SCHEME)
    return HH_N ** D, time.perf_counter() - t0


def oracle_all_cores(D):
    """The oracle as it stands (single-threaded) on every host core at once:
    one process per core, each running the same sample; throughput = points x
    steps of all processes / the slowest process's time."""
    import multiprocessing as mp

    n = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(n) as pool:
        res = pool.map(_oracle_sample_worker, [D] * n)
    wall = time.perf_counter() - t0
    pts = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return pts / slowest, n, slowest, wall


def cpu_model():
    """The host CPU's model name (lscpu), else what /proc/cpuinfo names."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.machine()


def run_reference(args):
    """The FP64 CPU oracle on the host cores (one thread) for the headline
    model: each timed step is HH_STEPS_PER_CALL time steps on a 12^4 grid (a
    bounded sample of the 12^8 workload: same model, axis length, scheme, dt
    and steps per iteration)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    o = hh_oracle(oracle, HH_REF_D)
    for _ in range(args.warmup):
        o.propagate(1, HH_DT, HH_SCHEME)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.propagate(HH_STEPS_PER_CALL, HH_DT, HH_SCHEME)
    el = time.perf_counter() - t0
    npts = HH_N ** HH_REF_D
    v = npts * HH_STEPS_PER_CALL * args.steps / el
    sample = (f"{args.steps} x {HH_STEPS_PER_CALL} time steps of the headline model on a {HH_N}^{HH_REF_D} grid (the oracle's cost "
              f"per point grows with the number of axes, so this favours it), single thread, {cpu_model()}")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(headline_config(args.gpus), l2="not applicable: the CPU oracle"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def cpu_baseline_and_error(mgmod, torch):
    """Oracle on a bounded sample (CPU_SAMPLE_STEPS steps) and the GPU on the
    same sample: returns the timing and the stated error vs the oracle."""
    import oracle

    fac, qc, pc = initial(mgmod)
    o = oracle.Grid(N_GRID, DQ, minv=MINV)
    o.set_potential(oracle.POT_ATOM_DIATOM, POT)
    o.set_separable(fac, qc, pc)
    t0 = time.perf_counter()
    o.propagate(CPU_SAMPLE_STEPS, DT, SCHEME)
    el = time.perf_counter() - t0
    psi_o, q_o, p_o, _ = o.get_state()
    g = mgmod.Propagator(N_GRID, DQ, minv=MINV)
    g.set_potential(mgmod.MG_POT_ATOM_DIATOM, POT)
    g.set_separable(fac, qc, pc)
    g.propagate(CPU_SAMPLE_STEPS, DT, SCHEME)
    psi, q, p, _ = g.get_state()
    npts = int(np.prod(N_GRID))
    err = {
        "psi_rel_l2": float(np.linalg.norm(psi - psi_o) / np.linalg.norm(psi_o)),
        "q_abs": float(np.abs(q - q_o).max()), "p_abs": float(np.abs(p - p_o).max()),
        "steps": CPU_SAMPLE_STEPS,
    }
    cpu = {"value": npts * CPU_SAMPLE_STEPS / el, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{CPU_SAMPLE_STEPS} time steps of the same 256x256 workload from its initial state, "
                     f"single thread, {el:.1f} s"}
    return cpu, err


def hh_propagator(mgmod, n, D, prec, dev=None):
    """Henon-Heiles (lambda = 0.111803) on an n^D grid with balanced windows
    (dq = sqrt(2 pi / n)), Gaussians at q = 2 with unit width."""
    dq = math.sqrt(2 * math.pi / n)
    g = mgmod.Propagator((n,) * D, (dq,) * D, precision=prec, device=dev)
    g.set_potential(mgmod.MG_POT_HENON_HEILES, [0.111803])
    g.set_separable([("gauss", 2.0, 0.0, 1.0)] * D, [2.0] * D, [0.0] * D)
    return g


def run_profile(args):
    """The timed launches of a workload alone, for profiler captures: the
    propagate kernel is launched warmup + steps times.  --profile-case
    hh8_fp64 (default): the headline, 12^8 FP64, HH_STEPS_PER_CALL time steps
    per call as timed;
    hh7_fp64 / hh7_fp32: Henon-Heiles on 12^7 (FP64) / 16^7 (FP32) grids, the
    small cases for full captures, with the same time steps per call; atom_diatom: the 256 x 256 workload,
    STEPS_PER_CALL steps per call; tc_dft16: the standalone 16-point DFT on
    TC_PROFILE_LINES lines, register form then 3xTF32 then BF16x3."""
    import torch
    import paper_1909_06412_gb300 as mg

    if args.profile_case == "tc_dft16":
        x, pre, post = dft16_inputs(torch, torch.device("cuda", 0), TC_PROFILE_LINES)
        y = torch.empty_like(x)
        st = torch.cuda.current_stream()
        for split in (0, 1, 2):
            for _ in range(args.warmup + args.steps):
                mg.mg_probe_tc_dft16(x, pre, post, split, False, st, out=y)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "case": args.profile_case, "lines": TC_PROFILE_LINES}))
        return
    if args.profile_case == "atom_diatom":
        fac, qc, pc = initial(mg)
        g = mg.Propagator(N_GRID, DQ, minv=MINV)
        g.set_potential(mg.MG_POT_ATOM_DIATOM, POT)
        g.set_separable(fac, qc, pc)
        call = lambda: g.propagate(STEPS_PER_CALL, DT, SCHEME)
    else:
        n, D, prec = {"hh8_fp64": (12, 8, mg.MG_FP64), "hh7_fp32": (16, 7, mg.MG_FP32_MIXED),
                      "hh7_fp64": (12, 7, mg.MG_FP64)}[args.profile_case]
        g = hh_propagator(mg, n, D, prec)
        k = HH_STEPS_PER_CALL  # the launch shape of the timed region
        call = lambda: g.propagate(k, HH_DT, HH_SCHEME)
    for _ in range(args.warmup + args.steps):
        call()
    g.sync()
    print(json.dumps({"profile_run": True, "case": args.profile_case, "launches": g.launches}))


def other_workloads(mgmod, torch, dev, flush):
    """The paper's other workload shapes, each timed over one propagate call
    after one warm-up call (state resident in HBM, L2 flushed before the call):
    3D harmonic 32^3 FP64 Strang; 8D Henon-Heiles 12^8 FP64 and 16^8 FP32,
    fourth-order Suzuki, dt = 0.01.  After the timed call: the drifts of the
    norm and the energy over it, and its reversibility error (the same number
    of steps back with -dt, then the distance to the state before the timed
    call, measured on the device)."""
    out = []
    cases = [
        ("3D harmonic 32^3 FP64, strang, dt=0.01", (32, 32, 32), (0.3,) * 3, mgmod.MG_FP64,
         mgmod.MG_POT_HARMONIC, list(np.diag(np.array([1.0, 1.2, 1.5]) ** 2).ravel()) + [0.0] * 3,
         [("gauss", q, p, w ** -0.5) for q, p, w in zip((1.0, -0.5, 0.8), (0.0, 0.5, -0.3), (1.0, 1.2, 1.5))],
         (1.0, -0.5, 0.8), (0.0, 0.5, -0.3), "strang", 1, 0.01, 200, 16),
        ("8D Henon-Heiles 12^8 FP64, suzuki4, dt=0.01", (12,) * 8, (math.sqrt(2 * math.pi / 12),) * 8,
         mgmod.MG_FP64, mgmod.MG_POT_HENON_HEILES, [0.111803], [("gauss", 2.0, 0.0, 1.0)] * 8,
         (2.0,) * 8, (0.0,) * 8, "suzuki4", 5, 0.01, 2, 16),
        ("8D Henon-Heiles 16^8 FP32 mixed, suzuki4, dt=0.01", (16,) * 8, (math.sqrt(2 * math.pi / 16),) * 8,
         mgmod.MG_FP32_MIXED, mgmod.MG_POT_HENON_HEILES, [0.111803], [("gauss", 2.0, 0.0, 1.0)] * 8,
         (2.0,) * 8, (0.0,) * 8, "suzuki4", 5, 0.01, 2, 8),
    ]
    for name, N, dq, prec, kind, pot, fac, q0, p0, scheme, stages, dt, steps, elem in cases:
        g = mgmod.Propagator(N, dq, precision=prec, device=dev)
        g.set_potential(kind, pot)
        g.set_separable(fac, q0, p0)
        g.propagate(1, dt, scheme)
        g.sync()
        n0, E0 = g.observables()[:2]
        psi0 = g.psi.clone()
        _, qs0, ps0, _ = g.get_state(want_psi=False)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(g.stream)
        g.propagate(steps, dt, scheme)
        e1.record(g.stream)
        g.sync()
        t = e0.elapsed_time(e1) / 1e3
        n1, E1 = g.observables()[:2]
        g.propagate(steps, -dt, scheme)
        g.sync()
        _, qs1, ps1, _ = g.get_state(want_psi=False)
        ref_norm = float(torch.linalg.vector_norm(psi0))
        psi0.sub_(g.psi)
        rev = float(torch.linalg.vector_norm(psi0)) / ref_norm
        del psi0
        npts = int(np.prod(N))
        ps = npts * steps * stages / t
        D = len(N)
        hbm_peak, _ = peaks()
        gbs = ps * 4 * elem / 1e9
        tf = ps * algorithmic_flops_per_point_stage(N, D) / 1e12 if prec == 0 else None
        out.append({
            "workload": name, "value": npts * steps / t, "unit": UNIT, "points": npts,
            "stages_per_step": stages, "ms_per_step": 1e3 * t / steps,
            "kernel_path": {0: "general", 1: "short-axis", 2: "short-axis, TMA copies"}.get(g.path, str(g.path)),
            "hbm_gbs_algorithmic": gbs, "hbm_frac_algorithmic": gbs / hbm_peak,
            "fp64_tflops_algorithmic": tf, "fp64_frac_algorithmic": tf / fp64_peak() if tf is not None else None,
            "norm_drift": n1 / n0 - 1, "energy_drift": E1 / E0 - 1,
            "reversibility": {"psi_rel_l2": rev, "q_abs": float(np.abs(qs1 - qs0).max()),
                              "p_abs": float(np.abs(ps1 - ps0).max()), "steps": steps},
        })
        g.close()
        del g
        torch.cuda.empty_cache()
    return out


def mixed_precision_leg(mgmod, torch, dev, args, flush):
    """The same workload with FP32 storage and transforms (FP64 phase
    arguments, reductions and centres): device throughput timed like the main
    line, and its error against the FP64 oracle on the CPU-baseline sample."""
    import oracle

    fac, qc, pc = initial(mgmod)
    g = mgmod.Propagator(N_GRID, DQ, minv=MINV, device=dev, precision=mgmod.MG_FP32_MIXED)
    g.set_potential(mgmod.MG_POT_ATOM_DIATOM, POT)
    g.set_separable(fac, qc, pc)
    for _ in range(max(3, args.warmup)):
        g.propagate(STEPS_PER_CALL, DT, SCHEME)
    g.sync()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(g.stream)
        g.propagate(STEPS_PER_CALL, DT, SCHEME)
        e1.record(g.stream)
        ms.append((e0, e1))
    g.sync()
    t = sum(a.elapsed_time(b) for a, b in ms) / 1e3
    npts = int(np.prod(N_GRID))
    g2 = mgmod.Propagator(N_GRID, DQ, minv=MINV, device=dev, precision=mgmod.MG_FP32_MIXED)
    g2.set_potential(mgmod.MG_POT_ATOM_DIATOM, POT)
    g2.set_separable(fac, qc, pc)
    g2.propagate(CPU_SAMPLE_STEPS, DT, SCHEME)
    psi, q, p, _ = g2.get_state()
    o = oracle.Grid(N_GRID, DQ, minv=MINV)
    o.set_potential(oracle.POT_ATOM_DIATOM, POT)
    o.set_separable(fac, qc, pc)
    o.propagate(CPU_SAMPLE_STEPS, DT, SCHEME)
    psi_o, q_o, p_o, _ = o.get_state()
    return {
        "dtype": "f32 storage/transforms, f64 phase arguments, reductions and centres",
        "value": npts * STEPS_PER_CALL * args.steps / t, "unit": UNIT,
        "ms_per_step": 1e3 * t / args.steps,
        "error_vs_oracle": {"psi_rel_l2": float(np.linalg.norm(psi - psi_o) / np.linalg.norm(psi_o)),
                            "q_abs": float(np.abs(q - q_o).max()), "p_abs": float(np.abs(p - p_o).max()),
                            "steps": CPU_SAMPLE_STEPS},
    }


def adjoint_leg(mgmod, torch, dev):
    """Cost of the reversible adjoint against the forward propagation it
    differentiates, on the two gradient workloads (FP64, sixth-order triple
    jump, 9 TVT stages per step): the atom-diatom model on a 128 x 128 grid
    (dR = 0.16, dr = 0.08, dt = 1 a.u.) and the 3D harmonic oscillator on a
    64^3 grid (dq = 0.3, dt = 0.01).  Each is timed over one forward call of
    ADJ_STEPS steps and the adjoint call that rewinds it."""
    out = []
    rbar = mgmod.mg_morse_mean(POT[0], POT[1], POT[2], 0.5 * AMU)
    om = np.array([1.0, 1.2, 1.5])
    cases = [
        ("atom-diatom 128x128 FP64, yoshida6, dt=1 a.u.", (128, 128), (0.08, 0.08), MINV,
         mgmod.MG_POT_ATOM_DIATOM, POT, initial(mgmod)[0], [8.0, rbar], [-10.0, 0.0], 1.0),
        ("3D harmonic 64^3 FP64, yoshida6, dt=0.01", (64, 64, 64), (0.3,) * 3, (1.0, 1.0, 1.0),
         mgmod.MG_POT_HARMONIC, list(np.diag(om ** 2).ravel()) + [0.0] * 3,
         [("gauss", q, p, w ** -0.5) for q, p, w in zip((1.0, -0.5, 0.8), (0.0, 0.5, -0.3), om)],
         (1.0, -0.5, 0.8), (0.0, 0.5, -0.3), 0.01),
    ]
    for name, N, dq, minv, kind, pot, fac, q0, p0, dt in cases:
        g = mgmod.Propagator(N, dq, minv=minv, device=dev)
        g.set_potential(kind, pot)
        g.set_separable(fac, q0, p0)
        D = len(N)
        ub = torch.zeros(int(np.prod(N)), dtype=torch.complex128, device=dev)
        qb, pb = np.eye(D)[0], np.zeros(D)
        # warm-up pair, then the timed pair
        g.propagate(2, dt, "yoshida6")
        g.adjoint(2, dt, "yoshida6", ub, qb, pb)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(g.stream)
        g.propagate(ADJ_STEPS, dt, "yoshida6")
        ev[1].record(g.stream)
        g.sync()
        g.adjoint(ADJ_STEPS, dt, "yoshida6", ub, qb, pb)
        ev[2].record(g.stream)
        g.sync()
        tf, ta = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
        out.append({"workload": name, "steps": ADJ_STEPS, "forward_s": tf, "adjoint_s": ta,
                    "adjoint_over_forward": ta / tf,
                    "note": "adjoint_s includes the host-side norm readout and cotangent upload of mg_adjoint",
                    "scope": "mg_adjoint: FP64 grids resident in the CTAs' shared memory, harmonic and "
                             "atom-diatom potentials"})
        g.close()
        del g
        torch.cuda.empty_cache()
    return out


ORDER_T = 32.0
ORDER_DTS = (2.0, 1.0, 0.5, 0.25)
ORDER_SCHEMES = (("strang", 1), ("yoshida4", 3), ("yoshida6", 9), ("yoshida8", 27), ("yoshida10", 81),
                 ("suzuki4", 5), ("suzuki6", 25))
ENSEMBLE_MEMBERS = 152
ENSEMBLE_STEPS = 20


def headline_propagator(mgmod, dev, precision=None):
    fac, qc, pc = initial(mgmod)
    g = mgmod.Propagator(N_GRID, DQ, minv=MINV, device=dev,
                         precision=mgmod.MG_FP64 if precision is None else precision)
    g.set_potential(mgmod.MG_POT_ATOM_DIATOM, POT)
    g.set_separable(fac, qc, pc)
    return g


def order_leg(mgmod, torch, dev):
    """Error against composition order and time step on the atom-diatom
    256 x 256 FP64 workload: every scheme runs to t = ORDER_T a.u. at each
    time step of ORDER_DTS.  As in the paper's convergence figures (Sec. III),
    the error of a run is its L2 distance to the run with half the time step,
    carried onto that run's grid by trigonometric interpolation (mg_regrid);
    the observed order is log2 of the ratio of successive errors."""
    out = []
    npts = int(np.prod(N_GRID))
    for scheme, stages in ORDER_SCHEMES:
        runs = []
        for dt in ORDER_DTS:
            g = headline_propagator(mgmod, dev)
            n = int(round(ORDER_T / dt))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(g.stream)
            g.propagate(n, dt, scheme)
            e1.record(g.stream)
            g.sync()
            runs.append((g, n, e0.elapsed_time(e1)))
        errs = []
        for k in range(len(runs) - 1):
            a, b = runs[k][0], runs[k + 1][0]
            _, qb, pb, _ = b.get_state(want_psi=False)
            a.regrid(qb, pb)
            ua, ub = a.get_state()[0], b.get_state()[0]
            errs.append(float(np.linalg.norm(ua - ub) / np.linalg.norm(ub)))
        orders = [math.log2(errs[k] / errs[k + 1]) if min(errs[k], errs[k + 1]) > 1e-11 else None
                  for k in range(len(errs) - 1)]
        out.append({"scheme": scheme, "stages_per_step": stages, "dt": list(ORDER_DTS[:-1]), "error": errs,
                    "observed_order": orders, "ms": [r[2] for r in runs[:-1]],
                    "gp_stages_per_s": [npts * r[1] * stages / (r[2] / 1e3) for r in runs[:-1]]})
        for g, _, _ in runs:
            g.close()
        del runs
        torch.cuda.empty_cache()
    return {"workload": f"collinear atom-diatom 256x256 FP64, t = {ORDER_T} a.u.", "results": out,
            "error_definition": "||psi(dt) - psi(dt/2)|| / ||psi(dt/2)||, psi(dt) interpolated onto the "
                                "grid of the dt/2 run"}


def ensemble_leg(mgmod, torch, dev):
    """The headline problem as an ensemble: ENSEMBLE_MEMBERS independent copies
    in one batched launch (mg_batch_*, FP64), one or two CTAs per member
    (thread-block clusters of 1 or 2) instead of the whole GPU per member.
    Reports whole-ensemble throughput, its FP64 roofline fraction and the
    distance of a member to the single-grid result."""
    npts = int(np.prod(N_GRID))
    ref = headline_propagator(mgmod, dev)
    ref.propagate(2 + ENSEMBLE_STEPS, DT, SCHEME)
    ref_psi = ref.get_state()[0]
    ref.close()
    out = {"workload": f"{ENSEMBLE_MEMBERS} independent members of the headline atom-diatom 256x256 FP64 run, "
                       f"{SCHEME}, dt = {DT} a.u.", "members": ENSEMBLE_MEMBERS, "steps": ENSEMBLE_STEPS}
    for cluster in (1, 2):
        gs = [headline_propagator(mgmod, dev) for _ in range(ENSEMBLE_MEMBERS)]
        try:
            b = mgmod.Batch(gs, cluster=cluster)
        except mgmod.MgError as e:  # a launch shape this GPU cannot place
            out[f"cluster_{cluster}"] = {"unavailable": str(e)}
            for g in gs:
                g.close()
            continue
        dts = np.full(ENSEMBLE_MEMBERS, DT)
        b.propagate(2, dts, SCHEME)
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(gs[0].stream)
        b.propagate(ENSEMBLE_STEPS, dts, SCHEME)
        e1.record(gs[0].stream)
        b.sync()
        t = e0.elapsed_time(e1) / 1e3
        err = max(float(np.linalg.norm(gs[i].get_state()[0] - ref_psi) / np.linalg.norm(ref_psi))
                  for i in (0, ENSEMBLE_MEMBERS - 1))
        v = npts * ENSEMBLE_STEPS * ENSEMBLE_MEMBERS / t
        tf = v * STAGES * algorithmic_flops_per_point_stage(N_GRID, 2) / 1e12
        out[f"cluster_{cluster}"] = {"value": v, "unit": UNIT, "s": t, "teams": b.info()["teams"],
                                     "fp64_tflops_algorithmic": tf, "fp64_frac_algorithmic": tf / fp64_peak(),
                                     "psi_rel_l2_vs_single_grid": err}
        b.close()
        for g in gs:
            g.close()
        del gs
        torch.cuda.empty_cache()
    return out


BATCH_STEPS = 200
BATCH_SEPARATE_STEPS = 20


def batch_problem_setup(mgmod, pr, precision):
    """One problem of the seeded batch workload as a Propagator."""
    g = mgmod.Propagator(pr["N"], pr["dq"], minv=1.0 / np.array(pr["mass"]), precision=precision)
    if pr["kind"] == "atom_diatom":
        g.set_potential(mgmod.MG_POT_ATOM_DIATOM, list(pr["pot"]))
    else:
        k, c = pr["pot"]
        g.set_potential(mgmod.MG_POT_HARMONIC, list(np.diag(k).ravel()) + list(c))
    batch_problem_initial(mgmod, g, pr)
    return g


def batch_problem_initial(mgmod, g, pr):
    """(Re)set a batch problem's initial state and grid centre."""
    if pr["kind"] == "atom_diatom":
        Dm, a, re, A, be = pr["pot"]
        R0, P0, sg = pr["gauss"][0]
        mr = pr["mass"][1]
        g.set_separable([("gauss", R0, P0, sg), ("morse", Dm, a, re, mr)],
                        [R0, mgmod.mg_morse_mean(Dm, a, re, mr)], [P0, 0.0])
    else:
        g.set_separable([("gauss", q, p, sg) for q, p, sg in pr["gauss"]],
                        [f[0] for f in pr["gauss"]], [f[1] for f in pr["gauss"]])


def batch_leg(mgmod, torch, dev):
    """Batched serving-style launch on the seeded 512-grid workload (256 2D
    grids of 64^2..256^2 points, harmonic or atom-diatom; 256 3D harmonic grids
    of 16^3..48^3; parameters within +-20% of the 3D harmonic and atom-diatom
    workloads): FP32 storage with FP64 reductions, suzuki4, one graph-replayed
    batched launch of BATCH_STEPS steps, with the launch knobs from the
    autotuner; against the same problems as 512 separate plain FP64
    mg_propagate launches of BATCH_SEPARATE_STEPS steps each."""
    import tempfile

    from paper_1909_06412_gb300 import autotune
    from tests import inputs

    probs = inputs.batch_problems()
    dts = np.array([pr["dt"] for pr in probs])
    pts = np.array([int(np.prod(pr["N"])) for pr in probs])
    gs = [batch_problem_setup(mgmod, pr, mgmod.MG_FP32_MIXED) for pr in probs]
    cache = os.path.join(tempfile.mkdtemp(), "autotune.json")
    t0 = time.perf_counter()
    s, tb, rm, entry = autotune.tune_batch(gs, BATCH_STEPS, dts, "suzuki4", trial_steps=4, cache_path=cache)
    tune_s = time.perf_counter() - t0
    MEASURED["batch_knobs_fp32"] = {"cluster": s["cluster"], "tile_bytes": tb, "radix_max": rm}
    out = {"workload": "seeded 512-grid batch (2D 64^2-256^2, 3D 16^3-48^3), FP32 storage + FP64 reductions, "
                       "suzuki4", "points": int(pts.sum()), "problems": len(probs),
           "autotune": {"settings": s, "trials": entry["trials"], "tuning_s": tune_s,
                        "trial_s_per_step_default": entry["default_seconds_per_step"],
                        "trial_s_per_step_tuned": entry["seconds_per_step"]}}
    for label, kw in (("default", {}), ("tuned", {"cluster": s["cluster"], "tile_bytes": tb, "radix_max": rm})):
        b = mgmod.Batch(gs, **kw)
        b.propagate(2, dts, "suzuki4")
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(gs[0].stream)
        b.propagate(BATCH_STEPS, dts, "suzuki4")
        e1.record(gs[0].stream)
        b.sync()
        t = e0.elapsed_time(e1) / 1e3
        out["batched_" + label] = {"value": float(pts.sum()) * BATCH_STEPS / t, "unit": UNIT, "s": t,
                                   "steps": BATCH_STEPS, "launches": b.info()["launches"]}
        b.close()
    # error of the batched FP32 result against the FP64 single-grid path
    # (itself pinned to the oracle), on every 64th problem after the runs above
    errs = []
    for i in range(0, len(probs), 64):
        ref = batch_problem_setup(mgmod, probs[i], mgmod.MG_FP64)
        ref.propagate(2 + BATCH_STEPS + 2 + BATCH_STEPS, dts[i], "suzuki4")
        a, b2 = gs[i].get_state()[0], ref.get_state()[0]
        errs.append(float(np.linalg.norm(a - b2) / np.linalg.norm(b2)))
        ref.close()
    out["batched_error_vs_fp64_single_grid"] = {"psi_rel_l2_max": max(errs), "problems_sampled": len(errs),
                                                "steps": 2 * (BATCH_STEPS + 2)}
    for g in gs:
        g.close()
    del gs
    torch.cuda.empty_cache()
    # 512 separate plain FP64 launches
    gd = [batch_problem_setup(mgmod, pr, mgmod.MG_FP64) for pr in probs]
    for g, dt in zip(gd, dts):
        g.propagate(1, dt, "suzuki4")
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(gd[0].stream)
    for g, dt in zip(gd, dts):
        g.propagate(BATCH_SEPARATE_STEPS, dt, "suzuki4")
    e1.record(gd[0].stream)
    torch.cuda.synchronize(dev)
    t = e0.elapsed_time(e1) / 1e3
    out["separate_fp64"] = {"value": float(pts.sum()) * BATCH_SEPARATE_STEPS / t, "unit": UNIT, "s": t,
                            "steps": BATCH_SEPARATE_STEPS, "launches": len(gd)}
    for g in gd:
        g.close()
    del gd
    torch.cuda.empty_cache()
    return out


TC_LINES = 1 << 22          # 64 M points: 512 MB in and 512 MB out, larger than L2
TC_PROFILE_LINES = 1 << 21


def dft16_inputs(torch, dev, nlines):
    """Seeded lines of 16 complex64 values and unit-modulus multipliers (the
    demodulation factor with the 1/16 of the transform pair, and a kinetic
    phase)."""
    g = np.random.default_rng(20190913)
    gen = torch.Generator(device=dev).manual_seed(20190913)
    x = torch.randn((nlines, 16), dtype=torch.complex64, device=dev, generator=gen)
    pre = np.exp(1j * g.uniform(-np.pi, np.pi, 16)) / 16
    post = np.exp(1j * g.uniform(-np.pi, np.pi, 16))
    return x, pre, post


def tc_dft16_leg(mgmod, torch, dev):
    """The 16-point line DFT of the FP32 16^D grids (eq:F_defintion along one
    axis, with its diagonal multipliers) as a standalone batched kernel in three
    forms: FP32 registers (the short-axis kernel's codelet), and the dense
    DFT-GEMM on the tensor cores (tcgen05.mma, kind::tf32 with 3xTF32 split
    products; kind::f16 with BF16x3).  Each is timed with CUDA events over 5
    launches on TC_LINES lines after 2 warm-up launches, and its error is taken
    against the FP64 product on 4096 sampled lines."""
    x, pre, post = dft16_inputs(torch, dev, TC_LINES)
    y = torch.empty_like(x)
    st = torch.cuda.current_stream(dev)
    sample = torch.arange(0, TC_LINES, TC_LINES // 4096, device=dev)
    xs = x[sample].cpu().numpy().astype(np.complex128)
    j = np.arange(16)
    F = np.exp(-2j * np.pi * np.outer(j, j) / 16)
    M = post.astype(np.complex64).astype(np.complex128)[:, None] * F * \
        pre.astype(np.complex64).astype(np.complex128)[None, :]
    ref = xs @ M.T
    npts = TC_LINES * 16
    out = {"workload": f"{TC_LINES} lines of 16 complex64 points ({npts * 8 / 1e9:.2f} GB in and out), "
                       "y = diag(post) F diag(pre) x", "bytes_per_point": 16,
           "dense_flops_per_point": 128}
    for split, name, mult in ((0, "register_fp32", 1), (1, "tcgen05_3xtf32", 3), (2, "tcgen05_bf16x3", 6)):
        for _ in range(2):
            mgmod.mg_probe_tc_dft16(x, pre, post, split, False, st, out=y)
        ms = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            mgmod.mg_probe_tc_dft16(x, pre, post, split, False, st, out=y)
            e1.record(st)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms) / 1e3
        err = float(np.abs(y[sample].cpu().numpy() - ref).max() / np.abs(ref).max())
        gbs = npts * 16 / t / 1e9
        out[name] = {"ms": 1e3 * t, "points_per_s": npts / t, "hbm_gbs": gbs,
                     "hbm_frac": gbs / peaks()[0],
                     "tensor_tflops": None if split == 0 else npts * 128 * mult / t / 1e12,
                     "max_rel_error_vs_fp64": err}
    best = min(("register_fp32", "tcgen05_3xtf32", "tcgen05_bf16x3"), key=lambda k: out[k]["ms"])
    out["fastest"] = best
    del x, y
    torch.cuda.empty_cache()
    return out


# Sec. III.A: 3D harmonic model (Table I), adaptive 32^3 (dq 0.4375, centred
# at the initial packet) against the fixed 128^3 grid with twice the q and p
# ranges, centred at the middle of the packet's sweep (the excited-state
# minimum q0); t_f = 50, dt = t_f / 2^9.
E2_TF, E2_STEPS, E2_CHECK = 50.0, 512, 128
# Sec. III.B: He-H2 scattering (eq:modified_secrest_johnson), VTV, dt = 0.1:
# adaptive and fixed 128 x 128 grids (q1 in (-14, 14), q2 in (0, 48)) against
# the fixed 128 x 2048 reference (q2 in (-50, 400)).
E7_DT, E7_STEPS, E7_CHECK = 0.1, 300, 10
ACC_SCHEME = "yoshida10"  # the tenth-order triple jump stands in for the unprinted optimal scheme


def adaptive_vs_fixed_leg(mgmod, torch, dev):
    """The accuracy of grid adaptation as the paper measures it (Figs. 3 and
    8): the distance ||psi_t - Psi_t|| between the adaptive-grid state and a
    fixed-grid reference on a larger, denser grid, the sparser state carried
    onto the denser grid by trigonometric interpolation (tests/grid_distance),
    and the difference of <q>.  Both runs use the same composition and dt."""
    from tests import grid_distance as gd
    from tests import inputs

    def grid_of(g):
        _, q, p, _ = g.get_state(want_psi=False)
        return {"N": list(g.N), "dq": list(g.dq), "q": list(q), "p": list(p)}

    def harmonic(N, dq, centre):
        P = inputs.DUSCHINSKY3D
        g = mgmod.Propagator(N, dq, minv=P["omega"], device=dev)
        g.set_potential(mgmod.MG_POT_HARMONIC, list(np.array(P["K"]).ravel()) + list(P["q0"]))
        g.set_separable([("gauss", 0.0, 0.0, 1.0)] * 3, list(centre), [0.0] * 3)
        return g

    out = {"scheme": ACC_SCHEME}
    # E2: 3D harmonic
    dt = E2_TF / E2_STEPS
    ga = harmonic((32,) * 3, (0.4375,) * 3, (0.0,) * 3)
    gf = harmonic((128,) * 3, (0.21875,) * 3, inputs.DUSCHINSKY3D["q0"])
    rows = []
    t_a = t_f = 0.0
    for k in range(E2_STEPS // E2_CHECK + 1):
        if k:
            for g, motion, acc in ((ga, mgmod.MG_GRID_ADAPTIVE, "a"), (gf, mgmod.MG_GRID_FIXED, "f")):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(g.stream)
                g.propagate(E2_CHECK, dt, ACC_SCHEME, mgmod.MG_TVT, motion)
                e1.record(g.stream)
                g.sync()
                if acc == "a":
                    t_a += e0.elapsed_time(e1) / 1e3
                else:
                    t_f += e0.elapsed_time(e1) / 1e3
        psi_a, psi_f = ga.get_state()[0], gf.get_state()[0]
        sa, sf = grid_of(ga), grid_of(gf)
        rows.append({"t": k * E2_CHECK * dt, "distance": gd.distance(psi_a, sa, psi_f, sf),
                     "dq_mean_max": float(np.abs(gd.mean_q(psi_a, sa) - gd.mean_q(psi_f, sf)).max()),
                     "grid_centre_q": sa["q"]})
    out["E2_harmonic_3d"] = {
        "workload": f"Sec. III.A model (Table I, K13 = +0.017): adaptive 32^3 (dq 0.4375, centred at 0) vs "
                    f"fixed 128^3 (dq 0.21875, centred at q0), {ACC_SCHEME} TVT, dt = t_f/{E2_STEPS}, "
                    f"t_f = {E2_TF}",
        "paper": "5e-11 at t = 0 and 2e-10 at t_f (optimal tenth-order scheme)",
        "rows": rows, "gpu_s_adaptive": t_a, "gpu_s_fixed": t_f}
    ga.close(); gf.close()
    del ga, gf
    torch.cuda.empty_cache()

    # E7: He-H2 scattering
    sj = [20.0, 0.158, 0.3]
    fac = [("gauss", 0.0, 0.0, 1.0), ("gauss", 24.0, -3.56, np.sqrt(8.0))]

    def scattering(N, lo2, hi2):
        dq = (28.0 / N[0], (hi2 - lo2) / N[1])
        qc2 = lo2 + (N[1] // 2) * dq[1]
        g = mgmod.Propagator(N, dq, minv=(1.0, 1.5), device=dev)
        g.set_potential(mgmod.MG_POT_SECREST_JOHNSON, sj)
        g.set_separable(fac, [0.0, qc2], [0.0, -3.56])
        return g

    runs = {"adaptive_128x128": (scattering((128, 128), 0.0, 48.0), mgmod.MG_GRID_ADAPTIVE),
            "fixed_128x128": (scattering((128, 128), 0.0, 48.0), mgmod.MG_GRID_FIXED),
            "reference_fixed_128x2048": (scattering((128, 2048), -50.0, 400.0), mgmod.MG_GRID_FIXED)}
    ref = runs["reference_fixed_128x2048"][0]
    rows = []
    secs = {k: 0.0 for k in runs}
    for k in range(E7_STEPS // E7_CHECK + 1):
        if k:
            for name, (g, motion) in runs.items():
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(g.stream)
                g.propagate(E7_CHECK, E7_DT, ACC_SCHEME, mgmod.MG_VTV, motion)
                e1.record(g.stream)
                g.sync()
                secs[name] += e0.elapsed_time(e1) / 1e3
        psi_r, sr = ref.get_state()[0], grid_of(ref)
        row = {"t": k * E7_CHECK * E7_DT}
        for name in ("adaptive_128x128", "fixed_128x128"):
            g = runs[name][0]
            psi, s = g.get_state()[0], grid_of(g)
            row[name] = {"distance": gd.distance(psi, s, psi_r, sr),
                         "dq_mean": list(gd.mean_q(psi, s) - gd.mean_q(psi_r, sr))}
        rows.append(row)
    first = {}
    for name in ("adaptive_128x128", "fixed_128x128"):
        over = [r["t"] for r in rows if r[name]["distance"] > 1e-3]
        first[name] = over[0] if over else None
    out["E7_scattering"] = {
        "first_t_error_above_1e-3": first,
        "workload": f"Sec. III.B He-H2 (eq:modified_secrest_johnson), {ACC_SCHEME} VTV, dt = {E7_DT}: adaptive "
                    f"and fixed 128 x 128 grids vs the fixed 128 x 2048 reference",
        "paper": "adaptive error < 1e-3 six times longer than the fixed grid's; <q> error small until t ~ 20",
        "rows": rows, "gpu_s": secs,
        "reference_tables_in_workspace": ref.tables_in_workspace}
    for g, _ in runs.values():
        g.close()
    del runs, ref
    torch.cuda.empty_cache()
    return out


# Equal stated error: every (precision, scheme, dt) of the atom-diatom 256^2
# workload run to EQ_T, its distance to an FP64 eighth-order run at dt 0.125,
# and per target error the fastest run of each precision that meets it.
EQ_T = 32.0
EQ_DTS = (2.0, 1.0, 0.5, 0.25)
EQ_SCHEMES = (("strang", 1), ("yoshida4", 3), ("suzuki4", 5), ("yoshida6", 9))
EQ_TARGETS = (1e-3, 1e-4, 1e-5, 1e-6, 1e-8, 1e-10)


def pick_fastest(runs, target):
    ok = [r for r in runs if r["error"] <= target]
    return min(ok, key=lambda r: r["s"]) if ok else None


def equal_error_leg(mgmod, torch, dev):
    """Mixed precision (FP32 storage and transforms) against plain FP64 at an
    equal stated error on the atom-diatom 256 x 256 workload: the time to reach
    t = EQ_T with an error below each target, choosing for each precision the
    fastest composition and time step that meets it."""
    from tests import grid_distance as gd

    def grid_of(g):
        _, q, p, _ = g.get_state(want_psi=False)
        return {"N": list(g.N), "dq": list(g.dq), "q": list(q), "p": list(p)}

    ref = headline_propagator(mgmod, dev)
    ref.propagate(int(round(EQ_T / 0.125)), 0.125, "yoshida8")
    psi_r, sr = ref.get_state()[0], grid_of(ref)
    ref.close()
    out = {"workload": f"collinear atom-diatom 256x256, t = {EQ_T} a.u.",
           "reference": "FP64 yoshida8, dt = 0.125 a.u.",
           "error_definition": "||psi - psi_ref||, psi carried onto the reference grid", "runs": []}
    for prec, pname in ((mgmod.MG_FP64, "fp64"), (mgmod.MG_FP32_MIXED, "fp32_mixed")):
        w = headline_propagator(mgmod, dev, prec)  # warm-up of this precision's kernels
        w.propagate(4, 1.0, "yoshida6")
        w.close()
        for scheme, stages in EQ_SCHEMES:
            for dt in EQ_DTS:
                g = headline_propagator(mgmod, dev, prec)
                n = int(round(EQ_T / dt))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(g.stream)
                g.propagate(n, dt, scheme)
                e1.record(g.stream)
                g.sync()
                psi = g.get_state()[0]
                out["runs"].append({"precision": pname, "scheme": scheme, "dt": dt, "stages": n * stages,
                                    "s": e0.elapsed_time(e1) / 1e3,
                                    "error": gd.distance(psi, grid_of(g), psi_r, sr)})
                g.close()
    rows = []
    for eps in EQ_TARGETS:
        a = pick_fastest([r for r in out["runs"] if r["precision"] == "fp64"], eps)
        b = pick_fastest([r for r in out["runs"] if r["precision"] == "fp32_mixed"], eps)
        rows.append({"target_error": eps, "fp64": a, "fp32_mixed": b,
                     "mixed_beats_fp64": None if a is None else (b is not None and b["s"] < a["s"]),
                     "fp64_s_over_mixed_s": a["s"] / b["s"] if a and b else None})
    out["at_equal_error"] = rows
    torch.cuda.empty_cache()
    return out


BATCH_EQ_STEPS = 40
BATCH_EQ_MULT = (1, 2, 4, 8)


def batch_equal_error_leg(mgmod, torch, dev, knobs32):
    """The batched launch at an equal stated error on the seeded 512-grid
    workload: FP64 and FP32 batches run the same simulated time with the
    problems' time steps multiplied by 1, 2, 4, 8 (BATCH_EQ_STEPS / k steps);
    errors on every 64th problem against the FP64 single-grid run of the same
    composition at the base time step (a higher-order reference would mix in
    the grids' truncation error, which depends on the grid's path: about 5e-6
    on the coarsest of these grids).  Also the FP64 batch against the 512
    separate FP64 launches over the same step count."""
    from paper_1909_06412_gb300 import autotune
    import tempfile
    from tests import inputs

    probs = inputs.batch_problems()
    dts = np.array([pr["dt"] for pr in probs])
    pts = np.array([int(np.prod(pr["N"])) for pr in probs])
    sample = list(range(0, len(probs), 64))
    refs = []
    for i in sample:
        r = batch_problem_setup(mgmod, probs[i], mgmod.MG_FP64)
        r.propagate(BATCH_EQ_STEPS, dts[i], "suzuki4")
        refs.append(r.get_state()[0])
        r.close()
    out = {"workload": "seeded 512-grid batch, suzuki4", "simulated_steps_at_base_dt": BATCH_EQ_STEPS,
           "reference": "FP64 single-grid suzuki4 at the base time step", "runs": []}
    for prec, pname in ((mgmod.MG_FP64, "fp64"), (mgmod.MG_FP32_MIXED, "fp32_mixed")):
        gs = [batch_problem_setup(mgmod, pr, prec) for pr in probs]
        if prec == mgmod.MG_FP64:
            cache = os.path.join(tempfile.mkdtemp(), "autotune64.json")
            s, tb, rm, _ = autotune.tune_batch(gs, BATCH_EQ_STEPS, dts, "suzuki4", trial_steps=4, cache_path=cache)
            knobs = {"cluster": s["cluster"], "tile_bytes": tb, "radix_max": rm}
            for g, pr in zip(gs, probs):
                batch_problem_initial(mgmod, g, pr)
        else:
            knobs = knobs32
        for k in BATCH_EQ_MULT:
            b = mgmod.Batch(gs, **knobs)
            n = BATCH_EQ_STEPS // k
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(gs[0].stream)
            b.propagate(n, dts * k, "suzuki4")
            e1.record(gs[0].stream)
            b.sync()
            t = e0.elapsed_time(e1) / 1e3
            err = max(float(np.linalg.norm(gs[i].get_state()[0] - ref) / np.linalg.norm(ref))
                      for i, ref in zip(sample, refs))
            out["runs"].append({"precision": pname, "dt_multiplier": k, "steps": n, "s": t, "error": err,
                                "value": float(pts.sum()) * n / t, "unit": UNIT})
            b.close()
            for g, pr in zip(gs, probs):
                batch_problem_initial(mgmod, g, pr)
        if prec == mgmod.MG_FP64:
            # the same problems as separate plain FP64 launches, same step count
            for g, dt in zip(gs, dts):
                g.propagate(1, dt, "suzuki4")
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(gs[0].stream)
            for g, dt in zip(gs, dts):
                g.propagate(BATCH_EQ_STEPS, dt, "suzuki4")
            e1.record(gs[0].stream)
            torch.cuda.synchronize(dev)
            t = e0.elapsed_time(e1) / 1e3
            bt = [r for r in out["runs"] if r["precision"] == "fp64" and r["dt_multiplier"] == 1][0]["s"]
            out["fp64_batch_vs_separate"] = {"steps": BATCH_EQ_STEPS, "separate_s": t, "batch_s": bt,
                                             "speedup": t / bt, "launches_separate": len(gs)}
        for g in gs:
            g.close()
        del gs
        torch.cuda.empty_cache()
    rows = []
    for eps in (1e-3, 1e-4, 1e-5, 1e-6, 1e-8):
        a = pick_fastest([r for r in out["runs"] if r["precision"] == "fp64"], eps)
        b = pick_fastest([r for r in out["runs"] if r["precision"] == "fp32_mixed"], eps)
        rows.append({"target_error": eps, "fp64": a, "fp32_mixed": b,
                     "mixed_beats_fp64": None if a is None else (b is not None and b["s"] < a["s"]),
                     "fp64_s_over_mixed_s": a["s"] / b["s"] if a and b else None})
    out["at_equal_error"] = rows
    return out


def fp64_peak():
    return MEASURED.get("fp64_tflops") or FP64_PEAK_TFLOPS


MEASURED = {}


def atom_diatom_leg(mg, torch, dev, args, flush):
    """The collinear atom-diatom workload (Sec. III.B model) on the 256 x 256
    FP64 grid, yoshida4, dt = 1 a.u.: STEPS_PER_CALL time steps per call, L2
    flushed before every timed call (its 1 MB state is L2-resident within a
    call), with its own roofline and error against the oracle."""
    npts = int(np.prod(N_GRID))
    g = headline_propagator(mg, dev)
    for _ in range(3):
        g.propagate(STEPS_PER_CALL, DT, SCHEME)
    g.sync()
    ms = []
    for _ in range(max(5, args.steps // 2)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(g.stream)
        g.propagate(STEPS_PER_CALL, DT, SCHEME)
        e1.record(g.stream)
        ms.append((e0, e1))
    g.sync()
    ms = [a.elapsed_time(b) for a, b in ms]
    g.close()
    t = statistics.mean(ms) / 1e3
    ps = npts * STEPS_PER_CALL * STAGES / t
    tf = ps * algorithmic_flops_per_point_stage(N_GRID, 2) / 1e12
    hbm_peak, _ = peaks()
    gbs = ps * algorithmic_bytes_per_point_stage() / 1e9
    cpu, err = cpu_baseline_and_error(mg, torch)
    return {"workload": "collinear atom-diatom 256x256 FP64, yoshida4 (3 stages per step), dt = 1 a.u.",
            "value": npts * STEPS_PER_CALL / t, "unit": UNIT, "ms_per_call": 1e3 * t,
            "time_steps_per_call": STEPS_PER_CALL, "calls": len(ms),
            "fp64_tflops_algorithmic": tf, "fp64_frac_algorithmic": tf / fp64_peak(),
            "hbm_frac_algorithmic": gbs / hbm_peak,
            "l2": "flushed before every timed call; the 1 MB state is L2-resident within a call",
            "error_vs_oracle": err, "cpu_baseline": cpu}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", action="store_true",
                    help="only the warm-up and timed propagate calls, as in the timed region (for ncu captures)")
    ap.add_argument("--profile-case", default="hh8_fp64",
                    choices=["hh8_fp64", "atom_diatom", "hh7_fp32", "hh7_fp64", "tc_dft16"])
    ap.add_argument("--headline-only", action="store_true", help="skip the secondary legs")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)

    import torch
    import paper_1909_06412_gb300 as mg

    rank, world, local, dist = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    warmup = max(3, args.warmup)

    # the FP64 FMA rate of this GPU: the roofline of the FP64 headline
    MEASURED["fp64_tflops"] = mg.mg_probe_fma_rate(mg.MG_FP64)
    MEASURED["fp32_tflops"] = mg.mg_probe_fma_rate(mg.MG_FP32_MIXED)

    g = hh_propagator(mg, HH_N, HH_D, mg.MG_FP64, dev)
    npts = g.npts
    stream = g.stream
    for _ in range(warmup):
        g.propagate(1, HH_DT, HH_SCHEME)
    g.sync()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # device-resident throughput: events on the library's stream around each
    # call; the 6.9 GB state is larger than L2, so nothing is flushed
    launches0 = g.launches
    times = []
    barrier()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.propagate(HH_STEPS_PER_CALL, HH_DT, HH_SCHEME)
            e1.record(stream)
            times.append((e0, e1))
        torch.cuda.synchronize(dev)
    barrier()
    wall = time.perf_counter() - wall0
    g.sync()
    launches = g.launches - launches0
    ms = [a.elapsed_time(b) for a, b in times]
    t_total, units = job_time_and_units(sum(ms) / 1e3, npts * HH_STEPS_PER_CALL * args.steps, dist, device=dev)
    value = units / t_total

    # end to end through the C-ABI with host buffers: every iteration uploads
    # the state from pinned host memory (mg_upload_u), propagates
    # HH_STEPS_PER_CALL time steps and reads the state back (mg_download_u)
    host = torch.empty(npts, dtype=torch.complex128, pin_memory=True)
    q, p, tt = g.download_u(host)
    barrier()
    e2e_t = []
    for _ in range(HH_E2E_ITERS):
        t0 = time.perf_counter()
        g.upload_u(host, q, p, tt)
        g.propagate(HH_STEPS_PER_CALL, HH_DT, HH_SCHEME)
        q, p, tt = g.download_u(host)
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = npts * HH_STEPS_PER_CALL * world / statistics.median(e2e_t)
    g.close()
    del g, host
    torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    hbm_peak, hbm_src = peaks()
    flops_ps = algorithmic_flops_per_point_stage((HH_N,) * HH_D, HH_D)
    t_launch = statistics.mean(ms) / 1e3
    ps = npts * HH_STAGES * HH_STEPS_PER_CALL / t_launch
    achieved_tf = flops_ps * ps / 1e12
    achieved_gbs = algorithmic_bytes_per_point_stage() * ps / 1e9
    # the oracle on a bounded sample of the same model: one time step on 12^5,
    # single-threaded and on every host core; and the GPU's error on it
    cpu_v, cpu_el = None, None
    import oracle

    o = hh_oracle(oracle, HH_CPU_D)
    t0 = time.perf_counter()
    o.propagate(1, HH_DT, HH_SCHEME)
    cpu_el = time.perf_counter() - t0
    cpu_v = HH_N ** HH_CPU_D / cpu_el
    all_v, ncores, all_slowest, _ = oracle_all_cores(HH_CPU_D)
    gs = hh_propagator(mg, HH_N, HH_CPU_D, mg.MG_FP64, dev)
    gs.propagate(1, HH_DT, HH_SCHEME)
    psi, qs, pss, _ = gs.get_state()
    psi_o, q_o, p_o, _ = o.get_state()
    gs.close()
    err = {"psi_rel_l2": float(np.linalg.norm(psi - psi_o) / np.linalg.norm(psi_o)),
           "q_abs": float(np.abs(qs - q_o).max()), "p_abs": float(np.abs(pss - p_o).max()),
           "sample": f"one time step of the same model on a {HH_N}^{HH_CPU_D} grid (same kernel family)"}
    cpu = {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"one time step of the headline model on a {HH_N}^{HH_CPU_D} grid ({cpu_el:.1f} s; the "
                     f"oracle's cost per point grows with the number of axes, so this favours it), single "
                     f"thread, {cpu_model()}",
           "all_cores": {"value": all_v, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": f"the same sample in {ncores} concurrent single-threaded oracle processes "
                                   f"(slowest {all_slowest:.1f} s)"}}

    secondary = {}
    if not args.headline_only:
        flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
        secondary["atom_diatom_256"] = atom_diatom_leg(mg, torch, dev, args, flush)
        secondary["mixed_precision"] = mixed_precision_leg(mg, torch, dev, args, flush)
        secondary["other_workloads"] = other_workloads(mg, torch, dev, flush)
        secondary["adjoint"] = adjoint_leg(mg, torch, dev)
        secondary["batch"] = batch_leg(mg, torch, dev)
        secondary["batch_equal_error"] = batch_equal_error_leg(mg, torch, dev, MEASURED["batch_knobs_fp32"])
        secondary["mixed_equal_error"] = equal_error_leg(mg, torch, dev)
        secondary["error_vs_order"] = order_leg(mg, torch, dev)
        secondary["ensemble"] = ensemble_leg(mg, torch, dev)
        secondary["dft16_tensor_cores"] = tc_dft16_leg(mg, torch, dev)
        secondary["adaptive_vs_fixed"] = adaptive_vs_fixed_leg(mg, torch, dev)
        del flush
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(headline_config(world),
                       l2="not flushed: the 6.9 GB state is larger than the 129 MB L2"),
        "gp_stages_per_s": value * HH_STAGES,
        "error_vs_oracle": err,
        "roofline": {
            "bound": "alu", "achieved": achieved_tf, "peak": fp64_peak(), "unit": "TFLOP/s",
            "frac": achieved_tf / fp64_peak(), "traffic": traffic_per_launch(),
            "kernel": f"k_propagate_short<double, 12> (persistent, one launch per {HH_STEPS_PER_CALL} time steps)",
            "flops_per_point_stage": flops_ps,
            "peak_source": "measured in this run: FP64 FMA rate (mg_probe_fma_rate, burst), "
                           f"nominal {FP64_PEAK_TFLOPS:.3f} = 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
            "fp32_fma_tflops_measured": MEASURED["fp32_tflops"],
            "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_gbs / hbm_peak, "peak_source": hbm_src,
                    "bytes_per_point_stage": algorithmic_bytes_per_point_stage()},
        },
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": npts * 16,
                "d2h_bytes_per_step": npts * 16,
                "note": f"mg_upload_u (pinned host psi) + mg_propagate ({HH_STEPS_PER_CALL} time steps) + "
                        f"mg_download_u (pinned host psi) per iteration, median of {HH_E2E_ITERS}"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "wall_s": wall,
    }
    line.update(secondary)
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
