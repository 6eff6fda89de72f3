"""Benchmark: grid points per second of one E_c^nl + v_nl evaluation
(Nq = 20, FP32 with FP64 energy) on the 180 x 180 x 72 double-wall nanotube
cell, through the C ABI of libvdwnl.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun) are independent
replicas: the method has no exchange between cells, so each rank evaluates
its own cell and the value is the points of all ranks over the slowest
rank's time (weak scaling).

--impl reference times the FP64 CPU oracle (the only other implementation:
the paper ships no code) on the host cores, on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "grid points/s for E_c^nl+v_nl (Nq=20, FP32)"
UNIT = "grid_points/s"
WORKLOAD = "dwnt_180x180x72_nq20"
HBM_FALLBACK = 6800.0


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


# algorithmic bytes per grid point of each stage (FP32 fields, complex64
# half spectrum with h = Nh/N1 of the points); the stage names are those of
# VdwNL.STAGES
def stage_bytes_per_point(Nq, N1):
    h = (N1 // 2 + 1) / N1
    return {
        "pointwise": 16 + 5 + Nq * 4 + 16,         # n, grad in; t, k, real theta, assembly coefficients out
        "planes_fwd": Nq * 4 + Nq * 8 * h,         # real theta in; theta(G) (x, z transformed) out
        "pencils_fwd": 2 * Nq * 8 * h,             # theta(G) in; y-transformed points in |G| order out
        "contract": 2 * Nq * 8 * h + 4 * h,        # theta(G) and |G| in, u(G) out
        "energy_final": 0.0,
        "pencils_inv": 2 * Nq * 8 * h,             # u(G) in |G| order in; y-transformed back out
        "planes_inv": Nq * 8 * h + Nq * 4,         # u(G) in; real u out
        "usum": Nq * 4 + 5 + 16 + 4 + 4,           # real u, t, k, coefficients in; v_loc and g out
        "w_planes": 4 + 12 + 3 * 8 * h,            # g, grad in; w(G) out
        "pencil_div": 3 * 8 * h + 8 * h,           # w(G) in, D.w(G) out
        "div_final": 8 * h + 4 + 4,                # D.w(G), v_loc in; v out
    }


def contract_flops_per_point(Nq, N1):
    """FP32 flops of the contraction per grid point: per half-spectrum point
    Nq(Nq+1)/2 cubic evaluations (3 FMA), the symmetric matrix-vector product
    (4 FMA per off-diagonal pair, 2 per diagonal one), the energy (2 FMA per
    field) and the 1/N scaling (2 products per field); 2 flops per FMA."""
    NP = Nq * (Nq + 1) // 2
    fma = 3 * NP + 4 * (NP - Nq) + 2 * Nq + 2 * Nq
    return (2 * fma + 2 * Nq) * (N1 // 2 + 1) / N1


# FP32 peak of the GPU from its unit counts: 152 SMs x 128 FP32 lanes x 2
# flops per FMA x the SM clock (2070 MHz at most)
FP32_LANES = 152 * 128


def fp32_peak_tflops(sm_mhz):
    return FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


# the sources of the plain path's kernels and of their launch configuration
PLAIN_SOURCES = ("api.cu", "common.cuh", "contract.cu", "fft.cuh", "pipeline.cu", "plane.cuh", "pointwise.cuh")


def source_sha1():
    """sha1 over the plain path's kernel sources (file name, then content, in
    name order); the learned path, the table generation and the
    no-allocation entry point live in other files."""
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_0812_0244_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f not in PLAIN_SOURCES:
            continue
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic(stage):
    """DRAM bytes per launch of a stage from the committed ncu capture, or None
    when there is none or the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_dwnt_180x180x72_nq20.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        parts = line.split()
        if len(parts) == 2 and not line.startswith("#"):
            vals[parts[0]] = parts[1]
    if vals.get("source_sha1") != source_sha1() or stage not in vals:
        return None
    return int(vals[stage])


def slowest_rank(x, world, dev=None):
    """The largest of each rank's x (max over the ranks of the process group;
    x itself for one rank): the timed region of a replica run is that of its
    slowest replica."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def b_alg(Nq):
    """Whole-call algorithmic bytes per point, 16 Nq + 76 (one HBM round trip
    of the Nq spectra per direction, inputs and outputs once)."""
    return 16 * Nq + 76


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

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
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, name):
        setattr(self, name, time.time())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for t, l in self.lines:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((t, float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return None
        t0, t1 = getattr(self, "start", 0), getattr(self, "stop", 1e30)
        inside = [r for r in rows if t0 <= r[0] <= t1]
        use = inside if inside else rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in use:
            for nm, val in zip(names, r[3][1:]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "reasons": sorted(reasons), "samples": len(use),
                "window": "timed region" if inside else "whole run (no sample fell inside the timed region)"}


ORACLE_SAMPLE = r"""
import os, sys, time, json
sys.path.insert(0, %r)
import numpy as np
import oracle as O
from paper_0812_0244_gb300 import synthetic as S
T = O.kernel_table(O.Params())
d = S.tube_density(int(sys.argv[1]), shape=(18, 180, 180), cell_ang=(25.0, 25.0, 2.46))
n = d["n"].astype(np.float32).astype(np.float64)
g = O.spectral_gradient(n, d["L"]).astype(np.float32).astype(np.float64)
t0 = time.time()
r = O.energy_potential(n, g, d["L"], T)
t1 = time.time()
print(json.dumps({"points": int(n.size), "t0": t0, "t1": t1, "E": r["E"]}))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate(procs=1, timeout=900):
    """Time the FP64 oracle (as it stands, one thread per process) on one
    axial period of the tube (180 x 180 x 18 points, the workload's grid
    spacing and density recipe, grad n = D n), in `procs` child processes at
    once, one sample each.  Returns (aggregate points/s, seconds of the
    overlapped window, points per sample)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SAMPLE % ROOT
    ps = [subprocess.Popen([sys.executable, "-c", code, str(i)], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True, env=env) for i in range(procs)]
    outs = []
    for p in ps:
        o, e = p.communicate(timeout=timeout)
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed: " + e[-2000:])
        outs.append(json.loads(o.strip().splitlines()[-1]))
    t0 = min(d["t0"] for d in outs)
    t1 = max(d["t1"] for d in outs)
    pts = outs[0]["points"]
    return procs * pts / (t1 - t0), t1 - t0, pts


def cpu_baselines():
    """The oracle on one core, then on every core of the process's affinity
    set (independent samples, one process per core)."""
    r1, s1, pts = oracle_rate(1)
    ncores = host_cores()
    rn, sn, _ = oracle_rate(ncores)
    return {"value": rn, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": "FP64 numpy/C oracle, E and v of one axial period of the tube (180x180x18 of the 180x180x72 "
                      "grid, %d points, grad n = D n) per process, %d single-threaded processes at once (%.1f s)"
                      % (pts, ncores, sn),
            "single_core": {"value": r1, "cores": 1, "seconds": s1}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    K = max(1, min(args.steps, 3))
    W = min(args.warmup, 1)
    ncores = host_cores()
    total_pts, total_s = 0, 0.0
    for i in range(W + K):
        rate, sec, pts = oracle_rate(ncores)
        if i >= W:
            total_pts += ncores * pts
            total_s += sec
    value = total_pts / total_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * total_s / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "one axial period (180x180x18 points) per host core"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": "FP64 numpy/C oracle, E and v of one axial period of the tube (180x180x18 "
                                       "of the 180x180x72 grid) in each of %d single-threaded processes, %d steps"
                                       % (ncores, K)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def learned_leg(ctx, n, g, E, v, flush, stream, K, E_plain, v_plain, natoms, ms_plain, N):
    """Time the learned 8-channel path (E and v) like the plain one and compare
    its energy and potential with the plain Nq = 20 results of the same density."""
    import torch
    from paper_0812_0244_gb300 import learned as LR
    from paper_0812_0244_gb300 import vdwnl
    if os.path.exists(LR.TRAINED_PATH):
        mdl = LR.load(LR.TRAINED_PATH)
        params = torch.tensor(mdl["params"], dtype=torch.float32, device=n.device)
        feat, base, kind = mdl["feat"], mdl["base"], "trained (%s)" % os.path.relpath(LR.TRAINED_PATH, ROOT)
        J, kmax = mdl["J"], mdl["k_max"]
    else:
        p8 = vdwnl.Params(Nq=8, q_1=LR.Q1_8, lam=LR.LAM_8)
        t8 = vdwnl.kernel_table(p8)
        t8["k_max"] = p8.k_max
        params = LR.init_params(0, t8, device=n.device)
        feat, base, kind = (-8.0, 4.0, 2.0, 3.0, 0.1), (LR.Q1_8, LR.LAM_8), "untrained initialisation"
        J, kmax = LR.J_KNOTS, LR.K_MAX
    ctx.learned_load(params, J, kmax, feat, base)
    # the network itself at every point (the training form), for reference
    for _ in range(3):
        ctx.learned_energy_potential(n, g, E, v)
    ms_direct = timed(lambda: ctx.learned_energy_potential(n, g, E, v), min(K, 20), flush, stream)
    E_direct = float(E[0])
    # inference: the network tabulated on the feature nodes
    ctx.learned_tabulate(LR.TAB_T, LR.TAB_D)
    for _ in range(3):
        ctx.learned_energy_potential(n, g, E, v)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for i in range(K):
        flush.zero_()
        starts[i].record(stream)
        ctx.learned_energy_potential(n, g, E, v)
        ends[i].record(stream)
    torch.cuda.synchronize()
    ms_l = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / K
    El = float(E[0])
    dv = (v.double() - v_plain.double())
    w = n.double()
    vrms = float(torch.sqrt((w * dv * dv).sum() / w.sum()) / torch.sqrt((w * v_plain.double() ** 2).sum() / w.sum()))
    vmax = float(dv.abs().max() / v_plain.double().abs().max())
    ctx.profile(True)
    ctx.learned_energy_potential(n, g, E, v)
    stages = {k: round(t, 4) for k, t in ctx.profile_read().items()}
    ctx.profile(False)
    return {"model": kind, "network": "tabulated on %d x %d feature nodes over [-%g, %g]^2, Catmull-Rom"
                                      % (LR.TAB_T, LR.TAB_T, LR.TAB_D, LR.TAB_D),
            "ms_per_step": ms_l, "value": N / (ms_l * 1e-3), "unit": UNIT,
            "speedup_vs_plain_nq20": ms_plain / ms_l, "stages_ms": stages,
            "network_at_every_point": {"ms_per_step": ms_direct, "speedup_vs_plain_nq20": ms_plain / ms_direct,
                                       "energy_minus_tabulated_mev_per_atom": (E_direct - El) / natoms
                                       * 27211.386245988},
            "energy_error_mev_per_atom_vs_plain_nq20": (El - E_plain) / natoms * 27211.386245988,
            "potential_vs_plain_nq20": {"density_weighted_rms_rel": vrms, "max_abs_rel": vmax},
            "tc_error": ctx.learned_status()}


def timed(fn, K, flush, stream):
    """Mean CUDA-event time (ms) of fn() over K calls, L2 flushed before each."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
    for i in range(K):
        flush.zero_()
        ev[2 * i].record(stream)
        fn()
        ev[2 * i + 1].record(stream)
    torch.cuda.synchronize()
    return sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(K)) / K


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-only", action="store_true",
                    help="time the plain call alone (no stage profile, other legs or host-buffer figure)")
    ap.add_argument("--learned-only", action="store_true",
                    help="time the plain call, then the learned leg alone (for profiling the learned kernels)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    # CPU baseline first (child processes, before this process touches the GPU)
    cpu = None
    if rank == 0 and world == 1 and not (args.no_cpu_baseline or args.plain_only or args.learned_only):
        cpu = cpu_baselines()

    import torch
    import torch.distributed as dist
    from paper_0812_0244_gb300 import synthetic as S
    from paper_0812_0244_gb300 import vdwnl

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    d = S.tube_density(rank)
    n_h = d["n"].astype(np.float32)
    N = n_h.size
    params = vdwnl.Params()
    ctx = vdwnl.VdwNL(params)
    ctx.plan(n_h.shape, d["L"])
    n = torch.tensor(n_h, device=dev)
    g = ctx.spectral_gradient(n)  # grad n = D n, the library's spectral derivative
    torch.cuda.synchronize()
    E = torch.empty(3, dtype=torch.float64, device=dev)
    v = torch.empty_like(n)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        ctx.energy_potential(n, g, E, v)
    torch.cuda.synchronize()

    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        clk.mark("start")
        for i in range(K):
            flush.zero_()
            starts[i].record(stream)
            ctx.energy_potential(n, g, E, v)
            ends[i].record(stream)
        torch.cuda.synchronize()
        clk.mark("stop")
        barrier()
    ms = slowest_rank(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / K, world, dev)
    value = world * N / (ms * 1e-3)  # the points of all replicas over the slowest one's time
    Eh = E.cpu().numpy()
    peak, peak_kind = measured_peaks()
    clocks = clk.summary() if rank == 0 else None
    base = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded double-wall tube density; grad n = D n by the library's "
                                "spectral derivative)",
        "config": {"workload": WORKLOAD, "grid": [180, 180, 72], "Nq": params.Nq, "cell_angstrom": [25, 25, 9.84],
                   "sites": int(d["natoms"]), "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed (256 MiB write) before every timed step", "energy_fp64": float(Eh[0])},
        # pointwise, forward planes, forward y pencils, contraction, energy
        # reduction (two passes), inverse y pencils, inverse planes, field sum,
        # w planes, divergence pencils, final planes
        "gpu_launches": 12 * K,
        "clocks": clocks,
    }
    if args.plain_only or args.learned_only:
        if args.learned_only:
            ctx.energy_potential(n, g, E, v)
            base["learned_m8"] = learned_leg(ctx, n, g, E, v, flush, stream, min(K, 5), float(E[0]), v.clone(),
                                             int(d["natoms"]), ms, N)
        if rank == 0:
            print(json.dumps(base), flush=True)
        ctx.close()
        if world > 1:
            dist.destroy_process_group()
        return

    # per-stage durations (separate, untimed iterations with stage events)
    ctx.profile(True)
    acc = {}
    reps = min(K, 50)
    for _ in range(reps):
        flush.zero_()
        ctx.energy_potential(n, g, E, v)
        for k2, t2 in ctx.profile_read().items():
            acc[k2] = acc.get(k2, 0.0) + t2 / reps
    ctx.profile(False)
    sb = stage_bytes_per_point(params.Nq, n_h.shape[2])
    top = max((k2 for k2 in acc if k2 != "energy_final"), key=lambda k2: acc[k2])
    achieved = sb[top] * N / (acc[top] * 1e-3) / 1e9
    traffic = captured_traffic(top)
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    alu_peak = fp32_peak_tflops(sm_mhz)
    alu_achieved = contract_flops_per_point(params.Nq, n_h.shape[2]) * N / (acc["contract"] * 1e-3) / 1e12

    # reference only: cuFFT (through torch.fft) on the transforms of one step:
    # Nq forward and Nq inverse real 3D transforms, plus 3 forward and 1
    # inverse for the gradient term (never on the product path)
    cufft_ms = None
    try:
        fields = torch.randn((params.Nq,) + n_h.shape, device=dev, dtype=torch.float32)
        wf = torch.randn((3,) + n_h.shape, device=dev, dtype=torch.float32)

        def cufft_step():
            th = torch.fft.rfftn(fields, dim=(1, 2, 3))
            torch.fft.irfftn(th, s=n_h.shape, dim=(1, 2, 3))
            wh = torch.fft.rfftn(wf, dim=(1, 2, 3))
            torch.fft.irfftn(wh[0], s=n_h.shape, dim=(0, 1, 2))
        for _ in range(3):
            cufft_step()
        cufft_ms = timed(cufft_step, 10, flush, stream)
        del fields, wf
    except Exception:
        cufft_ms = None

    # the same call with the finite-difference gradient (the paper's own
    # operator; the chain term is a stencil instead of three transforms)
    fd_ms = None
    try:
        # grad = None: the library's central-difference gradient, inside the call
        for _ in range(3):
            ctx.energy_potential_fd(n, None, E, v)
        fd_ms = timed(lambda: ctx.energy_potential_fd(n, None, E, v), min(K, 100), flush, stream)
    except Exception:
        fd_ms = None

    # the whole functional: revPBE exchange and LDA correlation beside the
    # nonlocal term (Eq. Exc), same density and gradient
    xc_ms = None
    try:
        for _ in range(3):
            ctx.xc_energy_potential(n, g, v)
        xc_ms = timed(lambda: ctx.xc_energy_potential(n, g, v), min(K, 100), flush, stream)
    except Exception:
        xc_ms = None

    # the autograd Function on the 256 x 256 x 96 tube: forward (energy only)
    # and backward (theta recomputed; dE/dn and dE/d grad n), n and grad n leaves
    ag_ms = None
    try:
        from paper_0812_0244_gb300.autograd import vdw_energy
        shape2 = (96, 256, 256)
        n64, L2, _ = S.tube_density_torch(3, shape=shape2, device="cuda")
        ctx2 = vdwnl.VdwNL(vdwnl.Params()).plan(shape2, L2)
        n2 = n64.to(torch.float32).contiguous()
        g2 = ctx2.spectral_gradient(n2)
        del n64
        n2.requires_grad_(True)
        g2.requires_grad_(True)

        def ag_step():
            vdw_energy(n2, g2, ctx2).backward()
            n2.grad = None
            g2.grad = None
        for _ in range(3):
            ag_step()
        ag_ms = timed(ag_step, min(K, 40), flush, stream)
        del ctx2, n2, g2
    except Exception:
        ag_ms = None

    # several densities per call (NEXT-3): B = 8 tube densities (outer wall
    # shifted and rotated), one launch per stage for the whole batch
    batched = None
    try:
        Bb = 8
        nb = []
        for b in range(Bb):
            n64b, _, _ = S.tube_density_torch(100 + b, shape=n_h.shape, shift_ang=0.3 * b, rot_deg=4.5 * b,
                                              device=dev)
            nb.append(n64b.to(torch.float32))
        nb = torch.stack(nb).contiguous()
        gb = torch.stack([ctx.spectral_gradient(nb[b]) for b in range(Bb)]).contiguous()
        vb = torch.empty_like(nb)
        Eb = torch.empty((Bb, 3), dtype=torch.float64, device=dev)
        ctx.plan_batch(Bb)
        for _ in range(3):
            ctx.energy_potential_batched(nb, gb, Eb, vb)
        b_ms = timed(lambda: ctx.energy_potential_batched(nb, gb, Eb, vb), min(K, 50), flush, stream)
        batched = {"B": Bb, "ms_per_call": b_ms, "ms_per_density": b_ms / Bb,
                   "value": Bb * N / (b_ms * 1e-3), "unit": UNIT,
                   "what": "vdw_energy_potential_batched: E and v of 8 tube densities per call"}
        ctx.plan_batch(1)
        del nb, gb, vb
    except Exception as ex:  # reported, never silently replaced
        batched = {"error": str(ex)[:200]}

    # plain potential of the same density, for the learned comparison
    ctx.energy_potential(n, g, E, v)
    v_plain = v.clone()
    E_plain = float(E[0])

    # learned reduced basis (M = 8 channels) on the same density: the trained
    # model if one is stored in the package, else its initialisation
    learned = None
    try:
        learned = learned_leg(ctx, n, g, E, v, flush, stream, min(K, 100), E_plain, v_plain, int(d["natoms"]), ms,
                              N)
    except Exception as ex:  # reported, never silently replaced
        learned = {"error": str(ex)[:200]}

    # end to end through the host-pointer entry point (pinned buffers)
    n_p = torch.from_numpy(n_h).pin_memory()
    g_p = g.cpu().pin_memory()
    v_p = torch.empty(n_h.shape, dtype=torch.float32).pin_memory()
    E_p = np.zeros(3)
    Ke = max(1, min(K, 50))
    for _ in range(2):
        ctx.energy_potential_host(n_p.numpy(), g_p.numpy(), E_p, v_p.numpy())
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(Ke):
        ctx.energy_potential_host(n_p.numpy(), g_p.numpy(), E_p, v_p.numpy())
    e2e_s = (time.perf_counter() - t0) / Ke
    barrier()
    e2e_s = slowest_rank(e2e_s, world, dev)

    if rank == 0:
        stage_frac = {k2: round(sb[k2] * N / (t2 * 1e-3) / 1e9 / peak, 4) for k2, t2 in acc.items() if sb[k2] > 0}
        line = dict(base)
        line.update({
            "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak,
                         "peak_kind": "%s hbm_gbs (MEASURED_PEAKS.json)" % peak_kind if peak_kind == "measured"
                         else "fallback 6.8 TB/s", "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "bytes_per_point": sb[top], "launch_ms": acc[top],
                         "alu": {"kernel": "contract", "flops_per_point": contract_flops_per_point(params.Nq,
                                                                                                  n_h.shape[2]),
                                 "achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
                                 "frac": alu_achieved / alu_peak,
                                 "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flops x %.0f MHz" % sm_mhz}},
            "step_roofline": {"bytes_per_point": b_alg(params.Nq),
                              "achieved_gbs": b_alg(params.Nq) * N / (ms * 1e-3) / 1e9,
                              "frac": b_alg(params.Nq) * N / (ms * 1e-3) / 1e9 / peak},
            "stages_ms": {k2: round(t2, 4) for k2, t2 in acc.items()},
            "stages_hbm_frac": stage_frac,
            "e2e": {"value": world * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 16 * N,
                    "d2h_bytes_per_step": 4 * N + 24},
            "cufft_reference": {"ms_per_step": cufft_ms,
                                "what": "torch.fft (cuFFT) on the step's %d forward + %d inverse real 3D transforms "
                                        "alone, no pointwise work or contraction; reference only"
                                        % (params.Nq + 3, params.Nq + 1)},
            "learned_m8": learned,
            "batched_b8": batched,
            "autograd_256x256x96": {"ms_per_step": ag_ms,
                                    "value": (256 * 256 * 96 / (ag_ms * 1e-3)) if ag_ms else None, "unit": UNIT,
                                    "what": "torch.autograd.Function forward (E) + backward (theta recomputed, "
                                            "dE/dn and dE/d grad n) on the 256x256x96 tube"},
            "xc_functional": {"ms_per_step": xc_ms, "value": (N / (xc_ms * 1e-3)) if xc_ms else None,
                              "unit": UNIT, "what": "vdw_xc_energy_potential: E_x^revPBE + E_c^LDA + E_c^nl "
                                                    "and the potential of E_xc, spectral gradient"},
            "fd_gradient_variant": {"ms_per_step": fd_ms, "value": (N / (fd_ms * 1e-3)) if fd_ms else None,
                                    "unit": UNIT, "what": "vdw_energy_potential_fd: central-difference gradient "
                                                          "(computed in the call), chain term by stencil"},
        })
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
