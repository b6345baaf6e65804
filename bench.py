#!/usr/bin/env python
"""Throughput benchmark of the preconditioned GLBE time step on GB300.

Default workload (one GPU): the square duct of 256 x 256 cross-section and
512 nodes streamwise (x periodic, half-way bounce-back walls on y and z),
body force F_x(y, z) = F0 (1 + 0.5 sin(2 pi y/L_y) cos(2 pi z/L_z)),
F0 = 1e-6, nu = 0.5, gamma = 0.1, D3Q19 MRT-GLBE, population deviations
stored in BF16 with FP32 collide arithmetic.  One bench step = 10 time steps
(one residual period: 9 plain fused steps, 1 fused step with the FP64
residual reduction and its finalize kernel).  Inputs (1.27 GB per population
buffer) are larger than L2, so no flush is needed.

The JSON line reports MLUPS (fluid-node updates per second, millions), the
roofline of the dominant kernel (the plain fused step) against the measured
HBM copy bandwidth, the end-to-end rate through the C-ABI with host buffers,
sampled SM clocks, the FP64 CPU oracle timed on a bounded sample, and
variants: FP32 / FP16 storage on the same duct, the fused D3Q19 + D3Q7 step
on the 128^3 Hartmann duct, and wall time to a 1e-8 residual at gamma = 0.1
vs gamma = 1 on the 64 x 64 x 8 Hartmann duct.

Multi-GPU (torchrun, N > 1): the duct is split into N slabs of z planes, one
per rank (strong scaling: the whole job is one duct); after every time step
each rank sends the populations crossing its slab faces to its neighbours
(NCCL point-to-point) and every 10 steps the FP64 residual sums are
all-reduced.  Timing is the max over ranks.  ``--replicas`` runs N
independent copies instead (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W19 = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12

DUCT = dict(nx=512, ny=256, nz=256, gamma=0.1, nu=0.5, F0=1e-6)

# DRAM bytes (read + write) of one plain step of the kernel the automatic
# choice launches (PLAIN_STEP_KERNEL), per fluid node, from `ncu --metrics
# dram__bytes_read.sum,dram__bytes_write.sum -c 1`: BF16 on one launch of the
# timed 512 x 256 x 256 duct itself (33,032,192 fluid nodes; 79.9 B against
# the algorithmic 80 B); F16 and F32
# on the 256 x 128 x 128 duct (4,064,256 fluid nodes), whose 335 MB state
# leaves part of the written data in L2 (below the algorithmic 80 / 156 B),
# scaled by fluid nodes.
STEP_TRAFFIC_B_PER_FLUID_NODE = {"bf16": (1409381888 + 1230580992) / 33032192,
                                 "f16": (175882752 + 119174144) / 4064256,
                                 "f32": (332382976 + 267721472) / 4064256}
# the kernels the automatic choice launches on the duct (x periodic, even nx, no induction)
PLAIN_STEP_KERNEL = {"bf16": "step_pair_kernel_dense", "f16": "step_pair_kernel_dense", "f32": "step_kernel"}
RESID_STEP_KERNEL = {"bf16": "step_pair_kernel_dense", "f16": "step_pair_kernel_dense", "f32": "step_kernel"}


def step_kernels(storage: str, variant: int):
    """(plain, residual) step kernel names for a flow-only duct step."""
    if variant == 0:
        return PLAIN_STEP_KERNEL[storage], RESID_STEP_KERNEL[storage]
    if variant == 1:
        return ("step_kernel" if storage == "f32" else "step_kernel_dense"), "step_kernel"
    if variant == 2:
        k = "step_pair_kernel" if storage == "f32" else "step_pair_kernel_dense"
        return k, k
    return "tile_kernel", "tile_kernel"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed bench steps (10 time steps each)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["glbe", "reference"], default="glbe")
    ap.add_argument("--storage", choices=["bf16", "f16", "f32"], default="bf16")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", type=int, default=0, help="kernel form: 0 automatic, 1 one node/thread, 2 paired")
    ap.add_argument("--workload", choices=["duct", "batch", "batch-single", "batch-small", "adjoint", "sweeps",
                                           "coupled", "cavity", "tts", "2d", "cpu-configs"],
                    default="duct",
                    help="duct: the timed duct step (default); batch: 64 seeded ducts solved to 1e-8 in one "
                         "launch; adjoint: steady and unrolled dQ/dF on the 128^3 Hartmann duct")
    ap.add_argument("--adjoint-n", type=int, default=128)
    ap.add_argument("--adjoint-tol", type=float, default=1e-5)
    ap.add_argument("--adjoint-fwd-tol", type=float, default=1e-7)
    ap.add_argument("--adjoint-max-steps", type=int, default=300_000)
    ap.add_argument("--adjoint-unrolled-steps", type=int, default=2000)
    ap.add_argument("--adjoint-K", type=int, default=100)
    ap.add_argument("--no-adjoint-fd", action="store_true")
    ap.add_argument("--batch-storage", choices=["f32", "f32c"], default="f32c",
                    help="f32c by default: with F32 storage these ducts stall near r = 3e-8 (measured)")
    ap.add_argument("--batch-max-steps", type=int, default=400_000,
                    help="level cap: the gamma = 1 ducts of up to 160 nodes need ~2e5 levels at nu = 0.1")
    ap.add_argument("--batch-tol", type=float, default=1e-8)
    ap.add_argument("--replicas", action="store_true",
                    help="with N > 1: N independent replicas of the duct instead of one duct split into N slabs")
    ap.add_argument("--forms2d", default="f32_mhd,bf16_mhd,f32c_mhd,f32_flow,bf16_flow",
                    help="2d workload: storage forms timed (storage_mhd or storage_flow)")
    ap.add_argument("--no-tts", action="store_true", help="2d workload: skip the time-to-solution part")
    ap.add_argument("--nx", type=int, default=None, help="override the duct size (profiling of a small case)")
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--nz", type=int, default=None)
    args = ap.parse_args()
    for k in ("nx", "ny", "nz"):
        if getattr(args, k) is not None:
            DUCT[k] = getattr(args, k)
    return args


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------
def dist_init(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    """Maximum of a scalar over all ranks (identity for one rank)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        # address the GPU by UUID: CUDA and nvidia-smi may number GPUs differently
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            self.gpu = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            self.gpu = str(device_index)
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def duct_solver(storage: str, device="cuda", variant: int = 0, collision: int = 0):
    import torch
    from paper_0809_4730_gb300.glbe import Solver
    from paper_0809_4730_gb300.inputs import duct_force_x
    d = DUCT
    G = Solver(d["nx"], d["ny"], d["nz"], wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=d["gamma"], nu=d["nu"],
               force_field=1, storage=storage, device=device, variant=variant, collision=collision)
    Fx = duct_force_x(d["nx"], d["ny"], d["nz"], d["F0"])[0].reshape(1, -1)
    F_host = torch.tensor(Fx, dtype=torch.float32).pin_memory()
    G.set_force(F_host.to(device))
    fluid = d["nx"] * (d["ny"] - 2) * (d["nz"] - 2)
    return G, F_host, fluid


def hartmann_duct_solver(n=128, Ha=10.0, gamma=0.1, device="cuda", storage="f32", variant=0, force_field=0,
                         nu=0.01, shape=None):
    """Hartmann duct of n^3 nodes (or shape = (nx, ny, nz)): x periodic,
    walls on y and z, B0 along y, nu = eta (0.01 by default), chi = 0.01
    (Pr_m = 0.01), F_x = 1e-6 uniform (or, with force_field = 3, a per-node
    field set by the caller), FP32."""
    from paper_0809_4730_gb300.glbe import Solver
    nx, ny, nz = shape if shape is not None else (n, n, n)
    eta = nu
    L = (ny - 2) / 2
    B0 = Ha * math.sqrt(nu * eta) / L
    F = (0.0, 0.0, 0.0) if force_field else (1e-6, 0, 0)
    G = Solver(nx, ny, nz, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=nu, F=F, induction=1,
               gamma_m=gamma, eta=eta, chi=0.01, mu=1.0, B0=(0, B0, 0), device=device, storage=storage,
               variant=variant, force_field=force_field)
    return G, nx * (ny - 2) * (nz - 2)


def bytes_per_node(storage: str, mhd: bool, force_comp: int) -> int:
    ss = 4 if storage == "f32" else 2
    b = 19 * ss * 2 + 4 * force_comp
    if mhd:
        b += 21 * ss * 2 + 3 * 4 * 2
    return b


def timed_steps(G, K, stream):
    """K bench steps of 10 time steps each on stream; returns (total ms,
    plain-kernel ms total, plain launches) from CUDA events recorded on the
    launching stream inside the timed region."""
    import torch
    assert G.t % 10 == 0
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for a, b, c in evs:
        a.record(stream)
        G.step(1)          # fused step with the residual reduction (+ finalize)
        b.record(stream)
        G.step(9)          # nine plain fused steps
        c.record(stream)
    end.record(stream)
    end.synchronize()
    total = start.elapsed_time(end)
    plain = sum(b.elapsed_time(c) for _, b, c in evs)
    return total, plain, 9 * K


def run_glbe(args, rank, ws):
    import torch
    stream = torch.cuda.current_stream()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        hbm_peak, peak_src = 6800.0, "fallback"

    G, F_host, fluid = duct_solver(args.storage, variant=args.variant)
    G.step(10 * args.warmup)
    G.residual()
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        total_ms, plain_ms, nplain = timed_steps(G, args.steps, stream)
        torch.cuda.synchronize()
    barrier(ws)
    info = G.residual()
    total_ms = max_over_ranks(total_ms, ws)
    updates = 10 * args.steps * fluid
    mlups = updates / (total_ms * 1e-3) / 1e6 * ws
    kern_ms = plain_ms / nplain
    bpn = bytes_per_node(args.storage, False, 1)
    achieved = bpn * fluid / (kern_ms * 1e-3) / 1e9
    line = {
        "metric": "MLUPS (fluid-node updates/s) and % of HBM roofline of the fused GLBE step",
        "value": round(mlups, 1),
        "unit": "MLUPS",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": f"square duct {DUCT['nx']}x{DUCT['ny']}x{DUCT['nz']} (x periodic, walls y/z), "
                        "Fx(y,z) = F0(1+0.5 sin cos), "
                        "F0=1e-6, nu=0.5, gamma=0.1, D3Q19 MRT-GLBE, " + args.storage + " deviation storage, "
                        "FP32 collide; 1 bench step = 10 time steps incl. FP64 residual",
            "nodes": DUCT["nx"] * DUCT["ny"] * DUCT["nz"],
            "fluid_nodes": fluid,
            "storage": args.storage,
            "l2": "inputs larger than L2 (no flush)",
            "parallelism": "replicas" if ws > 1 else "single GPU",
        },
        "roofline": {
            "bound": "hbm",
            "achieved": round(achieved, 1),
            "peak": hbm_peak,
            "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4),
            "traffic": (round(STEP_TRAFFIC_B_PER_FLUID_NODE[args.storage] * fluid)
                        if args.variant == 0 and args.storage in STEP_TRAFFIC_B_PER_FLUID_NODE else None),
            "traffic_note": ("bytes of one launch, ncu capture (-c 1) on this 512x256x256 duct"
                             if args.storage == "bf16" else
                             "bytes per launch, ncu capture on the 256x128x128 duct scaled by fluid nodes"),
            "kernel": "%s (plain fused collide+stream; %s on residual levels)" % step_kernels(args.storage,
                                                                                           args.variant),
            "bytes_per_node": bpn,
            "kernel_ms": round(kern_ms, 5),
            "peak_source": peak_src,
        },
        "gpu_launches": 11 * args.steps,
        "residual_at_end": {"t": info.t, "r": info.r},
        "clocks": clk.summary(),
    }
    # end to end through the C-ABI with host buffers: every bench step uploads
    # its force field from pinned memory, runs 10 steps and reads back the
    # residual record (which synchronises).  The upload of step k+1's field
    # is issued right after step k is enqueued, so the library's staged copy
    # overlaps step k's kernels; the first upload is not overlapped.
    from paper_0809_4730_gb300.glbe import glbe_set_force_host
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    glbe_set_force_host(G.ctx, F_host)
    for k in range(args.steps):
        G.step(10)
        if k + 1 < args.steps:
            glbe_set_force_host(G.ctx, F_host)
        G.residual()
    t1 = time.perf_counter()
    e2e_s = max_over_ranks(t1 - t0, ws)
    line["e2e"] = {"value": round(updates / e2e_s / 1e6 * ws, 1), "unit": "MLUPS",
                   "h2d_bytes_per_step": F_host.numel() * 4, "d2h_bytes_per_step": 16 * 8}
    G.close()
    del G
    torch.cuda.empty_cache()

    refs = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], refs = cpu_baseline()
    if not args.no_variants:
        line["variants"] = variants(args, hbm_peak, stream)
        if refs is not None:
            line["steady_error"], line["time_to_solution"] = duct64_study(refs)
    return line


def run_coupled(args, rank, ws):
    """The fused D3Q19 + D3Q7 step on the large coupled grid: the Hartmann
    physics (Ha = 10, gamma = 0.1, Pr_m = 0.01) on nx x ny x nz (default
    512 x 256 x 256), x periodic, walls on y and z, --storage f32 or bf16;
    bench steps of 10 time steps as for the duct."""
    import torch
    stream = torch.cuda.current_stream()
    try:
        hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        hbm = 6800.0
    st = args.storage
    G, fluid = hartmann_duct_solver(storage=st, shape=(DUCT["nx"], DUCT["ny"], DUCT["nz"]), variant=args.variant)
    G.step(10 * args.warmup)
    G.sync()
    with ClockSampler(torch.cuda.current_device()) as clk:
        total_ms, plain_ms, nplain = timed_steps(G, args.steps, stream)
    kern_ms = plain_ms / nplain
    bpn = bytes_per_node(st, True, 0)
    achieved = bpn * fluid / (kern_ms * 1e-3) / 1e9
    G.close()
    return {"metric": "MLUPS of the fused D3Q19 + D3Q7 step (lagged Lorentz force)",
            "value": round(10 * args.steps * fluid / (total_ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"Hartmann duct {DUCT['nx']}x{DUCT['ny']}x{DUCT['nz']}, Ha=10, gamma=0.1, "
                                   f"Pr_m=0.01, {st} storage", "fluid_nodes": fluid},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "bytes_per_node": bpn, "kernel_ms": round(kern_ms, 5)},
            "clocks": clk.summary()}


def run_sharded(args, rank, ws):
    """One 512 x 256 x 256 duct split along z into ws slabs, slab `rank` on
    this GPU; every time step is the fused step plus the exchange of the
    crossing populations with the neighbouring ranks."""
    import torch
    from paper_0809_4730_gb300.glbe import Solver
    from paper_0809_4730_gb300.inputs import duct_force_x
    from paper_0809_4730_gb300.slabs import RankSlab, SolverSlab, global_planes, plan, slab_params
    stream = torch.cuda.current_stream()
    d = DUCT
    slabs = plan(d["nz"], ws, 1, 1)
    s = slabs[rank]
    kw = dict(wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=d["gamma"], nu=d["nu"], force_field=1,
              storage=args.storage, variant=args.variant)
    G = Solver(d["nx"], d["ny"], s.nz_local, **slab_params(kw, s))
    Fx = duct_force_x(d["nx"], d["ny"], d["nz"], d["F0"])[0]
    zs = global_planes(s, d["nz"])
    G.set_force(torch.tensor(Fx[zs].reshape(1, -1), dtype=torch.float32, device="cuda"))
    R = RankSlab(slabs, rank, SolverSlab(G))
    fluid_total = d["nx"] * (d["ny"] - 2) * (d["nz"] - 2)
    R.step(10 * args.warmup)
    R.residual()
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            R.step(10)
        e1.record(stream)
        e1.synchronize()
    barrier(ws)
    ms = max_over_ranks(e0.elapsed_time(e1), ws)
    info = R.residual()
    updates = 10 * args.steps * fluid_total
    G.close()
    return {
        "metric": "MLUPS (fluid-node updates/s) and % of HBM roofline of the fused GLBE step",
        "value": round(updates / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"square duct {d['nx']}x{d['ny']}x{d['nz']} split into {ws} z slabs, "
                               f"{args.storage} deviation storage; 1 bench step = 10 time steps, each followed by "
                               "the halo exchange (NCCL send/recv), FP64 all-reduce of the residual sums",
                   "fluid_nodes": fluid_total, "storage": args.storage, "parallelism": f"z slabs x{ws}",
                   "l2": "inputs larger than L2 (no flush)"},
        # per time step: the fused step, a pack and an unpack per ghost face;
        # per bench step the residual finalize (one or two kernels)
        "gpu_launches": args.steps * (10 * (1 + 2 * (s.ghost_lo + s.ghost_hi)) + 2),
        "residual_at_end": {"t": info.t, "r": info.r},
        "clocks": clk.summary(),
    }


def variants(args, hbm_peak, stream):
    import torch
    out = {}
    for st, variant in (("f32", 0), ("f16", 0), ("bf16", 0), ("bf16", 2), ("f32", 2), ("f32", -1)):
        if st == args.storage and variant == 0:
            continue
        G, _, fluid = duct_solver(st, variant=max(variant, 0), collision=1 if variant == -1 else 0)
        G.step(30)
        G.sync()
        total_ms, plain_ms, nplain = timed_steps(G, 5, stream)
        kern_ms = plain_ms / nplain
        bpn = bytes_per_node(st, False, 1)
        out[f"duct_{st}" + ("_paired" if variant == 2 else "") + ("_srt" if variant == -1 else "")] = {
                             "mlups": round(50 * fluid / (total_ms * 1e-3) / 1e6, 1),
                             "kernel_ms": round(kern_ms, 5), "bytes_per_node": bpn,
                             "hbm_frac": round(bpn * fluid / (kern_ms * 1e-3) / 1e9 / hbm_peak, 4)}
        G.close()
        del G
        torch.cuda.empty_cache()
    # fused D3Q19 + D3Q7 on the 128^3 Hartmann duct (FP32 and BF16 storage)
    for st, variant in (("f32", 0), ("f32", 2), ("bf16", 0)):
        G, fluid = hartmann_duct_solver(storage=st, variant=variant)
        G.step(30)
        G.sync()
        total_ms, plain_ms, nplain = timed_steps(G, 5, stream)
        kern_ms = plain_ms / nplain
        bpn = bytes_per_node(st, True, 0)
        key = f"mhd_duct_128_{st}" + ("_paired" if variant == 2 else "")
        out[key] = {"mlups": round(50 * fluid / (total_ms * 1e-3) / 1e6, 1), "kernel_ms": round(kern_ms, 5),
                    "bytes_per_node": bpn, "hbm_frac": round(bpn * fluid / (kern_ms * 1e-3) / 1e9 / hbm_peak, 4)}
        G.close()
        del G
        torch.cuda.empty_cache()
    # the fused coupled step on the large coupled grid: the Hartmann physics
    # (Ha = 10, gamma = 0.1, Pr_m = 0.01) on 512 x 256 x 256
    for st in ("f32", "bf16"):
        G, fluid = hartmann_duct_solver(storage=st, shape=(512, 256, 256))
        G.step(30)
        G.sync()
        total_ms, plain_ms, nplain = timed_steps(G, 3, stream)
        kern_ms = plain_ms / nplain
        bpn = bytes_per_node(st, True, 0)
        out[f"mhd_duct_512x256x256_{st}"] = {
            "mlups": round(30 * fluid / (total_ms * 1e-3) / 1e6, 1), "kernel_ms": round(kern_ms, 5),
            "bytes_per_node": bpn, "hbm_frac": round(bpn * fluid / (kern_ms * 1e-3) / 1e9 / hbm_peak, 4)}
        G.close()
        del G
        torch.cuda.empty_cache()
    out["batch_64_ducts_bounded"] = batch_bounded(hbm_peak)
    try:
        out["adjoint_steady_128_bounded"] = adjoint_bounded(hbm_peak)
    except Exception as e:       # reported in the line, not fatal to it
        out["adjoint_steady_128_bounded"] = {"error": str(e)[:300]}
    out["time_to_1e-8_hartmann_64x64x8"] = time_to_solution()
    # the 2D lattices: the fused D2Q9 + D2Q5 step on the 4096^2 Hartmann channel
    for st in ("f32", "bf16"):
        G, fluid = channel2d_solver(st, True)
        G.step(30)
        G.sync()
        total_ms, plain_ms, nplain = timed_steps(G, 3, stream)
        kern_ms = plain_ms / nplain
        bpn = bytes_per_node_2d(st, True)
        out[f"d2q9_d2q5_4096x4096_{st}"] = {
            "mlups": round(30 * fluid / (total_ms * 1e-3) / 1e6, 1), "kernel_ms": round(kern_ms, 5),
            "bytes_per_node": bpn, "hbm_frac": round(bpn * fluid / (kern_ms * 1e-3) / 1e9 / hbm_peak, 4)}
        G.close()
        del G
        torch.cuda.empty_cache()
    return out


def batch_bounded(hbm_peak: float, levels: int = 200):
    """The 64-duct batch (F32C) marched a fixed number of levels in one
    persistent launch (no domain converges that early): aggregate MLUPS and
    the fraction of the HBM roofline at the algorithmic bytes of each domain
    (F32C: 19 x 6 x 2 B per flow node; coupled nodes add 21 x 6 x 2 B of the
    vector lattice and 24 B of lagged Lorentz force; the residual snapshot,
    24 B read + written once per 10 levels, adds 4.8 B per level)."""
    import torch
    from paper_0809_4730_gb300.glbe import Batch
    doms, meta = batch_domains("f32c")
    B = Batch(doms)
    bt, bps, sps = B.autotune(10)
    st, res, sec = B.solve(1e-300, levels, use_graph=True)
    upd, byt = 0, 0.0
    for m in meta:
        fluid = m["n"] * (m["n"] - 2) ** 2
        bpn = 19 * 6 * 2 + 4.8 + ((21 * 6 * 2 + 24) if m["Ha"] > 0 else 0)
        upd += fluid * levels
        byt += fluid * levels * bpn
    B.close()
    del B
    torch.cuda.empty_cache()
    return {"levels": levels, "mlups": round(upd / sec / 1e6, 1), "seconds": round(sec, 4),
            "achieved_gbs": round(byt / sec / 1e9, 1), "hbm_frac": round(byt / sec / 1e9 / hbm_peak, 4),
            "launch": {"block_threads": bt, "blocks_per_sm": bps}, "status": st,
            "note": "one persistent cooperative launch over all 64 domains, F32C storage, device time"}


def batch_against_single(levels: int = 200, steps: int = 100):
    """The cost of batching: device time per level of the 64-duct F32C batch
    in one persistent launch (autotuned, CUDA graph) against the sum over the
    same 64 ducts of one single-context plain step each (CUDA events around
    `steps` steps per duct; the smallest ducts are launch-bound there)."""
    import torch
    from paper_0809_4730_gb300.glbe import Batch, Solver
    doms, meta = batch_domains("f32c")
    B = Batch(doms)
    bt, bps, _ = B.autotune(10)
    _, _, sec = B.solve(1e-300, levels, use_graph=True)
    B.close()
    del B
    torch.cuda.empty_cache()
    total, per = 0.0, []
    for m in meta:
        n = m["n"]
        kw = dict(wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=m["gamma"], nu=0.1, F=(1e-6, 0, 0), storage="f32c")
        if m["Ha"] > 0:
            L = (n - 2) / 2
            kw.update(induction=1, gamma_m=m["gamma"], eta=0.1, chi=0.01, mu=1.0,
                      B0=(0, m["Ha"] * math.sqrt(0.1 * 0.1) / L, 0))
        G = Solver(n, n, n, **kw)
        G.step(21)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        G.step(steps)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        total += ms
        per.append({"n": n, "Ha": m["Ha"], "gamma": m["gamma"], "ms": round(ms, 4)})
        G.close()
    return {"metric": "device ms per level: 64-duct F32C batch in one launch vs the ducts as single contexts",
            "batch_ms_per_level": round(sec / levels * 1e3, 4), "single_sum_ms_per_level": round(total, 4),
            "batch_over_single": round(sec / levels * 1e3 / total, 4), "launch": {"block_threads": bt,
                                                                                  "blocks_per_sm": bps},
            "higher_is_better": False, "data": "synthetic", "dtype": "f32", "per_domain": per}


def batch_small(n: int = 96, levels: int = 20):
    """A small batch for profiling the persistent kernel: four n^3 F32C
    ducts (two flow, two coupled at Ha = 5; gamma = gamma_m = 0.1, nu = eta =
    0.1, chi = 0.01, F_x = 1e-6), `levels` levels in one launch of 256-thread
    blocks, two per SM, without a CUDA graph; and the same ducts as single
    contexts."""
    import torch
    from paper_0809_4730_gb300.glbe import Batch, Solver, make_params

    def kw(Ha):
        k = dict(wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=0.1, nu=0.1, F=(1e-6, 0, 0), storage="f32c")
        if Ha > 0:
            L = (n - 2) / 2
            k.update(induction=1, gamma_m=0.1, eta=0.1, chi=0.01, mu=1.0, B0=(0, Ha * math.sqrt(0.1 * 0.1) / L, 0))
        return k

    has = (0.0, 5.0, 0.0, 5.0)
    B = Batch([make_params(n, n, n, **kw(h)) for h in has])
    B.set_launch(256, 2)
    _, _, sec = B.solve(1e-300, levels, use_graph=False)
    B.close()
    del B
    single = 0.0
    for h in has:
        G = Solver(n, n, n, **kw(h))
        G.step(21)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        G.step(100)
        e1.record()
        e1.synchronize()
        single += e0.elapsed_time(e1) / 100
        G.close()
    return {"metric": "device ms per level: four %d^3 F32C ducts (two coupled) in one batch launch vs single "
                      "contexts" % n, "batch_ms_per_level": round(sec / levels * 1e3, 4),
            "single_sum_ms_per_level": round(single, 4), "higher_is_better": False, "data": "synthetic",
            "dtype": "f32", "launch": {"block_threads": 256, "blocks_per_sm": 2, "levels": levels}}


def adjoint_bounded(hbm_peak: float, n: int = 128, fwd_steps: int = 500, iters: int = 500):
    """The steady adjoint iteration of the adjoint workload (n^3 Hartmann
    duct, F32C state, FP32 cotangents), bounded: glbe_adjoint_steady for
    `iters` iterations at the state `fwd_steps` steps from rest (an iteration
    costs the same at any state; the full workload first solves to 1e-7).
    Device time per iteration, including the one linearisation launch and
    the finalize every 10 iterations."""
    import torch
    G, F, fluid = adjoint_duct(n)
    G.step(fwd_steps)
    G.adjoint_steady(None, tol=1e-30, max_iters=10)      # workspace allocated outside the timed region
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    _, st, it, _ = G.adjoint_steady(None, tol=1e-30, max_iters=iters)
    e1.record(stream)
    e1.synchronize()
    # stopped by max_iters (a multiple of 10): all `iters` iterations ran; `it`
    # is the last level whose gradient change was evaluated
    per_it = e0.elapsed_time(e1) / 1e3 / iters
    bpn = adjoint_bytes_per_node(True)
    G.close()
    del G, F
    torch.cuda.empty_cache()
    return {"iterations": iters, "last_evaluated": it, "ms_per_iteration": round(per_it * 1e3, 4),
            "bytes_per_node": bpn,
            "mlups": round(fluid / per_it / 1e6, 1), "hbm_frac": round(bpn * fluid / per_it / 1e9 / hbm_peak, 4),
            "status": st, "note": "stopped at max_iters by design (status 4); one linearisation launch included"}


def hartmann_analytic(ny, Ha, F=1e-6, nu=0.01):
    """Insulating-wall Hartmann profile with the walls half-way between the
    solid and first fluid rows (half-width L = (ny - 2)/2)."""
    L = (ny - 2) / 2
    A = F * L * L / (nu * Ha * math.tanh(Ha))
    return [A * (1 - math.cosh(Ha * (y - (ny - 1) / 2) / L) / math.cosh(Ha)) for y in range(ny)]


def time_to_solution():
    """Wall time to r <= 1e-8 on the 64x64x8 Hartmann duct (Pr_m = 0.01,
    nu = eta = 0.01, Ha = 5, 10, 20) at gamma = gamma_m = 0.025, 0.05, 0.1 and 1, same
    GPU, FP32 arithmetic with compensated (F32C) storage, with the error of
    the converged u against the analytic profile."""
    import torch
    from paper_0809_4730_gb300.glbe import Solver
    res = {}
    nu, eta, chi = 0.01, 0.01, 0.01
    for Ha in (5.0, 10.0, 20.0):
        B0 = Ha * math.sqrt(nu * eta) / 31.0
        ua = hartmann_analytic(64, Ha)
        r_ha = {}
        for gamma in (0.025, 0.05, 0.1, 1.0):
            G = Solver(64, 64, 8, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(1e-6, 0, 0),
                       induction=1, gamma_m=gamma, eta=eta, chi=chi, mu=1.0, B0=(0, B0, 0), storage="f32c")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, steps, r = G.solve(1e-8, 3_000_000)
            t1 = time.perf_counter()
            _, u, _ = G.fields()
            G.sync()
            ux = u[0].reshape(8, 64, 64)[0, :, 0].double().cpu().tolist()
            err = max(abs(ux[y] - ua[y]) for y in range(1, 63)) / max(ua)
            r_ha[f"gamma_{gamma}"] = {"status": st, "steps": steps, "r": r, "wall_s": round(t1 - t0, 4),
                                      "err_vs_analytic": err}
            G.close()
        b = r_ha["gamma_1.0"]
        for g in ("0.1", "0.05", "0.025"):
            a = r_ha[f"gamma_{g}"]
            r_ha[f"speedup_wall_gamma_{g}"] = round(b["wall_s"] / a["wall_s"], 2) if a["wall_s"] > 0 else None
            r_ha[f"speedup_steps_gamma_{g}"] = round(b["steps"] / max(1, a["steps"]), 2)
        res[f"Ha_{int(Ha)}"] = r_ha
    return res


# ---------------------------------------------------------------------------
# FP64 CPU oracle (the baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample():
    """A bounded sample of the duct workload the CPU oracle can time: an
    8-node-long slab of the same 256 x 256 cross-section (x periodic, the
    force is x-invariant)."""
    import numpy as np
    import oracle
    from paper_0809_4730_gb300.inputs import duct_force_x
    d = DUCT
    nx = 8
    cfg = oracle.Config(nx, d["ny"], d["nz"], wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=d["gamma"], nu=d["nu"])
    F = duct_force_x(nx, d["ny"], d["nz"], d["F0"]).reshape(3, -1).T.copy()
    S = oracle.Solver(cfg, Fext=F)
    fluid = nx * (d["ny"] - 2) * (d["nz"] - 2)
    return S, fluid, f"oracle FP64 on an {nx}x{d['ny']}x{d['nz']} slab of the duct"


DUCT64_GAMMAS = (1.0, 0.5, 0.1, 0.05)


def duct64_oracle_columns():
    """The 64^3 copy of the duct (same F_x(y, z) and nu, H = 64): its steady
    state is x-invariant, so the oracle marches the 1 x 64 x 64 column, the
    same discrete problem, at each gamma of the sweep: timed to r <= 1e-8
    (steps and wall time of the FP64 CPU method), then on to r <= 1e-11 for
    the converged reference field."""
    import numpy as np
    import oracle
    from paper_0809_4730_gb300.inputs import duct_force_x
    n = 64
    Fx = duct_force_x(1, n, n, DUCT["F0"])[0].reshape(-1)
    Fext = np.zeros((n * n, 3))
    Fext[:, 0] = Fx
    out = {}
    for gamma in DUCT64_GAMMAS:
        S = oracle.Solver(oracle.Config(1, n, n, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=DUCT["nu"]),
                          Fext=Fext)
        t0 = time.perf_counter()
        S.run(3_000_000, tol=1e-8)
        dt = time.perf_counter() - t0
        t8 = S.t
        S.run(3_000_000, tol=1e-11)
        _, u, _, _ = S.fields()
        out[gamma] = {"steps_1e-8": t8, "wall_s_1e-8_column": round(dt, 3),
                      "mlups": round(n * n * t8 / dt / 1e6, 3), "col": u[:, 0].reshape(n, n)}
    return out


def cpu_baseline(target_s: float = 10.0):
    """The CPU leg: the FP64 oracle timed on a bounded sample of the duct
    (value), and on the 64^3 duct copy's column per gamma, whose converged
    fields are the references of the GPU steady errors (returned apart)."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    S, fluid, desc = oracle_sample()
    t0 = time.perf_counter()
    S.run(2)
    dt = max(1e-6, time.perf_counter() - t0)
    n = max(2, min(400, int(target_s / (dt / 2))))
    t0 = time.perf_counter()
    S.run(n)
    dt = time.perf_counter() - t0
    refs = duct64_oracle_columns()
    cols = {f"gamma_{g}": {k: v for k, v in r.items() if k != "col"} for g, r in refs.items()}
    return ({"value": round(n * fluid / dt / 1e6, 3), "unit": "MLUPS", "cores": oracle.get_threads(),
             "kind": "oracle", "sample": f"{desc}, {n} time steps, {dt:.1f} s",
             "duct64_column_to_1e-8": cols}, refs)


def duct64_study(refs):
    """GPU side of the 64^3 duct copy, against the oracle references:
    (1) steady error of each storage form at gamma = 0.1 after 4000 steps
    (relative L-infinity of u_x over the fluid nodes); (2) time to r <= 1e-8
    with compensated storage at each gamma of the sweep: steps, device wall
    time, error against the converged oracle field, and the gain over
    gamma = 1 at the same physical nu."""
    import numpy as np
    import torch
    from paper_0809_4730_gb300.glbe import Solver
    from paper_0809_4730_gb300.inputs import duct_force_x
    n = 64
    Ff = torch.tensor(duct_force_x(n, n, n, DUCT["F0"])[0].reshape(1, -1), dtype=torch.float32, device="cuda")

    def make(st, gamma):
        G = Solver(n, n, n, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=DUCT["nu"], force_field=1,
                   storage=st)
        G.set_force(Ff)
        return G

    def err(G, col):
        _, u, _ = G.fields()
        torch.cuda.synchronize()
        ux = u[0].double().cpu().numpy().reshape(n, n, n)[1:-1, 1:-1, :]
        c = col[1:-1, 1:-1]
        return float(np.abs(ux - c[:, :, None]).max() / np.abs(c).max())

    steady = {"workload": "64^3 duct copy, gamma = 0.1, 4000 steps from rest, rel. L-inf error of u_x against "
                          "the converged FP64 oracle"}
    for st in ("f32c", "f32", "f16", "bf16", "f16sr", "bf16sr"):
        G = make(st, 0.1)
        G.step(4000)
        info = G.residual()
        steady[st] = {"error": err(G, refs[0.1]["col"]), "r": info.r}
        G.close()
    stream = torch.cuda.current_stream()
    tts = {"workload": "64^3 duct copy (nu = 0.5, F0 = 1e-6), F32C storage, glbe_solve to r <= 1e-8 from rest"}
    for gamma in DUCT64_GAMMAS:
        G = make("f32c", gamma)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        status, steps, r = G.solve(1e-8, 500_000)
        e1.record(stream)
        e1.synchronize()
        tts[f"gamma_{gamma}"] = {"status": status, "steps": steps, "r": r, "wall_s": round(e0.elapsed_time(e1) / 1e3, 4),
                                 "error_vs_oracle": err(G, refs[gamma]["col"]),
                                 "oracle_steps_1e-8": refs[gamma]["steps_1e-8"]}
        G.close()
    base = tts["gamma_1.0"]
    for gamma in DUCT64_GAMMAS[1:]:
        a = tts[f"gamma_{gamma}"]
        a["gain_wall_vs_gamma_1"] = round(base["wall_s"] / a["wall_s"], 2) if a["wall_s"] > 0 else None
        a["gain_steps_vs_gamma_1"] = round(base["steps"] / max(1, a["steps"]), 2)
    return steady, tts


def run_reference(args, rank, ws):
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    S, fluid, desc = oracle_sample()
    S.run(10 * args.warmup)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.run(10)
    dt = time.perf_counter() - t0
    mlups = 10 * args.steps * fluid / dt / 1e6
    return {
        "impl": "reference",
        "metric": "MLUPS (fluid-node updates/s) and % of HBM roofline of the fused GLBE step",
        "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "square duct 512x256x256 (bounded sample: 8x256x256 slab), Fx(y,z), nu=0.5, "
                               "gamma=0.1, D3Q19 MRT-GLBE, FP64 CPU oracle", "parallelism": "cpu"},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": f"{desc}, {10 * args.steps} time steps"},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def batch_domains(storage: str):
    """64 cubic ducts (x periodic, walls y and z) with seeded edge lengths
    uniform in 32..160, (gamma, Ha) from {1, 0.1, 0.05} x {0, 5, 20} assigned
    round-robin after a seeded shuffle, nu = eta = 0.1, chi = 0.01
    (Pr_m = chi nu/eta = 0.01), F_x = 1e-6 uniform, Ha = 0 without the
    induction lattice."""
    import random
    from paper_0809_4730_gb300.glbe import make_params
    from paper_0809_4730_gb300.inputs import batch_sizes
    sizes = [int(n) for n in batch_sizes(64, 32, 160, seed=0)]
    combos = [(g, h) for g in (1.0, 0.1, 0.05) for h in (0.0, 5.0, 20.0)]
    order = list(range(len(combos)))
    random.Random(0).shuffle(order)
    doms, meta = [], []
    nu = eta = 0.1
    for k, n in enumerate(sizes):
        gamma, Ha = combos[order[k % len(order)]]
        kw = dict(wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=nu, F=(1e-6, 0, 0), storage=storage)
        if Ha > 0:
            L = (n - 2) / 2
            kw.update(induction=1, gamma_m=gamma, eta=eta, chi=0.01, mu=1.0, B0=(0, Ha * math.sqrt(nu * eta) / L, 0))
        doms.append(make_params(n, n, n, **kw))
        meta.append(dict(n=n, gamma=gamma, Ha=Ha))
    return doms, meta


def run_batch(args, rank, ws):
    import torch
    from paper_0809_4730_gb300.glbe import Batch
    doms, meta = batch_domains(args.batch_storage)
    B = Batch(doms)
    bt, bps, sps = B.autotune(20)
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        st, res, sec = B.solve(args.batch_tol, args.batch_max_steps, use_graph=True)
    sec = max_over_ranks(sec, ws)
    # node updates: each domain marched to its convergence level + 1 (or the cap)
    updates = 0
    for m, r in zip(meta, res):
        fluid = m["n"] * (m["n"] - 2) ** 2
        steps = (r["steps"] + 1) if r["converged"] else args.batch_max_steps
        updates += fluid * steps
    per = [dict(m, converged=r["converged"], steps=r["steps"], seconds=round(r["seconds"], 4), r=r["r"])
           for m, r in zip(meta, res)]
    by = {}
    for q in per:
        key = f"gamma_{q['gamma']}"
        by.setdefault(key, []).append((q["seconds"], q["steps"]) if q["converged"] else None)

    def median(xs):
        xs = sorted(xs)
        return xs[len(xs) // 2] if xs else None
    # per-solve time: device seconds from the launch start to the domain's
    # convergence (all domains share the launch), and its level count
    summary = {k: {"converged": sum(x is not None for x in v), "of": len(v),
                   "median_s": median([x[0] for x in v if x is not None]),
                   "median_steps": median([x[1] for x in v if x is not None])} for k, v in by.items()}
    B.close()
    return {
        "metric": f"aggregate MLUPS of the batched steady solve (64 ducts, one persistent launch) to r <= "
                  f"{args.batch_tol:g}",
        "value": round(updates / sec / 1e6 * ws, 1), "unit": "MLUPS", "n_gpus": ws, "steps": 1, "warmup": 0,
        "ms_per_step": round(sec * 1e3, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "64 cubic ducts n~U{32..160} (seed 0), gamma x Ha in {1,0.1,0.05} x {0,5,20} "
                               "round-robin after seeded shuffle, nu=eta=0.1, chi=0.01, Fx=1e-6, "
                               + args.batch_storage + " storage", "nodes": sum(m["n"] ** 3 for m in meta),
                   "launch": {"block_threads": bt, "blocks_per_sm": bps, "autotune_s_per_step": sps}},
        "status": st, "tol": args.batch_tol, "max_steps": args.batch_max_steps, "per_gamma": summary,
        "converged": sum(1 for r in res if r["converged"]), "diverged": sum(1 for r in res if r["nonfinite"]),
        "domains": per, "clocks": clk.summary(),
    }


# ---------------------------------------------------------------------------
# Stability and preconditioning sweeps (Sec. 5: Poiseuille stability,
# Hartmann gamma_m studies), many small problems per persistent launch
# ---------------------------------------------------------------------------
SWEEP_NU = (0.002, 0.005, 0.02, 0.05)
SWEEP_UMAX = (0.005, 0.01, 0.02, 0.04)
SWEEP_GAMMA = (1.0, 0.5, 0.2, 0.1, 0.05, 0.02, 0.01, 0.005)


def channel_params(nu: float, umax: float, gamma: float, H: int = 32, storage: str = "f32c"):
    """Plane channel 1 x (H + 2) x 1 (walls at y = 0, H + 1; half-way walls
    H apart), uniform F_x giving the Poiseuille maximum u_max = F H^2/(8 nu)."""
    from paper_0809_4730_gb300.glbe import make_params
    F = 8.0 * nu * umax / (H * H)
    return make_params(1, H + 2, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(F, 0, 0),
                       storage=storage)


def stability_map(nus=SWEEP_NU, umaxs=SWEEP_UMAX, gammas=SWEEP_GAMMA, max_steps=100_000, tol=1e-8):
    """All (nu, u_max, gamma) channels in one persistent launch.  A domain is
    unstable when its velocity becomes non-finite; gamma_min(nu, u_max) is
    the smallest gamma of the sweep whose channel stayed finite (None if
    none did)."""
    from paper_0809_4730_gb300.glbe import Batch
    pts = [(nu, um, g) for nu in nus for um in umaxs for g in gammas]
    B = Batch([channel_params(*q) for q in pts])
    st, res, sec = B.solve(tol, max_steps, use_graph=True)
    B.close()
    cells = {}
    for (nu, um, g), r in zip(pts, res):
        c = cells.setdefault((nu, um), {})
        c[g] = "diverged" if r["nonfinite"] else ("converged" if r["converged"] else "finite")
        c[f"steps_{g}"] = r["steps"]
    out = {"seconds": round(sec, 3), "domains": len(pts), "max_steps": max_steps, "tol": tol, "map": []}
    for (nu, um), c in cells.items():
        stable = [g for g in gammas if c[g] != "diverged"]
        out["map"].append({"nu": nu, "u_max": um, "Ma": um * math.sqrt(3.0), "gamma_min": min(stable) if stable
                           else None, "status": {str(g): c[g] for g in gammas},
                           "steps": {str(g): c[f"steps_{g}"] for g in gammas}})
    return out


def hartmann_channel(Ha: float, gamma: float, gamma_m: float, H: int = 62, nu: float = 0.01,
                     storage: str = "f32c"):
    """Hartmann channel 1 x (H + 2) x 1 of the Hartmann workload (walls on y,
    B0 along y, nu = eta = 0.01, chi = 0.01, F_x = 1e-6)."""
    from paper_0809_4730_gb300.glbe import make_params
    B0 = Ha * math.sqrt(nu * nu) / (H / 2)
    return make_params(1, H + 2, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(1e-6, 0, 0),
                       induction=1, gamma_m=gamma_m, eta=nu, chi=0.01, mu=1.0, B0=(0, B0, 0), storage=storage)


GAMMA_M_SWEEP = (1.0, 0.5, 0.2, 0.1, 0.05, 0.02)


def gamma_m_sweep(Ha: float = 10.0, gammas=(0.05, 1.0), gms=GAMMA_M_SWEEP, max_steps=2_000_000, tol=1e-8):
    """Steps to r <= tol of the Hartmann channel for every (gamma, gamma_m)
    pair, all in one persistent launch."""
    from paper_0809_4730_gb300.glbe import Batch
    pts = [(g, gm) for g in gammas for gm in gms]
    B = Batch([hartmann_channel(Ha, g, gm) for g, gm in pts])
    st, res, sec = B.solve(tol, max_steps, use_graph=True)
    B.close()
    out = {"Ha": Ha, "seconds": round(sec, 3), "tol": tol}
    for (g, gm), r in zip(pts, res):
        out.setdefault(f"gamma_{g}", {})[f"gamma_m_{gm}"] = (r["steps"] if r["converged"] else
                                                            ("diverged" if r["nonfinite"] else None))
    for g in gammas:
        row = {k: v for k, v in out[f"gamma_{g}"].items() if isinstance(v, int)}
        out[f"gamma_{g}"]["fastest"] = min(row, key=row.get) if row else None
    return out


def srt_mrt_stability(nus=(0.0005, 0.001, 0.002, 0.005, 0.01), umax=0.05, gamma=0.1, steps=50_000):
    """The preconditioned SRT-LBE and the MRT-GLBE on the same channel at
    decreasing viscosity (u_max = 0.05, gamma = 0.1): which stay finite."""
    from paper_0809_4730_gb300.glbe import GLBE_ERR_DIVERGED, GlbeError, Solver
    out = {"u_max": umax, "gamma": gamma, "steps": steps}
    H = 32
    for coll, name in ((0, "mrt"), (1, "srt")):
        row = {}
        for nu in nus:
            F = 8.0 * nu * umax / (H * H)
            G = Solver(1, H + 2, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(F, 0, 0),
                       storage="f32", collision=coll)
            G.step(steps)
            try:
                info = G.residual()
                row[str(nu)] = "finite" if math.isfinite(info.r) else "diverged"
            except GlbeError as e:
                row[str(nu)] = "diverged" if e.status == GLBE_ERR_DIVERGED else "error"
            G.close()
        out[name] = row
    for name in ("mrt", "srt"):
        ok = [float(k) for k, v in out[name].items() if v == "finite"]
        out[f"{name}_nu_min_stable"] = min(ok) if ok else None
    return out


def run_sweeps(args, rank, ws):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    smap = stability_map()
    gms = gamma_m_sweep()
    srt = srt_mrt_stability()
    return {"metric": "stability and preconditioning sweeps (batched persistent launches)", "value": None,
            "unit": None, "n_gpus": ws, "higher_is_better": True, "data": "synthetic", "dtype": "f32",
            "config": {"workload": "plane channels 1x34x1 over (nu, u_max, gamma); Hartmann channel 1x64x1, "
                                   "Ha=10, over (gamma, gamma_m); SRT vs MRT channel at u_max=0.05, gamma=0.1"},
            "stability_map": smap, "gamma_m_sweep": gms, "srt_vs_mrt": srt,
            "wall_s": round(time.perf_counter() - t0, 2)}


# ---------------------------------------------------------------------------
# 3D lid-driven cavity (Sec. 5): 64^3 fluid nodes (W = 64 between half-way
# walls), lid along x at U0 = 0.0235, nu = 0.015 (Re = 100); MHD case with B0
# along y (parallel to the lid, normal to its motion), Ha = 45
# (B0 = Ha sqrt(nu eta)/(W/2)), eta = 0.015, Pr_m = chi nu/eta = 5.625e-7, on
# an extended magnetic domain of CAV_EXT nodes around the cavity
# ---------------------------------------------------------------------------
CAV_W, CAV_U, CAV_NU, CAV_EXT = 64, 0.0235, 0.015, 16


def cavity_solver(gamma: float, mhd: bool, storage: str = "f32c", nu: float = CAV_NU, collision: int = 0):
    from paper_0809_4730_gb300.glbe import Solver
    if not mhd:
        n = CAV_W + 2
        return Solver(n, n, n, wall_lo=(1, 1, 1), wall_hi=(1, 1, 1), gamma=gamma, nu=nu, U_lid=(CAV_U, 0, 0),
                      storage=storage, collision=collision), n ** 3
    n = CAV_W + 2 + 2 * CAV_EXT
    lo, hi = 1 + CAV_EXT, n - 2 - CAV_EXT
    eta, Ha = 0.015, 45.0
    B0 = Ha * math.sqrt(nu * eta) / (CAV_W / 2)
    G = Solver(n, n, n, wall_lo=(1, 1, 1), wall_hi=(1, 1, 1), gamma=gamma, nu=nu, U_lid=(CAV_U, 0, 0),
               box=((lo, lo, lo), (hi, hi, hi)), induction=1, gamma_m=gamma, eta=eta, chi=5.625e-7 * eta / nu,
               mu=1.0, B0=(0, B0, 0), storage=storage, collision=collision)
    return G, n ** 3


def run_tts(args, rank, ws):
    """Time to r <= 1e-8 on the full 512 x 256 x 256 duct (F32C storage, the
    duct's nu = 0.5) at gamma = 1, 0.5, 0.1 and 0.05: steps, device time,
    and (CPU leg) the error of the converged field against the FP64 oracle
    on the 1 x 256 x 256 column at gamma = 0.1 -- the duct's steady state is
    x-invariant, so the column is the same discrete problem."""
    import numpy as np
    import torch
    from paper_0809_4730_gb300.glbe import Solver
    from paper_0809_4730_gb300.inputs import duct_force_x
    stream = torch.cuda.current_stream()
    d = DUCT
    Fx = torch.tensor(duct_force_x(d["nx"], d["ny"], d["nz"], d["F0"])[0].reshape(1, -1), dtype=torch.float32,
                      device="cuda")
    out = {"metric": "steps and device time to r <= 1e-8, 512x256x256 duct, F32C", "n_gpus": ws,
           "higher_is_better": False, "data": "synthetic", "dtype": "f32"}
    fields = {}
    for gamma in (1.0, 0.5, 0.1, 0.05):
        G = Solver(d["nx"], d["ny"], d["nz"], wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=gamma, nu=d["nu"],
                   force_field=1, storage="f32c")
        G.set_force(Fx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        st, steps, r = G.solve(1e-8, 400_000)
        e1.record(stream)
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        out[f"gamma_{gamma}"] = {"status": st, "steps": steps, "r": r, "seconds": round(sec, 3)}
        print(f"tts gamma {gamma}: {out[f'gamma_{gamma}']}", file=sys.stderr, flush=True)
        if gamma == 0.1:
            _, u, _ = G.fields()
            fields[gamma] = u[0].reshape(d["nz"], d["ny"], d["nx"]).double().cpu().numpy()
        G.close()
    base = out["gamma_1.0"]
    for gamma in (0.5, 0.1, 0.05):
        a = out[f"gamma_{gamma}"]
        if a["status"] == 0 and base["status"] == 0:
            a["gain_steps_vs_gamma_1"] = round(base["steps"] / a["steps"], 2)
            a["gain_time_vs_gamma_1"] = round(base["seconds"] / a["seconds"], 2)
    if not args.no_cpu_baseline:
        # CPU leg: the oracle on the x-invariant column at gamma = 0.1
        import oracle
        oracle.set_threads(os.cpu_count() or 1)
        ny, nz = d["ny"], d["nz"]
        F = duct_force_x(1, ny, nz, d["F0"])[0].reshape(-1)
        Fext = np.zeros((ny * nz, 3))
        Fext[:, 0] = F
        S = oracle.Solver(oracle.Config(1, ny, nz, wall_lo=(0, 1, 1), wall_hi=(0, 1, 1), gamma=0.1, nu=d["nu"]),
                          Fext=Fext)
        t0 = time.perf_counter()
        S.run(3_000_000, tol=1e-8)
        t8, w8 = S.t, time.perf_counter() - t0
        S.run(3_000_000, tol=1e-11)
        _, ou, _, _ = S.fields()
        col = ou[:, 0].reshape(nz, ny)[1:-1, 1:-1]
        ux = fields[0.1][1:-1, 1:-1, :]
        out["gamma_0.1"]["error_vs_oracle"] = float(np.abs(ux - col[:, :, None]).max() / np.abs(col).max())
        out["cpu_baseline"] = {"kind": "oracle", "cores": oracle.get_threads(), "sample": "1x256x256 column, gamma 0.1",
                               "steps_1e-8": t8, "seconds_1e-8": round(w8, 2),
                               "value": round(ny * nz * t8 / w8 / 1e6, 3), "unit": "MLUPS"}
    return out


def cpu_configs():
    """CPU baseline of the small configurations, the FP64 oracle on this
    host: the 4 x 32 x 4 Poiseuille channel (gamma = 0.1, tau = 0.8 on the
    stress rows, i.e. nu = gamma (tau - 1/2)/3; gamma = 1 at the same nu) to
    r <= 1e-10, and the 64 x 64 x 8 Hartmann duct (walls on y, periodic x
    and z: its steady state is the 1 x 64 x 1 column's) at Ha = 5, 10, 20,
    gamma = gamma_m in {1, 0.1}, Pr_m = 0.01, to r <= 1e-8.  Steps, wall
    time, MLUPS of the column, error against the closed forms.  One thread
    (the problems are a few hundred nodes)."""
    import numpy as np
    import oracle
    oracle.set_threads(1)
    out = {"kind": "oracle", "cores": 1}
    nu1 = 0.1 * (0.8 - 0.5) / 3
    rows = {}
    for gamma in (1.0, 0.1):
        cfg = oracle.Config(4, 32, 4, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu1, F=(1e-6, 0, 0))
        S = oracle.Solver(cfg)
        t0 = time.perf_counter()
        S.run(20_000_000, tol=1e-10)
        w = time.perf_counter() - t0
        _, u, _, _ = S.fields()
        y = np.arange(32, dtype=float)
        ana = 1e-6 * (y - 0.5) * (30.5 - y) / (2 * nu1)
        ux = u.reshape(4, 32, 4, 3)[0, 1:-1, 0, 0]
        rows[f"gamma_{gamma}"] = {"steps": S.t, "seconds": round(w, 3), "mlups": round(512 * S.t / w / 1e6, 2),
                                  "err_vs_analytic": float(np.abs(ux - ana[1:-1]).max() / ana.max())}
    out["poiseuille_4x32x4_to_1e-10"] = rows
    rows = {}
    for Ha in (5.0, 10.0, 20.0):
        for gamma in (1.0, 0.1):
            nu = eta = 0.01
            ny = 64
            L = (ny - 2) / 2
            B0 = Ha * nu / L
            cfg = oracle.Config(1, ny, 1, wall_lo=(0, 1, 0), wall_hi=(0, 1, 0), gamma=gamma, nu=nu, F=(1e-6, 0, 0),
                                induction=True, gamma_m=gamma, eta=eta, chi=0.01, mu=1.0, B0=(0, B0, 0))
            S = oracle.Solver(cfg)
            t0 = time.perf_counter()
            S.run(20_000_000, tol=1e-8)
            w = time.perf_counter() - t0
            _, u, _, _ = S.fields()
            yy = np.arange(ny) - (ny - 1) / 2
            A = 1e-6 * L ** 2 / (nu * Ha * np.tanh(Ha))
            ua = A * (1 - np.cosh(Ha * yy / L) / np.cosh(Ha))
            rows[f"Ha_{Ha:g}_gamma_{gamma}"] = {
                "steps": S.t, "seconds": round(w, 3), "mlups": round(62 * S.t / w / 1e6, 2),
                "err_vs_analytic": float(np.abs(u[1:-1, 0] - ua[1:-1]).max() / ua.max())}
    out["hartmann_64x64x8_column_to_1e-8"] = rows
    return out


def run_cavity(args, rank, ws):
    """Convergence of the cavity against gamma (Sec. 5: without and with the
    magnetic field, gamma = gamma_m), F32C storage, steps and device time to
    r <= 1e-6 (the FP32 collide arithmetic at the lid edges keeps r near
    1e-7), and the stability of the preconditioned SRT-LBE against the
    GLBE at decreasing viscosity on the MHD cavity."""
    import torch
    from paper_0809_4730_gb300.glbe import GLBE_ERR_DIVERGED, GlbeError
    stream = torch.cuda.current_stream()
    out = {"metric": "cavity: steps and device time to r <= 1e-6 against gamma; SRT vs GLBE stability",
           "n_gpus": ws, "higher_is_better": False, "data": "synthetic", "dtype": "f32",
           "config": {"workload": f"lid-driven cavity {CAV_W}^3 fluid nodes, U0={CAV_U}, nu={CAV_NU} (Re=100); "
                                  f"MHD: Ha=45, eta=0.015, Pr_m=5.625e-7, B0 along y, extended magnetic domain "
                                  f"of {CAV_EXT} nodes"}}
    for mhd, gammas in ((False, (1.0, 0.5, 0.2, 0.1)), (True, (1.0, 0.2, 0.1, 0.05))):
        res = {}
        for g in gammas:
            G, nodes = cavity_solver(g, mhd)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            try:
                st, steps, r = G.solve(1e-6, 600_000)
            except GlbeError as e:          # a diverged march is a result, not a failure of the bench
                st, steps, r = e.status, G.t, float("nan")
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            res[f"gamma_{g}"] = {"status": st, "steps": steps, "r": r, "seconds": round(sec, 3),
                                 "mlups": round(nodes * steps / max(sec, 1e-9) / 1e6, 1)}
            print(f"cavity {'mhd' if mhd else 'hydro'} gamma {g}: {res[f'gamma_{g}']}", file=sys.stderr, flush=True)
            G.close()
        base = res["gamma_1.0"]
        for g in gammas[1:]:
            a = res[f"gamma_{g}"]
            if a["status"] == 0 and base["status"] == 0:
                a["gain_steps_vs_gamma_1"] = round(base["steps"] / max(1, a["steps"]), 2)
                a["gain_time_vs_gamma_1"] = round(base["seconds"] / max(a["seconds"], 1e-9), 2)
        out["mhd" if mhd else "hydro"] = res
    stab = {}
    for coll, name, gam in ((0, "glbe_mrt", 1.0), (1, "srt", 1.0), (0, "glbe_mrt", 0.1), (1, "srt", 0.1)):
        row = {}
        for nu in (0.005, 0.015, 0.05, 0.166):
            G, _ = cavity_solver(gam, True, storage="f32", nu=nu, collision=coll)
            G.step(20_000)
            try:
                info = G.residual()
                row[str(nu)] = "finite" if math.isfinite(info.r) else "diverged"
            except GlbeError as e:
                row[str(nu)] = "diverged" if e.status == GLBE_ERR_DIVERGED else "error"
            print(f"cavity stability {name} gamma {gam} nu {nu}: {row[str(nu)]}", file=sys.stderr, flush=True)
            G.close()
        stab[f"{name}_gamma_{gam}"] = row
    out["stability_mhd_cavity_20000_steps"] = stab
    return out


# ---------------------------------------------------------------------------
# two-dimensional lattices (D2Q9 + D2Q5)
# ---------------------------------------------------------------------------
D2 = {"nx": 4096, "ny": 4096}
# DRAM bytes of one plain coupled F32 launch on the 4096 x 4096 channel (ncu,
# one pass, -c 1: read 1409227776 + write 1376905216 B) per fluid node
TRAFFIC_2D_F32_MHD_B_PER_NODE = (1409227776 + 1376905216) / (4096 * 4094)


def channel2d_solver(storage: str, mhd: bool, nx: int = D2["nx"], ny: int = D2["ny"], Ha: float = 10.0,
                     gamma: float = 0.1, nu: float = 0.01, F: float = 1e-6, variant: int = 0):
    """2D Hartmann channel (the Sec. 5 physics on the D2Q9 + D2Q5 lattices):
    x periodic, walls on y, B0 along y, nu = eta, chi = 0.01, uniform F_x."""
    from paper_0809_4730_gb300.glbe import Solver2D
    kw = dict(wall_lo=(0, 1), wall_hi=(0, 1), gamma=gamma, nu=nu, F=(F, 0.0), storage=storage, variant=variant)
    if mhd:
        L = (ny - 2) / 2
        kw.update(induction=1, gamma_m=gamma, eta=nu, chi=0.01, mu=1.0, B0=(0.0, Ha * nu / L))
    return Solver2D(nx, ny, **kw), nx * (ny - 2)


def bytes_per_node_2d(storage: str, mhd: bool) -> int:
    vb = {"f32": 4, "bf16": 2, "f32c": 6}[storage]
    return 9 * vb * 2 + ((10 * vb * 2 + 2 * 4 * 2) if mhd else 0)


def cpu_baseline_2d(target_s: float = 10.0):
    """The 2D oracle on a bounded sample: a 512 x 130 coupled channel."""
    from oracle import d2
    cores = os.cpu_count() or 1
    S = d2.Solver2(d2.Config2(512, 130, wall_lo=(0, 1), wall_hi=(0, 1), gamma=0.1, nu=0.01, F=(1e-6, 0),
                              induction=True, gamma_m=0.1, eta=0.01, chi=0.01, mu=1.0, B0=(0, 10 * 0.01 / 64)))
    t0 = time.perf_counter()
    S.run(10)
    dt = max(1e-6, time.perf_counter() - t0)
    n = max(10, min(20_000, int(target_s / (dt / 10))))
    t0 = time.perf_counter()
    S.run(n)
    dt = time.perf_counter() - t0
    return {"value": round(n * 512 * 128 / dt / 1e6, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"512x130 coupled D2Q9+D2Q5 channel, {n} time steps, {dt:.1f} s"}


def run_2d(args, rank, ws):
    """The 2D forms (D2Q9 GLBE + D2Q5 induction): MLUPS and HBM roofline of
    the fused step on a 4096 x 4096 Hartmann channel (F32, BF16, F32C; with
    and without the induction lattice), and steps and device time to
    r <= 1e-8 on the 64 x 64 Hartmann cross-section of config 2 at
    gamma = 1, 0.1, 0.05 (F32C) with the error against the analytic profile
    and, in the CPU leg, against the converged FP64 oracle."""
    from paper_0809_4730_gb300.glbe import GlbeError
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    try:
        hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        hbm = 6800.0
    forms = {}
    nx2, ny2 = args.nx or D2["nx"], args.ny or D2["ny"]
    for key in args.forms2d.split(","):
        parts = key.split("_")          # storage_kind[_vN]
        st, mhd = parts[0], parts[1] == "mhd"
        var = int(parts[2][1:]) if len(parts) > 2 else 0
        G, fluid = channel2d_solver(st, mhd, nx=nx2, ny=ny2, variant=var)
        G.step(10 * args.warmup)
        G.sync()
        with ClockSampler(torch.cuda.current_device()) as clk:
            total_ms, plain_ms, nplain = timed_steps(G, args.steps, stream)
        kern_ms = plain_ms / nplain
        bpn = bytes_per_node_2d(st, mhd)
        achieved = bpn * fluid / (kern_ms * 1e-3) / 1e9
        forms[key] = {
            "mlups": round(10 * args.steps * fluid / (total_ms * 1e-3) / 1e6, 1),
            "ms_per_step": round(total_ms / args.steps, 4), "kernel_ms": round(kern_ms, 5),
            "bytes_per_node": bpn, "achieved_gbs": round(achieved, 1), "frac": round(achieved / hbm, 4),
            "clocks": clk.summary()}
        print(f"2d {key}: {forms[key]}", file=sys.stderr, flush=True)
        G.close()
    head = forms.get("f32_mhd") or next(iter(forms.values()))
    kernels = {k: ("step2d_pair_kernel" if (k.split("_")[0] in ("f32", "bf16") and k.endswith("_v2"))
                   else "step2d_kernel") for k in forms}
    line = {"metric": "MLUPS of the fused D2Q9 + D2Q5 step (lagged Lorentz force)", "value": head["mlups"],
            "unit": "MLUPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "dtype": "f32",
            "data": "synthetic", "vs_baseline": None,
            "config": {"workload": f"2D Hartmann channel {nx2}x{ny2}, Ha=10, gamma=0.1, Pr_m=0.01, "
                                   f"F32 storage", "l2": "state larger than L2 (2.9 GB at 4096x4096), no flush"},
            "roofline": {"bound": "hbm", "achieved": head["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                         "frac": head["frac"], "bytes_per_node": head["bytes_per_node"],
                         "kernel_ms": head["kernel_ms"],
                         "traffic": (round(TRAFFIC_2D_F32_MHD_B_PER_NODE * nx2 * (ny2 - 2))
                                     if "f32_mhd" in forms and (nx2, ny2) == (D2["nx"], D2["ny"]) else None),
                         "traffic_note": "bytes of one plain launch, ncu capture (-c 1) on this 4096x4096 channel",
                         "kernel": kernels.get("f32_mhd", "step2d_kernel")},
            "gpu_launches": 11 * args.steps, "clocks": head["clocks"], "forms": forms}
    if args.no_tts:
        return line
    # time to r <= 1e-8 on the 2D cross-section of the Hartmann duct of
    # config 2 (64 x 64, walls on y, Ha = 10, Pr_m = 0.01; x-invariant steady state)
    ny, Ha = 64, 10.0
    L = (ny - 2) / 2
    y = np.arange(ny) - (ny - 1) / 2
    A = 1e-6 * L ** 2 / (0.01 * Ha * np.tanh(Ha))
    ua = A * (1 - np.cosh(Ha * y / L) / np.cosh(Ha))
    tts, cols = {}, {}
    for gamma in (1.0, 0.1, 0.05):
        G, _ = channel2d_solver("f32c", True, nx=64, ny=ny, gamma=gamma)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        try:
            st, steps, r = G.solve(1e-8, 2_000_000)
        except GlbeError as e:            # a diverged march is a result, not a failure of the bench
            st, steps, r = e.status, G.t, float("nan")
        e1.record(stream)
        e1.synchronize()
        _, u, _ = G.fields()
        ux = u[0].reshape(ny, 64).double().cpu().numpy()
        cols[gamma] = ux
        err = float(np.abs(ux[1:-1] - ua[1:-1, None]).max() / ua.max())
        tts[f"gamma_{gamma}"] = {"status": st, "steps": steps, "r": r,
                                 "seconds": round(e0.elapsed_time(e1) / 1e3, 4), "error_vs_analytic": err}
        print(f"2d tts gamma {gamma}: {tts[f'gamma_{gamma}']}", file=sys.stderr, flush=True)
        G.close()
    for gamma in (0.1, 0.05):
        a, b = tts[f"gamma_{gamma}"], tts["gamma_1.0"]
        if a["status"] == 0 and b["status"] == 0:
            a["gain_steps_vs_gamma_1"] = round(b["steps"] / a["steps"], 2)
            a["gain_time_vs_gamma_1"] = round(b["seconds"] / a["seconds"], 2)
    line["time_to_1e-8_hartmann_64x64"] = tts
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import d2
        line["cpu_baseline"] = cpu_baseline_2d()
        S = d2.Solver2(d2.Config2(1, ny, wall_lo=(0, 1), wall_hi=(0, 1), gamma=0.1, nu=0.01, F=(1e-6, 0),
                                  induction=True, gamma_m=0.1, eta=0.01, chi=0.01, mu=1.0, B0=(0, Ha * 0.01 / L)))
        t0 = time.perf_counter()
        S.run(3_000_000, tol=1e-8)
        t8, w8 = S.t, time.perf_counter() - t0
        S.run(3_000_000, tol=1e-12)
        _, ou, _ = S.fields()
        ref = ou[1:-1, 0]
        tts["gamma_0.1"]["error_vs_oracle"] = float(np.abs(cols[0.1][1:-1] - ref[:, None]).max() / np.abs(ref).max())
        tts["oracle_column_gamma_0.1"] = {"steps_1e-8": t8, "seconds_1e-8": round(w8, 3)}
    return line


ADJ_NU = 0.05   # nu = eta of the adjoint workload (0.01 diverged at gamma = 0.1: u_max 0.04, Re ~ 500)


def adjoint_duct(n: int, storage: str = "f32c"):
    """The adjoint workload: n^3 Hartmann duct (Ha = 10, gamma = 0.1,
    nu = eta = 0.05, chi = 0.01) driven by the seeded per-node Gaussian force
    F_x ~ N(F0, (0.2 F0)^2), F_y, F_z ~ N(0, (0.2 F0)^2), F0 = 1e-6 (seed 1).
    Compensated FP32 storage: with F32 the residual stalls above 1e-8 (storage
    round-off ~1e-10 against |u| ~ 1e-2)."""
    import torch
    from paper_0809_4730_gb300.inputs import gaussian_force
    G, fluid = hartmann_duct_solver(n, Ha=10.0, gamma=0.1, storage=storage, force_field=3, nu=ADJ_NU)
    F = torch.tensor(gaussian_force(n, n, n, seed=1).reshape(3, -1), dtype=torch.float32, device="cuda")
    G.set_force(F)
    return G, F, fluid


# DRAM bytes of one plain steady-adjoint launch per fluid node: `ncu --metrics
# dram__bytes_read.sum,dram__bytes_write.sum -k regex:adjoint_kernel -s 41 -c 1` on the 128^3
# bench duct (2,032,128 fluid nodes), read + write
ADJ_TRAFFIC_B_PER_FLUID_NODE = (479625472 + 339030016) / 2032128


def adjoint_bytes_per_node(mhd: bool, storage: str = "f32c", steady: bool = True) -> int:
    """Algorithmic bytes of one adjoint step per fluid node.  Steady form:
    the linearisation rows of the fixed state (16 x 4 B with the induction
    lattice, 7 x 4 B without), cotangent gather and store 43 x 4 B each
    (19 without), gradient 3 x 4 B.  Unrolled form: the forward gather
    (19 f + 21 g) x 4 B (F32) or 6 B (F32C), lagged Lorentz force and force
    field 3 x 4 B each in place of the rows."""
    vb = 6 if storage == "f32c" else 4
    if steady:
        return (16 * 4 + 43 * 4 * 2 + 12) if mhd else (7 * 4 + 19 * 4 * 2 + 12)
    if mhd:
        return 40 * vb + 12 + 12 + 43 * 4 * 2 + 12
    return 19 * vb + 12 + 19 * 4 * 2 + 12


def run_adjoint(args, rank, ws):
    import torch
    n = args.adjoint_n
    stream = torch.cuda.current_stream()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    G, F, fluid = adjoint_duct(n)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, steps, r = G.solve(args.adjoint_fwd_tol, args.adjoint_max_steps)
    e1.record(stream)
    e1.synchronize()
    fwd_s = e0.elapsed_time(e1) / 1e3
    print(f"adjoint workload: forward status {st} at level {steps}, r = {r:.3g}, {fwd_s:.2f} s", file=sys.stderr,
          flush=True)
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        dQ, ast, it, ar = G.adjoint_steady(None, tol=args.adjoint_tol, max_iters=args.adjoint_max_steps)
        e1.record(stream)
        e1.synchronize()
    adj_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, ws)
    print(f"steady adjoint: status {ast}, {it} iterations, r = {ar:.3g}, {adj_s:.2f} s", file=sys.stderr, flush=True)
    per_it = adj_s / max(it, 1)
    bpn = adjoint_bytes_per_node(True)
    achieved = bpn * fluid / per_it / 1e9
    # unrolled transient from rest: 2000 steps, checkpoints every 100
    H, _, _ = adjoint_duct(n)
    e0.record(stream)
    dQu = H.adjoint_unrolled(args.adjoint_unrolled_steps, args.adjoint_K)
    e1.record(stream)
    e1.synchronize()
    unr_s = e0.elapsed_time(e1) / 1e3
    print(f"unrolled adjoint: {unr_s:.2f} s", file=sys.stderr, flush=True)
    # full-size property check: directional derivative along a seeded field
    # against a central difference of two steady solves
    fd = None
    if not args.no_adjoint_fd:
        # a same-sign direction (random signs would cancel below the FP32
        # resolution of Q): dF_x = 5e-8 U(0.5, 1.5) per node, 5% of F0
        gen = torch.Generator(device="cuda").manual_seed(7)
        dF = torch.zeros(3, G.N, device="cuda", dtype=torch.float32)
        dF[0] = 5e-8 * (0.5 + torch.rand(G.N, generator=gen, device="cuda"))
        qs = []
        for sgn in (1.0, -1.0):
            K2, _, _ = adjoint_duct(n)
            K2.set_force(F + sgn * dF)
            K2.solve(args.adjoint_fwd_tol, args.adjoint_max_steps)
            _, u, _ = K2.fields()      # 0 on solid nodes
            qs.append(float(u[0].double().sum() / n))
            K2.close()
        fd_val = (qs[0] - qs[1]) / 2.0
        ad_val = float((dQ.double() * dF.double()).sum())
        fd = {"directional_fd": fd_val, "directional_adjoint": ad_val, "Q": (qs[0] + qs[1]) / 2,
              "rel_diff": abs(fd_val - ad_val) / max(abs(fd_val), 1e-300),
              "direction": "dF_x = 5e-8 U(0.5,1.5) per node (seed 7), central difference of two steady solves"}
    G.close()
    H.close()
    mlups = fluid * it / adj_s / 1e6 * ws
    return {
        "metric": "steady adjoint throughput (MLUPS of transposed collide-stream steps) and time to dQ/dF",
        "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": ws, "steps": it, "warmup": 0,
        "ms_per_step": round(per_it * 1e3, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"adjoint: {n}^3 Hartmann duct Ha=10, gamma=0.1, nu=eta={ADJ_NU}, chi=0.01, "
                               "per-node Gaussian force (F0=1e-6, sigma=0.2 F0, seed 1), Q=(1/Lx) sum u_x, "
                               "F32C storage, FP32 cotangents", "inputs_vs_L2": "state > L2 (no flush)"},
        "forward": {"status": st, "level": steps, "r": r, "tol": args.adjoint_fwd_tol, "seconds": round(fwd_s, 3)},
        "steady_adjoint": {"status": ast, "iterations": it, "r": ar, "seconds": round(adj_s, 3),
                           "tol": args.adjoint_tol},
        "unrolled_adjoint": {"steps": args.adjoint_unrolled_steps, "K": args.adjoint_K, "seconds": round(unr_s, 3),
                             "max_abs_dQdF": float(dQu.abs().max())},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 3),
                     "traffic": None if ADJ_TRAFFIC_B_PER_FLUID_NODE is None
                     else round(ADJ_TRAFFIC_B_PER_FLUID_NODE * fluid),
                     "note": "per iteration of glbe_adjoint_steady (adjoint kernel + finalize every 10 + host "
                             f"polling), {bpn} B per fluid node, peak of measured; traffic: bytes of one plain launch, ncu "
                             "capture on the 128^3 duct scaled by fluid nodes"},
        "full_size_check": fd, "clocks": clk.summary(),
    }


def main():
    args = parse()
    if args.impl == "reference":
        # CPU oracle: rank 0 alone runs it; other ranks exit without work
        rank = int(os.environ.get("RANK", "0"))
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        if rank == 0:
            print(json.dumps(run_reference(args, rank, ws)), flush=True)
        return
    rank, ws = dist_init(args)
    if args.workload == "batch":
        line = run_batch(args, rank, ws)
    elif args.workload == "batch-single":
        line = batch_against_single()
    elif args.workload == "batch-small":
        line = batch_small()
    elif args.workload == "sweeps":
        line = run_sweeps(args, rank, ws)
    elif args.workload == "coupled":
        line = run_coupled(args, rank, ws)
    elif args.workload == "cavity":
        line = run_cavity(args, rank, ws)
    elif args.workload == "tts":
        line = run_tts(args, rank, ws)
    elif args.workload == "adjoint":
        line = run_adjoint(args, rank, ws)
    elif args.workload == "2d":
        line = run_2d(args, rank, ws)
    elif args.workload == "cpu-configs":
        line = {"metric": "FP64 oracle on the small configurations (CPU baseline)", "data": "synthetic",
                "cpu_baseline": cpu_configs()}
    elif ws > 1 and not args.replicas:
        line = run_sharded(args, rank, ws)
    else:
        line = run_glbe(args, rank, ws)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
