"""Throughput benchmark: converged Dey--Mittra eigenpairs per second on one GB300.

Workload (the paper's spherical-cavity test, Sec. 6.2, at the larger grid of the
plain-method configuration): a PEC sphere of radius 1 in [-1.1, 1.1]^3 on a
128^3 Yee grid, centre moved by a seeded sub-cell offset, the 10 electromagnetic
modes nearest sigma = 5 (the 10 lowest), residual <= 1e-8.  One step = geometry
+ multigrid setup + Krylov--Schur eigensolve + FP64 certification of every
returned eigenpair.  The headline uses the mixed-precision form (FP32 V-cycle
inside FP64 FGMRES / FP64 Krylov--Schur); the plain FP64 multigrid is timed in
the same run for comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas (one
per rank, no data-path collective), so scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "eigenpairs/s @1e-8 residual vs plain FP64 MG; V-cycle HBM GB/s % of peak"
UNIT = "eigenpairs/s"
RHO_TOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="sphere", choices=["sphere", "ellipsoid", "batch", "ninecell"],
                    help="sphere: 128^3 PEC sphere, 10 modes (the headline); ellipsoid: seeded ellipsoid on 192^3, "
                         "16 modes; batch: 48 seeded cavities of 32^3-96^3 with 1-4 shifts each, batched solve; "
                         "ninecell: synthetic 9-cell cavity on 96x96x1152, 20 modes, with and without the learned "
                         "smoother")
    ap.add_argument("--grid", type=int, default=None)
    ap.add_argument("--nev", type=int, default=None)
    ap.add_argument("--sigma", type=float, default=5.0)
    ap.add_argument("--precision", default="f32", choices=["f64", "f32", "bf16"])
    ap.add_argument("--count", type=int, default=0, help="batch: solve only the first COUNT cavities")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain FP64 comparison step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    a = ap.parse_args()
    if a.grid is None:
        a.grid = {"sphere": 128, "ellipsoid": 192, "batch": 0, "ninecell": 96}[a.workload]
    if a.nev is None:
        a.nev = {"sphere": 10, "ellipsoid": 16, "batch": 0, "ninecell": 20}[a.workload]
    return a


def workload(args):
    import workloads as W
    if args.workload == "ellipsoid":
        return W.ellipsoid_workload(args.grid, seed=W.SEED_BASE + 3, sigma=args.sigma, nev=args.nev)
    return W.sphere_workload(args.grid, radius=1.0, half_width=1.1, sigma=args.sigma, nev=args.nev,
                             offset_seed=W.SEED_BASE + 2)


def describe(args, w):
    if args.workload == "ellipsoid":
        ax = tuple(round(float(v), 4) for v in w.meta.get("semi_axes", ()))
        return (f"PEC ellipsoid, seeded semi-axes {ax}, {args.grid}^3 Yee cells, sigma={args.sigma}, "
                f"{args.nev} modes nearest sigma, residual<={RHO_TOL}")
    return (f"PEC sphere R=1 in [-1.1,1.1]^3, {args.grid}^3 Yee cells, seeded centre offset "
            f"{tuple(round(float(v), 5) for v in w.meta['center'])}, sigma={args.sigma}, "
            f"{args.nev} lowest modes, residual<={RHO_TOL}")


def config_of(args, w, extra=None):
    c = {"workload": describe(args, w),
         "grid": [args.grid] * 3, "nev": args.nev, "sigma": args.sigma,
         "mg_precision": args.precision, "outer_precision": "f64",
         "l2": "inputs larger than L2 (solver working set of several GB per step)"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# distributed helpers (replicas; host-side logic shared with the CPU tests)
# ---------------------------------------------------------------------------

def progress(msg):
    """One line of progress on stderr (the JSON result stays alone on stdout)."""
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(backend):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return dist


def aggregate(local_units, local_seconds, device=None):
    """(units summed over ranks, max seconds over ranks) -- the whole-job
    throughput is units / max seconds."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_units), float(local_seconds)
    t = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    s = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(t.item()), float(s.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(p[1]) for p in self.samples if p[1].replace(".", "").isdigit()]
        mx = [float(p[2]) for p in self.samples if p[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for p in self.samples:
            for n, v in zip(names, p[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# roofline of the dominant kernel
# ---------------------------------------------------------------------------

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def nvtx_mark(start):
    """Open (start) or close the NVTX range "timed" around the timed steps; a
    no-op where NVTX is unavailable."""
    try:
        import torch
        if start:
            torch.cuda.nvtx.range_push("timed")
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def stencil_bytes_per_cell(name):
    """Bytes per grid cell of one vector-stencil launch that streams every cell
    once: x (3 values) read, y (3) written, f (3) read for resid and jacobi;
    coefficients A (3), L (3), 1/V (1) and 1/D (3, jacobi only)."""
    parts = name.split("_")
    prec, mode = parts[2], parts[3]
    tv = {"f64": 8, "f32": 4, "bf16": 2}[prec]
    tc = 8 if prec == "f64" else 4
    vec = 3 * tv * (2 + (1 if mode in ("resid", "jacobi") else 0))
    coef = tc * (7 + (3 if mode == "jacobi" else 0))
    return vec + coef


def stencil_bytes_per_open_face(name):
    """Algorithmic bytes per OPEN face of one vector-stencil launch (conductor
    regions excluded): the face's x, y and (resid / jacobi) f, its A and 1/D
    (jacobi), about one edge fraction L and a third of a 1/V per face."""
    parts = name.split("_")
    prec, mode = parts[2], parts[3]
    tv = {"f64": 8, "f32": 4, "bf16": 2}[prec]
    tc = 8 if prec == "f64" else 4
    vec = tv * (2 + (1 if mode in ("resid", "jacobi") else 0))
    coef = tc * (2 + (1 if mode == "jacobi" else 0)) + tc / 3.0
    return vec + coef


# Algorithmic FP64 operations of one K - sigma A evaluation per open face:
# about 66 per cell of 3 faces (two curls, the grad-div and the shift).
APPLY_FLOPS_PER_FACE = 22.0
FP64_PEAK_TFLOPS = 1.204      # FP64 FMA-loop probe on a GB300 (measured rate, TFLOP/s)


# DRAM bytes (read + write) per launch of the fine-level stencil, from an ncu
# capture of that kernel on the same cavity: (trace name, level-0 tile shape,
# workload, grid) -> bytes.  profiles/stencil_jacobi_sphere128.md has the
# capture and its command; a shape without a capture reports null.
PROFILED_TRAFFIC = {
    ("vec_stencil_f32_jacobi_L0", 0, "sphere", 128): 90_759_424 + 5_890_304,
}


def roofline(stats, open_faces, hbm_peak, peak_kind, precision="f32", traffic=None):
    """Fine-level V-cycle smoothing stencil (the metric's V-cycle kernel):
    algorithmic bytes per launch (open faces only) over its event-timed mean
    duration."""
    name = f"vec_stencil_{precision}_jacobi_L0"
    if name not in stats:
        cands = {k: v for k, v in stats.items() if k.startswith("vec_stencil") and k.endswith("_L0")}
        if not cands:
            return None
        name = max(cands.items(), key=lambda kv: kv[1][1])[0]
    launches, ms = stats[name]
    avg_s = ms / launches * 1e-3
    bytes_per_launch = stencil_bytes_per_open_face(name) * open_faces
    achieved = bytes_per_launch / avg_s / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4), "traffic": traffic,
            "bytes_per_launch": int(bytes_per_launch), "avg_launch_us": round(avg_s * 1e6, 2), "launches": launches,
            "peak_kind": f"{peak_kind} (copy)", "unit_of_work": "open face"}


def roofline_fp64_apply(stats, open_faces):
    """The FP64 outer K - sigma A apply: bounded by GB300's FP64 pipes."""
    name = "vec_stencil_f64_apply_L0"
    if name not in stats:
        return None
    launches, ms = stats[name]
    avg_s = ms / launches * 1e-3
    tf = APPLY_FLOPS_PER_FACE * open_faces / avg_s / 1e12
    return {"kernel": name, "bound": "alu", "achieved": round(tf, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": round(tf / FP64_PEAK_TFLOPS, 4), "avg_launch_us": round(avg_s * 1e6, 2), "launches": launches,
            "peak_kind": "measured FP64 FMA probe"}


# ---------------------------------------------------------------------------
# native (GPU) arm
# ---------------------------------------------------------------------------

def run_native(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_3794_gb300 as dm

    w = workload(args)
    g = w.grid
    stream = torch.cuda.Stream()
    ctx = dm.Context(local, stream=stream.cuda_stream)
    phi_host = np.ascontiguousarray(w.phi.ravel())
    with torch.cuda.stream(stream):
        phi_dev = torch.from_numpy(phi_host).to(f"cuda:{local}")
    torch.cuda.synchronize()
    nf = dm.face_count(g.nx, g.ny, g.nz)
    B_dev = torch.empty((args.nev, nf), dtype=torch.float64, device=f"cuda:{local}")

    def step(precision, host_io=False):
        phi = phi_host if host_io else phi_dev
        geom = dm.Geometry(ctx, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, phi, g.origin)
        vec = "host" if host_io else "device"
        k2, B, rep, st = dm.eigensolve(ctx, geom, args.sigma, args.nev, vectors=vec,
                                       out=None if host_io else B_dev, precision=precision)
        geom.close()
        return k2, rep, st

    def converged(rep, st):
        return rep["n_converged"] if (st == 0 and rep["rho_max"] <= RHO_TOL) else 0

    for _ in range(args.warmup):
        step(args.precision)
    # ---- timed region: inputs resident in HBM ----
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = ctx.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    units = 0
    reps = []
    nvtx_mark(True)      # an NVTX range "timed", for profilers that filter on it
    for _ in range(args.steps):
        k2, rep, st = step(args.precision)
        units += converged(rep, st)
        reps.append(rep)
    nvtx_mark(False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = ctx.launches - l0
    local_s = e0.elapsed_time(e1) * 1e-3
    tot_units, max_s = aggregate(units, local_s, device=f"cuda:{local}")
    value = tot_units / max_s
    # ---- end-to-end through the public API with host buffers ----
    t0 = time.perf_counter()
    units_e2e = 0
    for _ in range(args.steps):
        k2h, reph, sth = step(args.precision, host_io=True)
        units_e2e += converged(reph, sth)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    tot_e2e, max_e2e = aggregate(units_e2e, e2e_s, device=f"cuda:{local}")
    # ---- one traced step: per-kernel event timings on the launching stream ----
    ctx.trace(True)
    k2t, rept, stt = step(args.precision)
    ctx.trace(False)
    stats = ctx.trace_stats()
    hbm, kind = peaks()
    open_faces = geom_open = None
    g0info = dm.Geometry(ctx, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, phi_dev, g.origin)
    open_faces = g0info.level_info(0)["open"]
    # tile shapes the autotuner chose for this cavity's levels (cached in the context, so no re-timing)
    op_info = dm.Operator(ctx, g0info, args.sigma, precision=args.precision)
    shapes = [op_info.stencil_shape(l) for l in range(op_info.num_levels - 1)]
    op_info.close()
    g0info.close()
    traffic = PROFILED_TRAFFIC.get((f"vec_stencil_{args.precision}_jacobi_L0", shapes[0] if shapes else -1,
                                    args.workload, args.grid))
    roof = roofline(stats, open_faces, hbm, kind, args.precision, traffic=traffic)
    roof64 = roofline_fp64_apply(stats, open_faces)
    # ---- plain FP64 multigrid on the same cavity ----
    plain = None
    if not args.no_compare and args.precision != "f64":
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        k2p, repp, stp = step("f64")
        p1.record(stream)
        torch.cuda.synchronize()
        ps = p0.elapsed_time(p1) * 1e-3
        plain = {"value": round(converged(repp, stp) / ps, 4), "unit": UNIT, "ms_per_step": round(ps * 1e3, 1),
                 "steps": 1, "inner_iters": repp["inner_iters"], "outer_iters": repp["outer_iters"],
                 "rho_max": repp["rho_max"],
                 "max_rel_k2_diff_vs_mixed": float(np.max(np.abs(k2p - k2) / np.abs(k2p)))}
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(max_s / args.steps * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32" if args.precision == "f32" else
        ("f64+bf16" if args.precision == "bf16" else "f64"), "data": "synthetic (seeded level set)",
        "config": config_of(args, w, {"parallelism": f"replicas x{world}"}),
        "e2e": {"value": round(tot_e2e / max_e2e, 4), "unit": UNIT,
                "h2d_bytes_per_step": int(phi_host.nbytes), "d2h_bytes_per_step": int(args.nev * nf * 8)},
        "gpu_launches": int(launches),
        "roofline": roof,
        "roofline_fp64_apply": roof64,
        "clocks": clk,
        "solver": {"inner_iters_per_step": reps[-1]["inner_iters"], "outer_iters": reps[-1]["outer_iters"],
                   "restarts": reps[-1]["restarts"], "proj_iters": reps[-1]["proj_iters"],
                   "mg_levels": reps[-1]["mg_levels"], "mg_complexity": round(reps[-1]["mg_complexity"], 3),
                   "rho_max": reps[-1]["rho_max"], "delta_max": reps[-1]["delta_max"],
                   "k2": [round(float(v), 10) for v in k2],
                   "inner_rate": None, "stencil_shapes": shapes,
                   # one shifted FGMRES solve (K - sigma A) x = A v per Krylov-Schur step
                   "solves_per_s": round(sum(r["outer_iters"] for r in reps) * world / max_s, 3)},
        "plain_f64": plain,
        "kernels_top": {k: {"launches": c, "ms": round(ms, 3)} for k, (c, ms) in
                        sorted(stats.items(), key=lambda kv: -kv[1][1])[:16]},
    }
    if reps[-1]["inner_iters"] and reps[-1]["outer_iters"]:
        it = reps[-1]["inner_iters"] / reps[-1]["outer_iters"]
        out["solver"]["inner_rate"] = round(1e-10 ** (1.0 / it), 3)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_batch(args):
    """The batched form: 48 seeded cavities (spheres and ellipsoids, 32^3 to
    96^3) with 1-4 shifts each, all (cavity, shift) eigensolves in one call of
    dm_eigensolve_batched over worker streams.  One step = geometry setup of
    every cavity + the batched solve; value = converged eigenpairs / s."""
    import numpy as np
    import torch
    import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_3794_gb300 as dm

    items = W.batch_workloads(48)[:args.count] if args.count else W.batch_workloads(48)
    stream = torch.cuda.Stream()
    ctx = dm.Context(local, stream=stream.cuda_stream)
    phis_host = [np.ascontiguousarray(w.phi.ravel()) for w, _, _ in items]
    with torch.cuda.stream(stream):
        phis_dev = [torch.from_numpy(p).to(f"cuda:{local}") for p in phis_host]
    torch.cuda.synchronize()
    npairs = sum(len(sh) * nev for _, sh, nev in items)

    def step(host_io=False):
        geoms = []
        jobs = []
        for (w, shifts, nev), ph, pd in zip(items, phis_host, phis_dev):
            g = w.grid
            geom = dm.Geometry(ctx, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, ph if host_io else pd, g.origin)
            geoms.append(geom)
            for sg in shifts:
                jobs.append({"geom": geom, "sigma": sg, "nev": nev, "precision": args.precision})
        out = dm.eigensolve_batched(ctx, jobs, streams=8)
        for geom in geoms:
            geom.close()
        return sum(rep["n_converged"] if (st == 0 and rep["rho_max"] <= RHO_TOL) else 0 for _, rep, st in out), out

    for _ in range(args.warmup):
        tw = time.perf_counter()
        _, out_w = step()
        progress(f"batch warm-up step {time.perf_counter() - tw:.1f} s")
        for (w, _, _), (_, rep, st) in zip([(w, sg, nv) for w, sh, nv in items for sg in sh], out_w):
            progress(f"  {w.name}: status {st}, {rep['n_converged']} converged, setup {rep['setup_seconds']:.2f} s, "
                     f"solve {rep['solve_seconds']:.2f} s, {rep['outer_iters']} outer / {rep['inner_iters']} inner / "
                     f"{rep['proj_iters']} projection iterations")
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = ctx.launches
    t0 = time.perf_counter()
    nvtx_mark(True)
    units = 0
    for _ in range(args.steps):
        u, out = step()
        units += u
    nvtx_mark(False)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    barrier()
    clk = clocks.stop()
    launches = ctx.launches - l0
    tot_units, max_s = aggregate(units, secs, device=f"cuda:{local}")
    t1 = time.perf_counter()
    units_e2e = 0
    for _ in range(args.steps):
        units_e2e += step(host_io=True)[0]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t1
    tot_e2e, max_e2e = aggregate(units_e2e, e2e_s, device=f"cuda:{local}")
    sizes = sorted({w.grid.nx for w, _, _ in items})
    res = {
        "metric": METRIC, "value": round(tot_units / max_s, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(max_s / args.steps * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+" + args.precision, "data": "synthetic (seeded level sets)",
        "config": {"workload": (f"batch of {len(items)} seeded cavities (spheres and ellipsoids, grids {sizes}), "
                                f"{sum(len(sh) for _, sh, _ in items)} (cavity, shift) solves, {npairs} eigenpairs "
                                f"requested per step, residual<={RHO_TOL}"),
                   "mg_precision": args.precision, "outer_precision": "f64", "streams": 8,
                   "l2": "inputs larger than L2 (48 cavities' solver state)", "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(tot_e2e / max_e2e, 4), "unit": UNIT,
                "h2d_bytes_per_step": int(sum(p.nbytes for p in phis_host)),
                "d2h_bytes_per_step": int(8 * npairs)},
        "gpu_launches": int(launches),
        "roofline": None,
        "clocks": clk,
        "solver": {"converged_per_step": units / max(args.steps, 1), "requested_per_step": npairs,
                   "solves_per_s": round(sum(len(sh) for _, sh, _ in items) * args.steps / max_s, 3)},
    }
    if rank == 0:
        print(json.dumps(res), flush=True)


def run_ninecell(args):
    """The learned-smoother configuration: the synthetic 9-cell cavity on a
    96 x 96 x 1152 grid (``--grid`` scales it), the 20 lowest modes (the
    accelerating passband and the next one) from a shift of the order of the
    smallest nonzero eigenvalue, FP32 V-cycle.  The network is trained on the GPU first (timed
    separately); each step then solves with the learned correction, and one
    step without it is timed for comparison."""
    import numpy as np
    import torch
    import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist_init("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1301_3794_gb300 as dm

    w = W.nine_cell_workload(nxy=args.grid, nz=12 * args.grid, nev=args.nev)
    g = w.grid
    stream = torch.cuda.Stream()
    ctx = dm.Context(local, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        phi_dev = torch.from_numpy(np.ascontiguousarray(w.phi.ravel())).to(f"cuda:{local}")
    torch.cuda.synchronize()
    geom = dm.Geometry(ctx, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, phi_dev, g.origin)
    op = dm.Operator(ctx, geom, w.sigma, precision=args.precision)
    net = dm.Learned(ctx, seed=11)
    t0 = time.perf_counter()
    hist = net.train(op, runs=2, epochs=6, lr=2e-3, seed=7)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    progress(f"ninecell training {train_s:.1f} s, loss {hist[0]:.4g} -> {hist[-1]:.4g}")

    def solve(learned):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        k2, _, rep, st = dm.eigensolve(ctx, geom, w.sigma, args.nev, vectors=None, precision=args.precision,
                                       learned=net if learned else None)
        ev1.record(stream)
        torch.cuda.synchronize()
        secs = ev0.elapsed_time(ev1) * 1e-3
        ok = rep["n_converged"] if (st == 0 and rep["rho_max"] <= RHO_TOL) else 0
        progress(f"ninecell solve (learned={learned}) {secs:.1f} s, status {st}, {ok} converged, "
                 f"{rep['outer_iters']} outer / {rep['inner_iters']} inner iterations")
        return ok, secs, rep, k2

    for _ in range(args.warmup):
        solve(True)
    clocks = ClockSampler(local)
    clocks.start()
    units, secs, reps = 0, 0.0, []
    nvtx_mark(True)
    for _ in range(args.steps):
        u, sec, rep, k2 = solve(True)
        units += u
        secs += sec
        reps.append(rep)
    nvtx_mark(False)
    clk = clocks.stop()
    up, sp, repp, k2p = solve(False)
    res = {
        "metric": METRIC, "value": round(units / secs, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+" + args.precision, "data": "synthetic (seeded level set)",
        "config": {"workload": (f"synthetic 9-cell elliptical cavity (cell 115.4 mm, equator 103.3 mm, iris 35 mm, "
                                f"beam pipes 2 cells), {g.nx}x{g.ny}x{g.nz} Yee cells, sigma={w.sigma:.1f} m^-2, "
                                f"{args.nev} modes nearest sigma, learned smoother in the preconditioner, "
                                f"residual<={RHO_TOL}"),
                   "mg_precision": args.precision, "outer_precision": "f64"},
        "gpu_launches": None, "roofline": None, "clocks": clk,
        "learned": {"train_seconds": round(train_s, 2), "loss_first_epoch": float(hist[0]),
                    "loss_last_epoch": float(hist[-1]),
                    "inner_iters_with": reps[-1]["inner_iters"], "inner_iters_without": repp["inner_iters"],
                    "learned_applied": reps[-1]["learned_applied"], "learned_fallbacks": reps[-1]["learned_fallbacks"],
                    "eigenpairs_per_s_without": round(up / sp, 4),
                    "max_rel_k2_diff": float(np.max(np.abs(np.asarray(k2) - np.asarray(k2p)) / np.abs(k2p)))},
        "solver": {"outer_iters": reps[-1]["outer_iters"], "proj_iters": reps[-1]["proj_iters"],
                   "rho_max": reps[-1]["rho_max"], "k2": [round(float(v), 6) for v in k2]},
    }
    if rank == 0:
        print(json.dumps(res), flush=True)


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

CPU_SAMPLE_GRID = 24


def oracle_step(args):
    """One bounded sample of the workload on the host: the oracle's sparse
    shift-invert eigensolve of the same cavity family (same radius, domain,
    offset seed, sigma and mode count) at 32^3 cells."""
    import workloads as W
    from oracle import eigen, geometry, operators
    w = W.sphere_workload(CPU_SAMPLE_GRID, radius=1.0, half_width=1.1, sigma=args.sigma, nev=args.nev,
                          offset_seed=W.SEED_BASE + 2)
    t0 = time.perf_counter()
    ops = operators.DMOperators(w.grid, geometry.fractions(w.phi))
    k2, B, _ = eigen.shift_invert_modes(ops, w.sigma, w.nev)
    ok = sum(1 for i in range(w.nev) if eigen.certificate(ops, k2[i], B[:, i])["rho"] <= RHO_TOL)
    return ok, time.perf_counter() - t0


def cpu_info():
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count()
    return cores


def cpu_baseline(args, reps=1):
    units = 0
    secs = 0.0
    for _ in range(reps):
        u, s = oracle_step(args)
        units += u
        secs += s
    return {"value": round(units / secs, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"oracle (scipy SuperLU + ARPACK shift-invert, single-threaded) on the same sphere family at "
                       f"{CPU_SAMPLE_GRID}^3 cells, {args.nev} modes, sigma={args.sigma}; {reps} solve(s), "
                       f"{secs:.1f} s; host has {cpu_info()} cores available")}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads as W
    for _ in range(args.warmup):
        oracle_step(args)
    units = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, _ = oracle_step(args)
        units += u
    secs = time.perf_counter() - t0
    value = units / secs
    w = workload(args)
    out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "impl": "reference", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded level set)",
           "config": config_of(args, w, {"parallelism": "host oracle", "sample_grid": [CPU_SAMPLE_GRID] * 3}),
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": (f"each step: the oracle's sparse shift-invert eigensolve of the same sphere "
                                       f"family at {CPU_SAMPLE_GRID}^3 cells ({args.nev} modes); "
                                       f"{cpu_info()} host cores available, SuperLU/ARPACK single-threaded")},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "ninecell":
        run_ninecell(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
