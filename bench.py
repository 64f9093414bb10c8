"""Throughput benchmark: converged Dey--Mittra eigenpairs per second on one GB300.

Headline workload (the mixed-precision configuration): a seeded PEC ellipsoid
(semi-axes U[0.6, 1.0]) on a 192^3 Yee grid with a seeded sub-cell offset, the
16 electromagnetic modes nearest sigma = 5, every returned pair certified at
rho = ||K b - k^2 A b|| / (k^2 ||A b||) <= 1e-8.  One step = geometry +
multigrid setup + Krylov--Schur eigensolve + FP64 certification.  The headline
runs the V-cycle in FP32 inside FP64 FGMRES / FP64 Krylov--Schur; the plain FP64
multigrid is timed over the same steps and warm-up in the same run, and a BF16
V-cycle beside it, with every eigenvalue's error against the FP64 result.
``--workload sphere|batch|ninecell`` runs the other configurations.

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
    ap.add_argument("--workload", default="ellipsoid", choices=["sphere", "ellipsoid", "batch", "ninecell"],
                    help="ellipsoid: seeded ellipsoid on 192^3, 16 modes, FP32 and BF16 V-cycles against the plain "
                         "FP64 multigrid (the headline); sphere: 128^3 PEC sphere, 10 modes; batch: 48 seeded "
                         "cavities of 32^3-96^3 with 1-4 shifts each, batched solve; ninecell: synthetic 9-cell "
                         "cavity on 96x96x1152, 20 modes, with and without the learned smoother")
    ap.add_argument("--grid", type=int, default=None)
    ap.add_argument("--nev", type=int, default=None)
    ap.add_argument("--sigma", type=float, default=5.0)
    ap.add_argument("--precision", default="f32", choices=["f64", "f32", "bf16"])
    ap.add_argument("--count", type=int, default=0, help="batch: solve only the first COUNT cavities")
    ap.add_argument("--streams", type=int, default=8, help="batch: worker streams of dm_eigensolve_batched")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain FP64 comparison arm")
    ap.add_argument("--bf16-steps", type=int, default=3, help="timed steps of the BF16 V-cycle arm (0: skip)")
    ap.add_argument("--inner-tol", type=float, default=1e-9, help="relative residual of each shifted solve (library default 1e-9)")
    ap.add_argument("--inner-restart", type=int, default=40, help="FGMRES restart length of the shifted solves")
    ap.add_argument("--band-sweeps", type=int, default=None,
                    help="Jacobi sweeps of the band smoother on the fine level (library default 24)")
    ap.add_argument("--band-sweeps-coarse", type=int, default=None,
                    help="sweeps of the band smoother below the fine level (library default 16)")
    ap.add_argument("--ritz-tol", type=float, default=None,
                    help="Krylov-Schur Ritz residual tolerance relative to |theta| (library default 1e-10)")
    ap.add_argument("--basis", type=int, default=None, help="Krylov-Schur basis size (library default)")
    ap.add_argument("--jacobi-sweeps", type=int, default=None,
                    help="damped Jacobi sweeps per smoothing step (library default 2)")
    ap.add_argument("--no-krylov-ff", action="store_true",
                    help="FP64 operator applies inside the shifted solves' FGMRES iterations (instead of float-float)")
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


def eig_overrides(args):
    """Eigensolver and multigrid settings given on the command line (the
    library's defaults otherwise)."""
    kw = mg_overrides(args)
    if getattr(args, "ritz_tol", None) is not None:
        kw["tol"] = args.ritz_tol
    if getattr(args, "basis", None) is not None:
        kw["basis"] = args.basis
    return kw


def mg_overrides(args):
    """Multigrid settings given on the command line (the library's defaults otherwise)."""
    kw = {}
    if args.band_sweeps is not None:
        kw["band_sweeps"] = args.band_sweeps
    if args.band_sweeps_coarse is not None:
        kw["band_sweeps_coarse"] = args.band_sweeps_coarse
    if args.jacobi_sweeps is not None:
        kw["jacobi_sweeps"] = args.jacobi_sweeps
    return kw


def config_of(args, w, extra=None):
    c = {"workload": describe(args, w),
         "grid": [args.grid] * 3, "nev": args.nev, "sigma": args.sigma, "inner_tol": args.inner_tol,
         "inner_restart": args.inner_restart, "krylov_apply": "f64" if args.no_krylov_ff else "float-float",
         "band_sweeps": [24 if args.band_sweeps is None else args.band_sweeps,
                         16 if args.band_sweeps_coarse is None else args.band_sweeps_coarse],
         "jacobi_sweeps": 2 if args.jacobi_sweeps is None else args.jacobi_sweeps,
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


# DRAM bytes (read + write) per launch from ncu captures of the same kernel:
# (trace name, workload, grid, level-0 stencil shape) -> bytes, the shape None
# for kernels that do not depend on it.  The profiles/ summaries hold the
# captures and their commands; a kernel or shape without a capture reports null.
#  - band smoother, fine level: the four size-class launches of one smoothing
#    step of the 128^3 ellipsoid read 103.5 MB and wrote 0.2 MB (25.9 MB per
#    launch); the 192^3 figure is that per-launch traffic scaled by the ratio of
#    the byte model's per-launch bytes (26.27 MB / 11.64 MB), the traffic
#    growing with the band's row copies as the byte model does.
PROFILED_TRAFFIC = {
    ("band_schwarz_f32_jacobi_L0", "ellipsoid", 128, None): 25_900_000,
    ("band_schwarz_f32_jacobi_L0", "ellipsoid", 192, None): 58_450_000,
}


def profiled_traffic(name, key):
    if not key:
        return None
    hit = PROFILED_TRAFFIC.get((name,) + tuple(key))
    return hit if hit is not None else PROFILED_TRAFFIC.get((name,) + tuple(key[:2]) + (None,))

# Algorithmic FP64 operations of one K - sigma A evaluation per open face:
# about 66 per cell of 3 faces (two curls, the grad-div and the shift).
APPLY_FLOPS_PER_FACE = 22.0


def rooflines(stats, hbm_peak, peak_kind, fp64_tflops, open_faces, top=8, key=None):
    """Per-kernel roofline of the top kernels by time in the traced step:
    achieved = the library's algorithmic bytes of the kernel's launches over
    their summed CUDA-event duration (on the library's stream).  The FP64
    operator apply is also given against the measured FP64 FMA rate."""
    total_ms = sum(v[1] for v in stats.values())
    out = []
    for name, (launches, ms, by) in sorted(stats.items(), key=lambda kv: -kv[1][1])[:top]:
        ent = {"kernel": name, "share": round(ms / total_ms, 4), "launches": launches,
               "avg_launch_us": round(ms / launches * 1e3, 2)}
        if by > 0:
            gbs = by / (ms * 1e-3) / 1e9
            ent.update({"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                        "frac": round(gbs / hbm_peak, 4), "bytes_per_launch": int(by / launches),
                        "peak_kind": f"{peak_kind} (copy)",
                        "traffic": profiled_traffic(name, key)})
        if name == "vec_stencil_f64_apply_L0" and fp64_tflops:
            tf = APPLY_FLOPS_PER_FACE * open_faces * launches / (ms * 1e-3) / 1e12
            ent["alu"] = {"bound": "alu", "achieved": round(tf, 4), "peak": round(fp64_tflops, 4),
                          "unit": "TFLOP/s", "frac": round(tf / fp64_tflops, 4),
                          "peak_kind": "measured FP64 FMA rate (dm_measure_fma_rates)"}
        out.append(ent)
    return out


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
    # the end-to-end leg's host buffers: pinned, as an application that streams
    # level sets in and eigenvectors out would hold them
    phi_pinned = torch.from_numpy(phi_host).pin_memory()
    B_pinned = torch.empty((args.nev, nf), dtype=torch.float64).pin_memory()

    sweep_kw = eig_overrides(args)

    def step(precision, host_io=False):
        phi = phi_pinned if host_io else phi_dev
        geom = dm.Geometry(ctx, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, phi, g.origin)
        vec = "host" if host_io else "device"
        k2, B, rep, st = dm.eigensolve(ctx, geom, args.sigma, args.nev, vectors=vec,
                                       out=B_pinned if host_io else B_dev, precision=precision,
                                       inner_tol=args.inner_tol, inner_restart=args.inner_restart,
                                       krylov_ff=0 if (args.no_krylov_ff or precision == "f64") else 1,
                                       **sweep_kw)
        geom.close()
        return k2, rep, st

    def converged(rep, st):
        return rep["n_converged"] if (st == 0 and rep["rho_max"] <= RHO_TOL) else 0

    def timed(precision, steps, warmup, label):
        """warmup untimed steps, then `steps` steps between CUDA events on the
        library's stream (barrier + synchronize on both sides)."""
        for i in range(warmup):
            t = time.perf_counter()
            step(precision)
            progress(f"{label} warm-up {i + 1}/{warmup}: {time.perf_counter() - t:.2f} s")
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = ctx.launches
        e0.record(stream)
        units, reps, per = 0, [], []
        for _ in range(steps):
            t = time.perf_counter()
            k2, rep, st = step(precision)
            units += converged(rep, st)
            reps.append(rep)
            per.append(time.perf_counter() - t)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        secs = e0.elapsed_time(e1) * 1e-3
        progress(f"{label}: {steps} steps in {secs:.2f} s, {units} pairs converged")
        return {"units": units, "secs": secs, "reps": reps, "k2": k2, "launches": ctx.launches - l0,
                "per_step_s": per}

    # ---- timed region of the headline: inputs resident in HBM ----
    clocks = ClockSampler(local)
    for i in range(args.warmup):
        t = time.perf_counter()
        step(args.precision)
        progress(f"warm-up {i + 1}/{args.warmup}: {time.perf_counter() - t:.2f} s")
    clocks.start()
    nvtx_mark(True)      # an NVTX range "timed", for profilers that filter on it
    main = timed(args.precision, args.steps, 0, f"mixed ({args.precision} V-cycle)")
    nvtx_mark(False)
    clk = clocks.stop()
    tot_units, max_s = aggregate(main["units"], main["secs"], device=f"cuda:{local}")
    value = tot_units / max_s
    reps = main["reps"]
    k2 = main["k2"]
    # ---- end-to-end through the public API with host buffers ----
    t0 = time.perf_counter()
    units_e2e = 0
    for _ in range(args.steps):
        k2h, reph, sth = step(args.precision, host_io=True)
        units_e2e += converged(reph, sth)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    tot_e2e, max_e2e = aggregate(units_e2e, e2e_s, device=f"cuda:{local}")
    progress(f"e2e: {args.steps} steps in {e2e_s:.2f} s")
    # ---- one traced step: per-kernel event timings and algorithmic bytes ----
    ctx.trace(True)
    step(args.precision)
    ctx.trace(False)
    stats = ctx.trace_stats(with_bytes=True)
    hbm, kind = peaks()
    fp64_tf, fp32_tf = ctx.fma_rates()
    g0info = dm.Geometry(ctx, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, phi_dev, g.origin)
    open_faces = g0info.level_info(0)["open"]
    # tile shapes the autotuner chose for this cavity's levels (cached in the context, so no re-timing)
    op_info = dm.Operator(ctx, g0info, args.sigma, precision=args.precision)
    shapes = [op_info.stencil_shape(l) for l in range(op_info.num_levels - 1)]
    op_info.close()
    g0info.close()
    roofs = rooflines(stats, hbm, kind, fp64_tf, open_faces, key=(args.workload, args.grid, shapes[0] if shapes else -1))
    # ---- plain FP64 multigrid on the same cavity, same steps and warm-up ----
    plain, errs = None, {}
    if not args.no_compare and args.precision != "f64":
        p64 = timed("f64", args.steps, args.warmup, "plain FP64 multigrid")
        k2p = p64["k2"]
        plain = {"value": round(p64["units"] / p64["secs"], 4), "unit": UNIT,
                 "ms_per_step": round(p64["secs"] / args.steps * 1e3, 1), "steps": args.steps,
                 "warmup": args.warmup, "per_step_s": [round(v, 3) for v in p64["per_step_s"]],
                 "inner_iters": p64["reps"][-1]["inner_iters"], "outer_iters": p64["reps"][-1]["outer_iters"],
                 "rho_max": p64["reps"][-1]["rho_max"]}
        errs[args.precision] = [float(v) for v in np.abs(k2 - k2p) / np.abs(k2p)]
        # the BF16 V-cycle beside it (a shorter run: its errors and its rate)
        if args.precision != "bf16" and args.bf16_steps > 0:
            b16 = timed("bf16", args.bf16_steps, 1, "bf16 V-cycle")
            errs["bf16"] = [float(v) for v in np.abs(b16["k2"] - k2p) / np.abs(k2p)]
            plain["bf16"] = {"value": round(b16["units"] / b16["secs"], 4), "unit": UNIT,
                             "ms_per_step": round(b16["secs"] / args.bf16_steps * 1e3, 1),
                             "steps": args.bf16_steps, "warmup": 1,
                             "inner_iters": b16["reps"][-1]["inner_iters"],
                             "rho_max": b16["reps"][-1]["rho_max"]}
    dominant = next((r for r in roofs if r.get("bound") == "hbm"), None)
    roof = None
    if dominant:
        roof = {k: dominant[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic",
                                         "bytes_per_launch", "avg_launch_us", "launches", "share", "peak_kind")}
        roof["unit_of_work"] = "the library's per-kernel byte model (open faces, band rows, compact vectors)"
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(max_s / args.steps * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32" if args.precision == "f32" else
        ("f64+bf16" if args.precision == "bf16" else "f64"), "data": "synthetic (seeded level set)",
        "config": config_of(args, w, {"parallelism": f"replicas x{world}"}),
        "e2e": {"value": round(tot_e2e / max_e2e, 4), "unit": UNIT,
                "h2d_bytes_per_step": int(phi_host.nbytes), "d2h_bytes_per_step": int(args.nev * nf * 8)},
        "gpu_launches": int(main["launches"]),
        "roofline": roof,
        "rooflines_top": roofs,
        "peaks_measured": {"fp64_tflops": round(fp64_tf, 4), "fp32_tflops": round(fp32_tf, 2),
                           "how": "dm_measure_fma_rates: FMA-chain loop, CUDA events, this run"},
        "clocks": clk,
        "solver": {"inner_iters_per_step": reps[-1]["inner_iters"], "outer_iters": reps[-1]["outer_iters"],
                   "restarts": reps[-1]["restarts"], "proj_iters": reps[-1]["proj_iters"],
                   "mg_levels": reps[-1]["mg_levels"], "mg_complexity": round(reps[-1]["mg_complexity"], 3),
                   "rho_max": reps[-1]["rho_max"], "delta_max": reps[-1]["delta_max"],
                   "k2": [round(float(v), 10) for v in k2],
                   "inner_rate": None, "stencil_shapes": shapes, "open_faces": int(open_faces),
                   "per_step_s": [round(v, 3) for v in main["per_step_s"]],
                   "setup_s": round(reps[-1].get("setup_seconds", 0.0), 3),
                   "solve_s": round(reps[-1].get("solve_seconds", 0.0), 3),
                   # one shifted FGMRES solve (K - sigma A) x = A v per Krylov-Schur step
                   "solves_per_s": round(sum(r["outer_iters"] for r in reps) * world / max_s, 3)},
        "plain_f64": plain,
        "rel_k2_error_vs_f64": errs,
        "kernels_top": {k: {"launches": c, "ms": round(ms, 3), "bytes": int(by)} for k, (c, ms, by) in
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
                jobs.append({"geom": geom, "sigma": sg, "nev": nev, "precision": args.precision,
                             "inner_tol": args.inner_tol, **eig_overrides(args)})
        out = dm.eigensolve_batched(ctx, jobs, streams=args.streams)
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
                   "mg_precision": args.precision, "outer_precision": "f64", "streams": args.streams,
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
    op = dm.Operator(ctx, geom, w.sigma, precision=args.precision, **mg_overrides(args))
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
                                       inner_tol=args.inner_tol, **eig_overrides(args),
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


def sample_workload(args):
    """The bounded host sample of the workload: the same cavity family (same
    seeds, shape recipe, sigma and mode count) at CPU_SAMPLE_GRID^3 cells."""
    import workloads as W
    if args.workload == "ellipsoid":
        return W.ellipsoid_workload(CPU_SAMPLE_GRID, seed=W.SEED_BASE + 3, sigma=args.sigma, nev=args.nev)
    return W.sphere_workload(CPU_SAMPLE_GRID, radius=1.0, half_width=1.1, sigma=args.sigma, nev=args.nev,
                             offset_seed=W.SEED_BASE + 2)


def oracle_step(args):
    """One bounded sample of the workload on the host: the oracle's sparse
    shift-invert eigensolve of the sample cavity, every pair certified."""
    from oracle import eigen, geometry, operators
    w = sample_workload(args)
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
            "sample": (f"oracle (scipy SuperLU + ARPACK shift-invert, single-threaded) on the same {args.workload} "
                       f"family at {CPU_SAMPLE_GRID}^3 cells, {args.nev} modes, sigma={args.sigma}; {reps} solve(s), "
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
                            "sample": (f"each step: the oracle's sparse shift-invert eigensolve of the same "
                                       f"{args.workload} family at {CPU_SAMPLE_GRID}^3 cells ({args.nev} modes); "
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
