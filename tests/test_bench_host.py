"""Host-side logic of bench.py: replica aggregation over two gloo ranks on CPU,
the roofline byte model, and the reference arm's JSON contract pieces."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_WORKER = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
bench.dist_init("gloo")
units, secs = bench.aggregate(10 * (rank + 1), 1.0 + rank)
bench.barrier()
print(json.dumps({"rank": rank, "units": units, "secs": secs}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_aggregate_two_gloo_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for o in outs:
        assert o["units"] == 30.0          # 10 + 20 eigenpairs over both replicas
        assert o["secs"] == 2.0            # slowest rank


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(7, 0.5) == (7.0, 0.5)


def test_rooflines_from_the_library_byte_models():
    import bench
    stats = {"band_schwarz_f32_jacobi_L0": (8, 4.0, 8 * 2.0e7),
             "vec_stencil_f64_apply_L0": (2, 1.0, 2 * 1.0e8),
             "k_gj_pivot": (1, 0.5, 0.0)}
    r = bench.rooflines(stats, 6794.8, "measured", 1.2, 10 ** 6)
    assert [e["kernel"] for e in r] == ["band_schwarz_f32_jacobi_L0", "vec_stencil_f64_apply_L0", "k_gj_pivot"]
    assert r[0]["share"] == pytest.approx(4.0 / 5.5, abs=1e-4)
    assert r[0]["achieved"] == pytest.approx(1.6e8 / 4e-3 / 1e9, rel=1e-3)
    assert r[0]["frac"] == pytest.approx(r[0]["achieved"] / 6794.8, abs=1e-4)
    assert r[0]["bytes_per_launch"] == 2 * 10 ** 7
    # a kernel without a byte model carries no HBM roofline
    assert "frac" not in r[2]
    # the FP64 apply is also measured against the FP64 FMA rate: 22 flops per open face
    alu = r[1]["alu"]
    assert alu["achieved"] == pytest.approx(22e6 * 2 / 1e-3 / 1e12, rel=1e-3) and alu["peak"] == 1.2
    assert json.loads(json.dumps(r)) == r


def test_profiled_traffic_reaches_only_the_captured_case():
    import bench
    saved = dict(bench.PROFILED_TRAFFIC)
    try:
        bench.PROFILED_TRAFFIC.clear()
        bench.PROFILED_TRAFFIC[("band_schwarz_f32_jacobi_L0", "ellipsoid", 192, 0)] = 12345
        stats = {"band_schwarz_f32_jacobi_L0": (8, 4.0, 8 * 2.0e7)}
        hit = bench.rooflines(stats, 6794.8, "measured", None, 10, key=("ellipsoid", 192, 0))
        miss = bench.rooflines(stats, 6794.8, "measured", None, 10, key=("ellipsoid", 192, 3))
        assert hit[0]["traffic"] == 12345 and miss[0]["traffic"] is None
        # a capture that holds for every stencil shape
        bench.PROFILED_TRAFFIC.clear()
        bench.PROFILED_TRAFFIC[("band_schwarz_f32_jacobi_L0", "ellipsoid", 192, None)] = 777
        anyshape = bench.rooflines(stats, 6794.8, "measured", None, 10, key=("ellipsoid", 192, 3))
        other = bench.rooflines(stats, 6794.8, "measured", None, 10, key=("ellipsoid", 128, 3))
        assert anyshape[0]["traffic"] == 777 and other[0]["traffic"] is None
    finally:
        bench.PROFILED_TRAFFIC.clear()
        bench.PROFILED_TRAFFIC.update(saved)


def test_host_sample_is_the_same_cavity_family():
    import argparse

    import bench
    a = argparse.Namespace(workload="ellipsoid", sigma=5.0, nev=16)
    w = bench.sample_workload(a)
    assert w.grid.nx == bench.CPU_SAMPLE_GRID and w.nev == 16 and "semi_axes" in w.meta
    a.workload = "sphere"
    assert "radius" in bench.sample_workload(a).meta
