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


def test_stencil_byte_model():
    import bench
    # FP64 apply: x, y (3 x 8 B each) + A, L, 1/V (7 x 8 B) = 104 B per cell
    assert bench.stencil_bytes_per_cell("vec_stencil_f64_apply_L0") == 104
    # FP32 Jacobi: x, f, y (3 x 4 B each) + A, L, 1/V, 1/D (10 x 4 B)
    assert bench.stencil_bytes_per_cell("vec_stencil_f32_jacobi_L0") == 36 + 40
    # per open face, FP32 Jacobi: x, f, y (4 B each) + A, 1/D (4 B each) + L (4 B) + 1/V / 3
    assert bench.stencil_bytes_per_open_face("vec_stencil_f32_jacobi_L0") == pytest.approx(12 + 12 + 4 / 3)
    r = bench.roofline({"vec_stencil_f32_jacobi_L0": (10, 1.0), "k_mdot_partial": (5, 100.0)}, 10 ** 6, 6758.5,
                       "measured", "f32")
    assert r["kernel"] == "vec_stencil_f32_jacobi_L0"
    assert r["achieved"] == pytest.approx((24 + 4 / 3) * 10 ** 6 / 1e-4 / 1e9, rel=1e-3)
    assert 0 < r["frac"] < 1
    f = bench.roofline_fp64_apply({"vec_stencil_f64_apply_L0": (4, 2.0)}, 10 ** 6)
    assert f["bound"] == "alu" and f["achieved"] == pytest.approx(22e6 / 5e-4 / 1e12)


def test_profiled_traffic_only_for_the_captured_shape():
    import bench
    key = ("vec_stencil_f32_jacobi_L0", 0, "sphere", 128)
    assert bench.PROFILED_TRAFFIC[key] == 90_759_424 + 5_890_304
    # another tile shape on level 0, or another cavity, has no capture: traffic stays null
    assert bench.PROFILED_TRAFFIC.get(("vec_stencil_f32_jacobi_L0", 3, "sphere", 128)) is None
    r = bench.roofline({"vec_stencil_f32_jacobi_L0": (10, 1.0)}, 10 ** 6, 6758.5, "measured", "f32",
                       traffic=bench.PROFILED_TRAFFIC[key])
    assert r["traffic"] == bench.PROFILED_TRAFFIC[key]
    assert json.loads(json.dumps(r)) == r
