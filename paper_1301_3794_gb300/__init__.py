"""GB300 Dey--Mittra cavity eigensolver (Bauer, Werner & Cary, arXiv:1301.3794).

Python binding of the C ABI in ``include/dmeig.h``: it only marshals arguments.
Every step of the solve runs in the CUDA kernels of ``libdmeig.so``; importing
this package fails loudly if that library has not been built.

Arrays may be numpy arrays (host) or torch tensors; CUDA tensors are passed to
the library as device pointers, so PyTorch serves as the device allocator.
Face vectors use the natural layout of the header: x-faces [nz][ny][nx+1],
y-faces [nz][ny+1][nx], z-faces [nz+1][ny][nx], concatenated and flattened.
"""
from __future__ import annotations

import ctypes as C
import weakref

import numpy as np

from . import _lib
from ._lib import EigParams, EigReport, MGParams, PREC, STATUS

__all__ = ["Context", "Geometry", "Operator", "Learned", "eigensolve", "eigensolve_batched", "certify", "DMError",
           "lib",
           "face_count",
           "edge_count", "cell_count"]

lib = _lib.load()


class DMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def face_count(nx, ny, nz):
    return (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1)


def edge_count(nx, ny, nz):
    return nx * (ny + 1) * (nz + 1) + (nx + 1) * ny * (nz + 1) + (nx + 1) * (ny + 1) * nz


def cell_count(nx, ny, nz):
    return nx * ny * nz


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _torch():
    import torch
    return torch


class _Arg:
    """Pointer to an input array plus whether it lives on the device."""

    def __init__(self, a, count=None):
        if _is_torch(a):
            if a.is_cuda:
                import torch
                self.keep = a.contiguous().to(torch.float64)
                self.ptr = C.c_void_p(self.keep.data_ptr())
                self.device = 1
            else:
                self.keep = np.ascontiguousarray(a.detach().numpy(), dtype=np.float64)
                self.ptr = C.c_void_p(self.keep.ctypes.data)
                self.device = 0
        else:
            self.keep = np.ascontiguousarray(a, dtype=np.float64)
            self.ptr = C.c_void_p(self.keep.ctypes.data)
            self.device = 0
        n = self.keep.numel() if _is_torch(self.keep) else self.keep.size
        if count is not None and n != count:
            raise ValueError(f"expected {count} values, got {n}")


def _out_like(arg, count):
    if arg.device:
        import torch
        t = torch.empty(count, dtype=torch.float64, device=arg.keep.device)
        return t, C.c_void_p(t.data_ptr())
    a = np.empty(count, dtype=np.float64)
    return a, C.c_void_p(a.ctypes.data)


class Context:
    """A CUDA device and stream; every call of the library issues on that stream."""

    def __init__(self, device=0, stream=None):
        h = C.c_void_p()
        sp = C.c_void_p(int(stream)) if stream is not None else None
        st = lib.dm_context_create(int(device), sp, C.byref(h))
        if st != 0:
            raise DMError(st, "context creation failed (device %d)" % device)
        self.h = h
        self.device = device

    def check(self, st, what=""):
        if st != 0:
            raise DMError(st, f"{what}: {lib.dm_last_error(self.h).decode()}")

    @property
    def launches(self):
        return lib.dm_context_launch_count(self.h)

    def trace(self, on=True):
        """Start (clearing earlier statistics) or stop per-kernel event timing."""
        self.check(lib.dm_trace_enable(self.h, int(bool(on))), "dm_trace_enable")

    def trace_stats(self, with_bytes=False):
        """{kernel name: (launches, total device ms)} recorded while tracing;
        with_bytes adds the summed algorithmic bytes of the launches."""
        out = {}
        buf = C.create_string_buffer(128)
        n = lib.dm_trace_count(self.h)
        for i in range(n):
            cnt = C.c_longlong()
            ms = C.c_double()
            self.check(lib.dm_trace_entry(self.h, i, buf, 128, C.byref(cnt), C.byref(ms)), "dm_trace_entry")
            if with_bytes:
                by = C.c_double()
                self.check(lib.dm_trace_entry_bytes(self.h, i, C.byref(by)), "dm_trace_entry_bytes")
                out[buf.value.decode()] = (cnt.value, ms.value, by.value)
            else:
                out[buf.value.decode()] = (cnt.value, ms.value)
        return out

    def fma_rates(self):
        """(FP64, FP32) FMA issue rates of the device in TFLOP/s (measured)."""
        r64, r32 = C.c_double(), C.c_double()
        self.check(lib.dm_measure_fma_rates(self.h, C.byref(r64), C.byref(r32)), "dm_measure_fma_rates")
        return r64.value, r32.value

    def _adopt(self, obj):
        """Record a geometry, operator or network made on this context: the C
        objects must be destroyed before their context."""
        if not hasattr(self, "_children"):
            self._children = weakref.WeakSet()
        self._children.add(obj)

    def close(self):
        if getattr(self, "h", None):
            live = list(getattr(self, "_children", ()))
            # operators point at their geometry and at a network: close them first
            for kind in (Operator, Learned, Geometry):
                for obj in live:
                    if isinstance(obj, kind):
                        obj.close()
            lib.dm_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Geometry:
    """Cut-cell fractions of a Yee grid and its multigrid levels."""

    WALL_KINDS = {"pec": 0, "pmc": 1}

    def __init__(self, ctx, nx, ny, nz, dx, dy, dz, phi, origin=(0.0, 0.0, 0.0), a_min=0.0, walls=None):
        """walls: None (every wall a conductor) or six of "pec" / "pmc" in the
        order x-low, x-high, y-low, y-high, z-low, z-high (dm_geometry_create_walls)."""
        self.ctx = ctx
        self.dims = (int(nx), int(ny), int(nz))
        self.spacing = (float(dx), float(dy), float(dz))
        arg = _Arg(phi, (nx + 1) * (ny + 1) * (nz + 1))
        org = (C.c_double * 3)(*origin)
        h = C.c_void_p()
        if walls is None:
            st = lib.dm_geometry_create(ctx.h, nx, ny, nz, dx, dy, dz, org, arg.ptr, arg.device, float(a_min),
                                        C.byref(h))
            ctx.check(st, "dm_geometry_create")
        else:
            walls = tuple(walls)
            if len(walls) != 6 or any(w not in self.WALL_KINDS for w in walls):
                raise ValueError("walls: six entries, each 'pec' or 'pmc'")
            wk = (C.c_int * 6)(*(self.WALL_KINDS[w] for w in walls))
            st = lib.dm_geometry_create_walls(ctx.h, nx, ny, nz, dx, dy, dz, org, arg.ptr, arg.device, float(a_min),
                                              wk, C.byref(h))
            ctx.check(st, "dm_geometry_create_walls")
        self.h = h
        ctx._adopt(self)

    @classmethod
    def from_fractions(cls, ctx, nx, ny, nz, dx, dy, dz, L, A, V):
        """A geometry from given edge, face and cell fractions (natural layouts)."""
        self = cls.__new__(cls)
        self.ctx = ctx
        self.dims = (int(nx), int(ny), int(nz))
        self.spacing = (float(dx), float(dy), float(dz))
        la = _Arg(L, edge_count(nx, ny, nz))
        aa = _Arg(A, face_count(nx, ny, nz))
        va = _Arg(V, cell_count(nx, ny, nz))
        if not (la.device == aa.device == va.device):
            raise ValueError("L, A and V must all be host arrays or all device tensors")
        h = C.c_void_p()
        st = lib.dm_geometry_create_from_fractions(ctx.h, nx, ny, nz, dx, dy, dz, la.ptr, aa.ptr, va.ptr, la.device,
                                                   C.byref(h))
        ctx.check(st, "dm_geometry_create_from_fractions")
        self.h = h
        ctx._adopt(self)
        return self

    @classmethod
    def from_workload(cls, ctx, w, a_min=0.0, phi=None):
        g = w.grid
        walls = getattr(w, "walls", None)
        if walls is not None and all(x == "pec" for x in walls):
            walls = None
        return cls(ctx, g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, w.phi.ravel() if phi is None else phi, g.origin, a_min,
                   walls=walls)

    @property
    def num_levels(self):
        return lib.dm_geometry_num_levels(self.h)

    def level_info(self, level=0):
        """Dims and counts of a level (cached: a level never changes)."""
        cache = self.__dict__.setdefault("_info", {})
        if level not in cache:
            dims = (C.c_int * 3)()
            counts = (C.c_longlong * 4)()
            self.ctx.check(lib.dm_geometry_level_info(self.h, level, dims, counts), "dm_geometry_level_info")
            cache[level] = {"dims": tuple(dims), "faces": counts[0], "edges": counts[1], "cells": counts[2],
                            "open": counts[3]}
        return dict(cache[level])

    def fractions(self, level=0):
        """(L, A, V) in natural layouts as numpy arrays."""
        info = self.level_info(level)
        L = np.empty(info["edges"])
        A = np.empty(info["faces"])
        V = np.empty(info["cells"])
        st = lib.dm_geometry_fractions(self.h, level, C.c_void_p(L.ctypes.data), C.c_void_p(A.ctypes.data),
                                       C.c_void_p(V.ctypes.data), 0)
        self.ctx.check(st, "dm_geometry_fractions")
        return L, A, V

    def close(self):
        if getattr(self, "h", None):
            lib.dm_geometry_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_params(max_coarse=4, band_sweeps=None, band_brick=8, omega_scale=1.7, power_iters=30, precision="f64",
              autotune=1, force_shape=-1, band_sweeps_coarse=None, symmetric_transform=0, dense_coarse=None,
              krylov_ff=1, jacobi_sweeps=None):
    """band_sweeps, band_sweeps_coarse: band-smoother sweeps on the fine level and below it
    (None: the library's defaults, 24 and 16);
    symmetric_transform: 1 for the V-cycle of Eq. fullMat2's symmetric form;
    krylov_ff: 1 to form the shifted solves' FGMRES operator applies in float-float;
    jacobi_sweeps: damped Jacobi sweeps per smoothing step (None: the library's default)."""
    p = MGParams()
    lib.dm_mg_params_default(C.byref(p))
    p.max_coarse = max_coarse
    if band_sweeps is not None:
        p.band_sweeps = int(band_sweeps)
    p.band_brick = band_brick
    p.omega_scale = omega_scale
    p.power_iters = power_iters
    p.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    p.autotune = int(autotune)
    p.stencil_shape = int(force_shape)
    if band_sweeps_coarse is not None:
        p.band_sweeps_coarse = int(band_sweeps_coarse)
    p.symmetric_transform = int(symmetric_transform)
    if dense_coarse is not None:
        p.dense_coarse = int(dense_coarse)
    p.krylov_ff = int(krylov_ff)
    if jacobi_sweeps is not None:
        p.jacobi_sweeps = int(jacobi_sweeps)
    return p


class Operator:
    """K - sigma A (Eq. discLaplDM) on every level with its V-cycle preconditioner."""

    def __init__(self, ctx, geom, sigma, **mg):
        self.ctx = ctx
        self.geom = geom
        self.sigma = float(sigma)
        self.mg = mg_params(**mg)
        h = C.c_void_p()
        ctx.check(lib.dm_operator_create(ctx.h, geom.h, self.sigma, C.byref(self.mg), C.byref(h)),
                  "dm_operator_create")
        self.h = h
        ctx._adopt(self)

    @property
    def num_levels(self):
        return lib.dm_operator_num_levels(self.h)

    def stencil_shape(self, level):
        return lib.dm_operator_stencil_shape(self.h, level)

    def omega(self, level, scalar=False):
        return lib.dm_operator_get_omega(self.h, level, int(scalar))

    def set_omega(self, level, omega, scalar=False):
        self.ctx.check(lib.dm_operator_set_omega(self.h, level, int(scalar), float(omega)), "set_omega")

    def _faces(self, level):
        return self.geom.level_info(level)["faces"]

    def _cells(self, level):
        return self.geom.level_info(level)["cells"]

    def apply(self, x, level=0):
        a = _Arg(x, self._faces(level))
        y, yp = _out_like(a, self._faces(level))
        self.ctx.check(lib.dm_operator_apply(self.h, level, a.ptr, yp, a.device), "dm_operator_apply")
        return y

    def apply_ff(self, x):
        """(K - sigma A) x on the fine level in float-float (dm_operator_apply_ff)."""
        a = _Arg(x, self._faces(0))
        y, yp = _out_like(a, self._faces(0))
        self.ctx.check(lib.dm_operator_apply_ff(self.h, a.ptr, yp, a.device), "dm_operator_apply_ff")
        return y

    def apply_noalloc(self, x, level=0, out=None):
        """(K - sigma A) x through dm_operator_apply_noalloc: x and the result are
        CUDA tensors; the call allocates nothing (see include/dmeig.h)."""
        import torch
        F = self._faces(level)
        dev = self.ctx.device

        def ok(t):
            return (_is_torch(t) and t.is_cuda and t.device.index == dev and t.dtype == torch.float64
                    and t.is_contiguous() and t.numel() == F)

        if not ok(x):
            raise ValueError(f"apply_noalloc: x must be a contiguous float64 tensor of {F} values on cuda:{dev}")
        if out is not None and not ok(out):
            raise ValueError(f"apply_noalloc: out must be a contiguous float64 tensor of {F} values on cuda:{dev}")
        y = torch.empty_like(x) if out is None else out
        self.ctx.check(lib.dm_operator_apply_noalloc(self.h, level, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())),
                       "dm_operator_apply_noalloc")
        return y

    def diagonal(self, level=0):
        d = np.empty(self._faces(level))
        self.ctx.check(lib.dm_operator_diagonal(self.h, level, C.c_void_p(d.ctypes.data), 0), "dm_operator_diagonal")
        return d

    def smooth(self, f, x, level=0):
        fa = _Arg(f, self._faces(level))
        xa = _Arg(x, self._faces(level))
        out = xa.keep.clone() if xa.device else xa.keep.copy()
        ptr = C.c_void_p(out.data_ptr()) if xa.device else C.c_void_p(out.ctypes.data)
        self.ctx.check(lib.dm_operator_smooth(self.h, level, fa.ptr, ptr, fa.device), "dm_operator_smooth")
        return out

    def restrict(self, r, level=0):
        a = _Arg(r, self._faces(level))
        y, yp = _out_like(a, self._faces(level + 1))
        self.ctx.check(lib.dm_operator_restrict(self.h, level, a.ptr, yp, a.device), "dm_operator_restrict")
        return y

    def prolong(self, ec, x, level=0):
        ea = _Arg(ec, self._faces(level + 1))
        xa = _Arg(x, self._faces(level))
        out = xa.keep.clone() if xa.device else xa.keep.copy()
        ptr = C.c_void_p(out.data_ptr()) if xa.device else C.c_void_p(out.ctypes.data)
        self.ctx.check(lib.dm_operator_prolong(self.h, level, ea.ptr, ptr, ea.device), "dm_operator_prolong")
        return out

    def vcycle(self, f):
        a = _Arg(f, self._faces(0))
        e, ep = _out_like(a, self._faces(0))
        self.ctx.check(lib.dm_operator_vcycle(self.h, a.ptr, ep, a.device), "dm_operator_vcycle")
        return e

    def scalar_vcycle(self, f):
        a = _Arg(f, self._cells(0))
        e, ep = _out_like(a, self._cells(0))
        self.ctx.check(lib.dm_operator_scalar_vcycle(self.h, a.ptr, ep, a.device), "dm_operator_scalar_vcycle")
        return e

    def solve(self, b, tol=1e-10, restart=40, maxit=400):
        a = _Arg(b, self._faces(0))
        x, xp = _out_like(a, self._faces(0))
        it = C.c_int()
        rr = C.c_double()
        st = lib.dm_operator_solve(self.h, a.ptr, xp, a.device, tol, restart, maxit, C.byref(it), C.byref(rr))
        if st not in (0, 2):
            self.ctx.check(st, "dm_operator_solve")
        return x, it.value, rr.value

    def project(self, x, tol=1e-12):
        a = _Arg(x, self._faces(0))
        y, yp = _out_like(a, self._faces(0))
        it = C.c_int()
        self.ctx.check(lib.dm_operator_project(self.h, a.ptr, yp, a.device, tol, C.byref(it)), "dm_operator_project")
        return y, it.value

    def set_learned(self, net):
        """Use (net) or stop using (None) the learned correction in the preconditioner."""
        self.ctx.check(lib.dm_operator_set_learned(self.h, net.h if net is not None else None), "set_learned")

    def close(self):
        if getattr(self, "h", None):
            lib.dm_operator_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Learned:
    """The learned smoother's network (3 conv layers, 8 -> 16 -> 16 -> 3 channels)."""

    def __init__(self, ctx, seed=0):
        self.ctx = ctx
        h = C.c_void_p()
        ctx.check(lib.dm_learned_create(ctx.h, int(seed), C.byref(h)), "dm_learned_create")
        self.h = h
        ctx._adopt(self)

    @staticmethod
    def num_params():
        return lib.dm_learned_num_params()

    def get_weights(self):
        w = np.empty(self.num_params(), dtype=np.float32)
        self.ctx.check(lib.dm_learned_get_weights(self.h, w.ctypes.data_as(C.POINTER(C.c_float))), "get_weights")
        return w

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.num_params()
        self.ctx.check(lib.dm_learned_set_weights(self.h, w.ctypes.data_as(C.POINTER(C.c_float))), "set_weights")

    def apply(self, geom, r):
        a = _Arg(r, geom.level_info(0)["faces"])
        y, yp = _out_like(a, geom.level_info(0)["faces"])
        self.ctx.check(lib.dm_learned_apply(self.h, geom.h, a.ptr, yp, a.device), "dm_learned_apply")
        return y

    def loss_grad(self, geom, X, E):
        fp = C.POINTER(C.c_float)
        X = np.ascontiguousarray(X, dtype=np.float32)
        E = np.ascontiguousarray(E, dtype=np.float32)
        loss = C.c_float()
        g = np.empty(self.num_params(), dtype=np.float32)
        self.ctx.check(lib.dm_learned_loss_grad(self.h, geom.h, X.ctypes.data_as(fp), E.ctypes.data_as(fp),
                                                C.byref(loss), g.ctypes.data_as(fp)), "dm_learned_loss_grad")
        return loss.value, g

    def train(self, op, runs=4, epochs=20, lr=1e-3, seed=1):
        hist = np.empty(epochs, dtype=np.float32)
        self.ctx.check(lib.dm_learned_train(self.h, op.h, runs, epochs, lr, int(seed),
                                            hist.ctypes.data_as(C.POINTER(C.c_float))), "dm_learned_train")
        return hist

    def train_step(self, op, r, lr=1e-3):
        """One Adam step on the residual r: returns (loss, gradient) before the update."""
        a = _Arg(r, op._faces(0))
        loss = C.c_float()
        g = np.empty(self.num_params(), dtype=np.float32)
        self.ctx.check(lib.dm_learned_train_step(self.h, op.h, a.ptr, a.device, float(lr), C.byref(loss),
                                                 g.ctypes.data_as(C.POINTER(C.c_float))), "dm_learned_train_step")
        return loss.value, g

    def close(self):
        if getattr(self, "h", None):
            lib.dm_learned_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eig_params(sigma, nev, tol=1e-10, inner_tol=None, proj_tol=1e-12, basis=0, max_restarts=100,
               inner_restart=40, inner_maxit=400, seed=1301, learned=None, max_seconds=0.0, rho_tol=1e-8,
               **mg):
    p = EigParams()
    lib.dm_eig_params_default(C.byref(p))
    p.sigma = float(sigma)
    p.nev = int(nev)
    p.tol = tol
    if inner_tol is not None:
        p.inner_tol = float(inner_tol)
    p.proj_tol = proj_tol
    p.basis = basis
    p.max_restarts = max_restarts
    p.inner_restart = inner_restart
    p.inner_maxit = inner_maxit
    p.seed = seed
    p.mg = mg_params(**mg)
    p.learned = learned.h if learned is not None else None
    p.max_seconds = float(max_seconds)
    p.rho_tol = float(rho_tol)
    return p


def eigensolve(ctx, geom, sigma, nev, vectors="host", out=None, **kw):
    """The nev electromagnetic eigenpairs nearest sigma.

    vectors: "host" (numpy [nev, F]), "device" (torch CUDA tensor [nev, F]) or None.
    Returns (k2 numpy[nev], B or None, report dict, status)."""
    p = eig_params(sigma, nev, **kw)
    F = geom.level_info(0)["faces"]
    k2 = np.empty(nev)
    B = None
    bptr = None
    dev = 0
    if vectors == "host":
        B = np.empty((nev, F)) if out is None else out
        if _is_torch(B):
            # a host tensor (pinned memory copies at full link speed)
            if B.is_cuda or B.dtype != _torch().float64 or not B.is_contiguous() or B.numel() != nev * F:
                raise ValueError(f"eigensolve: out must be a contiguous float64 host tensor of {nev} x {F} values")
            bptr = C.c_void_p(B.data_ptr())
        else:
            bptr = C.c_void_p(B.ctypes.data)
    elif vectors == "device":
        import torch
        B = torch.empty((nev, F), dtype=torch.float64, device=f"cuda:{ctx.device}") if out is None else out
        bptr = C.c_void_p(B.data_ptr())
        dev = 1
    rep = EigReport()
    st = lib.dm_eigensolve(ctx.h, geom.h, C.byref(p), k2.ctypes.data_as(C.POINTER(C.c_double)), bptr, dev,
                           C.byref(rep))
    if st != 0 and not (st == 3 or (st == 2 and rep.outer_iters > 0)):
        # DM_ERR_NO_CONVERGENCE with a filled report is a partial result and
        # DM_ERR_TIMEOUT a stopped one (both returned with their status);
        # anything else is an error
        ctx.check(st, "dm_eigensolve")
    return k2, B, rep.as_dict(), st


def eigensolve_batched(ctx, jobs, streams=8):
    """Solve many (geometry, sigma, nev, options) jobs in one call.

    jobs: list of dicts with keys geom, sigma, nev and optional eigensolve
    options (precision, tol, ...).  Returns a list of (k2, report, status)."""
    from ._lib import BatchItem
    n = len(jobs)
    arr = (BatchItem * n)()
    keep = []
    for i, job in enumerate(jobs):
        opts = {k: v for k, v in job.items() if k not in ("geom", "sigma", "nev")}
        p = eig_params(job["sigma"], job["nev"], **opts)
        k2 = np.empty(job["nev"])
        keep.append(k2)
        arr[i].geom = job["geom"].h
        arr[i].params = p
        arr[i].k2_out = k2.ctypes.data_as(C.POINTER(C.c_double))
        arr[i].b_out = None
        arr[i].b_on_device = 0
        arr[i].status = -1
    st = lib.dm_eigensolve_batched(ctx.h, n, arr, int(streams))
    if st not in (0, 2):
        ctx.check(st, "dm_eigensolve_batched")
    return [(keep[i], arr[i].report.as_dict(), arr[i].status) for i in range(n)]


def certify(ctx, geom, k2, B):
    """(rho, delta, rq) of the given eigenpairs (B: [n, F] numpy or CUDA tensor)."""
    n = len(k2)
    F = geom.level_info(0)["faces"]
    a = _Arg(B, n * F)
    k = np.ascontiguousarray(k2, dtype=np.float64)
    rho, delta, rq = np.empty(n), np.empty(n), np.empty(n)
    dp = C.POINTER(C.c_double)
    st = lib.dm_certify(ctx.h, geom.h, n, k.ctypes.data_as(dp), a.ptr, a.device, rho.ctypes.data_as(dp),
                        delta.ctypes.data_as(dp), rq.ctypes.data_as(dp))
    ctx.check(st, "dm_certify")
    return rho, delta, rq
