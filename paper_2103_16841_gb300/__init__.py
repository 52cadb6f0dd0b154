"""GB300 space-time Galerkin BEM for the retarded single layer of the 3D wave
equation (Poelz & Schanz, "On the space-time discretization of variational
retarded potential boundary integral equations").

Thin Python layer over the C ABI of libstbem.so (include/stbem.h). The CUDA
library does all computation; PyTorch is used only for device memory and
streams where the caller passes device tensors. Importing this package does
not load the library; the first object created does, and fails loudly when
the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _lib
from ._lib import BemError, DATA_PULSE, DATA_SIN2_UNIFORM

__all__ = ["Context", "Mesh", "Operator", "Request", "inner_potentials", "BemError", "DATA_PULSE", "DATA_SIN2_UNIFORM"]


class Context:
    """bem_context: binds one CUDA device and owns the library's stream."""

    def __init__(self, device: int = 0):
        self._L = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(self._L.bem_context_create(int(device), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._L.bem_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alu_peaks(self):
        """Measured FP32 and FP64 FMA throughput of the device, TFLOP/s."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _lib.check(self._L.bem_alu_peaks(self.h, ctypes.byref(a), ctypes.byref(b)))
        return {"fp32_tflops": a.value, "fp64_tflops": b.value}

    def selftest_bounded_wait(self):
        """bem_selftest_bounded_wait: (status, ms waited); status 5
        (BEM_ERR_DEVICE_TIMEOUT) is the expected outcome."""
        ms = ctypes.c_double()
        st = self._L.bem_selftest_bounded_wait(self.h, ctypes.byref(ms))
        return int(st), ms.value

    def set_tuning(self, mode=1, cache_path=None):
        """bem_context_set_tuning: 1 = time the quadrature's launch shape per
        shape class on first assembly (kept in cache_path if given), 0 = off."""
        path = None if cache_path is None else os.fsencode(cache_path)
        _lib.check(self._L.bem_context_set_tuning(self.h, int(mode), path))

    @staticmethod
    def version():
        return _lib.load().bem_version().decode()


class Mesh:
    """bem_mesh: a space-time tetrahedral mesh of Gamma x [0, T]."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.h = handle
        n = np.zeros(3, dtype=np.int64)
        _lib.check(ctx._L.bem_mesh_info(self.h, _lib.lptr(n[0:1]), _lib.lptr(n[1:2]), _lib.lptr(n[2:3])))
        self.n_tet, self.n_columns, self.n_surfaces = (int(v) for v in n)

    @classmethod
    def from_tets(cls, ctx, sv_xyz, stv_sv, stv_t, tets):
        sv_xyz = np.ascontiguousarray(sv_xyz, dtype=np.float64)
        stv_sv = np.ascontiguousarray(stv_sv, dtype=np.int32)
        stv_t = np.ascontiguousarray(stv_t, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        h = ctypes.c_void_p()
        _lib.check(ctx._L.bem_mesh_create(ctx.h, sv_xyz.shape[0], _lib.dptr(sv_xyz), stv_sv.shape[0],
                                          _lib.iptr(stv_sv), _lib.dptr(stv_t), tets.shape[0], _lib.iptr(tets),
                                          ctypes.byref(h)))
        return cls(ctx, h)

    @classmethod
    def from_prisms(cls, ctx, sv_xyz, tri, time_nodes):
        sv_xyz = np.ascontiguousarray(sv_xyz, dtype=np.float64)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        tn = np.ascontiguousarray(time_nodes, dtype=np.float64)
        h = ctypes.c_void_p()
        _lib.check(ctx._L.bem_mesh_create_prisms(ctx.h, sv_xyz.shape[0], _lib.dptr(sv_xyz), tri.shape[0],
                                                 _lib.iptr(tri), tn.shape[1] - 1, _lib.dptr(tn), ctypes.byref(h)))
        return cls(ctx, h)

    @classmethod
    def from_spacetime(cls, ctx, m):
        """From a paper_2103_16841_gb300.inputs.SpaceTimeMesh."""
        return cls.from_tets(ctx, m.svert, m.stv_sv, m.stv_t, m.tets)

    def close(self):
        if getattr(self, "h", None):
            self.ctx._L.bem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """bem_operator: the assembled energetic single-layer Galerkin matrix."""

    def __init__(self, ctx: Context, mesh: Mesh, precision: str = "fp64", m_q: int = 3, n_theta: int = 0,
                 store_fp32: bool = True, matrix_free: bool = False, trial_space: str = "p0"):
        self.ctx, self.mesh = ctx, mesh
        o = _lib.OpOpts(_lib.PREC[precision], int(m_q), int(n_theta), int(bool(store_fp32)), int(bool(matrix_free)),
                        _lib.TRIAL[trial_space])
        h = ctypes.c_void_p()
        _lib.check(ctx._L.bem_operator_create(ctx.h, mesh.h, ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        self.n = mesh.n_tet

    def stats(self):
        a = np.zeros(3, dtype=np.int64)
        ms = np.zeros(1)
        _lib.check(self.ctx._L.bem_operator_stats(self.h, _lib.lptr(a[0:1]), _lib.lptr(a[1:2]), _lib.lptr(a[2:3]),
                                                  _lib.dptr(ms)))
        return {"nnz": int(a[0]), "stored": int(a[1]), "blocks": int(a[2]), "assemble_ms": float(ms[0])}

    def inner_integrals(self):
        """Inner integrals of one assembly (bem_operator_work)."""
        n = np.zeros(1, dtype=np.int64)
        _lib.check(self.ctx._L.bem_operator_work(self.h, _lib.lptr(n)))
        return int(n[0])

    def tuning(self):
        """The quadrature's launch shape (bem_operator_tuning)."""
        per, budget, how = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = np.zeros(8)
        _lib.check(self.ctx._L.bem_operator_tuning(self.h, ctypes.byref(per), ctypes.byref(budget), ctypes.byref(how),
                                                   _lib.dptr(ms)))
        # candidate "b<budget>x<CTAs per SM>": its sample time
        return {"ctas_per_sm": per.value, "budget_ctas": budget.value, "tuned": ["default", "timed", "cache"][how.value],
                "sample_ms": {"b%dx%d" % (2 if k >= 4 else 4, k % 4 + 1): float(v) for k, v in enumerate(ms) if v > 0}}

    def check(self):
        """(number of non-finite stored values, largest |value|)"""
        n = np.zeros(1, dtype=np.int64)
        mx = np.zeros(1)
        _lib.check(self.ctx._L.bem_operator_check(self.h, _lib.lptr(n), _lib.dptr(mx)))
        return int(n[0]), float(mx[0])

    def timings(self):
        ms = np.zeros(4)
        _lib.check(self.ctx._L.bem_operator_timings(self.h, _lib.dptr(ms)))
        return {"outer_points_ms": ms[0], "pattern_ms": ms[1], "offsets_ms": ms[2], "quadrature_ms": ms[3]}

    def reassemble(self, stream=None):
        _lib.check(self.ctx._L.bem_operator_reassemble(self.h, _stream_ptr(stream)))

    def export_pattern(self):
        nnz = self.stats()["nnz"]
        rowptr = np.zeros(self.n + 1, dtype=np.int64)
        cols = np.zeros(max(nnz, 1), dtype=np.int32)
        _lib.check(self.ctx._L.bem_operator_export_pattern(self.h, _lib.lptr(rowptr), _lib.iptr(cols)))
        return rowptr, cols[:nnz]

    def pattern_rows(self, rows, cap=None):
        """Admissible columns (ascending) of the listed rows."""
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        cap = int(cap or self.n)
        counts = np.zeros(rows.shape[0], dtype=np.int64)
        cols = np.zeros(rows.shape[0] * cap, dtype=np.int32)
        _lib.check(self.ctx._L.bem_operator_pattern_rows(self.h, rows.shape[0], _lib.iptr(rows), cap,
                                                         _lib.lptr(counts), _lib.iptr(cols)))
        return [cols[k * cap: k * cap + min(cap, counts[k])].copy() for k in range(rows.shape[0])]

    def export_dense(self):
        A = np.zeros((self.n, self.n))
        _lib.check(self.ctx._L.bem_operator_export_dense(self.h, _lib.dptr(A)))
        return A

    def entries(self, ij):
        ij = np.ascontiguousarray(np.asarray(ij, dtype=np.int32).reshape(-1, 2))
        out = np.zeros(ij.shape[0])
        _lib.check(self.ctx._L.bem_operator_entries(self.h, ij.shape[0], _lib.iptr(ij), _lib.dptr(out)))
        return out

    def rhs(self, kind, params=None):
        if params is not None:
            params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 5)
            nrhs = params.shape[0]
            pp = _lib.dptr(params)
        else:
            nrhs = 1
            pp = ctypes.POINTER(ctypes.c_double)()
        b = np.zeros(nrhs * self.n)
        _lib.check(self.ctx._L.bem_rhs(self.h, int(kind), nrhs, pp, _lib.dptr(b)))
        return b.reshape(nrhs, self.n).T.copy()

    def rhs_points(self, level=0, n_gauss=8):
        """Quadrature points (t, x, y, z) [n_pts, 4] and weights [n_pts] of the
        right-hand side for arbitrary data (bem_rhs_points)."""
        n = ctypes.c_int64()
        _lib.check(self.ctx._L.bem_rhs_points(self.h, int(level), int(n_gauss), ctypes.byref(n), None, None))
        pts = np.zeros((n.value, 4))
        w = np.zeros(n.value)
        _lib.check(self.ctx._L.bem_rhs_points(self.h, int(level), int(n_gauss), ctypes.byref(n), _lib.dptr(pts),
                                              _lib.dptr(w)))
        return pts, w

    def rhs_from_samples(self, g, level=0, n_gauss=8):
        """b [n] or [n, nrhs] from samples g [n_pts] or [n_pts, nrhs] of the data
        at the points of rhs_points(level, n_gauss)."""
        g = np.asarray(g, dtype=np.float64)
        vec = g.ndim == 1
        G = np.ascontiguousarray((g[:, None] if vec else g).T)
        nrhs = G.shape[0]
        b = np.zeros(nrhs * self.n)
        _lib.check(self.ctx._L.bem_rhs_from_samples(self.h, int(level), int(n_gauss), _lib.dptr(G), nrhs,
                                                    _lib.dptr(b)))
        b = b.reshape(nrhs, self.n).T.copy()
        return b[:, 0] if vec else b

    def solve_refined(self, op_hi, b, tol=1e-10, restart=50, maxit=2000, inner="tf32", max_refine=20,
                      allow_unconverged=False):
        """bem_solve_refined: refinement with op_hi's FP64 residual and inner
        solves on this (mixed) operator. Host b [n] or [n, nrhs]."""
        b = np.asarray(b, dtype=np.float64)
        vec = b.ndim == 1
        B = np.ascontiguousarray((b[:, None] if vec else b).T)
        nrhs = B.shape[0]
        W = np.zeros_like(B)
        o = _lib.SolveOpts(float(tol), int(restart), int(maxit), _lib.DTYPE[inner], int(max_refine))
        info = (_lib.SolveInfo * nrhs)()
        st = self.ctx._L.bem_solve_refined(op_hi.h, self.h, _lib.dptr(B), _lib.dptr(W), nrhs, ctypes.byref(o), info)
        _lib.check(st, allow=(4,) if allow_unconverged else ())
        infos = [{"iterations": i.iterations, "refinements": i.refinements, "converged": bool(i.converged),
                  "rel_residual": i.rel_residual, "solve_ms": i.solve_ms} for i in info]
        w = W.T.copy()
        return (w[:, 0] if vec else w), infos

    def solve_async(self, b, w, tol=1e-8, restart=50, maxit=2000, inner="fp64", max_refine=10, stream=None):
        """Starts bem_solve_async on contiguous CUDA float64 tensors b, w of shape
        [n] or [nrhs, n]; returns a Request."""
        import torch
        for t in (b, w):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("b and w must be contiguous CUDA float64 tensors")
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        o = _lib.SolveOpts(float(tol), int(restart), int(maxit), _lib.DTYPE[inner], int(max_refine))
        h = ctypes.c_void_p()
        _lib.check(self.ctx._L.bem_solve_async(self.h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                               nrhs, ctypes.byref(o), _stream_ptr(stream), ctypes.byref(h)))
        return Request(self.ctx, h, nrhs)

    def matvec(self, x, y=None, stream=None, dtype=None):
        """y = A x for torch CUDA float64 tensors of shape [n] or [nrhs, n].
        dtype None: bem_matvec; "fp64" / "fp32" / "tf32" / "bf16": the
        arithmetic of bem_matvec_dtype."""
        import torch
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
            raise ValueError("x must be a contiguous CUDA float64 tensor")
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        if y is None:
            y = torch.empty_like(x)
        if dtype is None:
            _lib.check(self.ctx._L.bem_matvec(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                              nrhs, _stream_ptr(stream)))
        else:
            _lib.check(self.ctx._L.bem_matvec_dtype(self.h, ctypes.c_void_p(x.data_ptr()),
                                                    ctypes.c_void_p(y.data_ptr()), nrhs, _lib.DTYPE[dtype],
                                                    _stream_ptr(stream)))
        return y

    def matvec_noalloc(self, x, y=None, stream=None):
        """y = A x like matvec, through the allocation-free entry point: the
        library allocates no device memory for it (n_tet * nrhs <= 2**20).
        Enqueued on `stream` (default: the library's stream) without a final
        synchronize; synchronize before reading y."""
        import torch
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
            raise ValueError("x must be a contiguous CUDA float64 tensor")
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        if y is None:
            y = torch.empty_like(x)
        _lib.check(self.ctx._L.bem_matvec_noalloc(self.h, ctypes.c_void_p(x.data_ptr()),
                                                  ctypes.c_void_p(y.data_ptr()), nrhs, _stream_ptr(stream)))
        return y

    def solve(self, b, tol=1e-8, restart=50, maxit=2000, inner="fp64", max_refine=10, allow_unconverged=False):
        """Host arrays b [n] or [n, nrhs]; returns (w, infos)."""
        b = np.asarray(b, dtype=np.float64)
        vec = b.ndim == 1
        B = np.ascontiguousarray((b[:, None] if vec else b).T)
        nrhs = B.shape[0]
        W = np.zeros_like(B)
        o = _lib.SolveOpts(float(tol), int(restart), int(maxit), _lib.DTYPE[inner], int(max_refine))
        info = (_lib.SolveInfo * nrhs)()
        st = self.ctx._L.bem_solve(self.h, _lib.dptr(B), _lib.dptr(W), nrhs, ctypes.byref(o), info)
        _lib.check(st, allow=(4,) if allow_unconverged else ())
        infos = [{"iterations": i.iterations, "refinements": i.refinements, "converged": bool(i.converged),
                  "rel_residual": i.rel_residual, "solve_ms": i.solve_ms} for i in info]
        w = W.T.copy()
        return (w[:, 0] if vec else w), infos

    def close(self):
        if getattr(self, "h", None):
            self.ctx._L.bem_operator_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Request:
    """bem_request: an asynchronous solve (Operator.solve_async)."""

    def __init__(self, ctx, handle, nrhs):
        self.ctx, self.h, self.nrhs = ctx, handle, nrhs

    def wait(self, timeout_s):
        """bem_request_wait: the solve's status and infos, or None (status
        BEM_ERR_DEVICE_TIMEOUT) if it is still running after timeout_s."""
        info = (_lib.SolveInfo * self.nrhs)()
        st = self.ctx._L.bem_request_wait(self.h, int(max(0.0, timeout_s) * 1e9), info)
        if st == 5:
            return None
        _lib.check(st, allow=(4, 9))
        return st, [{"iterations": i.iterations, "refinements": i.refinements, "converged": bool(i.converged),
                     "rel_residual": i.rel_residual, "solve_ms": i.solve_ms} for i in info]

    def cancel(self):
        _lib.check(self.ctx._L.bem_request_cancel(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.ctx._L.bem_request_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """bem_batch: the operators of many small meshes assembled by one
    persistent launch per pass and solved as one block-diagonal system."""

    def __init__(self, ctx: Context, meshes, precision="mixed", m_q=3, n_theta=0, store_fp32=True):
        self.ctx = ctx
        self.meshes = list(meshes)          # the meshes must outlive the batch
        o = _lib.OpOpts(_lib.PREC[precision], int(m_q), int(n_theta), int(bool(store_fp32)), 0, 0)
        arr = (ctypes.c_void_p * len(self.meshes))(*[mm.h.value for mm in self.meshes])
        h = ctypes.c_void_p()
        _lib.check(ctx._L.bem_batch_create(ctx.h, len(self.meshes), arr, ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        self.n_tet = [Mesh_info(ctx, mm)[0] for mm in self.meshes]

    def stats(self):
        n = ctypes.c_int32()
        nt, nnz = ctypes.c_int64(), ctypes.c_int64()
        ms = ctypes.c_double()
        _lib.check(self.ctx._L.bem_batch_stats(self.h, ctypes.byref(n), ctypes.byref(nt), ctypes.byref(nnz),
                                               ctypes.byref(ms)))
        return {"n_ops": n.value, "n_tet": nt.value, "nnz": nnz.value, "assemble_ms": ms.value}

    def solve(self, params_list, tol=1e-8, restart=50, maxit=2000, inner="fp32", max_refine=10,
              allow_unconverged=False):
        """params_list: one [nrhs_i, 5] pulse array per mesh. Returns (list of
        w_i [n_tet_i, nrhs_i], list of per-RHS info lists)."""
        nrhs = np.array([np.asarray(p).reshape(-1, 5).shape[0] for p in params_list], dtype=np.int32)
        prm = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1, 5)
                                                   for p in params_list]))
        total = int(sum(n * k for n, k in zip(self.n_tet, nrhs)))
        w = np.zeros(total)
        infos = (_lib.SolveInfo * int(nrhs.sum()))()
        o = _lib.SolveOpts(float(tol), int(restart), int(maxit), _lib.DTYPE[inner], int(max_refine))
        st = self.ctx._L.bem_batch_solve(self.h, DATA_PULSE, _lib.iptr(nrhs), _lib.dptr(prm), ctypes.byref(o),
                                         _lib.dptr(w), infos)
        _lib.check(st, allow=(4,) if allow_unconverged else ())
        ws, inf, off, row = [], [], 0, 0
        for n, k in zip(self.n_tet, nrhs):
            ws.append(w[off:off + n * k].reshape(k, n).T.copy())
            inf.append([{"iterations": infos[row + q].iterations, "refinements": infos[row + q].refinements,
                         "converged": bool(infos[row + q].converged), "rel_residual": infos[row + q].rel_residual,
                         "solve_ms": infos[row + q].solve_ms} for q in range(k)])
            off += n * k
            row += k
        return ws, inf

    def close(self):
        if getattr(self, "h", None):
            self.ctx._L.bem_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def Mesh_info(ctx, mesh):
    nt, nc, ns = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _lib.check(ctx._L.bem_mesh_info(mesh.h, ctypes.byref(nt), ctypes.byref(nc), ctypes.byref(ns)))
    return nt.value, nc.value, ns.value


class Server:
    """bem_server: continuous batching of Dirichlet solves on one device.

    submit() copies a request (space-time mesh + data) and returns its ticket;
    poll() returns finished requests as dicts with the densities w
    [nrhs, n_tet] (caller panel order) and their timings."""

    def __init__(self, ctx: Context, hbm_budget=0, max_slots=4, precision="mixed", inner="fp32", tol=1e-8,
                 restart=50, maxit=2000, max_refine=10, cache_operators=False):
        self.ctx = ctx
        o = _lib.ServerOpts(int(hbm_budget), int(max_slots), _lib.PREC[precision], _lib.DTYPE[inner],
                            int(restart), int(maxit), int(max_refine), float(tol), int(bool(cache_operators)), 0)
        h = ctypes.c_void_p()
        _lib.check(ctx._L.bem_server_create(ctx.h, ctypes.byref(o), ctypes.byref(h)))
        self.h = h

    def submit(self, m, kind=DATA_PULSE, params=None, nrhs=1):
        """m: inputs.SpaceTimeMesh; params [nrhs, 5] for DATA_PULSE."""
        sv = np.ascontiguousarray(m.svert, dtype=np.float64)
        stv_sv = np.ascontiguousarray(m.stv_sv, dtype=np.int32)
        stv_t = np.ascontiguousarray(m.stv_t, dtype=np.float64)
        tets = np.ascontiguousarray(m.tets, dtype=np.int32)
        prm = None
        if kind == DATA_PULSE:
            prm = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 5)
            nrhs = prm.shape[0]
        job = _lib.Job(sv.shape[0], _lib.dptr(sv), stv_sv.shape[0], _lib.iptr(stv_sv), _lib.dptr(stv_t),
                       tets.shape[0], _lib.iptr(tets), int(kind), int(nrhs),
                       _lib.dptr(prm) if prm is not None else ctypes.POINTER(ctypes.c_double)())
        t = ctypes.c_uint64()
        _lib.check(self.ctx._L.bem_server_submit(self.h, ctypes.byref(job), ctypes.byref(t)))
        return int(t.value)

    def poll(self, max_items=64, timeout_ms=0):
        buf = (_lib.Completion * max_items)()
        n = ctypes.c_int32()
        _lib.check(self.ctx._L.bem_server_poll(self.h, buf, int(max_items), ctypes.byref(n), int(timeout_ms)))
        out = []
        for c in buf[:n.value]:
            w = None
            if c.w:
                w = np.ctypeslib.as_array(c.w, shape=(c.nrhs * c.n_tet,)).copy().reshape(c.nrhs, c.n_tet)
            out.append({"ticket": int(c.ticket), "status": int(c.status), "w": w, "iterations": int(c.iterations),
                        "refinements": int(c.refinements), "rel_residual": float(c.rel_residual),
                        "queue_ms": float(c.queue_ms), "latency_ms": float(c.latency_ms),
                        "reserved_bytes": int(c.reserved_bytes), "cache_hit": bool(c.cache_hit)})
            _lib.check(self.ctx._L.bem_server_release(self.h, c.ticket))
        return out

    def wait(self, tickets, timeout_s=600.0):
        """Poll until every ticket in `tickets` has completed; returns {ticket: dict}."""
        import time as _time
        want, got = set(tickets), {}
        t_end = _time.time() + timeout_s
        while want - set(got):
            if _time.time() > t_end:
                raise TimeoutError(f"server requests not finished: {sorted(want - set(got))}")
            for r in self.poll(timeout_ms=200):
                got[r["ticket"]] = r
        return got

    def stats(self):
        st = _lib.ServerStats()
        _lib.check(self.ctx._L.bem_server_stats_get(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_ if k != "reserved"}

    def close(self):
        if getattr(self, "h", None):
            self.ctx._L.bem_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def inner_potentials(ctx: Context, x4, tets, tet_sv, precision="fp64", n_theta=0):
    """V 1_sigma(x) for arrays of apexes x4 [n,4] and panels tets [n,4,4] (t,x,y,z)."""
    x4 = np.ascontiguousarray(x4, dtype=np.float64).reshape(-1, 4)
    tets = np.ascontiguousarray(tets, dtype=np.float64).reshape(-1, 4, 4)
    sv = np.ascontiguousarray(tet_sv, dtype=np.int32).reshape(-1, 4)
    out = np.zeros(x4.shape[0])
    _lib.check(ctx._L.bem_inner_potentials(ctx.h, x4.shape[0], _lib.dptr(x4), _lib.dptr(tets), _lib.iptr(sv),
                                           _lib.PREC[precision], int(n_theta), _lib.dptr(out)))
    return out


# cudaStreamLegacy: the legacy default stream named explicitly (a NULL stream
# argument means the library context's own stream)
_CUDA_STREAM_LEGACY = 1


def _stream_ptr(stream):
    """cudaStream_t of `stream`; None gives torch's current stream, so that the
    library's work is ordered with the torch operations around the call."""
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return ctypes.c_void_p(h if h else _CUDA_STREAM_LEGACY)


class ClusterTree:
    """bem_cluster_tree: the host-side lit-panel search of Sec. 3.3 (binary
    cluster tree with bounding balls, Algorithm ApproximateLitLeaves). Needs
    no GPU. m: a space-time mesh of inputs (vertices stv_xyzt(), panels tets)."""

    def __init__(self, m, n_min=8):
        L = _lib.load()
        self._L = L
        X = np.ascontiguousarray(m.stv_xyzt(), dtype=np.float64)
        T = np.ascontiguousarray(m.tets, dtype=np.int32)
        h = ctypes.c_void_p()
        _lib.check(L.bem_cluster_tree_create(X.shape[0], _lib.dptr(X), T.shape[0], _lib.iptr(T), int(n_min),
                                             ctypes.byref(h)))
        self.h = h
        self.n_tet = T.shape[0]

    def info(self):
        a = np.zeros(2, dtype=np.int64)
        d = np.zeros(1, dtype=np.int32)
        _lib.check(self._L.bem_cluster_tree_info(self.h, _lib.lptr(a[0:1]), _lib.lptr(a[1:2]), _lib.iptr(d)))
        return {"nodes": int(a[0]), "leaves": int(a[1]), "depth": int(d[0])}

    def query(self, x):
        """X_N(x) (panel ids, caller numbering) and the number of clusters tested."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros(self.n_tet, dtype=np.int32)
        n, v = np.zeros(1, dtype=np.int64), np.zeros(1, dtype=np.int64)
        _lib.check(self._L.bem_cluster_tree_query(self.h, _lib.dptr(x), self.n_tet, _lib.iptr(out), _lib.lptr(n),
                                                  _lib.lptr(v)))
        return out[:int(n[0])].copy(), int(v[0])

    def close(self):
        if getattr(self, "h", None):
            self._L.bem_cluster_tree_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
