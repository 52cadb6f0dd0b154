"""FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never imports it, and the two share no code: the only thing they
have in common is the plain input arrays produced by
``paper_2103_16841_gb300.inputs``.

The C source ``stbem_oracle.c`` states, function by function, which passage
of the paper it follows. This wrapper compiles it with gcc on first use (or
when ``build()`` is called) and exposes it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libstbem_oracle.so")
_SRC = os.path.join(_HERE, "stbem_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            lib.orc_inner.argtypes = [D, D]
            lib.orc_inner.restype = ctypes.c_double
            lib.orc_tet_geometry.argtypes = [D, D, D, D, D]
            lib.orc_midpoint_rule.argtypes = [ctypes.c_int, D]
            lib.orc_midpoint_rule.restype = ctypes.c_int
            lib.orc_pattern_pair.argtypes = [ctypes.c_int, D, I, ctypes.c_int, I, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.orc_pattern_pair.restype = ctypes.c_int
            lib.orc_entries.argtypes = [ctypes.c_int, D, I, ctypes.c_int, I, ctypes.c_int, ctypes.c_int, I, D,
                                        ctypes.c_int, ctypes.c_int]
            lib.orc_pattern_dense.argtypes = [ctypes.c_int, D, I, ctypes.c_int, I, ctypes.c_int, ctypes.POINTER(ctypes.c_ubyte)]
            lib.orc_pattern_rows.argtypes = [ctypes.c_int, D, I, ctypes.c_int, I, ctypes.c_int, ctypes.c_int, I,
                                             ctypes.c_int, I, I]
            lib.orc_rhs.argtypes = [ctypes.c_int, D, I, ctypes.c_int, I, ctypes.c_int, ctypes.c_int, D, D]
            lib.orc_lu_solve.argtypes = [ctypes.c_int, D, ctypes.c_int, D]
            lib.orc_lu_solve.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _threads(n):
    return int(n) if n else max(1, os.cpu_count() or 1)


def inner(x, tet):
    """V 1_sigma(x) for apex x=(t,x,y,z) and panel vertices tet[4][4] (with 1/(4 pi))."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    tet = np.ascontiguousarray(tet, dtype=np.float64)
    return lib.orc_inner(_d(x), _d(tet))


def tet_geometry(tet):
    lib = _load()
    tet = np.ascontiguousarray(tet, dtype=np.float64)
    nu = np.zeros(4)
    cn = np.zeros((4, 4))
    area = np.zeros(4)
    vol = np.zeros(1)
    lib.orc_tet_geometry(_d(tet), _d(nu), _d(cn), _d(area), _d(vol))
    return nu, cn, area, float(vol[0])


def midpoint_rule(m):
    lib = _load()
    xi = np.zeros(2 * m * m)
    n = lib.orc_midpoint_rule(m, _d(xi))
    return xi[: 2 * n].reshape(n, 2)


class Mesh:
    """Oracle view of a mesh: space-time vertices (t,x,y,z), spatial ids, tets."""

    def __init__(self, X, sv, tets):
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.sv = np.ascontiguousarray(sv, dtype=np.int32)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)

    @classmethod
    def from_spacetime(cls, m):
        return cls(m.stv_xyzt(), m.stv_sv, m.tets)

    @property
    def n_tet(self):
        return self.tets.shape[0]

    def _args(self):
        return (self.X.shape[0], _d(self.X), _i(self.sv), self.tets.shape[0], _i(self.tets))

    def pattern_pair(self, i, j, mq=3):
        return bool(_load().orc_pattern_pair(*self._args(), int(mq), int(i), int(j)))

    def pattern(self, mq=3):
        n = self.n_tet
        P = np.zeros((n, n), dtype=np.uint8)
        _load().orc_pattern_dense(*self._args(), int(mq), P.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        return P

    def pattern_rows(self, rows, mq=3, cap=None):
        """Admissible columns of the listed rows: list of int arrays."""
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        cap = int(cap or self.n_tet)
        counts = np.zeros(rows.shape[0], dtype=np.int32)
        cols = np.zeros((rows.shape[0], cap), dtype=np.int32)
        _load().orc_pattern_rows(*self._args(), int(mq), rows.shape[0], _i(rows), cap, _i(counts), _i(cols))
        return [cols[r, : counts[r]].copy() for r in range(rows.shape[0])]

    def entries(self, pairs, mq=3, use_pattern=True, nthreads=None):
        pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        out = np.zeros(pairs.shape[0])
        _load().orc_entries(*self._args(), int(mq), pairs.shape[0], _i(pairs), _d(out), int(bool(use_pattern)),
                            _threads(nthreads))
        return out

    def matrix(self, mq=3, use_pattern=True, nthreads=None):
        n = self.n_tet
        if use_pattern:
            P = self.pattern(mq)
            ij = np.argwhere(P != 0).astype(np.int32)
        else:
            ij = np.array([(i, j) for i in range(n) for j in range(n)], dtype=np.int32)
        vals = self.entries(ij, mq, use_pattern=False, nthreads=nthreads)
        A = np.zeros((n, n))
        A[ij[:, 0], ij[:, 1]] = vals
        return A

    def rhs(self, kind, params=None, nrhs=1):
        if params is not None:
            params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 5)
            nrhs = params.shape[0]
        b = np.zeros(self.n_tet * nrhs)
        pp = _d(params) if params is not None else ctypes.POINTER(ctypes.c_double)()
        _load().orc_rhs(*self._args(), int(kind), int(nrhs), pp, _d(b))
        return b.reshape(nrhs, self.n_tet).T.copy()


def lu_solve(A, B):
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    B = np.array(B, dtype=np.float64, copy=True)
    vec = B.ndim == 1
    B = np.ascontiguousarray(B.reshape(A.shape[0], -1))
    rc = _load().orc_lu_solve(A.shape[0], _d(A), B.shape[1], _d(B))
    if rc != 0:
        raise np.linalg.LinAlgError("singular matrix")
    return B[:, 0].copy() if vec else B
