"""Oracle: plain sequential FP64 SurfaceNets on the CPU (``sn_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The library in
``paper_2401_14906_gb300`` never imports this package, and this package never
imports the library; they share no code.

``extract`` follows the paper's definitions (Sec. 2.1-2.3, 3.3) cell by cell and
edge by edge; ``smooth`` applies Eq. 1 with the double buffer of Sec. 2.4 and the
per-cell constraint box of Sec. 2.2.  The C source documents each step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sn_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_TYPE = {np.dtype(np.uint8): 1, np.dtype(np.uint16): 2, np.dtype(np.uint32): 4}


class _OrMesh(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_quads", ctypes.c_int64), ("n_stencil", ctypes.c_int64),
                ("points", ctypes.POINTER(ctypes.c_double)), ("cells", ctypes.POINTER(ctypes.c_int32)),
                ("quads", ctypes.POINTER(ctypes.c_int32)), ("quad_labels", ctypes.POINTER(ctypes.c_uint32)),
                ("stencil_offsets", ctypes.POINTER(ctypes.c_int64)),
                ("stencil_ids", ctypes.POINTER(ctypes.c_int32)),
                ("face_masks", ctypes.POINTER(ctypes.c_uint8))]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to this file with gcc (no-op when up to date)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.or_extract.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.POINTER(_OrMesh)]
            lib.or_extract.restype = ctypes.c_int
            lib.or_smooth.argtypes = [ctypes.POINTER(_OrMesh), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.or_triangulate.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.or_triangulate.restype = ctypes.c_int
            lib.or_smooth.restype = ctypes.c_int
            lib.or_free.argtypes = [ctypes.POINTER(_OrMesh)]
            lib.or_free.restype = None
            _lib = lib
    return _lib


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


class OracleMesh:
    """Extraction result in canonical order (numpy arrays, copied out of C)."""

    def __init__(self, m: _OrMesh, label_dtype):
        n, q, s = m.n_points, m.n_quads, m.n_stencil
        self.n_points, self.n_quads, self.n_stencil = int(n), int(q), int(s)
        self.points = _arr(m.points, 3 * n, np.float64).reshape(n, 3)
        self.cells = _arr(m.cells, 3 * n, np.int32).reshape(n, 3)
        self.quads = _arr(m.quads, 4 * q, np.int32).reshape(q, 4)
        self.quad_labels = _arr(m.quad_labels, 2 * q, np.uint32).reshape(q, 2).astype(label_dtype)
        self.stencil_offsets = _arr(m.stencil_offsets, n + 1, np.int64)
        self.stencil_ids = _arr(m.stencil_ids, s, np.int32)
        self.face_masks = _arr(m.face_masks, n, np.uint8)


def extract(labels: np.ndarray, spacing=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0), selected=None,
            background=0) -> OracleMesh:
    """Steps 1-5 on a (nz, ny, nx) label array; returns an OracleMesh."""
    lib = _load()
    lab = np.ascontiguousarray(labels)
    if lab.dtype not in _TYPE or lab.ndim != 3:
        raise ValueError("labels must be a 3-D uint8/uint16/uint32 array")
    nz, ny, nx = lab.shape
    dims = (ctypes.c_int64 * 3)(nx, ny, nz)
    sp = (ctypes.c_double * 3)(*[float(s) for s in spacing])
    org = (ctypes.c_double * 3)(*[float(o) for o in origin])
    sel_ptr, nsel = None, 0
    if selected is not None:
        sel = np.ascontiguousarray(np.asarray(selected, dtype=np.uint32))
        sel_ptr = sel.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        nsel = int(sel.size)
    m = _OrMesh()
    rc = lib.or_extract(lab.ctypes.data, _TYPE[lab.dtype], dims, sp, org, sel_ptr, nsel, int(background),
                        ctypes.byref(m))
    if rc != 0:
        raise RuntimeError(f"or_extract failed with code {rc}")
    try:
        return OracleMesh(m, lab.dtype)
    finally:
        lib.or_free(ctypes.byref(m))


def smooth(mesh: OracleMesh, spacing=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0), iterations=16, relaxation=0.5,
           constraint=1.0, sphere=False):
    """Step 6 (Eq. 1, double-buffered; box or sphere constraint).  Returns (offsets, points), FP64 (n, 3)."""
    lib = _load()
    m = _OrMesh()
    m.n_points, m.n_quads, m.n_stencil = mesh.n_points, mesh.n_quads, mesh.n_stencil
    cells = np.ascontiguousarray(mesh.cells, dtype=np.int32)
    so = np.ascontiguousarray(mesh.stencil_offsets, dtype=np.int64)
    si = np.ascontiguousarray(mesh.stencil_ids, dtype=np.int32)
    if si.size == 0:
        si = np.zeros(1, dtype=np.int32)
    m.cells = cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    m.stencil_offsets = so.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    m.stencil_ids = si.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    n = mesh.n_points
    off = np.zeros((max(n, 1), 3), dtype=np.float64)
    pts = np.zeros((max(n, 1), 3), dtype=np.float64)
    sp = (ctypes.c_double * 3)(*[float(s) for s in spacing])
    org = (ctypes.c_double * 3)(*[float(o) for o in origin])
    rc = lib.or_smooth(ctypes.byref(m), sp, org, int(iterations), float(relaxation), float(constraint),
                       1 if sphere else 0, off.ctypes.data, pts.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"or_smooth failed with code {rc}")
    return off[:n], pts[:n]


TRI_METHODS = {"greedy": 0, "shortest": 1, "min_area": 2, "coplanar": 3}


def triangulate(points, quads, method="shortest"):
    """Step 7 on float32 points (n, 3) and quads (q, 4).

    Returns (triangles (2q, 3) int32, alt (q,) bool: split along v1-v3, metrics (q, 2) float32 compared)."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float32)
    qd = np.ascontiguousarray(quads, dtype=np.int32)
    nq = qd.shape[0]
    tris = np.zeros((max(2 * nq, 1), 3), dtype=np.int32)
    alt = np.zeros(max(nq, 1), dtype=np.uint8)
    m02 = np.zeros(max(nq, 1), dtype=np.float32)
    m13 = np.zeros(max(nq, 1), dtype=np.float32)
    rc = lib.or_triangulate(pts.ctypes.data if pts.size else None, qd.ctypes.data if qd.size else None, nq,
                            TRI_METHODS[method], tris.ctypes.data, alt.ctypes.data, m02.ctypes.data, m13.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"or_triangulate failed with code {rc}")
    return tris[:2 * nq], alt[:nq].astype(bool), np.stack([m02[:nq], m13[:nq]], axis=1)
