"""Thin ctypes binding of libsn.so with the same names as the C ABI (include/sn.h).

Argument marshalling only: every step of extraction and smoothing runs in the
library's CUDA kernels.  PyTorch is used for device memory and streams.  If
libsn.so is missing or cannot be loaded, every call raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsn.so")

SN_OK, SN_EINVAL, SN_ENOMEM, SN_EOVERFLOW, SN_ECUDA, SN_ETIMEOUT = range(6)
SN_U8, SN_U16, SN_U32 = 1, 2, 4

_lock = threading.Lock()
_lib = None


class SNError(RuntimeError):
    def __init__(self, status, detail):
        self.status = status
        super().__init__(f"{status_string(status)} ({detail})" if detail else status_string(status))


class sn_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class sn_slab_part(ctypes.Structure):
    _fields_ = [("first_point", ctypes.c_int64), ("n_points", ctypes.c_int64), ("first_quad", ctypes.c_int64),
                ("n_quads", ctypes.c_int64), ("first_stencil", ctypes.c_int64), ("n_stencil", ctypes.c_int64)]


# every symbol declared in include/sn.h, with its ctypes signature
_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "sn_extract": (ctypes.c_int, [_P, ctypes.c_int, _I64P, _DP, _DP, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int64,
                                  ctypes.c_uint32, _P, ctypes.POINTER(_P)]),
    "sn_labels_upload": (ctypes.c_int, [_P, ctypes.c_int, _I64P, ctypes.POINTER(_P)]),
    "sn_extract_labels": (ctypes.c_int, [_P, _DP, _DP, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int64,
                                         ctypes.c_uint32, _P, ctypes.POINTER(_P)]),
    "sn_labels_wait": (ctypes.c_int, [_P]),
    "sn_labels_free": (None, [_P, _P]),
    "sn_smooth": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_float, ctypes.c_float]),
    "sn_smooth_ex": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_int]),
    "sn_triangulate": (ctypes.c_int, [_P, ctypes.c_int]),
    "sn_mesh_triangles": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "sn_mesh_counts": (ctypes.c_int, [_P, _I64P, _I64P, _I64P]),
    "sn_mesh_device_arrays": (ctypes.c_int, [_P] + [ctypes.POINTER(_P)] * 6),
    "sn_mesh_face_masks": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "sn_mesh_cells": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "sn_mesh_record_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "sn_mesh_copy_to_host": (ctypes.c_int, [_P] + [_P] * 6),
    "sn_mesh_copy_to_host_async": (ctypes.c_int, [_P] + [_P] * 6),
    "sn_mesh_wait": (ctypes.c_int, [_P]),
    "sn_free": (None, [_P]),
    "sn_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sn_last_error": (ctypes.c_char_p, []),
    "sn_smooth_static": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                        _P, _P]),
    "sn_extract_smooth_batch": (ctypes.c_int, [ctypes.c_int64, _P, _P, _I64P, _DP, _DP, ctypes.c_uint32,
                                               ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_int, _P,
                                               ctypes.POINTER(_P)]),
    "sn_learner_create": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "sn_learner_free": (None, [_P]),
    "sn_learner_set_params": (ctypes.c_int, [_P, _P]),
    "sn_learner_get_params": (ctypes.c_int, [_P, _P]),
    "sn_learner_add_examples": (ctypes.c_int, [_P, _P, ctypes.c_float]),
    "sn_learner_n_examples": (ctypes.c_int, [_P, _I64P]),
    "sn_learner_set_engine": (ctypes.c_int, [_P, ctypes.c_int]),
    "sn_learner_train": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)]),
    "sn_smooth_learned": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_int]),
    "sn_learn_features": (ctypes.c_int, [_P, ctypes.c_float, _P]),
    "sn_learn_forward": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "sn_learn_gradient": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P]),
    "sn_learner_step": (ctypes.c_int, [_P, _P, ctypes.c_float, ctypes.c_float]),
    "sn_profile_enable": (None, [ctypes.c_int]),
    "sn_trim_memory": (ctypes.c_int, []),
    "sn_profile_read": (ctypes.c_int, [ctypes.POINTER(sn_kernel_time), ctypes.c_int, ctypes.c_int]),
    "sn_slab_part_of": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.POINTER(sn_slab_part)]),
    "sn_slab_stitch": (ctypes.c_int, [_P, ctypes.POINTER(sn_slab_part), ctypes.c_int64, ctypes.c_int64, _P, _P, _P,
                                      _P]),
    "sn_debug_set_spin_limit": (None, [ctypes.c_int]),
    "sn_debug_fail_allocation": (None, [ctypes.c_int64]),
    "sn_debug_set_point_limit": (None, [ctypes.c_int64]),
    "sn_debug_reset": (None, []),
}


def load(path: str | None = None):
    """Load libsn.so (build it first with paper_2401_14906_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libsn.so not found at {p}: build it with "
                                   "`python -m paper_2401_14906_gb300.build` (nvcc, sm_103a)")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(s):
    return load().sn_status_string(int(s)).decode()


def sn_last_error():
    return load().sn_last_error().decode()


def _check(rc):
    if rc != SN_OK:
        raise SNError(rc, sn_last_error())


_NP_TYPE = {np.dtype(np.uint8): SN_U8, np.dtype(np.uint16): SN_U16, np.dtype(np.uint32): SN_U32}
_NP_OF = {SN_U8: np.uint8, SN_U16: np.uint16, SN_U32: np.uint32}


def _torch():
    import torch
    return torch


def _label_info(labels):
    """(pointer, type code, dims (nx,ny,nz), is_cuda, keepalive) for a (nz,ny,nx) array/tensor."""
    if isinstance(labels, np.ndarray):
        a = np.ascontiguousarray(labels)
        if a.dtype not in _NP_TYPE or a.ndim != 3:
            raise ValueError("labels must be a 3-D uint8/uint16/uint32 array shaped (nz, ny, nx)")
        nz, ny, nx = a.shape
        return a.ctypes.data, _NP_TYPE[a.dtype], (nx, ny, nz), False, a
    torch = _torch()
    t = labels
    tmap = {torch.uint8: SN_U8, torch.uint16: SN_U16, torch.uint32: SN_U32}
    if t.dtype not in tmap or t.dim() != 3:
        raise ValueError("labels must be a 3-D uint8/uint16/uint32 tensor shaped (nz, ny, nx)")
    if not t.is_contiguous():
        t = t.contiguous()
    nz, ny, nx = t.shape
    return t.data_ptr(), tmap[t.dtype], (nx, ny, nz), t.is_cuda, t


def _stream_handle(stream, is_cuda):
    if stream is None:
        if is_cuda:
            return _torch().cuda.current_stream().cuda_stream
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Mesh:
    """Owner of an sn_mesh*; freed by free() or when garbage-collected."""

    def __init__(self, handle, label_type, dims, spacing, origin):
        self._h = ctypes.c_void_p(handle)
        self.label_type = label_type
        self.dims = dims
        self.spacing = tuple(spacing)
        self.origin = tuple(origin)

    @property
    def handle(self):
        if not self._h:
            raise ValueError("mesh has been freed")
        return self._h

    def free(self):
        if self._h:
            load().sn_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def counts(self):
        return sn_mesh_counts(self)


def sn_extract(labels, spacing=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0), selected=None, background=0,
               stream=None) -> Mesh:
    """Extract the shared quad mesh of a (nz, ny, nx) label map (device tensor or host array)."""
    lib = load()
    ptr, tcode, dims, is_cuda, keep = _label_info(labels)
    d = (ctypes.c_int64 * 3)(*dims)
    sp = (ctypes.c_double * 3)(*[float(s) for s in spacing])
    org = (ctypes.c_double * 3)(*[float(o) for o in origin])
    sel_ptr, nsel, sel_keep = None, 0, None
    if selected is not None:
        sel_keep = np.ascontiguousarray(np.asarray(selected, dtype=np.uint32))
        sel_ptr = sel_keep.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        nsel = int(sel_keep.size)
    out = ctypes.c_void_p()
    rc = lib.sn_extract(ctypes.c_void_p(ptr), tcode, d, sp, org, sel_ptr, nsel, int(background),
                        ctypes.c_void_p(_stream_handle(stream, is_cuda)), ctypes.byref(out))
    del keep, sel_keep
    _check(rc)
    return Mesh(out.value, tcode, dims, spacing, origin)


class Labels:
    """Owner of an sn_labels* (a label map copied to the device ahead of its extraction).  The host
    array or pinned tensor it was uploaded from is kept alive until free()."""

    def __init__(self, handle, label_type, dims, keep):
        self._h = ctypes.c_void_p(handle)
        self.label_type = label_type
        self.dims = dims
        self._keep = keep

    @property
    def handle(self):
        if not self._h:
            raise ValueError("labels have been freed")
        return self._h

    def wait(self):
        _check(load().sn_labels_wait(self.handle))

    def free(self, stream=None):
        """Stream-ordered release: after the copy and the work already queued on `stream`
        (default: torch's current stream)."""
        if self._h:
            load().sn_labels_free(self._h, ctypes.c_void_p(_stream_handle(stream, True)))
            self._h = ctypes.c_void_p(None)
            self._keep = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sn_labels_upload(labels) -> Labels:
    """Start copying a host (nz, ny, nx) label map (numpy array, or a pinned CPU tensor for an
    asynchronous copy) to the device; returns at once."""
    ptr, tcode, dims, is_cuda, keep = _label_info(labels)
    if is_cuda:
        raise ValueError("sn_labels_upload takes host labels; pass device labels to sn_extract directly")
    out = ctypes.c_void_p()
    _check(load().sn_labels_upload(ctypes.c_void_p(ptr), tcode, (ctypes.c_int64 * 3)(*dims), ctypes.byref(out)))
    return Labels(out.value, tcode, dims, keep)


def sn_extract_labels(labels: Labels, spacing=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0), selected=None, background=0,
                      stream=None) -> Mesh:
    """sn_extract over an uploaded map; the stream waits for the upload on the device."""
    sp = (ctypes.c_double * 3)(*[float(s) for s in spacing])
    org = (ctypes.c_double * 3)(*[float(o) for o in origin])
    sel_ptr, nsel, sel_keep = None, 0, None
    if selected is not None:
        sel_keep = np.ascontiguousarray(np.asarray(selected, dtype=np.uint32))
        sel_ptr = sel_keep.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        nsel = int(sel_keep.size)
    out = ctypes.c_void_p()
    rc = load().sn_extract_labels(labels.handle, sp, org, sel_ptr, nsel, int(background),
                                  ctypes.c_void_p(_stream_handle(stream, True)), ctypes.byref(out))
    del sel_keep
    _check(rc)
    return Mesh(out.value, labels.label_type, labels.dims, spacing, origin)


SN_CONSTRAINT_BOX, SN_CONSTRAINT_SPHERE = 0, 1
SN_TRI = {"greedy": 0, "shortest": 1, "min_area": 2, "coplanar": 3}


def sn_smooth(mesh: Mesh, iterations=16, relaxation=0.5, constraint_distance=1.0):
    _check(load().sn_smooth(mesh.handle, int(iterations), float(relaxation), float(constraint_distance)))


def sn_smooth_ex(mesh: Mesh, iterations=16, relaxation=0.5, constraint_distance=1.0, sphere=False):
    _check(load().sn_smooth_ex(mesh.handle, int(iterations), float(relaxation), float(constraint_distance),
                               SN_CONSTRAINT_SPHERE if sphere else SN_CONSTRAINT_BOX))


def sn_triangulate(mesh: Mesh, method="shortest"):
    _check(load().sn_triangulate(mesh.handle, SN_TRI[method]))


def sn_mesh_triangles(mesh: Mesh):
    """The mesh's triangles as a borrowed torch tensor (2*n_quads, 3), or None before sn_triangulate."""
    torch = _torch()
    p = ctypes.c_void_p()
    _check(load().sn_mesh_triangles(mesh.handle, ctypes.byref(p)))
    if not p.value:
        return None
    _, q, _ = sn_mesh_counts(mesh)
    return torch.as_tensor(_CudaArray(p.value, (2 * q, 3), "<i4"), device="cuda")


def sn_mesh_counts(mesh: Mesh):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().sn_mesh_counts(mesh.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def sn_mesh_copy_to_host(mesh: Mesh):
    """All output arrays as numpy arrays (waits for the mesh's stream)."""
    n, q, s = sn_mesh_counts(mesh)
    out = {
        "points": np.empty((n, 3), np.float32),
        "quads": np.empty((q, 4), np.int32),
        "quad_labels": np.empty((q, 2), _NP_OF[mesh.label_type]),
        "stencil_offsets": np.empty(n + 1, np.int64),
        "stencil_ids": np.empty(s, np.int32),
        "offsets": np.empty((n, 3), np.float32),
    }
    order = ["points", "quads", "quad_labels", "stencil_offsets", "stencil_ids", "offsets"]
    _check(load().sn_mesh_copy_to_host(mesh.handle, *[ctypes.c_void_p(out[k].ctypes.data) for k in order]))
    return out


def sn_mesh_copy_to_host_async(mesh: Mesh, out):
    """Starts copying into the caller's pinned buffers `out` (a dict with any of the keys of
    sn_mesh_copy_to_host, numpy or torch pinned); sn_mesh_wait(mesh) completes it."""
    order = ["points", "quads", "quad_labels", "stencil_offsets", "stencil_ids", "offsets"]

    def ptr(v):
        if v is None:
            return None
        return ctypes.c_void_p(v.data_ptr() if hasattr(v, "data_ptr") else v.ctypes.data)
    _check(load().sn_mesh_copy_to_host_async(mesh.handle, *[ptr(out.get(k)) for k in order]))


def sn_mesh_wait(mesh: Mesh):
    _check(load().sn_mesh_wait(mesh.handle))


class _CudaArray:
    """Zero-copy view of a borrowed device pointer for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def sn_mesh_device_arrays(mesh: Mesh):
    """Borrowed device arrays as torch tensors (valid until the mesh is freed)."""
    torch = _torch()
    n, q, s = sn_mesh_counts(mesh)
    ptrs = [ctypes.c_void_p() for _ in range(6)]
    _check(load().sn_mesh_device_arrays(mesh.handle, *[ctypes.byref(p) for p in ptrs]))
    lt = {SN_U8: "|u1", SN_U16: "<u2", SN_U32: "<u4"}[mesh.label_type]
    spec = [("points", (n, 3), "<f4"), ("quads", (q, 4), "<i4"), ("quad_labels", (q, 2), lt),
            ("stencil_offsets", (n + 1,), "<i8"), ("stencil_ids", (s,), "<i4"), ("offsets", (n, 3), "<f4")]
    out = {}
    for (name, shape, ts), p in zip(spec, ptrs):
        out[name] = torch.as_tensor(_CudaArray(p.value, shape, ts), device="cuda")
    fm = ctypes.c_void_p()
    _check(load().sn_mesh_face_masks(mesh.handle, ctypes.byref(fm)))
    out["face_masks"] = torch.as_tensor(_CudaArray(fm.value, (n,), "|u1"), device="cuda")
    return out


def sn_mesh_cells(mesh: Mesh):
    """Each point's generating cell as a borrowed int64 tensor (n_points, 3) of (cx, cy, cz), unpacked on the device."""
    torch = _torch()
    p = ctypes.c_void_p()
    _check(load().sn_mesh_cells(mesh.handle, ctypes.byref(p)))
    n, _, _ = sn_mesh_counts(mesh)
    packed = torch.as_tensor(_CudaArray(p.value, (n,), "<i8"), device="cuda")
    m21 = (1 << 21) - 1
    return torch.stack([(packed & m21) - 1, ((packed >> 21) & m21) - 1, ((packed >> 42) & m21) - 1], dim=1)


def sn_mesh_face_masks_host(mesh: Mesh):
    t = sn_mesh_device_arrays(mesh)["face_masks"]
    return t.cpu().numpy()


SN_STATIC_MAX_POINTS = 1048576


def sn_smooth_static(stencil_offsets, stencil_ids, face_masks, n_points, iterations, relaxation,
                     constraint_distance, offsets, stream=None):
    """Smoothing sweeps on caller-owned device tensors, allocating nothing (see include/sn.h)."""
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    _check(load().sn_smooth_static(ptr(stencil_offsets), ptr(stencil_ids), ptr(face_masks), int(n_points),
                                   int(iterations), float(relaxation), float(constraint_distance), ptr(offsets),
                                   ctypes.c_void_p(_stream_handle(stream, True))))


def sn_profile_enable(on=True):
    load().sn_profile_enable(1 if on else 0)


def sn_trim_memory():
    """Return the library's unused pooled device memory on the current device to the system."""
    _check(load().sn_trim_memory())


def sn_profile_read(reset=False):
    """{kernel name: (launches, total_ms)} accumulated since the last reset."""
    lib = load()
    buf = (sn_kernel_time * 64)()
    n = lib.sn_profile_read(buf, 64, 1 if reset else 0)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n, 64))}


# ------------------------------------------------------------ batched maps
SN_BATCH_GRAPH, SN_BATCH_TUNE = 1, 2


def sn_extract_smooth_batch(maps, spacing=None, origin=None, background=0, iterations=16, relaxation=0.5,
                            constraint_distance=1.0, graph=True, tune=True, stream=None):
    """Extract and smooth a list of (nz, ny, nx) label maps (device tensors or host arrays) in one call.

    Returns a list of Mesh objects, one per map."""
    lib = load()
    n = len(maps)
    infos = [_label_info(m) for m in maps]
    ptrs = (ctypes.c_void_p * max(n, 1))(*[ctypes.c_void_p(i[0]) for i in infos])
    types = (ctypes.c_int * max(n, 1))(*[i[1] for i in infos])
    dims = (ctypes.c_int64 * max(3 * n, 1))(*[d for i in infos for d in i[2]])
    sp = org = None
    if spacing is not None:
        sp = (ctypes.c_double * (3 * n))(*[float(v) for s3 in spacing for v in s3])
    if origin is not None:
        org = (ctypes.c_double * (3 * n))(*[float(v) for o3 in origin for v in o3])
    out = (ctypes.c_void_p * max(n, 1))()
    flags = (SN_BATCH_GRAPH if graph else 0) | (SN_BATCH_TUNE if tune else 0)
    is_cuda = any(i[3] for i in infos)
    rc = lib.sn_extract_smooth_batch(n, ctypes.cast(ptrs, ctypes.c_void_p), ctypes.cast(types, ctypes.c_void_p),
                                     dims, sp, org, int(background), int(iterations), float(relaxation),
                                     float(constraint_distance), flags,
                                     ctypes.c_void_p(_stream_handle(stream, is_cuda or True)), out)
    keep = infos  # noqa: F841 -- the label buffers must live until the call has enqueued its work
    _check(rc)
    res = []
    for k in range(n):
        res.append(Mesh(out[k], infos[k][1], infos[k][2], spacing[k] if spacing is not None else (1.0, 1.0, 1.0),
                        origin[k] if origin is not None else (0.0, 0.0, 0.0)))
    return res


# ------------------------------------------------------- learned proposal
SN_LEARN_FEATURES, SN_LEARN_PARAMS = 32, 6467


class Learner:
    """Owner of an sn_learner* (parameters, AdamW state, examples on the device)."""

    def __init__(self, stream=None):
        out = ctypes.c_void_p()
        _check(load().sn_learner_create(ctypes.c_void_p(_stream_handle(stream, True)), ctypes.byref(out)))
        self._h = out

    @property
    def handle(self):
        if not self._h:
            raise ValueError("learner has been freed")
        return self._h

    def free(self):
        if self._h:
            load().sn_learner_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sn_learner_create(stream=None) -> Learner:
    return Learner(stream)


def sn_learner_set_params(learner: Learner, params):
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    if p.size != SN_LEARN_PARAMS:
        raise ValueError(f"expected {SN_LEARN_PARAMS} parameters")
    _check(load().sn_learner_set_params(learner.handle, ctypes.c_void_p(p.ctypes.data)))


def sn_learner_get_params(learner: Learner):
    p = np.empty(SN_LEARN_PARAMS, np.float32)
    _check(load().sn_learner_get_params(learner.handle, ctypes.c_void_p(p.ctypes.data)))
    return p


def sn_learner_add_examples(learner: Learner, mesh: Mesh, constraint_distance=1.0):
    _check(load().sn_learner_add_examples(learner.handle, mesh.handle, float(constraint_distance)))


SN_LEARN_ENGINE_MMA_SYNC, SN_LEARN_ENGINE_TCGEN05 = 0, 1


def sn_learner_set_engine(learner: Learner, engine):
    """engine: "mma_sync" (default) or "tcgen05" -- the tensor-core kernel of the proposal."""
    code = {"mma_sync": SN_LEARN_ENGINE_MMA_SYNC, "tcgen05": SN_LEARN_ENGINE_TCGEN05}.get(engine, engine)
    _check(load().sn_learner_set_engine(learner.handle, int(code)))


def sn_learner_n_examples(learner: Learner):
    n = ctypes.c_int64()
    _check(load().sn_learner_n_examples(learner.handle, ctypes.byref(n)))
    return n.value


def sn_learner_train(learner: Learner, epochs, batch, lr, weight_decay=0.0, seed=0):
    """Returns the mean squared error of the last minibatch."""
    loss = ctypes.c_float()
    _check(load().sn_learner_train(learner.handle, int(epochs), int(batch), float(lr), float(weight_decay),
                                   int(seed) & (2 ** 64 - 1), ctypes.byref(loss)))
    return loss.value


def sn_smooth_learned(mesh: Mesh, learner: Learner, corrections=2, relaxation=0.5, constraint_distance=1.0,
                      sphere=False):
    _check(load().sn_smooth_learned(mesh.handle, learner.handle, int(corrections), float(relaxation),
                                    float(constraint_distance), SN_CONSTRAINT_SPHERE if sphere else SN_CONSTRAINT_BOX))


def sn_learn_features(mesh: Mesh, constraint_distance=1.0):
    """Features of every point: a device int16 tensor (n_points, 32) holding BF16 bit patterns."""
    torch = _torch()
    n, _, _ = sn_mesh_counts(mesh)
    x = torch.empty((max(n, 1), SN_LEARN_FEATURES), dtype=torch.int16, device="cuda")
    _check(load().sn_learn_features(mesh.handle, float(constraint_distance), ctypes.c_void_p(x.data_ptr())))
    return x[:n]


def sn_learn_forward(learner: Learner, x):
    """y (n, 3) float32 device tensor = MLP(x) for device BF16-bit rows x (n, 32)."""
    torch = _torch()
    x = x.contiguous()
    n = x.shape[0]
    y = torch.empty((max(n, 1), 3), dtype=torch.float32, device="cuda")
    _check(load().sn_learn_forward(learner.handle, ctypes.c_void_p(x.data_ptr()), n, ctypes.c_void_p(y.data_ptr())))
    return y[:n]


def sn_learn_gradient(learner: Learner, x, t):
    """(gradient float32 device tensor (SN_LEARN_PARAMS,), sum of squared errors) for rows x, targets t (n, 3)."""
    torch = _torch()
    x, t = x.contiguous(), t.contiguous().float()
    g = torch.zeros(SN_LEARN_PARAMS, dtype=torch.float32, device="cuda")
    sse = torch.zeros(1, dtype=torch.float32, device="cuda")
    _check(load().sn_learn_gradient(learner.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                    x.shape[0], ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(sse.data_ptr())))
    return g, sse


def sn_learner_step(learner: Learner, grads, lr, weight_decay=0.0):
    _check(load().sn_learner_step(learner.handle, ctypes.c_void_p(grads.data_ptr()), float(lr), float(weight_decay)))


# ------------------------------------------------------------ failure injection
def sn_debug_set_spin_limit(n: int):
    """Polls after which the row scan's look-back gives up (< 0: at once); see include/sn.h."""
    load().sn_debug_set_spin_limit(int(n))


def sn_debug_fail_allocation(k: int):
    """Make the k-th library allocation from now fail (k < 0: off)."""
    load().sn_debug_fail_allocation(int(k))


def sn_debug_set_point_limit(n: int):
    """Extractions of more than n points return SN_EOVERFLOW (n < 0: INT32_MAX)."""
    load().sn_debug_set_point_limit(int(n))


def sn_debug_reset():
    """Restore the default spin limit, allocation behaviour and point limit."""
    load().sn_debug_reset()


def sn_mesh_record_bytes(mesh) -> int:
    """Bytes per point of the sweeps' neighbour record: 8, 12, or 0 (the CSR stencil)."""
    b = ctypes.c_int()
    _check(load().sn_mesh_record_bytes(mesh.handle, ctypes.byref(b)))
    return b.value


# ------------------------------------------------------------------ z-slabs
def sn_slab_part_of(mesh, cz_lo, cz_hi, k_lo, k_hi):
    """Owned ranges of a slab mesh: points of cell slices [cz_lo, cz_hi), quads of first sample slices
    [k_lo, k_hi) (slab coordinates).  Returns an sn_slab_part."""
    part = sn_slab_part()
    _check(load().sn_slab_part_of(mesh.handle, int(cz_lo), int(cz_hi), int(k_lo), int(k_hi), ctypes.byref(part)))
    return part


def sn_slab_stitch(mesh, part, global_first_point, global_first_stencil, stream=None):
    """The owned quads, stencil offsets and stencil ids with global ids, as new device tensors."""
    torch = _torch()
    quads = torch.empty((part.n_quads, 4), dtype=torch.int32, device="cuda")
    so = torch.empty(part.n_points, dtype=torch.int64, device="cuda")
    si = torch.empty(part.n_stencil, dtype=torch.int32, device="cuda")
    _check(load().sn_slab_stitch(mesh.handle, ctypes.byref(part), int(global_first_point), int(global_first_stencil),
                                 ctypes.c_void_p(quads.data_ptr()), ctypes.c_void_p(so.data_ptr()),
                                 ctypes.c_void_p(si.data_ptr()), ctypes.c_void_p(_stream_handle(stream, True))))
    return quads, so, si
