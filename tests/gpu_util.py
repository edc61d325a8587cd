"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and
compare it with the oracle element by element."""
from __future__ import annotations

import numpy as np

import oracle

# Tolerances.  Integer arrays and the unsmoothed points (a single FP32 rounding
# of the FP64 cell centre) must be bit-exact.  Smoothed offsets are FP32 and
# must be within 1e-5 voxel of the FP64 oracle (the stated target).  Smoothed
# world points are compared per axis within 1e-5 * spacing plus one FP32 ulp of
# the coordinate (the final rounding to float).
OFFSET_TOL = 1e-5


def run_gpu(labels, spacing=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0), selected=None, background=0, iterations=16,
            relaxation=0.5, constraint=1.0, on_device=True, sphere=False, triangulate=None, record_bytes=None):
    import torch

    from paper_2401_14906_gb300 import sn
    if on_device == "uploaded":  # copied ahead by sn_labels_upload, then sn_extract_labels
        up = sn.sn_labels_upload(np.ascontiguousarray(labels))
        m = sn.sn_extract_labels(up, spacing, origin, selected=selected, background=background)
        up.free()
    elif on_device == "offset":  # device labels one element into a buffer: off every 16-byte boundary
        a = np.ascontiguousarray(labels)
        flat = np.zeros(a.size + 1, a.dtype)
        flat[1:] = a.ravel()
        t = torch.from_numpy(flat.view({1: np.uint8, 2: np.int16, 4: np.int32}[a.dtype.itemsize])).cuda()
        t = t.view({1: torch.uint8, 2: torch.uint16, 4: torch.uint32}[a.dtype.itemsize])
        src = t[1:].view(a.shape)
        assert src.data_ptr() % 16 != 0
    elif on_device:
        t = torch.from_numpy(np.ascontiguousarray(labels).view(
            {1: np.uint8, 2: np.int16, 4: np.int32}[labels.dtype.itemsize])).cuda()
        t = t.view({1: torch.uint8, 2: torch.uint16, 4: torch.uint32}[labels.dtype.itemsize])
        src = t
    else:
        src = np.ascontiguousarray(labels)
    if on_device != "uploaded":
        m = sn.sn_extract(src, spacing, origin, selected=selected, background=background)
    if record_bytes is not None:
        assert sn.sn_mesh_record_bytes(m) == record_bytes
    ext = sn.sn_mesh_copy_to_host(m)
    ext["face_masks"] = sn.sn_mesh_face_masks_host(m)
    smo = None
    if iterations is not None:
        sn.sn_smooth_ex(m, iterations, relaxation, constraint, sphere=sphere)
        smo = sn.sn_mesh_copy_to_host(m)
        if triangulate:
            smo["triangles"] = {}
            for method in triangulate:
                sn.sn_triangulate(m, method)
                smo["triangles"][method] = sn.sn_mesh_triangles(m).cpu().numpy()
    m.free()
    return ext, smo


def compare_extract(gpu, ref):
    assert gpu["points"].shape[0] == ref.n_points
    assert gpu["quads"].shape[0] == ref.n_quads
    assert gpu["stencil_ids"].shape[0] == ref.n_stencil
    np.testing.assert_array_equal(gpu["points"], ref.points.astype(np.float32))
    np.testing.assert_array_equal(gpu["quads"], ref.quads)
    np.testing.assert_array_equal(gpu["quad_labels"], ref.quad_labels)
    np.testing.assert_array_equal(gpu["stencil_offsets"], ref.stencil_offsets)
    np.testing.assert_array_equal(gpu["stencil_ids"], ref.stencil_ids)
    np.testing.assert_array_equal(gpu["face_masks"], ref.face_masks)
    assert np.all(gpu["offsets"] == 0.0)


def compare_smooth(gpu, ref_off, ref_pts, spacing, constraint, sphere=False):
    off = gpu["offsets"].astype(np.float64)
    err = np.abs(off - ref_off)
    assert err.size == 0 or err.max() <= OFFSET_TOL, f"max offset error {err.max():.3e} voxel"
    h = 0.5 * constraint
    if sphere:
        assert np.all(np.sqrt((off ** 2).sum(axis=1)) <= h * (1 + 1e-6))
    else:
        assert np.all(np.abs(gpu["offsets"]) <= np.float32(h))
    pts = gpu["points"].astype(np.float64)
    tol = OFFSET_TOL * np.asarray(spacing)[None, :] + np.spacing(np.abs(ref_pts).astype(np.float32)).astype(
        np.float64)
    assert np.all(np.abs(pts - ref_pts) <= tol)


TRI_TIE = 1e-4  # relative margin below which a triangulation choice is a near-tie


def compare_triangles(gpu_tris, quads, ref_tris, ref_alt, ref_metric, exact):
    """Triangles must match the oracle's; on smoothed points a near-tie may go either way if the split is valid."""
    g = gpu_tris.reshape(-1, 2, 3)
    r = ref_tris.reshape(-1, 2, 3)
    same = np.all(g == r, axis=(1, 2))
    if exact:
        assert np.all(same), f"{np.count_nonzero(~same)} quads split differently"
        return
    m = ref_metric.astype(np.float64)
    scale = np.maximum(np.maximum(np.abs(m[:, 0]), np.abs(m[:, 1])), 1e-30)
    tie = (np.abs(m[:, 0] - m[:, 1]) <= TRI_TIE * scale) | np.isnan(m).any(axis=1)
    assert np.all(same | tie), f"{np.count_nonzero(~(same | tie))} quads split differently"
    # every differing (near-tie) quad must still be split along one of its diagonals
    q = quads[~same]
    alt = np.stack([q[:, 0], q[:, 1], q[:, 3], q[:, 1], q[:, 2], q[:, 3]], axis=1).reshape(-1, 2, 3)
    std = np.stack([q[:, 0], q[:, 1], q[:, 2], q[:, 0], q[:, 2], q[:, 3]], axis=1).reshape(-1, 2, 3)
    gd = g[~same]
    assert np.all(np.all(gd == alt, axis=(1, 2)) | np.all(gd == std, axis=(1, 2)))


def parity(labels, spacing=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0), selected=None, background=0, iterations=16,
           relaxation=0.5, constraint=1.0, on_device=True, sphere=False, triangulate=None, record_bytes=None):
    gpu_e, gpu_s = run_gpu(labels, spacing, origin, selected, background, iterations, relaxation, constraint,
                           on_device, sphere, triangulate, record_bytes)
    ref = oracle.extract(labels, spacing, origin, selected, background)
    compare_extract(gpu_e, ref)
    if iterations is not None:
        ref_off, ref_pts = oracle.smooth(ref, spacing, origin, iterations, relaxation, constraint, sphere=sphere)
        compare_smooth(gpu_s, ref_off, ref_pts, spacing, constraint, sphere)
        for method in (triangulate or ()):
            pts32 = (ref.points if iterations == 0 else ref_pts).astype(np.float32)
            tris, alt, metric = oracle.triangulate(pts32, ref.quads, method)
            compare_triangles(gpu_s["triangles"][method], ref.quads, tris, alt, metric, exact=iterations == 0)
    return ref
