"""Batched extraction + smoothing (sn_extract_smooth_batch) through the C ABI.

* A subset of the 256 seeded maps of uneven sizes (uint8/uint16, ellipsoids and
  Voronoi partitions, edges 32-256) against the FP64 oracle: integers bit-exact,
  offsets within 1e-5 voxel.
* The first 48 maps against the single-map calls: bit-identical outputs (the
  same kernels run; tile heights and streams change nothing), with and without
  the graph and the tuner.
* Graph mode over three calls of one layout with new contents (the update of
  the kept executable graph).
* One batch that takes every counting form (direct, staged, element-wise,
  two-kernel) and both emission forms (batched tiles, map by map), uint32
  included, against the oracle.
* Degenerate batches: empty, maps without surfaces, host and device labels mixed.
"""
import numpy as np
import pytest

import oracle
import sn_synth
from gpu_util import compare_extract, compare_smooth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_14906_gb300 import build
    build.build()


def _sn():
    from paper_2401_14906_gb300 import sn
    return sn


def _dev(labels):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(labels).view(
        {1: np.uint8, 2: np.int16, 4: np.int32}[labels.dtype.itemsize])).cuda()
    return t.view({1: torch.uint8, 2: torch.uint16, 4: torch.uint32}[labels.dtype.itemsize])


def _host(m):
    sn = _sn()
    out = sn.sn_mesh_copy_to_host(m)
    out["face_masks"] = sn.sn_mesh_face_masks_host(m)
    return out


def _subset():
    """The 10 smallest maps of the 256, plus map 0 and map 1."""
    vol = [int(np.prod(sn_synth.config5_params(i)[0])) for i in range(256)]
    idx = sorted(range(256), key=lambda i: vol[i])[:10]
    return sorted(set(idx) | {0, 1})


def test_batch_subset_matches_oracle():
    sn = _sn()
    idx = _subset()
    ws = [sn_synth.config5_map(i) for i in idx]
    meshes = sn.sn_extract_smooth_batch([_dev(w.labels) for w in ws], iterations=16, relaxation=0.5,
                                        constraint_distance=1.0)
    for w, m in zip(ws, meshes):
        got = _host(m)
        m.free()
        ref = oracle.extract(w.labels)
        assert got["points"].shape[0] == ref.n_points
        off, pts = oracle.smooth(ref, iterations=16, relaxation=0.5, constraint=1.0)
        compare_smooth(got, off, pts, (1.0, 1.0, 1.0), 1.0)
        np.testing.assert_array_equal(got["quads"], ref.quads)
        np.testing.assert_array_equal(got["quad_labels"], ref.quad_labels)
        np.testing.assert_array_equal(got["stencil_offsets"], ref.stencil_offsets)
        np.testing.assert_array_equal(got["stencil_ids"], ref.stencil_ids)
        np.testing.assert_array_equal(got["face_masks"], ref.face_masks)


def test_batch_unsmoothed_matches_oracle():
    sn = _sn()
    idx = _subset()[:6]
    ws = [sn_synth.config5_map(i) for i in idx]
    meshes = sn.sn_extract_smooth_batch([_dev(w.labels) for w in ws], iterations=0)
    for w, m in zip(ws, meshes):
        got = _host(m)
        m.free()
        compare_extract(got, oracle.extract(w.labels))


@pytest.mark.parametrize("graph,tune", [(True, True), (False, False), (True, False), (False, True)])
def test_batch_equals_single_map_calls(graph, tune):
    sn = _sn()
    ws = [sn_synth.config5_map(i) for i in range(48)]
    labs = [_dev(w.labels) for w in ws]
    meshes = sn.sn_extract_smooth_batch(labs, iterations=16, relaxation=0.5, constraint_distance=1.0, graph=graph,
                                        tune=tune)
    for t, m in zip(labs, meshes):
        got = _host(m)
        m.free()
        one = sn.sn_extract(t)
        sn.sn_smooth(one, 16, 0.5, 1.0)
        want = _host(one)
        one.free()
        for k in want:
            np.testing.assert_array_equal(got[k], want[k], err_msg=k)


def test_graph_batches_of_one_layout_with_new_contents():
    """Graph mode keeps one executable graph per layout and updates it with the
    next call's buffers and grid sizes: contents that differ between calls
    (rolled and relabelled volumes of the same shapes) still match single calls."""
    sn = _sn()
    base = [sn_synth.config5_map(i).labels for i in range(6)]
    for turn in range(3):
        labs = [np.ascontiguousarray(np.roll(b, 3 * turn + i, axis=i % 3)) for i, b in enumerate(base)]
        if turn == 2:
            labs = [np.where(b > 0, (b.astype(np.int64) * 7 + 1) % 250 + 1, 0).astype(b.dtype) for b in labs]
        dev = [_dev(b) for b in labs]
        meshes = sn.sn_extract_smooth_batch(dev, iterations=8, relaxation=0.5, constraint_distance=1.0, graph=True)
        for t, m in zip(dev, meshes):
            got = _host(m)
            m.free()
            one = sn.sn_extract(t)
            sn.sn_smooth(one, 8, 0.5, 1.0)
            want = _host(one)
            one.free()
            for k in want:
                np.testing.assert_array_equal(got[k], want[k], err_msg=k)


@pytest.mark.parametrize("graph,tune", [(False, False), (True, True)])
def test_batch_of_every_counting_and_emission_form(graph, tune):
    """uint32 maps alongside uint8/uint16 ones, chosen so that one batch takes every form of the batched kernels and
    their fallbacks (with the batch's 16 KB counting slots): rows on 16-byte boundaries (direct counting), rows off
    them and a map one element into its buffer (staged counting), uint32 rows of 6004 bytes (element-wise counting),
    of 8404 bytes (no counting tile fits: the two-kernel form; 66 words per row, so the emission runs map by map) and
    of 20 KB (the same).  Every map against the FP64 oracle."""
    import torch
    sn = _sn()
    rng = np.random.default_rng(77)
    maps = [sn_synth.ellipsoids((64, 40, 23), 4, 3.0, 10.0, np.uint32, seed=1),
            sn_synth.ellipsoids((67, 45, 19), 5, 3.0, 10.0, np.uint32, seed=2),
            sn_synth.ellipsoids((33, 30, 28), 3, 3.0, 9.0, np.uint8, seed=3),
            sn_synth.ellipsoids((75, 21, 17), 4, 2.5, 8.0, np.uint16, seed=4)]
    for nx, ny, nz in ((1501, 4, 5), (2101, 4, 5), (5000, 3, 3)):
        a = (rng.random((nz, ny, nx)) < 0.2).astype(np.uint32) * rng.integers(1, 9, size=(nz, ny, nx)).astype(
            np.uint32)
        maps.append(a)
    devs = [_dev(m) for m in maps]
    off = sn_synth.ellipsoids((48, 26, 20), 4, 3.0, 9.0, np.uint32, seed=5)
    flat = torch.zeros(off.size + 1, dtype=torch.int32, device="cuda")
    flat[1:] = torch.from_numpy(off.view(np.int32).ravel()).cuda()
    devs.append(flat.view(torch.uint32)[1:].view(off.shape))
    maps.append(off)
    meshes = sn.sn_extract_smooth_batch(devs, iterations=6, relaxation=0.5, constraint_distance=1.0, graph=graph,
                                        tune=tune)
    for lab, m in zip(maps, meshes):
        got = _host(m)
        m.free()
        ref = oracle.extract(lab)
        assert got["points"].shape[0] == ref.n_points and got["quads"].shape[0] == ref.n_quads
        for k, want in (("quads", ref.quads), ("quad_labels", ref.quad_labels), ("face_masks", ref.face_masks),
                        ("stencil_offsets", ref.stencil_offsets), ("stencil_ids", ref.stencil_ids)):
            np.testing.assert_array_equal(got[k], want, err_msg=k)
        off_ref, pts_ref = oracle.smooth(ref, iterations=6, relaxation=0.5, constraint=1.0)
        compare_smooth(got, off_ref, pts_ref, (1.0, 1.0, 1.0), 1.0)


def test_batch_of_degenerate_shapes():
    """Extents of 1 along each axis and along all three, with every label type, in one batch: the batched counting,
    scan and emission tiles at their smallest (one row, one slice, one word), against the oracle."""
    sn = _sn()
    rng = np.random.default_rng(123)
    shapes = [(1, 1, 1), (1, 7, 1), (9, 1, 1), (1, 1, 12), (3, 2, 1), (1, 5, 6), (33, 1, 4), (2, 40, 1)]
    maps = []
    for n, (nz, ny, nx) in enumerate(shapes):
        dt = (np.uint8, np.uint16, np.uint32)[n % 3]
        maps.append(rng.integers(0, 3, size=(nz, ny, nx)).astype(dt))
    meshes = sn.sn_extract_smooth_batch([_dev(m) for m in maps], iterations=3, relaxation=0.5,
                                        constraint_distance=1.0)
    for lab, m in zip(maps, meshes):
        got = _host(m)
        m.free()
        ref = oracle.extract(lab)
        assert got["points"].shape[0] == ref.n_points and got["quads"].shape[0] == ref.n_quads
        for k, want in (("quads", ref.quads), ("quad_labels", ref.quad_labels), ("face_masks", ref.face_masks),
                        ("stencil_offsets", ref.stencil_offsets), ("stencil_ids", ref.stencil_ids)):
            np.testing.assert_array_equal(got[k], want, err_msg=k)
        if ref.n_points:
            off_ref, pts_ref = oracle.smooth(ref, iterations=3, relaxation=0.5, constraint=1.0)
            compare_smooth(got, off_ref, pts_ref, (1.0, 1.0, 1.0), 1.0)


def test_degenerate_batches():
    sn = _sn()
    assert sn.sn_extract_smooth_batch([]) == []
    flat = np.full((5, 6, 7), 3, np.uint16)               # one label everywhere: no label change
    empty = np.zeros((4, 4, 4), np.uint8)                 # background only: nothing at all
    w = sn_synth.config5_map(3)
    maps = [flat, _dev(empty), _dev(w.labels), w.labels]  # host and device labels mixed
    meshes = sn.sn_extract_smooth_batch(maps, iterations=4)
    counts = [m.counts for m in meshes]
    assert counts[1] == (0, 0, 0)
    assert counts[2] == counts[3] and counts[2][0] > 0
    ref = oracle.extract(flat)
    assert counts[0] == (ref.n_points, ref.n_quads, ref.n_stencil)
    for m in meshes:
        m.free()


def test_batch_rejects_bad_arguments():
    sn = _sn()
    with pytest.raises(sn.SNError):
        sn.sn_extract_smooth_batch([np.zeros((2, 2, 2), np.uint8)], iterations=-1)
    with pytest.raises(sn.SNError):
        sn.sn_extract_smooth_batch([np.zeros((2, 2, 2), np.uint8)], relaxation=float("nan"))
