"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Integer outputs and unsmoothed points are bit-exact; smoothed offsets are
within 1e-5 voxel.  Sizes span several 32-bit words per row, ragged row tails,
every label width, selected-label modes and the degenerate cases.
"""
import numpy as np
import pytest

import oracle
import sn_synth
from gpu_util import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_14906_gb300 import build
    build.build()


def test_config1_full():
    w = sn_synth.config1()
    ref = parity(w.labels, w.spacing, w.origin, iterations=w.iterations, relaxation=w.relaxation,
                 constraint=w.constraint)
    assert ref.n_points > 5000


@pytest.mark.parametrize("nx", [1, 2, 31, 32, 33, 63, 64, 65, 100, 127, 129, 1023, 1024, 1025])
def test_ragged_rows(nx):
    rng = np.random.default_rng(nx)
    lab = (rng.random((5, 4, nx)) < 0.3).astype(np.uint16) * rng.integers(1, 5, size=(5, 4, nx)).astype(np.uint16)
    parity(lab, iterations=5)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.uint32])
@pytest.mark.parametrize("seed", range(4))
def test_random_maps(dtype, seed):
    rng = np.random.default_rng(1000 + seed)
    shape = tuple(int(s) for s in rng.integers(1, 40, size=3))
    lab = rng.integers(0, 4, size=shape).astype(dtype)
    parity(lab, spacing=(0.7, 1.3, 2.0), origin=(-5.0, 3.0, 100.0), iterations=7, relaxation=0.6, constraint=0.8)


@pytest.mark.parametrize("nx", [16, 48, 64, 128])
def test_uint8_rows_on_16_byte_boundaries(nx):
    """uint8 maps whose rows are 16-byte aligned take the packed counting form."""
    lab = sn_synth.ellipsoids((nx, 37, 29), 5, 3.0, 11.0, np.uint8, seed=nx)
    parity(lab, iterations=6)


@pytest.mark.parametrize("dtype,nx", [(np.uint8, 80), (np.uint8, 208), (np.uint16, 72), (np.uint16, 200),
                                      (np.uint16, 360), (np.uint32, 68), (np.uint32, 164)])
def test_packed_rows_with_words_not_dividing_a_warp(dtype, nx):
    """Rows on 16-byte boundaries (the packed counting form) with 3-12 words per row: a warp's lanes span row
    ends, so the sample after a word comes from the next lane or, for the warp's last lane, from shared memory."""
    rng = np.random.default_rng(nx)
    lab = rng.integers(0, 3, size=(6, 9, nx)).astype(dtype)
    parity(lab, iterations=3)
    parity(lab, selected=[1], background=0, iterations=2)


@pytest.mark.parametrize("dtype,nx", [(np.uint8, 17), (np.uint8, 45), (np.uint8, 145), (np.uint8, 1001),
                                      (np.uint16, 9), (np.uint16, 73), (np.uint16, 257), (np.uint32, 5),
                                      (np.uint32, 67), (np.uint32, 301)])
def test_rows_off_16_byte_boundaries(dtype, nx):
    """Rows whose length is not a multiple of 16 bytes: the counting tile copies the 16-byte aligned span around
    each slice block (its start moves from slice to slice) and moves the rows to a 16-byte pitch before the
    packed compares.  70 rows and 19 slices span several row tiles and z-tiles; the selected-label form
    classifies the moved rows."""
    lab = sn_synth.ellipsoids((nx, 70, 19), 6, 3.0, 12.0, dtype, seed=nx)
    parity(lab, iterations=4)
    parity(lab, selected=[1, 3], iterations=2)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.uint32])
def test_labels_starting_off_16_byte_boundaries(dtype):
    """A label map one element into its buffer: rows of 64 samples, but no row on a 16-byte boundary."""
    lab = sn_synth.ellipsoids((64, 50, 21), 5, 3.0, 12.0, dtype, seed=7)
    parity(lab, iterations=3, on_device="offset")


def test_long_unaligned_rows_use_the_scalar_counting_form():
    """uint32 rows of 8404 bytes: too long for the staged form within a slot, so the tile copies and compares
    them element by element (and the emission uses the per-row kernels: 66 words per row)."""
    rng = np.random.default_rng(5)
    lab = (rng.random((4, 5, 2101)) < 0.2).astype(np.uint32) * rng.integers(1, 9, size=(4, 5, 2101)).astype(
        np.uint32)
    parity(lab, iterations=2)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.uint32])
def test_uploaded_labels(dtype):
    """Labels copied ahead by sn_labels_upload, then extracted by sn_extract_labels."""
    lab = sn_synth.ellipsoids((45, 38, 30), 5, 4.0, 13.0, dtype, seed=21)
    parity(lab, iterations=6, on_device="uploaded")
    parity(lab, selected=[1, 3], background=0, iterations=3, on_device="uploaded")


def test_uploads_ahead_of_extraction_match_direct_calls():
    """Three pinned maps uploaded before any extraction, one of them extracted twice, all freed in stream
    order: each mesh equals the one sn_extract gives for the same map."""
    import torch
    from paper_2401_14906_gb300 import sn
    maps = [sn_synth.ellipsoids((64, 48, 40), 6, 4.0, 14.0, np.uint16, seed=30 + k) for k in range(3)]
    pinned = [torch.from_numpy(m.view(np.int16)).pin_memory().view(torch.uint16) for m in maps]
    ups = [sn.sn_labels_upload(p) for p in pinned]
    for k in (0, 1, 2, 1):
        m, ref = sn.sn_extract_labels(ups[k]), sn.sn_extract(maps[k])
        a, b = sn.sn_mesh_copy_to_host(m), sn.sn_mesh_copy_to_host(ref)
        assert a["points"].shape[0] > 100
        for key in a:
            np.testing.assert_array_equal(a[key], b[key])
        m.free()
        ref.free()
    ups[2].wait()
    for u in ups:
        u.free()


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16, np.uint32])
def test_ellipsoids_each_dtype(dtype):
    lab = sn_synth.ellipsoids((70, 45, 38), 6, 4.0, 15.0, dtype, seed=9)
    parity(lab, iterations=16)


def test_selected_bitmap_mode():
    lab = sn_synth.ellipsoids((60, 50, 40), 8, 4.0, 14.0, np.uint16, seed=4)
    parity(lab, selected=[2, 5, 7], background=0, iterations=9)
    parity(lab, selected=[1, 2, 3, 4, 5, 6, 7, 8], background=0, iterations=3)


def test_selected_sorted_mode_large_u32_labels():
    base = sn_synth.ellipsoids((48, 40, 36), 6, 4.0, 14.0, np.uint32, seed=5)
    lab = np.where(base > 0, base.astype(np.uint64) * 700_000_000 % (2**32 - 3) + 2, 0).astype(np.uint32)
    vals = sorted(set(np.unique(lab).tolist()) - {0})
    parity(lab, selected=vals[::2], background=0, iterations=4)
    parity(lab, selected=vals[1:4], background=7, iterations=4)


def test_background_value_nonzero_and_max_labels():
    for dtype in (np.uint8, np.uint16, np.uint32):
        top = np.iinfo(dtype).max
        lab = np.full((9, 8, 37), top, dtype=dtype)
        lab[2:6, 1:7, 3:30] = top - 1
        lab[4, 4, 10:20] = 0
        parity(lab, background=int(top), iterations=4)
        parity(lab, selected=[int(top) - 1], background=int(top), iterations=4)


def test_degenerate_and_empty():
    for shape in [(1, 1, 1), (1, 1, 40), (1, 33, 1), (2, 1, 1), (1, 2, 2), (3, 1, 70)]:
        lab = (np.arange(int(np.prod(shape))).reshape(shape) % 3).astype(np.uint8)
        parity(lab, iterations=3)
    ref = parity(np.zeros((6, 7, 8), np.uint16), iterations=5)
    assert ref.n_points == 0
    z, y, x = np.mgrid[0:7, 0:6, 0:45]
    parity(((x + y + z) % 2).astype(np.uint8), iterations=5)


def _record_bytes(lab):
    from paper_2401_14906_gb300 import sn
    m = sn.sn_extract(lab)
    b = sn.sn_mesh_record_bytes(m)
    m.free()
    return b


@pytest.mark.parametrize("shape,want", [
    ((3, 120, 120), 8),    # small fields
    ((3, 260, 260), 8),    # -z/+z distances of ~68k ids: 18-bit z fields, 10-bit y fields
    ((3, 200, 2000), 12),  # ~400k points per slice and ~2k per row: 2 + 2*12 + 2*20 > 64 bits (tiled emission)
    ((3, 2, 16000), 12),   # rows of ~16k points: 15-bit y fields (per-row emission)
    ((3, 3, 20000), 0),    # rows of ~20k points: -y/+y distances beyond 15 bits, the sweeps read the CSR
])
def test_sweep_record_widths(shape, want):
    """Checkerboards whose point density fixes the sweep record: 8 bytes with per-mesh field widths,
    12 bytes with 32-bit -z/+z distances, or the CSR stencil."""
    z, y, x = np.mgrid[0:shape[0], 0:shape[1], 0:shape[2]]
    lab = ((x + y + z) % 2).astype(np.uint16)
    assert _record_bytes(lab) == want
    parity(lab, iterations=5)


def test_very_wide_rows_use_the_per_row_kernels():
    # 3100 uint32 labels per row (12.4 KB) do not fit the shared-memory row tile
    rng = np.random.default_rng(77)
    lab = rng.integers(0, 3, size=(3, 4, 3100)).astype(np.uint32)
    parity(lab, iterations=4)


def test_host_labels_are_copied():
    lab = sn_synth.ellipsoids((50, 40, 30), 5, 4.0, 12.0, np.uint16, seed=6)
    parity(lab, iterations=8, on_device=False)


@pytest.mark.parametrize("dims,dtype", [((64, 64, 64), np.uint16), ((97, 61, 133), np.uint8), ((40, 33, 257), np.uint32)])
def test_host_labels_uploaded_in_slabs(dims, dtype):
    """Host labels large enough to be copied in slabs that the counting pass follows slab by slab."""
    lab = sn_synth.ellipsoids(dims, 6, 5.0, 18.0, dtype, seed=11)
    parity(lab, iterations=4, on_device=False)


def test_zero_iterations_and_zero_relaxation():
    lab = sn_synth.ellipsoids((40, 40, 40), 4, 4.0, 12.0, np.uint16, seed=8)
    parity(lab, iterations=0)
    parity(lab, iterations=5, relaxation=0.0)
    parity(lab, iterations=6, relaxation=1.0, constraint=0.0)


@pytest.mark.parametrize("iterations", [1, 2, 3])
@pytest.mark.parametrize("sphere", [False, True])
def test_first_sweeps(iterations, sphere):
    """Sweeps 1 and 2 run as one launch whose offsets after sweep 1 come from the neighbour records; one,
    two and three sweeps, box and ball, 8- and 12-byte records."""
    lab = sn_synth.ellipsoids((52, 47, 40), 5, 4.0, 15.0, np.uint16, seed=31)
    parity(lab, spacing=(1.0, 0.9, 1.3), iterations=iterations, relaxation=0.7, constraint=0.8, sphere=sphere)
    z, y, x = np.mgrid[0:3, 0:200, 0:2000]
    parity(((x + y + z) % 2).astype(np.uint16), iterations=iterations, sphere=sphere, record_bytes=12)


def test_sphere_constraint():
    lab = sn_synth.ellipsoids((60, 52, 44), 6, 5.0, 16.0, np.uint16, seed=12)
    parity(lab, iterations=16, sphere=True)
    parity(lab, spacing=(0.8, 0.8, 0.8), iterations=7, relaxation=0.9, constraint=0.6, sphere=True)


TRI = ("greedy", "shortest", "min_area", "coplanar")


def test_triangulation_unsmoothed_exact():
    lab = sn_synth.ellipsoids((64, 64, 64), 6, 6.0, 20.0, np.uint16, seed=13)
    parity(lab, spacing=(0.9, 1.1, 1.7), iterations=0, triangulate=TRI)


def test_triangulation_smoothed():
    w = sn_synth.config1()
    parity(w.labels, iterations=16, triangulate=TRI)
    lab = sn_synth.atlas((96, 80, 72), n_seeds=12, seed=14)
    parity(lab, spacing=(1.0, 1.0, 2.0), iterations=9, sphere=True, triangulate=TRI)


def test_trim_memory_between_calls():
    """sn_trim_memory returns the pool's unused blocks; meshes alive across it keep their memory, and the next
    extraction allocates afresh."""
    import torch
    from paper_2401_14906_gb300 import sn
    lab = sn_synth.ellipsoids((60, 50, 40), 5, 3.0, 12.0, np.uint16, seed=9)
    t = torch.from_numpy(lab.view(np.int16)).cuda().view(torch.uint16)
    keep = sn.sn_extract(t)
    sn.sn_extract(t).free()
    torch.cuda.synchronize()
    sn.sn_trim_memory()
    got = sn.sn_mesh_copy_to_host(keep)
    keep.free()
    ref = oracle.extract(lab)
    np.testing.assert_array_equal(got["quads"], ref.quads)
    parity(lab, iterations=4)


def test_determinism():
    from gpu_util import run_gpu
    lab = sn_synth.ellipsoids((64, 64, 64), 6, 6.0, 20.0, np.uint16, seed=10)
    a = run_gpu(lab)
    b = run_gpu(lab)
    for k in a[0]:
        np.testing.assert_array_equal(a[0][k], b[0][k])
    for k in a[1]:
        np.testing.assert_array_equal(a[1][k], b[1][k])


def test_config2_full_size():
    w = sn_synth.config2()
    ref = parity(w.labels, w.spacing, w.origin, iterations=w.iterations, relaxation=w.relaxation,
                 constraint=w.constraint)
    assert ref.n_points > 1_000_000


def test_config3_full_size():
    # 1024x1024x512 uint32, 50,000 Voronoi cells with (1,1,4) spacing and 5% gaps:
    # ~1.4e8 points; the sweep record packs 11-bit -y/+y and 20-bit -z/+z
    # distances into 8 bytes
    w = sn_synth.config3()
    ref = parity(w.labels, w.spacing, w.origin, iterations=w.iterations, relaxation=w.relaxation,
                 constraint=w.constraint, record_bytes=8)
    assert ref.n_points > 100_000_000


def test_async_copy_out_matches_sync_copy():
    """sn_mesh_copy_to_host_async into pinned buffers, overlapping the next map's extraction, then sn_mesh_wait."""
    import torch
    from paper_2401_14906_gb300 import sn
    labs = [sn_synth.ellipsoids((70, 50, 40), 5, 5.0, 15.0, np.uint16, seed=s) for s in (21, 22)]
    meshes, outs = [], []
    for lab in labs:
        m = sn.sn_extract(lab)                       # host labels
        sn.sn_smooth(m, 16, 0.5, 1.0)
        n, q, s = m.counts
        out = {"points": torch.empty((n, 3), dtype=torch.float32).pin_memory(),
               "quads": torch.empty((q, 4), dtype=torch.int32).pin_memory(),
               "quad_labels": torch.empty((q, 2), dtype=torch.int16).pin_memory(),
               "stencil_offsets": torch.empty(n + 1, dtype=torch.int64).pin_memory(),
               "stencil_ids": torch.empty(s, dtype=torch.int32).pin_memory(),
               "offsets": torch.empty((n, 3), dtype=torch.float32).pin_memory()}
        sn.sn_mesh_copy_to_host_async(m, out)
        meshes.append(m)
        outs.append(out)
    for m, out in zip(meshes, outs):
        sn.sn_mesh_wait(m)
        want = sn.sn_mesh_copy_to_host(m)
        for k, v in out.items():
            got = v.numpy()
            if k == "quad_labels":
                got = got.view(np.uint16)
            np.testing.assert_array_equal(got, want[k], err_msg=k)
    # freeing with a copy in flight: the memory goes back after the copy
    m = sn.sn_extract(labs[0])
    sn.sn_smooth(m, 16, 0.5, 1.0)
    n = m.counts[0]
    pts = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    sn.sn_mesh_copy_to_host_async(m, {"points": pts})
    sn.sn_mesh_wait(m)
    m.free()
    np.testing.assert_array_equal(pts.numpy(), outs[0]["points"].numpy())
