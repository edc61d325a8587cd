"""z-slab decomposition on one GPU: every rank's slab is extracted and smoothed by
the library in turn (the allgather becomes a list), and the stitched mesh must
equal the whole-volume GPU mesh bit for bit.  The cell-local offsets do not
depend on where a slab starts, and with dyadic spacing and origin neither do
the world points."""
import numpy as np
import pytest

import sn_synth
from paper_2401_14906_gb300 import slabs
from slab_util import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_14906_gb300 import build
    build.build()


def whole(lab, spacing, origin, iterations, relaxation, constraint):
    return slabs.gpu_extract(lab, spacing, origin, 0, iterations, relaxation, constraint)


@pytest.mark.parametrize("world", [2, 3, 4])
def test_ellipsoids(world):
    lab = sn_synth.ellipsoids((64, 48, 40), 8, 3.0, 14.0, np.uint16, seed=3)
    args = ((1.0, 1.0, 1.0), (0.0, 0.0, 0.0), 16, 0.5, 1.0)
    assert_same(slabs.emulate(lab, *args, world), whole(lab, *args))


@pytest.mark.parametrize("world", [2, 5])
def test_anisotropic_voronoi_u32(world):
    lab = sn_synth.voronoi((48, 40, 60), 40, np.uint32, seed=5)
    args = ((1.0, 1.0, 4.0), (-8.0, 2.0, 16.0), 8, 0.5, 1.0)
    assert_same(slabs.emulate(lab, *args, world), whole(lab, *args))


def test_atlas_four_ranks():
    w = sn_synth.config2((256, 256, 256))
    args = (w.spacing, w.origin, 16, 0.5, 1.0)
    assert_same(slabs.emulate(w.labels, *args, 4), whole(w.labels, *args))


@pytest.mark.parametrize("world", [1, 2, 3])
def test_device_path(world):
    """The device-resident path (sn_slab_part_of, sn_slab_stitch, concatenation on the GPU) gives the
    same global mesh as the whole-volume run."""
    lab = sn_synth.ellipsoids((64, 48, 40), 8, 3.0, 14.0, np.uint16, seed=3)
    args = ((1.0, 1.0, 1.0), (0.0, 0.0, 0.0), 16, 0.5, 1.0)
    assert_same(slabs.emulate_device(lab, *args, world), whole(lab, *args))
    lab = sn_synth.voronoi((48, 40, 60), 40, np.uint32, seed=5)
    args = ((1.0, 1.0, 4.0), (-8.0, 2.0, 16.0), 8, 0.5, 1.0)
    assert_same(slabs.emulate_device(lab, *args, 4), whole(lab, *args))


def _rank_main(rank, world, port, path):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_2401_14906_gb300 import build, sn
    build.build()
    sn.load()
    lab = sn_synth.voronoi((48, 40, 60), 40, np.uint32, seed=5)
    spacing, origin = (1.0, 1.0, 4.0), (-8.0, 2.0, 16.0)
    p = slabs.slab_plan(lab.shape[0], world, 8)[rank]
    dev = torch.from_numpy(np.ascontiguousarray(lab[p["s0"]:p["s1"]]).view(np.int32)).cuda().view(torch.uint32)
    part, totals = slabs.run_rank_device(dev, spacing, origin, 8, 0.5, 1.0, rank, world, lab.shape[0],
                                         slabs.torch_allgather)
    host = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in part.items()}
    np.savez(path % rank, totals=totals, **{k: v for k, v in host.items() if isinstance(v, np.ndarray)})
    dist.destroy_process_group()


def test_two_gloo_ranks_with_the_library(tmp_path):
    """Two processes, each running the library's extraction, smoothing and stitching for its slab on the
    GPU and exchanging counts through a gloo allgather; their parts concatenate to the whole-volume mesh.
    (The ranks share one GPU; their kernels never wait on each other.)"""
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    path = str(tmp_path / "part%d.npz")
    mp.spawn(_rank_main, args=(2, port, path), nprocs=2, join=True)
    parts = [dict(np.load(path % r)) for r in range(2)]
    lab = sn_synth.voronoi((48, 40, 60), 40, np.uint32, seed=5)
    want = whole(lab, (1.0, 1.0, 4.0), (-8.0, 2.0, 16.0), 8, 0.5, 1.0)
    got = {k: np.concatenate([p[k] for p in parts]) for k in
           ("points", "offsets", "cells", "quads", "stencil_ids")}
    got["quad_labels"] = np.concatenate([p["quad_labels"] for p in parts]).view(np.uint32)
    got["stencil_offsets"] = np.concatenate([p["stencil_offsets"] for p in parts] +
                                            [np.array([parts[0]["totals"][2]], np.int64)])
    assert_same(got, want)
