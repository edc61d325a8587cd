"""z-slab decomposition (paper_2401_14906_gb300/slabs.py) on the CPU.

The per-rank extractor is the oracle, so these tests check the host-side logic:
the slab plan, the ownership of points and quads, the exchange (an exclusive
scan over the ranks' owned counts, through a real torch.distributed allgather on
gloo for world size 2) and the id remapping.  The stitched mesh must equal the
whole-volume oracle mesh: integer arrays exactly, offsets and points
identical up to the oracle's FP64 rounding of absolute world coordinates."""
import os
import socket
import tempfile

import numpy as np
import pytest

import sn_synth
from paper_2401_14906_gb300 import slabs
from slab_util import assert_same, oracle_extract, oracle_whole

ARGS = dict(spacing=(1.0, 1.0, 2.0), origin=(0.0, 0.0, 0.0), iterations=4, relaxation=0.5, constraint=1.0)


def _map():
    return sn_synth.ellipsoids((23, 19, 30), 6, 3.0, 9.0, np.uint16, seed=21)


def test_plan_covers_every_slice_once():
    for nz in (2, 5, 17, 64):
        for world in range(1, min(nz, 6) + 1):
            plan = slabs.slab_plan(nz, world, 3)
            assert plan[0]["k0"] == 0 and plan[-1]["k1"] == nz and plan[0]["c0"] == -1 and plan[-1]["c1"] == nz
            for p, q in zip(plan, plan[1:]):
                assert p["k1"] == q["k0"] and p["c1"] == q["c0"]
            for p in plan:
                assert p["s0"] <= max(0, p["k0"] - 1 - 5) and p["s1"] >= min(nz, p["k1"] + 5)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_emulated_ranks_match_whole_volume(world):
    lab = _map()
    whole = oracle_whole(lab, **ARGS)
    got = slabs.emulate(lab, ARGS["spacing"], ARGS["origin"], ARGS["iterations"], ARGS["relaxation"],
                        ARGS["constraint"], world, extract=oracle_extract)
    assert_same(got, whole, float_tol=1e-12)


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        part = slabs.run_rank(_map(), ARGS["spacing"], ARGS["origin"], ARGS["iterations"], ARGS["relaxation"],
                              ARGS["constraint"], rank, world, oracle_extract, slabs.torch_allgather)
        np.savez(os.path.join(outdir, "part%d.npz" % rank), **{k: np.asarray(v) for k, v in part.items()})
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_gloo_two_ranks_allgather_and_stitch():
    import torch.multiprocessing as mp
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True, start_method="spawn")
        parts = [dict(np.load(os.path.join(d, "part%d.npz" % r))) for r in range(world)]
    assert parts[0]["first_point"] == 0 and parts[1]["first_point"] == len(parts[0]["points"])
    got = slabs.assemble(parts)
    assert_same(got, oracle_whole(_map(), **ARGS), float_tol=1e-12)
