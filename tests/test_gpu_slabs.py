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
