"""sn_smooth_static: smoothing that allocates no device memory.

Some callers cannot call cudaMalloc (programs that reserve all device memory
through their own allocator, real-time pipelines that must not allocate after
start-up, plugins inside an application that owns the GPU's memory).  This
entry point keeps its ping-pong buffer in a fixed array inside the library.
These tests call it through the C ABI twice in a row -- on two different meshes
with different parameters, so the second call runs on whatever the first left in
the shared array -- and compare each result with sn_smooth's and with the FP64
oracle's, within the offset tolerance of the other parity tests.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
import sn_synth
from gpu_util import OFFSET_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_14906_gb300 import build
    build.build()
    from paper_2401_14906_gb300 import sn as binding
    binding.load()
    return binding


def _mesh_and_reference(sn, labels, iterations, relaxation, constraint):
    import torch
    t = torch.from_numpy(labels.view(np.int16)).cuda().view(torch.uint16)
    m = sn.sn_extract(t)
    sn.sn_smooth(m, iterations, relaxation, constraint)
    ref = sn.sn_mesh_copy_to_host(m)["offsets"]
    return m, ref


def test_two_calls_in_a_row_match_sn_smooth(sn):
    import torch
    cases = [
        (sn_synth.ellipsoids((64, 64, 64), 6, 6.0, 20.0, np.uint16, seed=21), 16, 0.5, 1.0),
        (sn_synth.ellipsoids((40, 36, 30), 3, 4.0, 12.0, np.uint16, seed=22), 7, 0.8, 0.6),
    ]
    prepared = []
    for lab, it, lam, d in cases:
        m, ref = _mesh_and_reference(sn, lab, it, lam, d)
        want, _ = oracle.smooth(oracle.extract(lab), iterations=it, relaxation=lam, constraint=d)
        assert want.shape == ref.shape
        prepared.append((m, ref, want, it, lam, d))
    assert prepared[1][1].shape[0] < prepared[0][1].shape[0]  # second call leaves stale data in the array
    stream = torch.cuda.current_stream()
    for m, ref, want, it, lam, d in prepared:
        arrs = sn.sn_mesh_device_arrays(m)
        n = int(ref.shape[0])
        assert 0 < n <= sn.SN_STATIC_MAX_POINTS
        out = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
        sn.sn_smooth_static(arrs["stencil_offsets"], arrs["stencil_ids"], arrs["face_masks"], n, it, lam, d, out,
                            stream=stream)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got.astype(np.float64) - ref.astype(np.float64)).max() <= OFFSET_TOL
        assert np.abs(got.astype(np.float64) - want).max() <= OFFSET_TOL
    for m, *_ in prepared:
        m.free()


def test_rejects_more_points_than_the_static_buffer(sn):
    import torch
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(sn.SNError) as e:
        sn.sn_smooth_static(dummy, dummy, dummy, sn.SN_STATIC_MAX_POINTS + 1, 4, 0.5, 1.0, dummy)
    assert e.value.status == sn.SN_EINVAL
    assert "SN_STATIC_MAX_POINTS" in sn.sn_last_error()
