"""Failure paths on the GPU, made to fire without faulting it (the paper's Sec. 4
reports memory exhaustion on the full connectome; these are the library's
answers to it and to a device-side wait that gives up):

* the row scan's look-back wait gives up (sn_debug_set_spin_limit): sn_extract
  returns SN_ETIMEOUT before any output is allocated or written;
* a device allocation fails (sn_debug_fail_allocation), at every allocation an
  extraction + smoothing makes in turn: SN_ENOMEM, nothing handed out;
* the mesh has more points than the limit (sn_debug_set_point_limit):
  SN_EOVERFLOW, single-map and batched.

After each, the library must still produce the oracle's mesh."""
import numpy as np
import pytest

import oracle
import sn_synth
from gpu_util import parity

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


@pytest.fixture(autouse=True)
def _reset(sn):
    sn.sn_debug_reset()
    yield
    sn.sn_debug_reset()


def _map():
    # 96 x 80 x 72: 81 x 73 = 5,913 cell rows, three scan tiles of 2,048
    return sn_synth.ellipsoids((96, 80, 72), 6, 5.0, 18.0, np.uint16, seed=41)


def _device(lab):
    import torch
    return torch.from_numpy(lab.view(np.int16)).cuda().view(torch.uint16)


def test_lookback_that_gives_up_returns_timeout(sn):
    lab = _map()
    t = _device(lab)
    sn.sn_debug_set_spin_limit(-1)
    with pytest.raises(sn.SNError) as e:
        sn.sn_extract(t)
    assert e.value.status == sn.SN_ETIMEOUT
    assert "look-back" in sn.sn_last_error()
    sn.sn_debug_reset()
    parity(lab, iterations=5)


def test_lookback_with_one_read(sn):
    """A limit of zero polls: each look-back reads a predecessor once.  Whether that read finds the
    predecessor's sums depends on timing, so both outcomes are valid; an extraction that succeeds must be
    exact, and the library must work afterwards."""
    lab = _map()
    t = _device(lab)
    ref = oracle.extract(lab)
    sn.sn_debug_set_spin_limit(0)
    outcomes = set()
    for _ in range(4):
        try:
            m = sn.sn_extract(t)
        except sn.SNError as e:
            assert e.status == sn.SN_ETIMEOUT, e
            outcomes.add("timeout")
            continue
        got = sn.sn_mesh_copy_to_host(m)
        m.free()
        np.testing.assert_array_equal(got["quads"], ref.quads)
        np.testing.assert_array_equal(got["stencil_ids"], ref.stencil_ids)
        outcomes.add("ok")
    assert outcomes
    sn.sn_debug_reset()
    parity(lab, iterations=3)


def test_every_allocation_failure_is_clean(sn):
    """Fail the k-th allocation for k = 0, 1, 2, ... until extract + smooth goes through."""
    lab = _map()
    t = _device(lab)
    failed = 0
    for k in range(64):
        sn.sn_debug_fail_allocation(k)
        try:
            m = sn.sn_extract(t)
            try:
                sn.sn_smooth(m, 6, 0.5, 1.0)
            finally:
                m.free()
        except sn.SNError as e:
            assert e.status == sn.SN_ENOMEM, e
            assert "injected" in sn.sn_last_error() or "host allocation" in sn.sn_last_error()
            failed += 1
            continue
        break
    else:
        pytest.fail("injected allocation failures never ran out")
    assert failed >= 3  # label-free device map: scratch, mesh handle, mesh outputs, smoothing buffer
    sn.sn_debug_reset()
    parity(lab, iterations=6)
    # host labels add the label copy allocation
    for k in range(64):
        sn.sn_debug_fail_allocation(k)
        try:
            sn.sn_extract(lab).free()
        except sn.SNError as e:
            assert e.status == sn.SN_ENOMEM
            continue
        break
    sn.sn_debug_reset()
    parity(lab, iterations=2, on_device=False)


def test_point_limit_overflow(sn):
    lab = _map()
    t = _device(lab)
    ref = oracle.extract(lab)
    sn.sn_debug_set_point_limit(ref.n_points - 1)
    with pytest.raises(sn.SNError) as e:
        sn.sn_extract(t)
    assert e.value.status == sn.SN_EOVERFLOW
    # batched: the map over the limit fails the call, nothing is handed out
    small = sn_synth.ellipsoids((20, 18, 16), 2, 2.0, 5.0, np.uint16, seed=42)
    with pytest.raises(sn.SNError) as e:
        sn.sn_extract_smooth_batch([_device(small), t], iterations=4, relaxation=0.5, constraint_distance=1.0)
    assert e.value.status == sn.SN_EOVERFLOW
    sn.sn_debug_set_point_limit(ref.n_points)
    m = sn.sn_extract(t)
    assert m.counts[0] == ref.n_points
    m.free()
    sn.sn_debug_reset()
    parity(lab, iterations=4)
