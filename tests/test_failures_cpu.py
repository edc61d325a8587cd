"""Failure paths that fire without a GPU: an injected host allocation failure
makes the entry points that allocate before touching the device return
SN_ENOMEM, release what they hold and leave the library usable.  (The paper's
Sec. 4 reports memory exhaustion on the full connectome; these are the
library's answers to it.)  The device-side forms -- a look-back wait that gives
up, a failing device allocation, a mesh over the point limit -- are in
test_gpu_failures.py."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2401_14906_gb300 import build, sn
    build.build()
    return sn.load()


@pytest.fixture(autouse=True)
def _reset(lib):
    lib.sn_debug_reset()
    yield
    lib.sn_debug_reset()


def _upload(lib):
    from paper_2401_14906_gb300 import sn
    arr = np.zeros((4, 5, 6), np.uint16)
    out = ctypes.c_void_p(7)
    rc = lib.sn_labels_upload(ctypes.c_void_p(arr.ctypes.data), sn.SN_U16, (ctypes.c_int64 * 3)(6, 5, 4),
                              ctypes.byref(out))
    return rc, out


def _release(lib, rc, out):
    from paper_2401_14906_gb300 import sn
    if rc == sn.SN_OK:  # on a machine with a GPU the upload may succeed
        lib.sn_labels_wait(out)
        lib.sn_labels_free(out, None)


def test_upload_handle_allocation_fails_cleanly(lib):
    from paper_2401_14906_gb300 import sn
    lib.sn_debug_fail_allocation(0)
    rc, out = _upload(lib)
    assert rc == sn.SN_ENOMEM
    assert out.value is None  # cleared on failure
    assert "host allocation" in sn.sn_last_error()
    # one-shot: the next call gets past the allocation (SN_ECUDA without a GPU, SN_OK with one)
    rc, out = _upload(lib)
    assert rc != sn.SN_ENOMEM
    _release(lib, rc, out)


def test_allocation_countdown_skips_the_first_allocations(lib):
    from paper_2401_14906_gb300 import sn
    lib.sn_debug_fail_allocation(1)
    rc1, out1 = _upload(lib)  # its handle allocation takes the countdown to 0
    assert rc1 != sn.SN_ENOMEM
    _release(lib, rc1, out1)
    if rc1 == sn.SN_OK:
        pytest.skip("a GPU is present: the upload's device allocation consumed the failure")
    rc2, out2 = _upload(lib)
    assert rc2 == sn.SN_ENOMEM and out2.value is None


def test_learner_create_fails_cleanly(lib):
    from paper_2401_14906_gb300 import sn
    lib.sn_debug_fail_allocation(0)
    out = ctypes.c_void_p(9)
    rc = lib.sn_learner_create(None, ctypes.byref(out))
    assert rc == sn.SN_ENOMEM
    assert out.value is None


def test_reset_turns_injection_off(lib):
    from paper_2401_14906_gb300 import sn
    lib.sn_debug_fail_allocation(0)
    lib.sn_debug_reset()
    rc, out = _upload(lib)
    assert rc != sn.SN_ENOMEM
    _release(lib, rc, out)
