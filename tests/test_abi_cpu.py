"""The C-ABI library builds, loads and exports every function include/sn.h declares;
argument validation fails cleanly with no GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_14906_gb300 import build, sn
    build.build()
    return sn.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(sn_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sn_extract", "sn_smooth", "sn_mesh_counts", "sn_mesh_device_arrays", "sn_mesh_copy_to_host",
                 "sn_free", "sn_status_string", "sn_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2401_14906_gb300 import sn
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in sn.SIGNATURES, f"binding lacks {name}"


def test_status_strings(lib):
    from paper_2401_14906_gb300 import sn
    for code in range(6):
        assert sn.status_string(code).startswith("SN_")


def _extract_rc(lib, labels=True, type_=2, dims=(4, 4, 4), spacing=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0),
                selected=None, nsel=0, background=0):
    arr = np.zeros(64, np.uint16)
    d = (ctypes.c_int64 * 3)(*dims)
    sp = (ctypes.c_double * 3)(*spacing)
    org = (ctypes.c_double * 3)(*origin)
    sel = None
    if selected is not None:
        s = np.asarray(selected, np.uint32)
        sel = s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    out = ctypes.c_void_p(123)
    rc = lib.sn_extract(ctypes.c_void_p(arr.ctypes.data if labels else 0), type_, d, sp, org, sel, nsel,
                        background, None, ctypes.byref(out))
    assert out.value is None  # cleared on failure
    return rc


def test_extract_argument_validation(lib):
    from paper_2401_14906_gb300 import sn
    E = sn.SN_EINVAL
    assert _extract_rc(lib, labels=False) == E
    assert _extract_rc(lib, type_=3) == E
    assert _extract_rc(lib, dims=(0, 4, 4)) == E
    assert _extract_rc(lib, dims=(4, -1, 4)) == E
    assert _extract_rc(lib, dims=(1 << 22, 4, 4)) == E
    assert _extract_rc(lib, spacing=(1.0, 0.0, 1.0)) == E
    assert _extract_rc(lib, spacing=(1.0, float("nan"), 1.0)) == E
    assert _extract_rc(lib, origin=(float("inf"), 0.0, 0.0)) == E
    assert _extract_rc(lib, background=70000) == E                      # does not fit uint16
    assert _extract_rc(lib, selected=[3, 0], nsel=2, background=0) == E  # selected == background
    assert _extract_rc(lib, selected=[70000], nsel=1) == E               # does not fit uint16
    assert _extract_rc(lib, selected=None, nsel=2) == E
    assert _extract_rc(lib, selected=[1], nsel=0) == E
    assert "background" in sn.sn_last_error() or sn.sn_last_error() != ""


def test_smooth_and_accessor_validation(lib):
    from paper_2401_14906_gb300 import sn
    assert lib.sn_smooth(None, 3, 0.5, 1.0) == sn.SN_EINVAL
    assert lib.sn_mesh_counts(None, None, None, None) == sn.SN_EINVAL
    assert lib.sn_mesh_copy_to_host(None, None, None, None, None, None, None) == sn.SN_EINVAL
    lib.sn_free(None)


def test_label_upload_validation(lib):
    """Argument errors of the upload calls are reported before any CUDA call."""
    from paper_2401_14906_gb300 import sn
    E = sn.SN_EINVAL
    arr = np.zeros(64, np.uint16)

    def up(ptr=True, type_=2, dims=(4, 4, 4), out=True):
        o = ctypes.c_void_p(123)
        rc = lib.sn_labels_upload(ctypes.c_void_p(arr.ctypes.data if ptr else 0), type_,
                                  (ctypes.c_int64 * 3)(*dims), ctypes.byref(o) if out else None)
        if out:
            assert o.value is None  # cleared on failure
        return rc
    assert up(ptr=False) == E
    assert up(type_=3) == E
    assert up(dims=(0, 4, 4)) == E
    assert up(dims=(4, 4, 1 << 22)) == E
    assert up(dims=(1 << 20, 1 << 20, 2)) == E  # 2^41 samples
    assert up(out=False) == E
    one = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    zero = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    o = ctypes.c_void_p(123)
    assert lib.sn_extract_labels(None, one, zero, None, 0, 0, None, ctypes.byref(o)) == E
    assert o.value is None
    assert lib.sn_labels_wait(None) == E
    lib.sn_labels_free(None, None)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2401_14906_gb300 import sn
    with pytest.raises(RuntimeError, match="libsn.so not found"):
        saved = sn._lib
        sn._lib = None
        try:
            sn.load(str(tmp_path / "missing.so"))
        finally:
            sn._lib = saved
