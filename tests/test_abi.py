"""The C ABI on the host (no GPU needed): the library loads, exports every
entry point include/blco.h declares, and rejects bad arguments before
touching the device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "blco.h")


@pytest.fixture(scope="module")
def blco():
    from paper_2201_12523_gb300 import build_lib

    build_lib.build()
    from paper_2201_12523_gb300 import blco as b

    return b


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(blco_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_expected_calls():
    names = declared_functions()
    for required in ["blco_build", "blco_mttkrp", "blco_cp_fwd", "blco_cp_bwd", "blco_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(blco):
    lib = ctypes.CDLL(blco.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(blco.EXPORTS) == declared_functions()


def test_default_opts(blco):
    o = blco.blco_default_opts()
    assert (o.max_nnz_per_block, o.line_bits, o.n_queues, o.device_budget_bytes, o.force_stream) == \
        (1 << 27, 64, 8, 0, 0)


def _status(fn, *args):
    return fn(*args)


def test_argument_validation_without_device(blco):
    lib = blco.lib()
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    # out == NULL
    assert lib.blco_build(None, None, 0, dims, 3, None, None, None) == blco.BLCO_ERR_ARG
    # bad order
    assert lib.blco_build(None, None, 0, dims, 0, None, None, ctypes.byref(h)) == blco.BLCO_ERR_ARG
    assert lib.blco_build(None, None, 0, dims, 9, None, None, ctypes.byref(h)) == blco.BLCO_ERR_ARG
    # negative nnz, missing arrays
    assert lib.blco_build(None, None, -1, dims, 3, None, None, ctypes.byref(h)) == blco.BLCO_ERR_ARG
    assert lib.blco_build(None, None, 5, dims, 3, None, None, ctypes.byref(h)) == blco.BLCO_ERR_ARG
    # bad options
    o = blco.blco_default_opts()
    o.line_bits = 65
    assert lib.blco_build(None, None, 0, dims, 3, ctypes.byref(o), None, ctypes.byref(h)) == blco.BLCO_ERR_ARG
    # unsupported shape: more than 128 index bits
    big = (ctypes.c_int64 * 5)(*([1 << 30] * 5))
    assert lib.blco_build(None, None, 0, big, 5, None, None, ctypes.byref(h)) == blco.BLCO_ERR_ARG
    assert b"128" in lib.blco_last_error()
    # NULL handles
    assert lib.blco_mttkrp(None, 0, None, 0, 32, None, None) == blco.BLCO_ERR_ARG
    assert lib.blco_cp_fwd(None, None, 0, 32, None, None) == blco.BLCO_ERR_ARG
    assert lib.blco_cp_bwd(None, 0, None, None, 0, 32, None, None) == blco.BLCO_ERR_ARG
    assert lib.blco_info(None, None) == blco.BLCO_ERR_ARG
    assert lib.blco_sync(None) == blco.BLCO_ERR_ARG
    assert lib.blco_convert(None, None, blco.BLCO_F32, 4, None) == blco.BLCO_ERR_ARG
    assert lib.blco_convert(None, None, blco.BLCO_BF16, -1, None) == blco.BLCO_ERR_ARG
    assert lib.blco_cpals_update(None, 3, 0, 16, None, 0, None, None, None, None, None) == blco.BLCO_ERR_ARG
    assert lib.blco_profile_enable(None, 1) == blco.BLCO_ERR_ARG
    lib.blco_destroy(None)  # no-op


def test_error_object_carries_status_and_message(blco):
    with pytest.raises(blco.BlcoError) as ei:
        blco._check("blco_x", blco.BLCO_ERR_INDEX)
    assert ei.value.status == blco.BLCO_ERR_INDEX and "BLCO_ERR_INDEX" in str(ei.value)


def test_header_is_plain_c(tmp_path):
    """include/blco.h is a C header: it compiles as C99 (no C++ or CUDA
    types in the signatures) and as C++."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    for lang, std in (("c", "c99"), ("c++", "c++11")):
        r = subprocess.run([gcc, "-fsyntax-only", "-x", lang, f"-std={std}", "-Wall", "-Werror", HEADER],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
