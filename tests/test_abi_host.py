"""The C-ABI library loads and exports every declared symbol; argument
validation that happens before any CUDA call works without a GPU."""
import ctypes

import pytest

from paper_1411_0436_gb300 import vspec


@pytest.fixture(scope="module")
def lib():
    return vspec.load()


def test_header_declares_the_boundary():
    names = vspec.declared_functions()
    for n in ["vspec_plan_create", "vspec_plan_destroy", "vspec_execute", "vspec_dump",
              "vspec_plan_info", "vspec_status_string", "vspec_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in vspec.declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/vspec.h but not exported"


def test_status_strings(lib):
    for code in range(-6, 1):
        assert vspec.vspec_status_string(code)
    assert vspec.vspec_status_string(-99) == "unknown status"


@pytest.mark.parametrize("args", [
    (15, 8, 2, 0, 1), (0, 8, 2, 0, 1), (1 << 21, 8, 2, 0, 1), (1000, 8, 2, 0, 1),
    (1024, 0, 2, 0, 1), (1024, 17, 2, 0, 1), (1024, 8, 3, 0, 1), (1024, 8, 0, 0, 1),
    (1024, 8, 2, 2, 1), (1024, 8, 2, 0, 3), (1024, 2, 2, 1, 0), (1024, -1, 2, 1, 0),
])
def test_plan_create_rejects_bad_arguments(lib, args):
    h = ctypes.c_void_p(123)
    assert lib.vspec_plan_create(ctypes.byref(h), *args) == vspec.ERR_INVALID_ARG
    assert h.value is None


def test_plan_create_ex_rejects_unknown_flags(lib):
    h = ctypes.c_void_p(123)
    assert lib.vspec_plan_create_ex(ctypes.byref(h), 1024, 8, 2, 0, 1, 1 << 7) == vspec.ERR_INVALID_ARG
    assert h.value is None


@pytest.mark.parametrize("nsub", [0, 17, -1])
def test_plan_create_sb_rejects_bad_subband_counts(lib, nsub):
    h = ctypes.c_void_p(5)
    assert lib.vspec_plan_create_sb(ctypes.byref(h), 4096, 8, 2, nsub, 0, 1, 0) == vspec.ERR_INVALID_ARG
    assert h.value is None


def test_null_arguments_are_rejected(lib):
    assert lib.vspec_plan_create(None, 1024, 8, 2, 0, 1) == vspec.ERR_INVALID_ARG
    assert lib.vspec_execute(None, 16, 1, 16, None) == vspec.ERR_INVALID_ARG
    assert lib.vspec_dump(None, 16, None, None) == vspec.ERR_INVALID_ARG
    assert lib.vspec_plan_info(None, None, None) == vspec.ERR_INVALID_ARG
    assert lib.vspec_plan_destroy(None) == vspec.OK


def test_tuning_rejects_null_arguments(lib):
    t = vspec.VspecTuning(1, 0, 1, 0, 0)
    assert lib.vspec_plan_get_tuning(None, None, None) == vspec.ERR_INVALID_ARG
    assert lib.vspec_plan_set_tuning(None, ctypes.byref(t)) == vspec.ERR_INVALID_ARG


def test_describe_rejects_null_arguments(lib):
    import ctypes
    buf = ctypes.create_string_buffer(8)
    assert lib.vspec_plan_describe(None, buf, 8) == vspec.ERR_INVALID_ARG


def test_wait_limit_arguments(lib):
    """Out-of-range wait limits are refused before any CUDA call; a negative
    value restores the default."""
    assert lib.vspec_set_wait_limit(ctypes.c_longlong(1 << 33)) == vspec.ERR_INVALID_ARG
    assert lib.vspec_set_wait_limit(ctypes.c_longlong(-1)) == vspec.OK
    assert lib.vspec_plan_inject_timeout(None) == vspec.ERR_INVALID_ARG
