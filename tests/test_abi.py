"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/hz.h declares (no GPU needed)."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def hz():
    from paper_2409_16172_gb300 import build
    build.build()
    from paper_2409_16172_gb300 import hz as _hz
    return _hz


def test_exports_every_header_symbol(hz):
    names = hz.header_symbols()
    assert len(names) >= 12, names
    for name in names:
        assert hasattr(hz.lib, name), f"{name} declared in hz.h but not exported"
        assert isinstance(getattr(hz.lib, name), ctypes._CFuncPtr)


def test_version_and_error_string_without_gpu(hz):
    assert "sm_103a" in hz.version()
    assert isinstance(hz.last_error(), str)


def test_allocator_argument_check(hz):
    # one of alloc / release without the other is rejected before any CUDA call
    st = hz.lib.hz_set_allocator(ctypes.c_void_p(1), None, None)
    assert st == 1
    assert "both" in hz.last_error()
    assert hz.lib.hz_set_allocator(None, None, None) == 0
