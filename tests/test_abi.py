"""The C-ABI library loads, exports every declared symbol, and validates
arguments / injects faults on the host without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2411_17804_gb300 import hai, _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hai_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return hai.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "hai_epic_image" in names and "hai_create" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_built_for_sm103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings(lib):
    assert hai.hai_status_string(0) == "HAI_OK"
    assert hai.hai_status_string(2) == "HAI_ERR_OFF_GRID"
    assert hai.hai_version() >= 100


def test_null_arguments_are_rejected(lib):
    assert lib.hai_create(0, None) == 1
    h = ctypes.c_void_p()
    assert lib.hai_layout_create(None, None, ctypes.byref(h)) == 1
    assert lib.hai_epic_image(None, None, None, 1, 1, 0, None, 0, None) == 1
    assert "NULL" in hai.hai_last_error()
    assert lib.hai_sync(None, None) == 1
    assert lib.hai_fft_correlate(None, None, 1, 64, 2, None, None) == 1
    assert lib.hai_station_epic_layout_create(None, None, 0, None, None) == 1
    assert lib.hai_xbf_layout_create(None, None, 0, 1, 1, None) == 1
    assert lib.hai_xbf_station_image(None, None, None, 1, None, 0, None) == 1
    assert lib.hai_epic_image_host(None, None, None, 1, 1, 0, None, 0, 0, None) == 1


def test_fault_injection_on_host(lib, monkeypatch):
    monkeypatch.setenv("HAI_FAULT", "launch,alloc")
    h = ctypes.c_void_p()
    assert lib.hai_create(0, ctypes.byref(h)) == 7          # HAI_ERR_NO_MEMORY
    assert "injected" in hai.hai_last_error()
    with pytest.raises(hai.HaiError) as e:
        hai.hai_create(0)
    assert e.value.status == 7
