"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point include/hx.h declares; without a GPU it refuses to
run (no CPU fallback).  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_2006_07964_gb300 import build, hx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header="hx.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hx_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return hx.load()


def test_header_declares_binding_names():
    assert sorted(hx.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_config_default_values(lib):
    cfg = hx.default_config()
    assert cfg.gamma == 1.4 and cfg.precision == hx.HX_FP64 and cfg.autotune == 1
    assert cfg.sutherland_s == pytest.approx(110.4 / 288.15)


def test_no_gpu_means_error_not_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hx.HxError) as ei:
        hx.Context()
    assert ei.value.name == "HX_ERR_CUDA"


def test_library_is_built_for_sm_103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_probe_library_exports_its_header():
    """libhx_probe.so (the benchmark's FMA peak probe) exports what
    include/hx_probe.h declares."""
    build.build()
    assert sorted(hx.PROBE_EXPORTS) == _declared("hx_probe.h")
    lib = ctypes.CDLL(hx.PROBE_PATH)
    for name in _declared("hx_probe.h"):
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)
