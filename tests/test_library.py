"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(tsr_[a-z0-9_]+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libtsr():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2203_12339_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("tsr_fit_pca_basis", "tsr_project_material", "tsr_precompute_transfer", "tsr_haar_compress",
                     "tsr_relight", "tsr_relight_backward", "tsr_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libtsr):
    missing = [n for n in _declared_functions() if not hasattr(libtsr, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu(libtsr):
    libtsr.tsr_version.restype = ctypes.c_int
    assert libtsr.tsr_version() == 100
    libtsr.tsr_last_error.restype = ctypes.c_char_p
    assert isinstance(libtsr.tsr_last_error(), bytes)


def test_argument_checks_run_before_any_device_work(libtsr):
    # NULL handles/pointers are rejected on the host with TSR_ERR_INVALID_ARG.
    f = libtsr.tsr_precompute_transfer
    f.restype = ctypes.c_int
    assert f(None, 100, None, None, None, 4, 1, None, None) == -1
    g = libtsr.tsr_haar_forward
    g.restype = ctypes.c_int
    assert g(None, 1, 4, None, None) == -1
    m = libtsr.tsr_relight_many
    m.restype = ctypes.c_int
    m.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    assert m(-1, None, 1, None, None, None, None) == -1
    assert m(2, None, 1, None, None, None, None) == -1
    handles = (ctypes.c_void_p * 2)(None, None)
    buf = ctypes.create_string_buffer(64)
    assert m(2, ctypes.cast(handles, ctypes.c_void_p), 1, ctypes.addressof(buf), ctypes.addressof(buf),
             ctypes.addressof(buf), None) == -1
    # batched Step 2: mesh sizes must be 10 nu^2 + 2; NULL handles rejected; nothing reaches the device
    libtsr.tsr_last_error.restype = ctypes.c_char_p
    cb = libtsr.tsr_haar_compress_batched
    cb.restype = ctypes.c_int
    cb.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                   ctypes.c_void_p, ctypes.c_void_p]
    offs = (ctypes.c_int64 * 3)(0, 642, 642 + 100)          # 100 is not of the chart form
    outs = (ctypes.c_void_p * 2)()
    assert cb(2, ctypes.addressof(offs), ctypes.addressof(buf), 4, 4, 0.1, ctypes.addressof(outs), None) == -1
    assert b"not 10 nu^2 + 2" in libtsr.tsr_last_error()
    offs_ok = (ctypes.c_int64 * 3)(0, 642, 642 + 2562)
    assert cb(2, ctypes.addressof(offs_ok), None, 4, 4, 0.1, ctypes.addressof(outs), None) == -1
    assert cb(2, ctypes.addressof(offs_ok), ctypes.addressof(buf), 17, 4, 0.1, ctypes.addressof(outs), None) == -1
    rb = libtsr.tsr_haar_recompress_batched
    rb.restype = ctypes.c_int
    rb.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    nulls = (ctypes.c_void_p * 2)(None, None)
    assert rb(2, ctypes.addressof(offs_ok), ctypes.addressof(buf), ctypes.addressof(nulls), None) == -1
    assert b"is NULL" in libtsr.tsr_last_error()


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2203_12339_gb300 import tsr
    monkeypatch.setattr(tsr, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(tsr, "_lib", None)
    with pytest.raises(RuntimeError):
        tsr.lib()


def test_compressed_load_rejects_bad_files_on_the_host(libtsr, tmp_path):
    """Checkpoint files are validated before any device work: missing, foreign, truncated and
    out-of-range files give TSR_ERR_INVALID_ARG and no handle."""
    import struct
    load = libtsr.tsr_compressed_load
    load.restype = ctypes.c_int
    load.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    libtsr.tsr_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p(1)
    assert load(str(tmp_path / "missing.tsr").encode(), ctypes.byref(out)) == -1 and not out.value
    foreign = tmp_path / "foreign.tsr"
    foreign.write_bytes(b"NOTATSRC" + b"\0" * 64)
    assert load(str(foreign).encode(), ctypes.byref(out)) == -1
    assert b"not a compressed transfer file" in libtsr.tsr_last_error()
    short = tmp_path / "short.tsr"
    short.write_bytes(b"TSRCMP01" + b"\0" * 10)
    assert load(str(short).encode(), ctypes.byref(out)) == -1
    assert b"truncated header" in libtsr.tsr_last_error()
    # K = 99: out of range
    bad = tmp_path / "bad.tsr"
    bad.write_bytes(b"TSRCMP01" + struct.pack("<8iq", 99, 4, 4, 4, 162, 1, 0, 0, 0))
    assert load(str(bad).encode(), ctypes.byref(out)) == -1
    assert b"header out of range" in libtsr.tsr_last_error()
    # a valid header (K = J = 1, nu = 1, P = 1, n_rows = 12, nnz = 2) but the arrays cut short
    cut = tmp_path / "cut.tsr"
    cut.write_bytes(b"TSRCMP01" + struct.pack("<8iq", 1, 1, 1, 1, 12, 0, 0, 0, 2) + b"\0" * 8)
    assert load(str(cut).encode(), ctypes.byref(out)) == -1
    assert b"truncated arrays" in libtsr.tsr_last_error()
    assert not out.value


def test_fault_injection_arguments_checked_on_the_host(libtsr):
    f = libtsr.tsr_fault_inject
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int]
    assert f(0, 1) == -1 and f(4, 1) == -1 and f(1, -1) == -1
    for kind in (1, 2, 3):
        assert f(kind, 0) == 0


def test_kernel_timing_toggle_and_empty_read_without_gpu(libtsr):
    libtsr.tsr_kernel_timing.restype = ctypes.c_int
    libtsr.tsr_kernel_timing_read.restype = ctypes.c_int
    assert libtsr.tsr_kernel_timing(1) == 0
    ms, n = ctypes.c_double(-1.0), ctypes.c_int(-1)
    assert libtsr.tsr_kernel_timing_read(ctypes.byref(ms), ctypes.byref(n)) == 0
    assert ms.value == 0.0 and n.value == 0
    assert libtsr.tsr_kernel_timing(0) == 0
