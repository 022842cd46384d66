"""The C ABI library builds, loads and exports every symbol include/xc.h declares.

No compute calls here: these run without a GPU.
"""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libxc():
    from paper_1801_09803_gb300 import build as b
    b.build()
    import paper_1801_09803_gb300 as xc
    return xc


def declared_functions():
    src = open(os.path.join(ROOT, "include", "xc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("xc_load_lines", "xc_partition_function", "xc_cross_section", "xc_cross_section_batched",
              "xc_cross_section_vjp"):
        assert f in names


def test_every_declared_symbol_is_exported(libxc):
    out = subprocess.run(["nm", "-D", "--defined-only", libxc.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (xc_[a-z0-9_]+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    assert sorted(libxc.EXPORTED_SYMBOLS) == declared_functions()
    L = libxc.lib()
    for f in declared_functions():
        assert hasattr(L, f)


def test_host_side_errors_without_compute(libxc):
    L = libxc.lib()
    assert L.xc_version().decode().startswith("xc")
    # NULL handle / NULL arguments are rejected before any CUDA call
    assert L.xc_load_lines(None, None, 0, 0, None) == 1
    assert b"handle" in L.xc_last_error()
    assert L.xc_num_lines(None, None) == 1
    assert L.xc_destroy(None) == 0
    assert L.xc_partition_function(None, None, 0, None, 0, None, None, 0, None) == 0  # nothing to do
    n = C.c_size_t()
    assert L.xc_num_lines(None, C.byref(n)) == 1


def test_create_without_device_fails_cleanly(libxc):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = libxc.lib().xc_create(C.byref(h), 0)
    assert rc in (1, 3)  # EINVAL (no such device) or ECUDA
    assert not h.value


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    import paper_1801_09803_gb300 as xc
    monkeypatch.setattr(xc, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(xc, "_lib", None)
    with pytest.raises(xc.XcError):
        xc.lib()
