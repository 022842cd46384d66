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


def _header():
    src = open(os.path.join(ROOT, "include", "xc.h")).read()
    return re.sub(r"/\*.*?\*/", "", src, flags=re.S)


def _enum_values():
    vals = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", _header(), flags=re.S):
        for name, v in re.findall(r"\b(XC_[A-Z0-9_]+)\s*=\s*([0-9]+)u?", body):
            vals[name] = int(v)
    return vals


def _struct_fields(name):
    m = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", _header(), flags=re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = re.match(r"((?:const\s+)?[a-z0-9_]+\s*\**)\s*(.*)", decl).groups()
        for n in names.split(","):
            n = n.strip()
            fields.append((n.lstrip("*"), ctype.replace(" ", "") + "*" * n.count("*")))
    return fields


_CT = {"int": C.c_int, "double": C.c_double, "int64_t": C.c_int64}


@pytest.mark.parametrize("cname,pyname", [("xc_condition", "XcCondition"), ("xc_grid", "XcGrid"),
                                          ("xc_opts", "XcOpts"), ("xc_broadener", "XcBroadener"),
                                          ("xc_lines", "XcLines")])
def test_binding_structs_match_the_header(cname, pyname):
    """Field names, order and C types of every struct the binding passes by pointer."""
    import paper_1801_09803_gb300 as xc
    py = getattr(xc, pyname)._fields_
    hdr = _struct_fields(cname)
    assert [n for n, _ in py] == [n for n, _ in hdr], (cname, py, hdr)
    for (n, t), (_, ct) in zip(py, hdr):
        if ct.endswith("*"):
            assert t in (C.c_void_p,) or issubclass(t, C._Pointer) or t is C.c_char_p, (cname, n, t, ct)
        else:
            assert t is _CT[ct], (cname, n, t, ct)


def test_binding_enums_match_the_header():
    import paper_1801_09803_gb300 as xc
    e = _enum_values()
    prof = {"doppler": "XC_DOPPLER", "lorentz": "XC_LORENTZ", "voigt_w4": "XC_VOIGT_W4",
            "voigt_gh_binned": "XC_VOIGT_GH_BINNED", "voigt_gh_sampled": "XC_VOIGT_GH_SAMPLED",
            "doppler_binned": "XC_DOPPLER_BINNED", "lorentz_binned": "XC_LORENTZ_BINNED", "voigt_vv": "XC_VOIGT_VV"}
    assert set(xc.PROFILES) == set(prof)
    for k, v in prof.items():
        assert xc.PROFILES[k] == e[v], k
    assert xc.PRECISIONS == {"fp64": e["XC_FP64_PLAIN"], "fp32": e["XC_FP32"]}
    assert xc.QUANTITIES == {"absorption": e["XC_ABSORPTION"], "emission": e["XC_EMISSION"]}
    assert xc.THRESHOLDS == {"constant": e["XC_THRESHOLD_CONSTANT"], "hitran": e["XC_THRESHOLD_HITRAN"]}
    assert xc.BROAD_TYPES == {"constant": e["XC_BROAD_CONSTANT"], "a0": e["XC_BROAD_A0"], "a1": e["XC_BROAD_A1"]}
    assert xc.XC_OPT_NO_TENSOR_CORES == e["XC_OPT_NO_TENSOR_CORES"]
    o = xc.make_opts("voigt_vv", "fp32", 5.0, vv_beta=True, vv_norm=True)
    assert o.vv_flags == e["XC_VV_BETA"] | e["XC_VV_NORMALISE"]
    assert (xc.XC_MEM_HOST, xc.XC_MEM_DEVICE) == (e["XC_MEM_HOST"], e["XC_MEM_DEVICE"])


@pytest.mark.parametrize("cname,pyname", [("xo_condition", "Condition"), ("xo_opts", "Opts"),
                                          ("xo_broadener", "Broadener")])
def test_oracle_structs_match_its_c_source(cname, pyname):
    """The oracle's ctypes structs against the C structs of oracle/xo.c (same parser)."""
    import oracle
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "oracle", "xo.c")).read(), flags=re.S)
    m = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*" + cname + r"\s*;", src, flags=re.S)
    assert m, cname
    hdr = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, names = re.match(r"((?:const\s+)?(?:long\s+long|[a-z0-9_]+)\s*\**)\s*(.*)", decl).groups()
        for n in names.split(","):
            n = n.strip()
            hdr.append((n.lstrip("*"), ctype.replace(" ", "") + "*" * n.count("*")))
    py = getattr(oracle, pyname)._fields_
    assert [n for n, _ in py] == [n for n, _ in hdr], (cname, py, hdr)
    ct = {"int": C.c_int, "double": C.c_double, "longlong": C.c_longlong}
    for (n, t), (_, c) in zip(py, hdr):
        if c.endswith("*"):
            assert t is C.c_void_p, (cname, n)
        else:
            assert t is ct[c], (cname, n, t, c)
