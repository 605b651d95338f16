"""CPU checks of the boundary: the compiled library loads, exports every
function include/mhdc.h declares, and the product package stays independent
of the oracle.  No compute call is made (no GPU here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\([^;{]*\)\s*;", src, flags=re.M):
            if not m.group(0).lstrip().startswith(("typedef", "return")):
                names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2105_04937_gb300 import build
    so = build.build()
    return C.CDLL(so)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mhdc_build", "hdc_build", "mhdc_spmv", "mhdc_spmm", "csr_spmv",
                     "mhdc_export", "mhdc_info", "mhdc_destroy", "mhdc_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in declared_functions() if not hasattr(built_lib, n)]
    assert not missing, missing


def test_status_codes_and_strerror(built_lib):
    built_lib.mhdc_strerror.restype = C.c_char_p
    hdr = open(os.path.join(ROOT, "include", "mhdc.h")).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"(MHDC_(?:OK|ERR_\w+))\s*=\s*(-?\d+)", hdr))
    assert codes["MHDC_OK"] == 0
    for name, code in codes.items():
        txt = built_lib.mhdc_strerror(code).decode()
        assert txt and txt != "unknown status", name
    assert built_lib.mhdc_strerror(12345).decode() == "unknown status"
    # host-only calls reject a missing handle without touching a device
    assert built_lib.mhdc_stats(None, None, None, None, None) == codes["MHDC_ERR_INVALID_ARG"]
    import paper_2105_04937_gb300 as m
    for name, code in codes.items():
        assert getattr(m, name) == code, name


def test_python_binding_names_match_abi():
    import paper_2105_04937_gb300 as m
    for n in declared_functions():
        if n == "mhdc_last_error":
            continue
        assert hasattr(m, n), n


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2105_04937_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "mhdc_oracle" not in src, f
    osrc = open(os.path.join(ROOT, "oracle", "mhdc_oracle.c")).read()
    assert "paper_2105_04937_gb300" not in osrc and "mhdc.h" not in osrc


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2105_04937_gb300 as m
    monkeypatch.setattr(m, "_lib", None)
    monkeypatch.setattr(m, "SO", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        m.lib()


def test_selector_weight_file_is_intact():
    import hashlib
    import struct
    path = os.path.join(ROOT, "paper_2105_04937_gb300", "selector_weights.bin")
    data = open(path, "rb").read()
    assert data[:8] == b"MHDCMLP1"
    assert hashlib.sha256(data[:-32]).digest() == data[-32:]
    F, H, O = struct.unpack("<iii", data[8:20])
    assert (F, O) == (64, 45)
    assert len(data) == 20 + 4 * (H * F + H + H * H + H + O * H + O) + 32
