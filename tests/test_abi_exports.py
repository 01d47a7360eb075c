"""The C-ABI library loads and exports every entry point include/lbf.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "lbf.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbf_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lbf_create", "lbf_nucleate", "lbf_step", "lbf_bubbles", "lbf_fields",
                 "lbf_destroy", "lbf_ledger", "lbf_set_cells"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1908_04262_gb300 import build as B
    from paper_1908_04262_gb300 import lbf

    path = lbf.LIB_PATH
    if not os.path.exists(path):
        try:
            B.build()
        except Exception as e:  # pragma: no cover - needs nvcc
            pytest.skip("library not built and nvcc unavailable: %s" % e)
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(lbf.EXPORTS) <= set(_declared())


def test_config_struct_matches_header_layout():
    """The ctypes mirror lists the fields of lbf_config in header order."""
    from paper_1908_04262_gb300 import lbf

    with open(os.path.join(ROOT, "include", "lbf.h")) as fh:
        src = fh.read()
    body = src[src.index("typedef struct {\n  int nx, ny, nz;"):src.index("} lbf_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.replace("typedef struct {", "").split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"^(int|double|void\s*\*)\s*", "", decl)
        for part in decl.split(","):
            names.append(re.sub(r"[\s*]|\[.*\]", "", part))
    assert names == [f for f, _ in lbf.Config._fields_]
