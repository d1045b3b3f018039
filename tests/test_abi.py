"""The C ABI library loads and exports every entry point declared in
include/rykov.h (no GPU needed: nothing is called but rk_version)."""
import ctypes
import os
import re

from paper_2303_10846_gb300 import build as B
from paper_2303_10846_gb300 import rykov

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rykov.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rk_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"
    assert sorted(rykov.EXPORTS) == sorted(names)
    assert lib.rk_version() == 102


def test_params_struct_layout_matches_header():
    # 13 doubles + 6 int32 + 1 double
    assert ctypes.sizeof(rykov.RkParams) == 13 * 8 + 6 * 4 + 8
    src = open(os.path.join(ROOT, "include", "rykov.h")).read()
    body = src[src.index("typedef struct rk_params"):src.index("} rk_params;")]
    fields = re.findall(r"(double|int32_t)\s+([^;]+);", body)
    names = []
    for _, decl in fields:
        names += [x.strip() for x in decl.split(",")]
    assert names == [f for f, _ in rykov.RkParams._fields_]


def test_header_documents_every_environment_switch():
    """Every RYKOV_* environment variable that the library reads is described in the
    header next to rk_create."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_2303_10846_gb300", "csrc")
    read = set()
    for f in os.listdir(csrc):
        with open(os.path.join(csrc, f)) as fh:
            read |= set(re.findall(r'getenv\("(RYKOV_[A-Z0-9_]+)"\)', fh.read()))
    with open(os.path.join(root, "include", "rykov.h")) as fh:
        header = fh.read()
    assert read, "no switches found"
    missing = sorted(v for v in read if v not in header)
    assert not missing, missing
