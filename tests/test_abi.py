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
