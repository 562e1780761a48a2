"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/*.h declares.  No compute call (CPU only)."""
import ctypes
import glob
import os
import re

import paper_2508_15532_b300 as rt
from paper_2508_15532_b300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(rt_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_declared_symbols():
    path = _build.build()
    L = ctypes.CDLL(path)
    names = declared_functions()
    assert {"rt_create_geodesic_grid", "rt_set_metric", "rt_set_fluid", "rt_step", "rt_moments"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(rt.EXPORTS) <= names


def test_config_struct_matches_header_order():
    text = open(os.path.join(ROOT, "include", "rt.h")).read()
    body = text[text.index("typedef struct {"):text.index("} rt_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(\w+)(?:\[\d\])*(?:\[\d\])?\s*[;,]", body)
    fields = [f for f in fields if f not in ("int", "double")]
    assert fields == [f[0] for f in rt.rt_config._fields_]
