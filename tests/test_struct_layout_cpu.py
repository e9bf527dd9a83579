"""The ctypes structures of the binding have the layout of the C structures in include/bt_selinv.h:
a plain C program compiled with gcc against the header prints sizeof and every field's offsetof
(it does not compile if a field the binding names is missing from the header), and the binding's
ctypes.sizeof / field offsets must agree, and name every field the header's structure has."""
import os
import re
import shutil
import subprocess

import ctypes
import pytest

from paper_2508_19138_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bt_selinv.h")
STRUCTS = ["bt_bt", "bt_bt_out", "bt_selinv_desc", "bt_stats", "bt_server_desc", "bt_request", "bt_server_stats"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("layout")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bt_selinv.h"', 'int main(void) {']
    for s in STRUCTS:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for name, _ in getattr(N, s)._fields_:
            lines.append(f'  printf("{s} {name} %zu\\n", offsetof({s}, {name}));')
    lines += ['  return 0;', '}']
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(d / "layout")
    subprocess.run([cc, "-std=c99", "-Wall", "-I", os.path.dirname(HEADER), str(src), "-o", exe], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for ln in out.splitlines():
        s, name, v = ln.split()
        layout[(s, name)] = int(v)
    return layout


@pytest.mark.parametrize("struct", STRUCTS)
def test_ctypes_layout_matches_header(c_layout, struct):
    cls = getattr(N, struct)
    assert ctypes.sizeof(cls) == c_layout[(struct, "size")]
    for name, _ in cls._fields_:
        assert getattr(cls, name).offset == c_layout[(struct, name)], name


def _header_fields(struct):
    """Field names of `typedef struct { ... } struct;` in the header (comments removed)."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + struct + r"\s*;", text)
    assert m, struct
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            nm = re.findall(r"[A-Za-z_]\w*", part.split("[")[0])
            names.append(nm[-1])
    return names


@pytest.mark.parametrize("struct", STRUCTS)
def test_binding_names_every_header_field_in_order(struct):
    assert [name for name, _ in getattr(N, struct)._fields_] == _header_fields(struct)


def test_binding_constants_match_header(tmp_path):
    """Every BT_* enumerator of the header has the binding's value, and the binding defines them all."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    names = []
    for body in re.findall(r"enum\s*\{([^{}]*)\}", text):
        names += re.findall(r"\b(BT_[A-Z0-9_]+)\s*=", body)
    assert len(names) >= 20
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "bt_selinv.h"\nint main(void) {\n' +
                   "".join(f'  printf("{n} %d\\n", (int){n});\n' for n in names) + "  return 0;\n}\n")
    exe = str(tmp_path / "consts")
    subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", exe], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    for ln in out.splitlines():
        n, v = ln.split()
        assert getattr(N, n) == int(v), n
