"""The ctypes binding against the C ABI header (no GPU, no library needed): every struct the
binding declares has the header's fields in the header's order, at the offsets and sizes a
C compiler gives them, and the binding's constants equal the header's enum values and
macros.  A field added to one side only, or a changed type, would otherwise make the
library write past the binding's buffer or the binding read the wrong field."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_2404_15249_gb300 as K

STRUCTS = {"kfbi_options": K.Options, "kfbi_solve_info": K.SolveInfo,
           "kfbi_ctx_info": K.CtxInfo, "kfbi_stage_times": K.StageTimes}


def header_text():
    with open(K.HEADER) as f:
        return f.read()


def header_fields(text, name):
    """Field names of `typedef struct { ... } name;` in declaration order."""
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "int N, M" / "double lo, hi" / "int dst_variant[4]" / "long long launches[...]"
        parts = decl.split(",")
        first = parts[0].split()[-1]
        for tok in [first] + [p.strip() for p in parts[1:]]:
            names.append(re.sub(r"\[.*\]", "", tok).lstrip("*"))
    return names


def test_struct_fields_match_the_header_in_order():
    text = header_text()
    for cname, py in STRUCTS.items():
        assert [f for f, _ in py._fields_] == header_fields(text, cname), cname


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    """sizeof / offsetof / field sizes and constants as the C compiler lays them out."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kfbi.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("S {cname} %zu %zu\\n", sizeof({cname}), _Alignof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("F {cname} {f} %zu %zu\\n", offsetof({cname}, {f}), '
                         f'sizeof((({cname}*)0)->{f}));')
    consts = [n for n in dir(K) if n.startswith("KFBI_") and isinstance(getattr(K, n), int)]
    for n in consts:
        lines.append(f'  printf("C {n} %lld\\n", (long long)({n}));')
    lines.append('  printf("C NSTAGES %lld\\n", (long long)KFBI_NSTAGES);')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = os.path.join(d, "abi.c"), os.path.join(d, "abi")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(K.HEADER), src, "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    lay = {"S": {}, "F": {}, "C": {}}
    for ln in out:
        t = ln.split()
        if not t:
            continue
        if t[0] == "S":
            lay["S"][t[1]] = (int(t[2]), int(t[3]))
        elif t[0] == "F":
            lay["F"][(t[1], t[2])] = (int(t[3]), int(t[4]))
        else:
            lay["C"][t[1]] = int(t[2])
    return lay


def test_struct_offsets_and_sizes_match_the_c_compiler(c_layout):
    for cname, py in STRUCTS.items():
        assert c_layout["S"][cname] == (ctypes.sizeof(py), ctypes.alignment(py)), cname
        for f, _ in py._fields_:
            d = getattr(py, f)
            assert c_layout["F"][(cname, f)] == (d.offset, d.size), (cname, f)


def test_binding_constants_equal_the_header(c_layout):
    consts = {n: getattr(K, n) for n in dir(K) if n.startswith("KFBI_") and isinstance(getattr(K, n), int)}
    assert len(consts) >= 10
    for n, v in consts.items():
        assert c_layout["C"][n] == v, n
    assert c_layout["C"]["NSTAGES"] == K.NSTAGES
