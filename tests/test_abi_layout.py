"""The ctypes binding against the C ABI header (no GPU, no library needed): every struct the
binding declares has the header's fields in the header's order, at the offsets and sizes a
C compiler gives them; the binding's constants equal the header's enum values and macros;
and every prototype has the binding's argument and return kinds.  A field added to one side only, or a changed type, would otherwise make the
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


_STRUCT_OF = {"kfbi_options": "Options", "kfbi_solve_info": "SolveInfo",
              "kfbi_ctx_info": "CtxInfo", "kfbi_stage_times": "StageTimes"}
_HANDLES = ("kfbi_ctx", "kfbi_batch")


def c_class(decl):
    """Kind of one C parameter or return type: int, double, int64, ptr, ptr:<Struct>,
    ptrptr (a handle out-pointer or an array of pointers), cstr, or None for void."""
    toks = [t for t in re.findall(r"[A-Za-z_]\w*|\*", decl) if t != "const"]
    stars = toks.count("*")
    ids = [t for t in toks if t != "*"]
    if len(ids) > 1:
        ids = ids[:-1]                                 # drop the parameter name
    base = " ".join(ids)
    if base == "void" and stars == 0:
        return None
    if base == "char" and stars == 1:
        return "cstr"
    if stars == 0:
        if base in _HANDLES:
            return "ptr"
        return {"int": "int", "kfbi_status": "int", "double": "double", "int64_t": "int64"}[base]
    if stars == 1 and base in _STRUCT_OF:
        return "ptr:" + _STRUCT_OF[base]
    if stars >= 2 or base in _HANDLES:
        return "ptrptr"
    return "ptr"


def py_class(t):
    if t is None:
        return None
    if t is ctypes.c_char_p:
        return "cstr"
    if t is ctypes.c_void_p:
        return "ptr"
    if t is ctypes.c_int:
        return "int"
    if t is ctypes.c_double:
        return "double"
    if t is ctypes.c_int64:
        return "int64"
    target = getattr(t, "_type_", None)
    if target is ctypes.c_void_p:
        return "ptrptr"
    if isinstance(target, type) and issubclass(target, ctypes.Structure):
        return "ptr:" + target.__name__
    return "ptr"


def test_function_signatures_match_the_header_prototypes():
    text = re.sub(r"/\*.*?\*/", "", header_text(), flags=re.S)
    protos = {m.group(2): (m.group(1), m.group(3)) for m in
              re.finditer(r"([A-Za-z_][\w\s\*]*?)\s*\b(kfbi_\w+)\s*\(([^)]*)\)\s*;", text)}
    assert set(protos) == set(K._SIGS), set(protos) ^ set(K._SIGS)
    for name, (ret, args) in protos.items():
        res, argtypes = K._SIGS[name]
        assert c_class(ret) == py_class(res), (name, ret, res)
        cargs = [] if args.strip() == "void" else [c_class(a) for a in args.split(",")]
        assert cargs == [py_class(a) for a in argtypes], (name, cargs)
