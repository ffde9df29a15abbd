"""The C-ABI library builds for sm_103a, loads, and exports every function include/mpk.h declares;
the binding's ctypes structs lay out exactly as the header's, and it declares every entry point
with the header's argument and return types."""
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "mpk.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mpk_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    import paper_2405_12525_gb300 as mpk
    return mpk.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("mpk_build_levels", "mpk_plan", "mpk_apply", "mpk_cheb_filter"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(mpk_[a-z0-9_]+)\b", out))
    missing = [f for f in _declared_functions() if f not in exported]
    assert not missing, missing


def test_binding_loads_and_lists_all_symbols(lib_path):
    import paper_2405_12525_gb300 as mpk
    lib = mpk.load()
    for f in _declared_functions():
        assert hasattr(lib, f), f
    assert sorted(mpk.EXPORTED_SYMBOLS) == _declared_functions()


def test_status_strings_without_gpu(lib_path):
    import paper_2405_12525_gb300 as mpk
    lib = mpk.load()
    assert lib.mpk_status_string(0) == b"ok"
    assert lib.mpk_status_string(4) == b"device wait timed out"


def _c_struct_fields(name: str):
    """Field names, in order, of `typedef struct { ... } name;` in the header."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", text).group(1)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "const int32_t *a, *b" -> a, b: the last identifier of each declarator
        head, *rest = decl.split(",")
        for d in [head] + rest:
            names.append(re.findall(r"[A-Za-z_][A-Za-z0-9_]*", d)[-1])
    return names


def test_binding_structs_match_the_header_layout(tmp_path):
    # the ctypes mirrors of the header's structs: same fields in the same order, and the offsets
    # and sizes a C compiler gives them (a mismatch would pass wrong options without an error)
    import ctypes
    import paper_2405_12525_gb300 as mpk
    structs = {"mpk_csr": mpk._Csr, "mpk_plan_opts": mpk._Opts, "mpk_plan_desc": mpk._Desc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for cname, cls in structs.items():
        assert _c_struct_fields(cname) == [f for f, _ in cls._fields_], cname
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu %zu\\n", offsetof({cname}, {f}), sizeof((({cname} *)0)->{f}));')
    lines += ["return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines))
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {}
    for ln in filter(None, out):
        parts = ln.split()
        c[tuple(parts[:2])] = tuple(int(v) for v in parts[2:])
    for cname, cls in structs.items():
        assert c[(cname, "sizeof")] == (ctypes.sizeof(cls),), cname
        for f, _ in cls._fields_:
            field = getattr(cls, f)
            assert c[(cname, f)] == (field.offset, field.size), (cname, f)


def _c_kind(decl: str) -> str:
    """Kind of a C parameter or return type of the header: ptr, i32, i64, f64 or void."""
    decl = decl.strip()
    if "*" in decl or re.match(r"(const\s+)?mpk_stream\b", decl):
        return "ptr"
    t = re.findall(r"[A-Za-z_][A-Za-z0-9_]*", decl)
    t = [w for w in t if w != "const"]
    base = t[0]
    return {"int32_t": "i32", "mpk_status": "i32", "int": "i32", "int64_t": "i64", "double": "f64",
            "void": "void"}[base]


def _ctypes_kind(t) -> str:
    import ctypes
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "ptr"  # POINTER(...) classes carry the pointee type in _type_
    return {ctypes.c_int32: "i32", ctypes.c_int: "i32", ctypes.c_int64: "i64", ctypes.c_double: "f64"}[t]


def test_binding_signatures_match_the_header_prototypes(lib_path):
    # every entry point's argument and return kinds as the header declares them, so that no
    # 32/64-bit integer, double or pointer is passed in the wrong register or width
    import paper_2405_12525_gb300 as mpk
    lib = mpk.load()
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = re.findall(r"(mpk_status|int64_t|void|const\s+char\s*\*)\s*(mpk_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text)
    assert {name for _, name, _ in protos} == set(_declared_functions())
    for ret, name, params in protos:
        f = getattr(lib, name)
        params = params.strip()
        want = [] if params in ("", "void") else [_c_kind(p) for p in params.split(",")]
        assert f.argtypes is not None, f"{name}: argument types not set by the binding"
        assert [_ctypes_kind(t) for t in f.argtypes] == want, name
        assert _ctypes_kind(f.restype) == ("ptr" if "*" in ret else _c_kind(ret)), name


def test_readme_c_example_compiles_and_links(lib_path, tmp_path):
    # the README's program that uses the C ABI without Python builds against the header and the
    # library as shown there (it is not run: that needs a GPU)
    readme = open(os.path.join(ROOT, "README.md")).read()
    section = readme.split("## Use from C", 1)[1]
    code = re.search(r"```c\n(.*?)```", section, flags=re.S).group(1)
    src = tmp_path / "example.c"
    src.write_text(code)
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cmd = ["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
           str(src), "-o", str(tmp_path / "example"), "-L", os.path.dirname(lib_path), "-lmpk",
           "-L", os.path.join(cuda, "lib64"), "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
