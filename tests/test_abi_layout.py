"""The binding against the C header.  Structures: a plain C program compiled
with gcc prints sizeof and offsetof of every field of feast_opts,
feast_stats and feast_problem, and each must equal the ctypes structure's
(same names, same order); a field added to one side only, or a changed type,
shifts an offset and fails here.  Functions: every prototype's return and
parameter types against the ctypes declarations.  No GPU is involved."""
import os
import shutil
import subprocess

import pytest

import paper_1605_08771_gb300 as fg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"feast_opts": fg.FeastOpts, "feast_stats": fg.FeastStats, "feast_problem": fg.FeastProblem}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    d = tmp_path_factory.mktemp("layout")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "feast.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        s, f, v = line.split()
        table[(s, f)] = int(v)
    return table


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_ctypes_structures_match_the_header(c_layout, cname):
    cls = STRUCTS[cname]
    assert c_layout[(cname, "sizeof")] == __import__("ctypes").sizeof(cls)
    for fname, _ in cls._fields_:
        assert c_layout[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_header_compiles_as_c_and_cpp(tmp_path):
    # the boundary is plain C: the header alone compiles as C11 and as C++17
    for comp, std, ext in (("gcc", "-std=c11", "c"), ("g++", "-std=c++17", "cpp")):
        if shutil.which(comp) is None:
            pytest.skip(f"{comp} not found")
        src = tmp_path / f"h.{ext}"
        src.write_text('#include "feast.h"\nint main(void) { feast_opts o; (void)o; return 0; }\n')
        subprocess.run([comp, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / f"h_{ext}.o")], check=True, capture_output=True)


def _prototypes():
    """{name: (return type, [parameter types])} of every function the header
    declares, comments stripped, parameter names dropped."""
    import re
    text = open(os.path.join(ROOT, "include", "feast.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = re.sub(r"#[^\n]*", " ", text)
    out = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w\s\*]*?)\s*\b(feast_\w+)\s*\(([^;{]*?)\)\s*;", text):
        ret = " ".join(ret.replace("*", " * ").split()).split("}")[-1].strip()
        ret = ret.split(";")[-1].strip()
        ps = []
        for p in params.split(","):
            p = " ".join(p.replace("*", " * ").split())
            if p in ("", "void"):
                continue
            toks = p.split()
            if toks[-1] != "*":
                toks = toks[:-1]   # drop the parameter name
            ps.append(" ".join(toks))
        out[name] = (ret, ps)
    return out


def _ctype_of(c):
    """The ctypes type a C parameter or return type must be marshalled as."""
    import ctypes
    base = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "double": ctypes.c_double, "void": None,
            "uint64_t": ctypes.c_uint64}
    toks = [t for t in c.split() if t != "const"]
    if toks.count("*") == 0:
        return base[toks[0]]
    if toks == ["char", "*"]:
        return ctypes.c_char_p
    return "pointer:" + " ".join(toks)


def test_ctypes_signatures_match_the_header():
    # every entry point's return type and parameter list, as the binding
    # declares them to ctypes, against the header's prototypes: a 32-bit int
    # passed where the C side reads int64_t, or a missing parameter, would
    # hand the library garbage without any error
    import ctypes
    try:
        L = fg.lib()
    except RuntimeError:
        fg.build_library()
        L = fg.lib()
    pointee = {"double *": ctypes.c_double, "int *": ctypes.c_int, "feast_ctx * *": ctypes.c_void_p,
               "feast_opts *": fg.FeastOpts,
               "feast_stats *": fg.FeastStats, "feast_problem *": fg.FeastProblem}
    protos = _prototypes()
    assert sorted(protos) == sorted(fg.EXPORTS)
    for name, (ret, params) in protos.items():
        f = getattr(L, name)
        want_ret = _ctype_of(ret)
        if isinstance(want_ret, str):
            assert f.restype == ctypes.c_void_p, (name, ret)
        else:
            assert f.restype == want_ret, (name, ret, f.restype)
        assert len(f.argtypes) == len(params), (name, params, f.argtypes)
        for i, (c, t) in enumerate(zip(params, f.argtypes)):
            want = _ctype_of(c)
            if isinstance(want, str):
                kind = want.split(":", 1)[1]
                if t is ctypes.c_void_p or t is ctypes.c_char_p:
                    continue   # any pointer may travel as void*
                assert kind in pointee and t == ctypes.POINTER(pointee[kind]), (name, i, c, t)
            else:
                assert t == want, (name, i, c, t)
