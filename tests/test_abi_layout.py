"""The binding's ctypes structures against the C header's layout: a plain C
program compiled with gcc prints sizeof and offsetof of every field of
feast_opts, feast_stats and feast_problem, and each must equal the ctypes
structure's (same names, same order).  A field added to one side only, or a
changed type, shifts an offset and fails here."""
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
