"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/hww.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_2512_19925_gb300 as hww

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_verbs():
    names = declared_functions()
    for verb in ("create_problem", "set_cross_sections", "set_ww_params", "run_step", "get_tallies",
                 "get_losm_solution", "destroy_problem"):
        assert verb in names


def test_library_exports_every_declared_symbol():
    path = hww._build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    assert set(hww.SYMBOLS) <= set(declared_functions())


def test_no_fallback_when_library_missing(tmp_path, monkeypatch):
    # the binding raises instead of computing anything itself
    monkeypatch.setattr(hww._build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(hww, "_lib", None)
    with pytest.raises(RuntimeError):
        hww.load(build_if_missing=False)


STRUCTS = [("hww_problem_desc", hww.ProblemDesc), ("hww_step_stats", hww.StepStats),
           ("hww_counters", hww.Counters), ("hww_batch_stats", hww.BatchStats)]


def test_struct_layouts_match_header(tmp_path):
    # the binding's ctypes mirrors of the public structs against the header,
    # compiled by the host C compiler: every field at the same offset, and
    # the same size (a field the binding lacks shows as a size difference)
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "hww.h"', "int main(void) {"]
    for cname, py in STRUCTS:
        lines.append('    printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('    printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for cname, py in STRUCTS:
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
