"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/bm.h declares (no compute calls: those need a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_29977_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("bm_analyze", "bm_factor", "bm_solve", "bm_query", "bm_destroy", "bm_workspace_bytes"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_the_same_symbols():
    from paper_2609_29977_gb300 import bm
    assert sorted(bm.EXPORTED_SYMBOLS) == declared_functions()


def test_host_only_entry_points(lib):
    from paper_2609_29977_gb300 import bm
    assert bm.bm_version() == 1
    assert "positive definite" in bm.bm_status_string(2)
    d = bm.make_desc(64, 64, 12, 4)
    n = bm.bm_workspace_bytes(d)
    # factors (3 blocks per stage) + level workspace (2) + vectors
    assert n >= 5 * 64 * 64 * 144 * 8
    assert bm.bm_workspace_bytes(bm.make_desc(0, 4, 4, 2)) == 0
    assert bm.bm_workspace_bytes(bm.make_desc(2, 4, 65, 2)) == 0


def header_structs():
    """(name, [field names in order]) of every `typedef struct { ... } name;`
    in include/bm.h."""
    src = open(os.path.join(ROOT, "include", "bm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = []
    for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(bm_\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"^((?:const\s+)?(?:unsigned\s+long\s+long|unsigned|double|int|size_t))\s+(.*)$", decl)
            assert m, "unparsed field declaration in %s: %r" % (name, decl)
            for d in m.group(2).split(","):
                fields.append(re.sub(r"\[.*\]", "", d).strip().lstrip("*").strip())
        out.append((name, fields))
    return out


def test_binding_structs_match_the_header(tmp_path):
    """Every struct of the C ABI has a ctypes twin in the binding with the
    same fields in the same order at the same offsets and sizes (the C side
    measured by a C compiler on include/bm.h)."""
    import shutil
    import subprocess
    from paper_2609_29977_gb300 import bm
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = header_structs()
    assert {n for n, _ in structs} >= {"bm_desc", "bm_info", "bm_qp_desc", "bm_server_desc", "bm_request",
                                       "bm_completion", "bm_server_stats"}
    lines = ['#include "bm.h"', "#include <stdio.h>", "#include <stddef.h>", "int main(void) {"]
    for name, fields in structs:
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f in fields:
            lines.append('  printf("%s.%s %%zu %%zu\\n", offsetof(%s, %s), sizeof(((%s *)0)->%s));'
                         % (name, f, name, f, name, f))
    lines += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I" + os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        key, *vals = line.split()
        got[key] = tuple(int(v) for v in vals)
    for name, fields in structs:
        py = getattr(bm, name)
        assert [f[0] for f in py._fields_] == fields, name
        assert ctypes.sizeof(py) == got[name][0], name
        for f in fields:
            assert (getattr(py, f).offset, getattr(py, f).size) == got["%s.%s" % (name, f)], (name, f)
