"""The C ABI on a host without a GPU: the library builds for sm_103a, loads,
and exports every entry point include/mace.h declares; the binding covers
them.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mace.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mace_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for required in ("mace_build_sysmatrix", "mace_init", "mace_iterate", "mace_reconstruct"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1911_09278_gb300 import build as gbuild
    lib = gbuild.build()
    L = ctypes.CDLL(lib)
    for name in declared():
        assert hasattr(L, name), name
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib]).decode()
    exported = set(re.findall(r"\bT (mace_[a-z_0-9]+)\b", out))
    assert set(declared()) <= exported


def test_binding_covers_the_header():
    import paper_1911_09278_gb300 as mace
    assert sorted(mace.EXPORTS) == declared()


def test_binding_has_no_cpu_fallback(tmp_path):
    """Without the built library the binding raises instead of computing."""
    import paper_1911_09278_gb300 as mace
    saved = mace._lib
    try:
        mace._lib = None
        with pytest.raises(RuntimeError):
            mace.load(str(tmp_path / "missing.so"))
    finally:
        mace._lib = saved


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.join(ROOT, "paper_1911_09278_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "mace_oracle" not in text, f


def _c_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in the header, in order."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", src).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"^(const\s+)?[a-z_0-9]+\s*", "", decl)  # drop the type
        for part in decl.split(","):
            fields.append(re.sub(r"[\s*]|\[.*\]", "", part))
    return fields


def test_structs_match_the_header(tmp_path):
    """The ctypes structures of the binding have the header's fields in the
    header's order, at the offsets and sizes a C compiler gives them."""
    import paper_1911_09278_gb300 as mace
    pairs = {"mace_geometry": mace.Geometry, "mace_partition": mace.Partition,
             "mace_params": mace.Params, "mace_sysmatrix_info": mace.SysmatrixInfo}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mace.h"', "int main(void) {"]
    for cname, py in pairs.items():
        fields = _c_struct_fields(cname)
        assert fields == [f for f, _ in py._fields_], cname
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in fields:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)]).decode().splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
