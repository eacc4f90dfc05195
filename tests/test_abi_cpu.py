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
