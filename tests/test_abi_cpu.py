"""CPU-side checks of the CUDA library: it builds, loads, and exports what the header declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            # a declaration: a line that starts with its return type and names a function
            names |= set(re.findall(r"^[A-Za-z_][\w \t\*]*?\b([a-z][a-z0-9_]*)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2010_04868_gb300 import build, stencil
    build.build()
    lib = stencil.load()
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert declared == set(stencil.EXPORTS)


def test_checked_build_exports_the_same_symbols_and_says_so():
    """The checked build (every kernel index tested before its access) links from the same sources; the
    query needs no GPU."""
    import ctypes
    from paper_2010_04868_gb300 import build, stencil
    build.build()
    chk = ctypes.CDLL(build.LIB_CHECKED)
    missing = [n for n in sorted(_declared()) if not hasattr(chk, n)]
    assert not missing, missing
    assert chk.stencil_checked_build() == 1
    assert stencil.load().stencil_checked_build() == 0


def test_strerror_covers_codes():
    from paper_2010_04868_gb300 import stencil
    for code in range(0, -7, -1):
        assert stencil.strerror(code) != "unknown error code"
    assert stencil.strerror(-99) == "unknown error code"


def test_missing_library_fails_loudly(tmp_path):
    from paper_2010_04868_gb300 import stencil
    saved = stencil._lib
    stencil._lib = None
    try:
        with pytest.raises(RuntimeError):
            stencil.load(str(tmp_path / "nope.so"))
    finally:
        stencil._lib = saved
