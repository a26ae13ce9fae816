"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/octax.h declares; the binding's struct layouts match the header."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names += re.findall(r"\b(octax_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_01764_gb300 import build

    path = build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2510_01764_gb300 import octax

    assert set(octax.EXPORTS) <= set(declared_functions())


def test_struct_layouts_match_header():
    from paper_2510_01764_gb300 import octax

    assert C.sizeof(octax.CTerm) == 8
    assert C.sizeof(octax.CClause) == 16
    assert octax.CGame.score.offset == 36 and octax.CGame.term.offset == 68
    assert C.sizeof(octax.CGame) == 144
    assert octax.RECORD_DTYPE.itemsize == 4416
    assert C.sizeof(octax.CLaunch) == 16


def test_binding_refuses_without_library(tmp_path):
    from paper_2510_01764_gb300 import octax

    saved = octax._lib
    octax._lib = None
    try:
        with pytest.raises(ImportError):
            octax.load_library(str(tmp_path / "missing.so"))
    finally:
        octax._lib = saved


def test_last_error_without_gpu(lib):
    lib.octax_last_error.restype = C.c_char_p
    assert isinstance(lib.octax_last_error(), bytes)
    lib.octax_num_envs.restype = C.c_int64
    lib.octax_num_envs.argtypes = [C.c_void_p]
    assert lib.octax_num_envs(None) == -1
