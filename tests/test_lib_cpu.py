"""CPU-side checks of the C ABI library: it builds, loads without a GPU, and
exports every entry point include/hdg.h declares (no compute calls)."""
import ctypes
import os
import re

from paper_2512_13619_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, 'include', 'hdg.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return set(re.findall(r'\b(hdg_[A-Za-z0-9_]+)\s*\(', src))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    names = declared()
    assert len(names) >= 18
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names == set(_lib.exported_symbols())


def test_status_strings_without_gpu():
    _lib.load()
    assert _lib.hdg_status_str(_lib.HDG_OK) == 'ok'
    assert _lib.hdg_status_str(_lib.HDG_ERR_SINGULAR) == 'singular block'


def test_invalid_create_rejected_on_host():
    """Argument checks run before any device call."""
    m = _lib.hdg_mesh()
    m.dim = 7
    st, h = _lib.hdg_problem_create(m, 1, 0)
    assert st == _lib.HDG_ERR_ARG and h is None
