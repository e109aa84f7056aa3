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


def test_null_handles_rejected_on_host():
    """Every entry point that takes a problem handle refuses NULL with
    HDG_ERR_ARG before touching the device (as include/hdg.h documents);
    the workspace estimate of a NULL mesh is 0."""
    L = _lib
    L.load()
    o = L.hdg_solver_opts()
    ph, _keep = L.physics([[[[0.0]]]])
    calls = {
        'hdg_condense': lambda: L.hdg_condense(None, 0, 1, *([None] * 11), 0),
        'hdg_condense_strided': lambda: L.hdg_condense_strided(None, 0, 1, [None] * 11, None, 0),
        'hdg_condense_hex': lambda: L.hdg_condense_hex(None, 0, 1, 3, None, None, ph, None, None, 0),
        'hdg_hex_blocks': lambda: L.hdg_hex_blocks(None, 1, 3, None, None, ph, [None] * 9, 0),
        'hdg_set_hex_generation': lambda: L.hdg_set_hex_generation(None, 1),
        'hdg_set_dirichlet': lambda: L.hdg_set_dirichlet(None, None, 0),
        'hdg_assemble': lambda: L.hdg_assemble(None, o),
        'hdg_setup_precond': lambda: L.hdg_setup_precond(None, o, None),
        'hdg_set_condense_mode': lambda: L.hdg_set_condense_mode(None, 1),
        'hdg_set_condense_chunk': lambda: L.hdg_set_condense_chunk(None, 4),
        'hdg_set_graphs': lambda: L.hdg_set_graphs(None, 1),
    }
    for name, call in calls.items():
        assert call() == L.HDG_ERR_ARG, name
    assert L.load().hdg_workspace_bytes(None, 1, None) == 0
    # the batched solve refuses a NULL problem in its list, an empty list and
    # options it does not run (a polynomial preconditioner), on the host
    assert L.hdg_solve_batch([None], o)[0] == L.HDG_ERR_ARG
    assert L.load().hdg_solve_batch(None, 0, ctypes.byref(o), None, None) == L.HDG_ERR_ARG
    o2 = L.hdg_solver_opts()
    o2.restart, o2.max_iters, o2.rtol, o2.poly = 30, 100, 1e-8, L.HDG_POLY_GMRES
    assert L.hdg_solve_batch([None], o2)[0] == L.HDG_ERR_ARG


def test_gemm_shape_checks_on_host():
    """hdg_gemm_f64 rejects inconsistent shapes and tensor-core shapes it
    cannot take (N < 16) before any device work."""
    L = _lib
    z = 1  # any non-null address: the checks fail before it is used
    assert L.hdg_gemm_f64(1, 8, 8, 8, z, 8, 64, z, 8, 64, z, 8, 64, 1.0, 0.0, 1) == L.HDG_ERR_ARG   # N < 16
    assert L.hdg_gemm_f64(0, 8, 8, 8, z, 4, 64, z, 8, 64, z, 8, 64, 1.0, 0.0, 1) == L.HDG_ERR_ARG   # lda < K
    assert L.hdg_gemm_f64(4, 8, 32, 8, z, 8, 64, z, 32, 256, z, 32, 256, 1.0, 0.0, 1) == L.HDG_ERR_ARG  # mode
    assert L.hdg_gemm_f64(0, 8, 8, 8, z, 8, 64, z, 8, 64, z, 8, 64, 1.0, 0.0, 0) == L.HDG_OK          # nothing to do
