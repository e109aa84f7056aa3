"""ctypes binding of libhdg.so: one Python function per C entry point of
include/hdg.h, with the same name and argument order.  Arguments are
marshalled only: numpy arrays pass their host pointer, torch tensors their
data pointer, ints are taken as raw addresses.  Functions return the integer
hdg_status (0 = HDG_OK); hdg_problem_create returns (status, handle).

Loading fails loudly (RuntimeError) when the compiled library is missing:
there is no fallback implementation.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, 'libhdg.so')

HDG_OK, HDG_ERR_ARG, HDG_ERR_OOM, HDG_ERR_BUDGET, HDG_ERR_SINGULAR, HDG_ERR_NOT_CONVERGED, HDG_ERR_BREAKDOWN, \
    HDG_ERR_NAN, HDG_ERR_TIMEOUT, HDG_ERR_CUDA, HDG_ERR_STATE = range(11)
HDG_FP64, HDG_FP32, HDG_BF16 = 0, 1, 2
HDG_PC_NONE, HDG_PC_BJ, HDG_PC_ASM = 0, 1, 2
HDG_POLY_NONE, HDG_POLY_GMRES, HDG_POLY_CHEBYSHEV = 0, 1, 2
HDG_ORTH_CGS, HDG_ORTH_MGS, HDG_ORTH_CGS2 = 0, 1, 2


class hdg_mesh(ctypes.Structure):
    _fields_ = [('dim', ctypes.c_int), ('n_lfe', ctypes.c_int), ('M', ctypes.c_int), ('PE', ctypes.c_int),
                ('PF', ctypes.c_int), ('n_elem', ctypes.c_int64), ('n_face', ctypes.c_int64),
                ('elem_face', ctypes.c_void_p), ('face_elem', ctypes.c_void_p), ('face_dirichlet', ctypes.c_void_p)]


class hdg_physics(ctypes.Structure):
    _fields_ = [('Cq', ctypes.c_void_p), ('Cu', ctypes.c_void_p), ('Rr', ctypes.c_void_p), ('tau', ctypes.c_double)]


class hdg_solver_opts(ctypes.Structure):
    _fields_ = [('restart', ctypes.c_int), ('max_iters', ctypes.c_int), ('rtol', ctypes.c_double),
                ('orth', ctypes.c_int), ('pc', ctypes.c_int), ('poly', ctypes.c_int), ('poly_degree', ctypes.c_int),
                ('inner_prec', ctypes.c_int), ('poly_prec', ctypes.c_int), ('inner_rtol', ctypes.c_double),
                ('max_outer', ctypes.c_int)]


class hdg_solve_info(ctypes.Structure):
    _fields_ = [('iters', ctypes.c_int), ('restarts', ctypes.c_int), ('outer', ctypes.c_int),
                ('converged', ctypes.c_int), ('rel_resid', ctypes.c_double)]


_V, _I, _I64, _D, _P = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
_SIGS = {
    'hdg_status_str': (ctypes.c_char_p, [_I]),
    'hdg_problem_create': (_I, [ctypes.POINTER(hdg_mesh), _I, _I, ctypes.POINTER(_V)]),
    'hdg_problem_destroy': (_I, [_V]),
    'hdg_problem_device_bytes': (ctypes.c_size_t, [_V]),
    'hdg_workspace_bytes': (ctypes.c_size_t, [ctypes.POINTER(hdg_mesh), _I, ctypes.POINTER(hdg_solver_opts)]),
    'hdg_condense': (_I, [_V, _I64, _I64] + [_P] * 11 + [_I, _V]),
    'hdg_condense_strided': (_I, [_V, _I64, _I64, ctypes.POINTER(_P), ctypes.POINTER(_I64), _I, _V]),
    'hdg_set_dirichlet': (_I, [_V, _P, _I, _V]),
    'hdg_assemble': (_I, [_V, ctypes.POINTER(hdg_solver_opts), _V]),
    'hdg_setup_precond': (_I, [_V, ctypes.POINTER(hdg_solver_opts), _P, _V]),
    'hdg_solve': (_I, [_V, ctypes.POINTER(hdg_solver_opts), _V, ctypes.POINTER(hdg_solve_info)]),
    'hdg_solve_batch': (_I, [ctypes.POINTER(_V), _I, ctypes.POINTER(hdg_solver_opts), _V,
                             ctypes.POINTER(hdg_solve_info)]),
    'hdg_get_trace': (_I, [_V, _P, _I, _V]),
    'hdg_recover': (_I, [_V, _P, _P, _I, _V]),
    'hdg_apply_K': (_I, [_V, _I, _P, _P, _V]),
    'hdg_apply_precond': (_I, [_V, ctypes.POINTER(hdg_solver_opts), _I, _P, _P, _V]),
    'hdg_get_condensed': (_I, [_V, _I64, _I64, _P, _P]),
    'hdg_get_face_rows': (_I, [_V, _I64, _I64, _P, _P, _P]),
    'hdg_get_poly': (_I, [_V, _P, _P, _I, ctypes.POINTER(_I)]),
    'hdg_set_timing': (_I, [_V, _I]),
    'hdg_get_timing': (_I, [_V, _I, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    'hdg_set_kernel_variant': (_I, [_V, _I]),
    'hdg_launch_count': (ctypes.c_longlong, []),
    'hdg_apply_K_noalloc': (_I, [_V, _I, _P, _P, _V]),
    'hdg_set_graphs': (_I, [_V, _I]),
    'hdg_last_error': (ctypes.c_char_p, []),
    'hdg_autotune': (_I, [_V, _I, _I, _V]),
    'hdg_gemm_f64': (_I, [_I, _I, _I, _I, _P, _I64, _I64, _P, _I64, _I64, _P, _I64, _I64, _D, _D, _I64, _V]),
    'hdg_set_condense_mode': (_I, [_V, _I]),
    'hdg_set_condense_chunk': (_I, [_V, _I64]),
    'hdg_get_tuning': (_I, [_V, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float),
                            ctypes.POINTER(ctypes.c_float)]),
    'hdg_tuning_candidates': (_I, [_V, _I, _I, ctypes.POINTER(_I), _I]),
    'hdg_set_tuning': (_I, [_V, _I, _I, ctypes.POINTER(_I)]),
    'hdg_condense_hex': (_I, [_V, _I64, _I64, _I, _P, _P, ctypes.POINTER(hdg_physics), _P, _P, _I, _V]),
    'hdg_hex_blocks': (_I, [_V, _I64, _I, _P, _P, ctypes.POINTER(hdg_physics), ctypes.POINTER(_P), _I, _V]),
    'hdg_set_hex_generation': (_I, [_V, _I]),
}

_lib = None


def load():
    """Load libhdg.so (built by paper_2512_13619_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError('libhdg.so is not built (%s); run __graft_entry__.build()' % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def ptr(a):
    """Address of a numpy array, a torch tensor, an int address or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, 'data_ptr'):
        return a.data_ptr()
    if hasattr(a, 'ctypes'):
        return a.ctypes.data
    raise TypeError('cannot take the address of %r' % type(a))


def stream_ptr(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def hdg_status_str(st):
    return load().hdg_status_str(st).decode()


def hdg_problem_create(mesh, nrhs, device):
    h = ctypes.c_void_p()
    st = load().hdg_problem_create(ctypes.byref(mesh), nrhs, device, ctypes.byref(h))
    return st, h.value


def hdg_problem_destroy(p):
    return load().hdg_problem_destroy(p)


def hdg_problem_device_bytes(p):
    return load().hdg_problem_device_bytes(p)


def hdg_workspace_bytes(mesh, nrhs, opts):
    return load().hdg_workspace_bytes(ctypes.byref(mesh), nrhs, ctypes.byref(opts) if opts is not None else None)


def hdg_condense(p, e0, count, Me, Bd, Cd, D, E, F, G, H, J, ru, ruh, on_device, stream=None):
    return load().hdg_condense(p, e0, count, *[ptr(a) for a in (Me, Bd, Cd, D, E, F, G, H, J, ru, ruh)],
                               int(on_device), stream_ptr(stream))


def hdg_condense_strided(p, e0, count, blocks, elem_stride, on_device, stream=None):
    arr = (_P * 11)(*[ptr(a) for a in blocks])
    st = (_I64 * 11)(*[int(x) for x in elem_stride]) if elem_stride is not None else None
    return load().hdg_condense_strided(p, e0, count, arr, st, int(on_device), stream_ptr(stream))


def physics(Cq, Cu=None, Rr=None, tau=1.0):
    """hdg_physics over host float64 arrays (returned with the arrays, which
    must outlive the call)."""
    import numpy as np
    keep = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None for a in (Cq, Cu, Rr)]
    ph = hdg_physics(*[ptr(a) for a in keep], float(tau))
    return ph, keep


def hdg_condense_hex(p, e0, count, nquad, verts, face_perm, phys, ru, ruh, on_device, stream=None):
    return load().hdg_condense_hex(p, e0, count, nquad, ptr(verts), ptr(face_perm), ctypes.byref(phys), ptr(ru),
                                   ptr(ruh), int(on_device), stream_ptr(stream))


def hdg_hex_blocks(p, count, nquad, verts, face_perm, phys, out, on_device, stream=None):
    arr = (_P * 9)(*[ptr(a) for a in out])
    return load().hdg_hex_blocks(p, count, nquad, ptr(verts), ptr(face_perm), ctypes.byref(phys), arr,
                                 int(on_device), stream_ptr(stream))


def hdg_set_hex_generation(p, sum_factorised):
    return load().hdg_set_hex_generation(p, int(sum_factorised))


def hdg_set_dirichlet(p, uhat_dirichlet, on_device, stream=None):
    return load().hdg_set_dirichlet(p, ptr(uhat_dirichlet), int(on_device), stream_ptr(stream))


def hdg_assemble(p, opts, stream=None):
    return load().hdg_assemble(p, ctypes.byref(opts), stream_ptr(stream))


def hdg_setup_precond(p, opts, v0, stream=None):
    return load().hdg_setup_precond(p, ctypes.byref(opts), ptr(v0), stream_ptr(stream))


def hdg_solve(p, opts, stream=None, info=None):
    return load().hdg_solve(p, ctypes.byref(opts), stream_ptr(stream), ctypes.byref(info) if info is not None else None)


def hdg_solve_batch(handles, opts, stream=None):
    """Returns (status, [hdg_solve_info per problem])."""
    n = len(handles)
    arr = (_V * n)(*handles)
    infos = (hdg_solve_info * n)()
    st = load().hdg_solve_batch(arr, n, ctypes.byref(opts), stream_ptr(stream), infos)
    return st, list(infos)


def hdg_get_trace(p, uhat, on_device, stream=None):
    return load().hdg_get_trace(p, ptr(uhat), int(on_device), stream_ptr(stream))


def hdg_recover(p, u, q, on_device, stream=None):
    return load().hdg_recover(p, ptr(u), ptr(q), int(on_device), stream_ptr(stream))


def hdg_apply_K(p, prec, x, y, stream=None):
    return load().hdg_apply_K(p, prec, ptr(x), ptr(y), stream_ptr(stream))


def hdg_apply_precond(p, opts, prec, x, y, stream=None):
    return load().hdg_apply_precond(p, ctypes.byref(opts), prec, ptr(x), ptr(y), stream_ptr(stream))


def hdg_get_condensed(p, e0, count, Kbar, rbar):
    return load().hdg_get_condensed(p, e0, count, ptr(Kbar), ptr(rbar))


def hdg_get_face_rows(p, f0, count, blocks, nbr, r):
    return load().hdg_get_face_rows(p, f0, count, ptr(blocks), ptr(nbr), ptr(r))


def hdg_get_poly(p, re, im, cap):
    n = ctypes.c_int()
    st = load().hdg_get_poly(p, ptr(re), ptr(im), cap, ctypes.byref(n))
    return st, n.value


def hdg_set_timing(p, enable):
    return load().hdg_set_timing(p, int(enable))


def hdg_get_timing(p, kind=0):
    t = ctypes.c_double()
    n = ctypes.c_int64()
    st = load().hdg_get_timing(p, kind, ctypes.byref(t), ctypes.byref(n))
    return st, t.value, n.value


def hdg_set_kernel_variant(p, variant):
    return load().hdg_set_kernel_variant(p, variant)


def hdg_launch_count():
    return load().hdg_launch_count()


def hdg_apply_K_noalloc(p, prec, x, y, stream=None):
    return load().hdg_apply_K_noalloc(p, prec, ptr(x), ptr(y), stream_ptr(stream))


def hdg_set_graphs(p, enable):
    return load().hdg_set_graphs(p, int(enable))


def hdg_last_error():
    return load().hdg_last_error().decode()


def hdg_autotune(p, reps=0, force=0, stream=None):
    return load().hdg_autotune(p, reps, int(force), stream_ptr(stream))


def hdg_get_tuning(p, op, prec):
    """Returns (status, (kind, sp, cps), us_tuned, us_default)."""
    c = (_I * 3)()
    a, b = ctypes.c_float(), ctypes.c_float()
    st = load().hdg_get_tuning(p, op, prec, c, ctypes.byref(a), ctypes.byref(b))
    return st, tuple(c), a.value, b.value


def hdg_tuning_candidates(p, op, prec):
    """Returns the list of (kind, sp, cps) candidates (empty on bad arguments)."""
    n = load().hdg_tuning_candidates(p, op, prec, None, 0)
    if n <= 0:
        return []
    c = (_I * (3 * n))()
    load().hdg_tuning_candidates(p, op, prec, c, n)
    return [tuple(c[3 * i:3 * i + 3]) for i in range(n)]


def hdg_set_tuning(p, op, prec, cfg):
    c = (_I * 3)(*cfg)
    return load().hdg_set_tuning(p, op, prec, c)


def hdg_gemm_f64(mode, M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, alpha, beta, count, stream=None):
    return load().hdg_gemm_f64(mode, M, N, K, ptr(A), lda, sA, ptr(B), ldb, sB, ptr(C), ldc, sC, float(alpha),
                               float(beta), count, stream_ptr(stream))


def hdg_set_condense_mode(p, mode):
    return load().hdg_set_condense_mode(p, mode)


def hdg_set_condense_chunk(p, elems):
    return load().hdg_set_condense_chunk(p, int(elems))
