"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle,
element by element on seeded inputs (Welter & Nguyen, Sec. 4.1-4.7)."""
import numpy as np
import pytest

from hdg_inputs import workloads as W
from oracle import krylov, precond
from oracle.condense import condense_local
from tests.gpu_helpers import need_gpu, rel, sparse_mv
from tests.oracle_helpers import OracleSystem

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U16 = 2.0 ** -8

SMALL = {
    'tri_k2': lambda: W.tri_poisson(n=3, k=2),
    'hex_k2': lambda: W.hex_poisson(n=3, k=2),
    'elast_R2': lambda: W.hex_elasticity(n=2, k=1, R=2),
    'cdr_M5_R4': lambda: W.hex_cdr(n=2, k=1, R=4),
    'elast_pert_k2_R8': lambda: W.hex_elasticity(n=2, k=2, R=8),
    'cdr_k2_R4': lambda: W.hex_cdr(n=2, k=2, R=4),     # b = 45: face rows span several staging chunks
    'hex_q4': lambda: W.hex_poisson(n=2, k=4),          # K = 375 > 192: tensor-core products in K slices
    'beam_k2': lambda: W.hex_beam(n=2, k=2),            # traction faces: boundary rows with one element
    'elast_q3_R2': lambda: W.hex_elasticity(n=2, k=3, R=2),   # Ebar 192 x 192, ASM patches 288 x 288:
                                                         # block inverses beyond one CTA's shared memory
    'tet_k2': lambda: W.tet_poisson(n=2, k=2),          # tetrahedra: N_lfe = 4, 7 slots, permuted face nodes
    'tet_obst_k3': lambda: W.tet_obstacle(n=4, k=3, hole=0.5),   # obstacle: Dirichlet inside, flux outside
}


def _problem(w, o=None, chunks=1):
    from paper_2512_13619_gb300 import driver
    o = o or driver.opts()
    p = driver.Problem.from_workload(w)
    bounds = np.linspace(0, w.n_elem, chunks + 1).astype(int)
    for a, b in zip(bounds[:-1], bounds[1:]):
        p.condense(w.blocks(a, b), a)
    p.set_dirichlet(w.uhat_dirichlet())
    return p


@pytest.mark.parametrize('name', sorted(SMALL))
def test_condensation_matches_oracle(name):
    """Kbar^e and rbar^e (Eq. w22) per element, FP64, to 1e-12."""
    need_gpu()
    w = SMALL[name]()
    p = _problem(w, chunks=2)
    Kg, rg = p.condensed()
    Ko, ro, _ = condense_local(w.blocks(), w.M, w.n_lfe)
    assert rel(Kg, Ko) < 1e-12
    assert rel(rg, ro) < 1e-12
    p.close()


@pytest.mark.parametrize('name', sorted(SMALL))
def test_assembly_matches_oracle(name):
    """Face rows of K (Sec. 4.2) equal the blocks of the oracle's
    K = sum_e R_e^T Kbar^e R_e; padding slots are zero; r equals."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = SMALL[name]()
    s = OracleSystem(w)
    p = _problem(w)
    p.assemble(driver.opts())
    blocks, nbr, r = p.face_rows()
    b = s.bsz
    K = s.K.toarray()
    seen = np.zeros_like(K, dtype=bool)
    scale = np.abs(K).max()
    for f in range(p.n_free):
        for sl in range(nbr.shape[1]):
            g = nbr[f, sl]
            if g < 0:
                assert np.all(blocks[f, sl] == 0.0)
                continue
            ref = K[f * b:(f + 1) * b, g * b:(g + 1) * b]
            assert np.abs(blocks[f, sl] - ref).max() <= 1e-12 * scale
            seen[f * b:(f + 1) * b, g * b:(g + 1) * b] = True
    assert np.all(K[~seen] == 0.0)          # every nonzero block is in some slot
    assert rel(r, s.r) < 1e-12
    p.close()


@pytest.mark.parametrize('name', sorted(SMALL))
def test_matvec_fp64_fp32_bf16(name):
    """y = K x (Sec. 4.3).  FP64: normwise 1e-13.  FP32/BF16 storage with FP32
    accumulation: |y - Kx| <= (u_store + (n+1) u_32) |K||x| elementwise,
    n = terms per row (the rounding bound of a dot product)."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = SMALL[name]()
    s = OracleSystem(w)
    p = _problem(w)
    p.assemble(driver.opts(poly_prec='bf16'))
    x = np.random.default_rng(7).standard_normal((p.n_dof, w.R))
    y_ref = sparse_mv(s.K, x)
    bound = sparse_mv(abs(s.K), np.abs(x))
    nterm = (2 * w.n_lfe - 1) * s.bsz
    y64 = p.apply_K(x, 'fp64')
    assert np.abs(y64 - y_ref).max() <= 1e-13 * np.abs(bound).max()
    y32 = p.apply_K(x, 'fp32')
    assert np.all(np.abs(y32 - y_ref) <= (U32 + (nterm + 1) * U32) * bound + 1e-300)
    y16 = p.apply_K(x, 'bf16')
    assert np.all(np.abs(y16 - y_ref) <= (U16 + (nterm + 1) * U32) * bound + 1e-300)
    p.close()


@pytest.mark.parametrize('name', ['hex_k2', 'elast_R2', 'cdr_M5_R4', 'elast_pert_k2_R8', 'beam_k2', 'elast_q3_R2',
                                  'tet_k2', 'tet_obst_k3'])
@pytest.mark.parametrize('pc', ['bj', 'asm'])
def test_bj_asm_apply(name, pc):
    """Block-Jacobi (Sec. 4.5) and ASM (Sec. 4.6) applies in FP64 against the
    oracle's inverses of K_ff and of R_e K R_e^T."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = SMALL[name]()
    s = OracleSystem(w)
    o = driver.opts(pc=pc)
    p = _problem(w)
    p.assemble(o)
    p.setup_precond(o)
    x = np.random.default_rng(8).standard_normal((p.n_dof, w.R))
    if pc == 'bj':
        Binv = precond.bj_setup(s.K, s.bsz)
        z_ref = np.column_stack([precond.bj_apply(Binv, x[:, r]) for r in range(w.R)])
    else:
        subs = precond.asm_setup(s.K, s.elem_dofs)
        z_ref = np.column_stack([precond.asm_apply(subs, x[:, r]) for r in range(w.R)])
    z = p.apply_precond(o, x, 'fp64')
    assert rel(z, z_ref) < 1e-10
    z32 = p.apply_precond(o, x, 'fp32')
    assert rel(z32, z_ref) < 1e-3
    p.close()


def test_gmres_bj_tri_poisson_to_1e10():
    """Unit square, 128 P^2 triangles (528 unknowns), BJ-GMRES(30) to 1e-10:
    the true relative residual of the GPU solution is <= 1e-10 and it equals
    the sparse direct solution within cond(K) * 1e-10; the iteration count is
    within 2 of the oracle's GMRES with the same rule."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = W.tri_poisson(8, 2)
    s = OracleSystem(w)
    o = driver.opts(restart=30, rtol=1e-10, pc='bj')
    p = _problem(w)
    p.assemble(o)
    p.setup_precond(o)
    st, info = p.solve(o)
    assert st == 0 and info.converged == 1
    x = p.free_trace()
    b = s.r[:, 0]
    assert np.linalg.norm(b - s.K @ x[:, 0]) / np.linalg.norm(b) <= 1e-10
    xd = s.direct()
    cond = np.linalg.cond(s.K.toarray())
    assert np.linalg.norm(x[:, 0] - xd) / np.linalg.norm(xd) <= cond * 1e-10
    Binv = precond.bj_setup(s.K, s.bsz)
    _, oi = krylov.gmres(lambda v: s.K @ v, lambda v: precond.bj_apply(Binv, v), b, m=30, rtol=1e-10)
    assert abs(info.iters - oi['iters']) <= 2
    # recovery (Eq. w19, w16) against the oracle's recovery of its own solution
    u, q = p.recover()
    uo, qo = s.recover(xd)
    assert rel(u, uo) < cond * 1e-9
    assert rel(q, qo) < cond * 1e-9
    p.close()


@pytest.mark.parametrize('orth', ['mgs', 'cgs2'])
@pytest.mark.parametrize('pc', ['asm', 'none'])
def test_gmres_variants_multi_rhs(orth, pc):
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = W.hex_elasticity(n=2, k=1, R=4)
    s = OracleSystem(w)
    o = driver.opts(restart=20, rtol=1e-9, pc=pc, orth=orth, max_iters=2000)
    p = _problem(w)
    p.assemble(o)
    p.setup_precond(o)
    st, info = p.solve(o)
    assert st == 0, info.rel_resid
    x = p.free_trace()
    for r in range(w.R):
        b = s.r[:, r]
        assert np.linalg.norm(b - s.K @ x[:, r]) / np.linalg.norm(b) <= 1e-9
    p.close()


def test_polynomial_setup_and_apply():
    """Harmonic Ritz values of Arnoldi(P) on M^{-1} K from the same seeded v0
    agree with the oracle's, and the GPU's polynomial apply agrees with the
    oracle's apply of its own values (p does not depend on the order)."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = W.hex_elasticity(n=2, k=1, R=2)
    s = OracleSystem(w)
    o = driver.opts(pc='bj', poly='gmres', degree=6)
    p = _problem(w)
    p.assemble(o)
    v0 = w.random_vector(31)
    p.setup_precond(o, v0)
    th = p.poly()
    Binv = precond.bj_setup(s.K, s.bsz)
    M = lambda v: precond.bj_apply(Binv, v)
    A = lambda v: M(s.K @ v)
    tho = precond.pp_setup(A, v0, 6)
    key = lambda t: (round(t.real, 6), round(t.imag, 6))
    assert np.allclose(sorted(th, key=key), sorted(tho, key=key), rtol=1e-8, atol=1e-10)
    x = np.random.default_rng(9).standard_normal((p.n_dof, w.R))
    z = p.apply_precond(o, x, 'fp64')
    zo = np.column_stack([precond.pp_apply(A, tho, M(x[:, r])) for r in range(w.R)])
    assert rel(z, zo) < 1e-7
    p.close()


def test_chebyshev_setup_and_apply():
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = W.hex_elasticity(n=2, k=1, R=2)
    s = OracleSystem(w)
    o = driver.opts(pc='asm', poly='chebyshev', degree=4)
    p = _problem(w)
    p.assemble(o)
    v0 = w.random_vector(31)
    p.setup_precond(o, v0)
    ab = p.poly().real
    subs = precond.asm_setup(s.K, s.elem_dofs)
    M = lambda v: precond.asm_apply(subs, v)
    A = lambda v: M(s.K @ v)
    a, b = precond.chebyshev_bounds(A, v0, 10)
    assert abs(ab[0] - a) < 1e-8 * abs(b) and abs(ab[1] - b) < 1e-8 * abs(b)
    x = np.random.default_rng(10).standard_normal((p.n_dof, w.R))
    z = p.apply_precond(o, x, 'fp64')
    zo = np.column_stack([precond.chebyshev_apply(A, a, b, 4, M(x[:, r])) for r in range(w.R)])
    assert rel(z, zo) < 1e-8
    p.close()


@pytest.mark.parametrize('pc,poly,deg', [('asm', 'chebyshev', 4), ('bj', 'gmres', 6), ('bj', None, 0)])
@pytest.mark.parametrize('mode', ['refinement', 'restarted', 'precond'])
def test_mixed_precision_reaches_1e8(pc, poly, deg, mode):
    """FP32 blocks with FP64 refinement (inner solves to 1e-4), or with FP64
    true residuals at the restarts of one GMRES (max_outer = -1), or FP64
    GMRES whose preconditioner alone is stored in FP32 and its polynomial's K
    in BF16 (max_outer = -2), reach a true FP64 relative residual of 1e-8;
    the error against the oracle's direct solution is <= cond * 1e-8."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = W.hex_elasticity(n=3, k=1, R=8)
    s = OracleSystem(w)
    mo = {'refinement': 20, 'restarted': -1, 'precond': -2}[mode]
    o = driver.opts(restart=30, rtol=1e-8, pc=pc, poly=poly, degree=deg, inner='fp32', inner_rtol=1e-4,
                    max_iters=3000, max_outer=mo, poly_prec='bf16' if mode == 'precond' else 'fp32')
    p = _problem(w)
    p.assemble(o)
    p.setup_precond(o, w.random_vector(31) if poly else None)
    st, info = p.solve(o)
    assert st == 0 and (info.outer >= 1 if mode == 'refinement' else info.outer == 0)
    x = p.free_trace()
    xd = np.column_stack([s.direct()[:, r] for r in range(w.R)]) if s.direct().ndim == 2 else s.direct()[:, None]
    cond = np.linalg.cond(s.K.toarray())
    for r in range(w.R):
        b = s.r[:, r]
        assert np.linalg.norm(b - s.K @ x[:, r]) / np.linalg.norm(b) <= 1e-8
        assert np.linalg.norm(x[:, r] - xd[:, r]) / np.linalg.norm(xd[:, r]) <= cond * 1e-8
    p.close()


@pytest.mark.parametrize('inner', ['fp64', 'fp32'])
def test_graph_cycles_equal_launch_by_launch(inner):
    """GMRES cycles replayed as CUDA graphs (conditional IF node per
    iteration) give bit-identical results to iteration-by-iteration launches
    (the reductions are deterministic)."""
    need_gpu()
    from paper_2512_13619_gb300 import driver, _lib as L
    w = W.hex_elasticity(n=2, k=1, R=2)
    o = driver.opts(restart=12, rtol=1e-9, pc='bj', inner=inner, max_iters=3000)
    sols = []
    for graphs in (1, 0, 1):
        p = _problem(w)
        p.assemble(o)
        p.setup_precond(o)
        assert L.hdg_set_graphs(p.h, graphs) == 0
        st, info = p.solve(o)
        assert st == 0
        sols.append((p.free_trace(), info.iters))
        p.close()
    assert np.array_equal(sols[0][0], sols[1][0]) and sols[0][1] == sols[1][1]
    assert np.array_equal(sols[0][0], sols[2][0])


@pytest.mark.parametrize('shared', ['all', 'geometry'])
def test_condense_strided_shared_blocks(shared):
    """hdg_condense_strided with blocks shared by all elements (stride 0)
    equals hdg_condense with per-element copies, on a structured mesh whose
    elements are identical."""
    need_gpu()
    from paper_2512_13619_gb300 import driver, _lib as L
    w = W.hex_convdiff(3, 2, 0.3, (0.6, 0.0, 0.8))
    full = w.blocks()
    _, one, strides, _ = W.structured_convdiff_inputs(3, 2, 0.3, (0.6, 0.0, 0.8))
    names = driver.BLOCK_NAMES
    if shared == 'geometry':     # only the q-equation blocks shared
        blocks = [one[k] if i < 3 else np.ascontiguousarray(full[k]) for i, k in enumerate(names)]
        strides = [0, 0, 0] + [full[k][0].size for k in names[3:]]
    else:
        blocks = [one[k] for k in names]
    p = driver.Problem.from_workload(w)
    assert L.hdg_condense_strided(p.h, 0, w.n_elem, blocks, strides, 0) == 0
    K1, r1 = p.condensed()
    p.close()
    p2 = driver.Problem.from_workload(w)
    p2.condense(full)
    K2, r2 = p2.condensed()
    p2.close()
    assert rel(K1, K2) < 1e-13 and rel(r1, r2) < 1e-13


@pytest.mark.parametrize('name', ['hex_k2', 'elast_R2', 'cdr_M5_R4', 'cdr_k2_R4', 'beam_k2', 'tet_obst_k3',
                                  'elast_pert_k2_R8'])
def test_every_tuning_candidate_matches_oracle(name):
    """Every launch configuration the autotuner may pick computes the same
    block-row products: K x at each storage precision (bounds as in the
    matvec test) and the FP64 BJ / ASM applies (1e-10 normwise, as in the
    apply test), against the
    oracle; then hdg_autotune picks one and the results stay within them."""
    need_gpu()
    from paper_2512_13619_gb300 import driver, _lib as L
    w = SMALL[name]()
    s = OracleSystem(w)
    x = np.random.default_rng(9).standard_normal((s.K.shape[0], w.R))
    y_ref = sparse_mv(s.K, x)
    bound = sparse_mv(abs(s.K), np.abs(x))
    nterm = (2 * w.n_lfe - 1) * s.bsz
    tol = {0: None, 1: U32 + (nterm + 1) * U32, 2: U16 + (nterm + 1) * U32}
    names = {0: 'fp64', 1: 'fp32', 2: 'bf16'}
    for pc in ('bj', 'asm'):
        o = driver.opts(pc=pc, poly_prec='bf16')
        p = _problem(w, o)
        p.assemble(o)
        p.setup_precond(o)
        if pc == 'bj':
            Binv = precond.bj_setup(s.K, s.bsz)
            z_ref = np.column_stack([precond.bj_apply(Binv, x[:, r]) for r in range(w.R)])
        else:
            subs = precond.asm_setup(s.K, s.elem_dofs)
            z_ref = np.column_stack([precond.asm_apply(subs, x[:, r]) for r in range(w.R)])
        ncand = 0
        for prec in (0, 1, 2):
            for cfg in L.hdg_tuning_candidates(p.h, 0, prec):
                assert L.hdg_set_tuning(p.h, 0, prec, cfg) == 0
                y = p.apply_K(x, names[prec])
                if prec == 0:
                    assert np.abs(y - y_ref).max() <= 1e-13 * np.abs(bound).max(), cfg
                else:
                    assert np.all(np.abs(y - y_ref) <= tol[prec] * bound + 1e-300), (prec, cfg)
                ncand += 1
        op = 1 if pc == 'bj' else 2
        for cfg in L.hdg_tuning_candidates(p.h, op, 0):
            assert L.hdg_set_tuning(p.h, op, 0, cfg) == 0
            z = p.apply_precond(o, x, 'fp64')
            assert rel(z, z_ref) < 1e-10, (pc, cfg)
            ncand += 1
        for cfg in L.hdg_tuning_candidates(p.h, op, 1):      # FP32 blocks, FP32 accumulation
            assert L.hdg_set_tuning(p.h, op, 1, cfg) == 0
            z = p.apply_precond(o, x, 'fp32')
            assert rel(z, z_ref) < 1e-3, (pc, cfg)
            ncand += 1
        assert ncand > 8
        assert L.hdg_autotune(p.h, 3, 1) == 0
        st, cfg, us, us0 = L.hdg_get_tuning(p.h, 0, 1)
        assert st == 0 and 0 < us <= us0
        assert np.all(np.abs(p.apply_K(x, 'fp32') - y_ref) <= tol[1] * bound + 1e-300)
        assert rel(p.apply_precond(o, x, 'fp64'), z_ref) < 1e-10
        p.close()


@pytest.mark.parametrize('pc,poly', [('bj', None), ('bj', 'gmres'), ('asm', None), ('asm', 'gmres')])
def test_beam_preconditioners_match_oracle(pc, poly):
    """Sec. 6.2 beam (10 x 2 x 2 hexahedra, Q^2, clamped at x = 0, traction
    at x = 5), GMRES(50) with classical Gram-Schmidt to 1e-6 as in the paper,
    with BJ, BJ-PP(10), ASM and ASM-PP(10) on the GPU: the true relative
    residual is <= 1e-6 and the iteration count is within 5% (at least 2) of
    the oracle's GMRES on the same system with the same start vector of the
    polynomial's Arnoldi cycle.  Runs of thousands of iterations (plain BJ)
    stall over many restarts, and there rounding alone moves the count: the
    oracle's own BJ count on this system is 3557 on an x86 host and 4137 on
    an Arm host (the same code, different BLAS rounding); those are compared
    within 25%."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = W.hex_beam(n=2, k=2)
    s = OracleSystem(w)
    deg = 10 if poly else 0
    o = driver.opts(restart=50, rtol=1e-6, pc=pc, poly=poly, degree=deg, max_iters=20000)
    p = _problem(w)
    p.assemble(o)
    v0 = w.random_vector(11)
    p.setup_precond(o, v0 if poly else None)
    st, info = p.solve(o)
    assert st == 0 and info.converged == 1
    x = p.free_trace()[:, 0]
    b = s.r[:, 0]
    assert np.linalg.norm(b - s.K @ x) / np.linalg.norm(b) <= 1e-6
    if pc == 'bj':
        Binv = precond.bj_setup(s.K, s.bsz)
        M = lambda v: precond.bj_apply(Binv, v)
    else:
        subs = precond.asm_setup(s.K, s.elem_dofs)
        M = lambda v: precond.asm_apply(subs, v)
    if poly:
        A = lambda v: M(s.K @ v)
        th = precond.pp_setup(A, v0, deg)
        Pinv = lambda v: precond.pp_apply(A, th, M(v))
    else:
        Pinv = M
    _, oi = krylov.gmres(lambda v: s.K @ v, Pinv, b, m=50, rtol=1e-6, maxit=20000)
    assert oi['converged']
    tol = max(2, 0.05 * oi['iters']) if oi['iters'] < 500 else 0.25 * oi['iters']
    assert abs(info.iters - oi['iters']) <= tol, (info.iters, oi['iters'])
    p.close()


@pytest.mark.parametrize('pc,deg', [('bj', 10), ('bj', 20), ('asm', 10), ('asm', 20)])
def test_tet_obstacle_polynomial_preconditioners_match_oracle(pc, deg):
    """Sec. 6.1's tetrahedral Poisson set-up (synthetic obstacle stand-in,
    3024 P^1 tetrahedra): BJ-PP(10/20) and ASM-PP(10/20), GMRES(50)-CGS to
    1e-6: true residual <= 1e-6, iteration count within 5% (at least 2) of the
    oracle's with the same polynomial start vector."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = W.tet_obstacle(n=8, k=1, hole=0.25)
    s = OracleSystem(w)
    o = driver.opts(restart=50, rtol=1e-6, pc=pc, poly='gmres', degree=deg, max_iters=3000)
    p = _problem(w)
    p.assemble(o)
    v0 = w.random_vector(11)
    p.setup_precond(o, v0)
    st, info = p.solve(o)
    assert st == 0 and info.converged == 1
    x = p.free_trace()[:, 0]
    b = s.r[:, 0]
    assert np.linalg.norm(b - s.K @ x) / np.linalg.norm(b) <= 1e-6
    if pc == 'bj':
        Binv = precond.bj_setup(s.K, s.bsz)
        M = lambda v: precond.bj_apply(Binv, v)
    else:
        subs = precond.asm_setup(s.K, s.elem_dofs)
        M = lambda v: precond.asm_apply(subs, v)
    A = lambda v: M(s.K @ v)
    th = precond.pp_setup(A, v0, deg)
    _, oi = krylov.gmres(lambda v: s.K @ v, lambda v: precond.pp_apply(A, th, M(v)), b, m=50, rtol=1e-6,
                         maxit=3000)
    assert oi['converged']
    assert abs(info.iters - oi['iters']) <= max(2, 0.05 * oi['iters']), (info.iters, oi['iters'])
    p.close()


def test_cycle_graphs_follow_a_new_polynomial_and_iteration_cap():
    """The GMRES cycles replay CUDA graphs that hold the polynomial's
    coefficients by value: after a second polynomial set-up (another start
    vector) the solve equals a fresh problem's solve with that vector, and a
    changed iteration cap takes effect."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = W.hex_elasticity(n=2, k=1, R=2)
    o = driver.opts(restart=20, rtol=1e-10, pc='bj', poly='gmres', degree=6, max_iters=2000)
    va, vb = w.random_vector(31), w.random_vector(77)
    p = _problem(w)
    p.assemble(o)
    p.setup_precond(o, va)
    st, _ = p.solve(o)
    assert st == 0
    p.setup_precond(o, vb)
    st, info = p.solve(o)
    xb = p.free_trace()
    q = _problem(w)
    q.assemble(o)
    q.setup_precond(o, vb)
    st2, info2 = q.solve(o)
    assert st == 0 and st2 == 0 and info.iters == info2.iters
    assert np.array_equal(xb, q.free_trace())
    o3 = driver.opts(restart=20, rtol=1e-10, pc='bj', poly='gmres', degree=6, max_iters=3)
    st3, info3 = p.solve(o3)
    assert info3.iters <= 3 and info3.converged == 0
    p.close()
    q.close()


@pytest.mark.parametrize('pc,poly,deg', [('bj', 'chebyshev', 4), ('asm', 'chebyshev', 4), ('bj', 'chebyshev', 1),
                                         ('bj', 'gmres', 5), ('bj', 'gmres', 6), ('asm', 'gmres', 7),
                                         ('none', 'gmres', 4)])
def test_low_precision_polynomial_apply(pc, poly, deg):
    """The polynomial preconditioner with FP32 blocks (M^{-1} and K), its
    recurrence fused into the epilogue of M^{-1} on FP32 state vectors,
    against the oracle's FP64 apply of the same polynomial (Sec. 4.7 /
    Chebyshev iteration): within the FP32 rounding of the degree+1 products
    (relative 1e-4), for every right-hand side."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = W.hex_elasticity(n=3, k=1, R=4)
    s = OracleSystem(w)
    o = driver.opts(pc=pc, poly=poly, degree=deg, inner='fp32', poly_prec='fp32')
    p = _problem(w)
    p.assemble(o)
    v0 = w.random_vector(31)
    p.setup_precond(o, v0)
    if pc == 'bj':
        Binv = precond.bj_setup(s.K, s.bsz)
        M = lambda v: precond.bj_apply(Binv, v)
    elif pc == 'asm':
        subs = precond.asm_setup(s.K, s.elem_dofs)
        M = lambda v: precond.asm_apply(subs, v)
    else:
        M = lambda v: v
    A = lambda v: M(s.K @ v)
    x = np.random.default_rng(12).standard_normal((p.n_dof, w.R))
    if poly == 'chebyshev':
        a, b = p.poly().real[:2]
        zo = np.column_stack([precond.chebyshev_apply(A, a, b, deg, M(x[:, r])) for r in range(w.R)])
    else:
        th = p.poly()
        zo = np.column_stack([precond.pp_apply(A, th, M(x[:, r])) for r in range(w.R)])
    z = p.apply_precond(o, x, 'fp32')
    for r in range(w.R):
        assert rel(z[:, r], zo[:, r]) < 1e-4, (r, rel(z[:, r], zo[:, r]))
    # the FP64 apply of the same set-up agrees with the oracle to FP64 rounding
    z64 = p.apply_precond(o, x, 'fp64')
    assert rel(z64, zo) < 1e-8
    p.close()


@pytest.mark.parametrize('name', ['elast_pert_k2_R8', 'cdr_M5_R4'])
@pytest.mark.parametrize('xkind', ['normal', 'scaled'])
def test_tensor_core_fp64_matvec_rowwise_bound(name, xkind):
    """The FP64 block-row product with R = 8 / 4 right-hand sides on the
    tensor cores (K and the gathered x as exact 8-digit expansions, the
    digit products summed exactly, the result rounded once) against the
    oracle's FP64 product, row by row: the error stays within
    4 * 2^-53 * ncol * max_j |K_ij| * max_j |x_jr| over the face row's
    columns j, the error bound of the scheme (the same form as FP64
    rounding of a dot product of ncol terms).  'scaled' gives the faces of x
    magnitudes 10^-4 .. 10^4, so the per-row exponents of x matter."""
    need_gpu()
    from paper_2512_13619_gb300 import driver, _lib as L
    w = SMALL[name]()
    s = OracleSystem(w)
    p = _problem(w)
    p.assemble(driver.opts())
    b = s.bsz
    nf = p.n_free
    blocks, nbr, _ = p.face_rows()
    rng = np.random.default_rng(21)
    x = rng.standard_normal((p.n_dof, w.R))
    if xkind == 'scaled':
        x *= np.repeat(10.0 ** rng.uniform(-4, 4, size=nf), b)[:, None]
    assert L.hdg_set_tuning(p.h, 0, 0, [6, 0, 0]) == 0          # the tensor-core kernel
    y = p.apply_K(x, 'fp64')
    y_ref = sparse_mv(s.K, x)
    xb = x.reshape(nf, b, w.R)
    for f in range(nf):
        cols = [g for g in nbr[f] if g >= 0]
        ncol = len(cols) * b
        kmax = np.abs(blocks[f, :len(cols)]).max(axis=(0, 2))                 # (b,) max_j |K_ij|
        xmax = np.abs(xb[cols]).max(axis=(0, 1))                              # (R,) max_j |x_jr|
        bound = 4 * 2.0 ** -53 * ncol * np.outer(kmax, xmax)
        err = np.abs(y[f * b:(f + 1) * b] - y_ref[f * b:(f + 1) * b])
        assert np.all(err <= bound + 1e-300), (f, float((err / (bound + 1e-300)).max()))
    p.close()
