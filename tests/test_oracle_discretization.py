"""Pins of the oracle's condensation / assembly / recovery against the
mathematics: manufactured-solution rates, the polynomial patch test, the
monolithic dense solve, symmetry, and structural counts (Welter & Nguyen,
Sec. 2.3-2.4, 4.1-4.2)."""
import json
import os

import numpy as np
import pytest

from hdg_inputs import workloads as W
from hdg_inputs import blocks as blk
from oracle.condense import condense_direct, condense_local
from oracle.assemble import monolithic_solve
from oracle.postprocess import postprocess_tri
from tests.oracle_helpers import OracleSystem, l2_errors

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')


def _solve_errors(w):
    s = OracleSystem(w)
    uh = s.direct()
    u, q = s.recover(uh)
    return s, u, q, l2_errors(w, s.b, u, q)


def test_tri_mms_rates_k2():
    """L2 errors of u and q decrease at order k+1 = 3 (P^2 triangles)."""
    errs = [_solve_errors(W.tri_poisson(n=n, k=2))[3] for n in (4, 8, 16)]
    for (eu0, eq0), (eu1, eq1) in zip(errs[:-1], errs[1:]):
        assert 2.85 < np.log2(eu0 / eu1) < 3.2
        assert 2.85 < np.log2(eq0 / eq1) < 3.2


def test_tri_postprocessing_superconvergence():
    """u* converges at order k+2 = 4."""
    errs = []
    for n in (4, 8, 16):
        w = W.tri_poisson(n=n, k=2)
        s, u, q, _ = _solve_errors(w)
        phs, coef, xq, wq = postprocess_tri(w.mesh, 2, u[:, :, 0], q[:, :, 0])
        us = np.einsum('qi,ei->eq', phs, coef)
        errs.append(np.sqrt((wq * (us - w.u_exact(xq)[..., 0]) ** 2).sum()))
    for e0, e1 in zip(errs[:-1], errs[1:]):
        assert 3.8 < np.log2(e0 / e1) < 4.3


@pytest.mark.parametrize('k', [1, 3])
def test_hex_mms_rates(k):
    """Q^k hexahedra: errors of u and q decrease at about order k+1."""
    ns = (2, 4) if k == 3 else (4, 8)
    errs = [_solve_errors(W.hex_poisson(n=n, k=k))[3] for n in ns]
    (eu0, eq0), (eu1, eq1) = errs
    assert np.log2(eu0 / eu1) > k + 0.5
    assert np.log2(eq0 / eq1) > k + 0.4


def _patch(mesh_w, k):
    """Replace the manufactured solution of a Poisson workload by a
    polynomial of degree k (in each variable for Q^k)."""
    D = mesh_w.D
    if D == 2:
        c = np.array([0.3, -1.2, 0.7, 0.5, -0.4, 0.9])
        def u(x):
            X, Y = x[..., 0], x[..., 1]
            return (c[0] + c[1] * X + c[2] * Y + c[3] * X * X + c[4] * X * Y + c[5] * Y * Y)[..., None]
        def qf(x):
            X, Y = x[..., 0], x[..., 1]
            return np.stack([c[1] + 2 * c[3] * X + c[4] * Y, c[2] + c[4] * X + 2 * c[5] * Y], -1)[..., None, :]
        lap = 2 * c[3] + 2 * c[5]
        f = lambda x: np.full(x.shape[:-1] + (1,), -lap)
    else:
        def u(x):
            X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
            return (0.5 + X * X * Y - 0.3 * Y * Z * Z + 0.2 * X * Y * Z)[..., None]
        def qf(x):
            X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
            return np.stack([2 * X * Y + 0.2 * Y * Z, X * X - 0.3 * Z * Z + 0.2 * X * Z,
                             -0.6 * Y * Z + 0.2 * X * Y], -1)[..., None, :]
        f = lambda x: -(2 * x[..., 1] - 0.6 * x[..., 1])[..., None]
    mesh_w.u_exact, mesh_w.q_exact, mesh_w.f_exact = u, qf, f
    return mesh_w


@pytest.mark.parametrize('case', ['tri', 'hex'])
def test_patch_test_exact(case):
    """HDG reproduces a polynomial solution in the discrete space exactly
    (consistency + uniqueness): errors at round-off level."""
    w = _patch(W.tri_poisson(n=3, k=2) if case == 'tri' else W.hex_poisson(n=2, k=2), 2)
    s, u, q, (eu, eq) = _solve_errors(w)
    assert eu < 1e-11 and eq < 1e-10


@pytest.mark.parametrize('make', [
    lambda: W.tri_poisson(n=4, k=2),
    lambda: W.hex_poisson(n=2, k=2),
    lambda: W.hex_elasticity(n=2, k=1, R=2),
    lambda: W.hex_cdr(n=2, k=1, R=2),
])
def test_condensed_then_recovered_equals_monolithic(make):
    """Condensation + trace solve + recovery equals the dense monolithic
    solve of Eq. matrixform to 1e-12 (relative)."""
    w = make()
    s = OracleSystem(w)
    uh = s.direct()
    if uh.ndim == 1:
        uh = uh[:, None]
    u, q = s.recover(uh)
    qm, um, uhm = monolithic_solve(s.b, w.mesh.elem_face, w.face_dirichlet, s.uD, w.M, w.n_lfe)
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(uh, uhm) < 1e-12
    assert rel(u, um) < 1e-12
    assert rel(q, qm) < 1e-12


def test_condensation_routes_agree():
    """Eq. 13b-c (dense local inverse) equals the route of Eqs. w15-w22."""
    w = W.hex_elasticity(n=2, k=2, R=3)
    b = w.blocks()
    K1, r1 = condense_direct(b, w.M, w.n_lfe)
    K2, r2, _ = condense_local(b, w.M, w.n_lfe)
    assert np.abs(K1 - K2).max() < 1e-12 * np.abs(K1).max()
    assert np.abs(r1 - r2).max() < 1e-12 * np.abs(r1).max()


@pytest.mark.parametrize('make', [lambda: W.hex_poisson(n=3, k=2), lambda: W.hex_elasticity(n=2, k=2, R=1)])
def test_trace_matrix_symmetric_definite(make):
    """For Poisson and elasticity K is symmetric and (with the sign of Eq.
    HDGd) negative definite."""
    s = OracleSystem(make())
    K = s.K.toarray()
    assert np.abs(K - K.T).max() < 1e-12 * np.abs(K).max()
    np.linalg.cholesky(-K)


def test_structural_counts_golden():
    """N_dof = M P_F N_F (Sec. 2.4) and the number of nonzero face blocks
    (each pair of free faces sharing an element) for the named workloads."""
    gold = json.load(open(os.path.join(GOLDEN, 'structural_counts.json')))
    for name, ref in gold['cases'].items():
        w = {'tri_poisson_8_k2': lambda: W.tri_poisson(8, 2),
             'hex_poisson_16_k3': lambda: W.hex_poisson(16, 3)}[name]()
        assert w.n_dof == ref['n_dof']
        assert w.n_free == ref['n_free_faces']
        fd = w.face_dirichlet
        nfree_e = (fd[w.mesh.elem_face] == 0).sum(axis=1)
        nnzb = int((nfree_e ** 2).sum() - w.n_free)
        assert nnzb == ref['n_nonzero_blocks']
    # and the oracle's assembled matrix has exactly that block pattern
    s = OracleSystem(W.tri_poisson(8, 2))
    b = s.bsz
    pat = (abs(s.K) > 0).toarray().reshape(s.K.shape[0] // b, b, -1, b).any(axis=(1, 3))
    assert int(pat.sum()) == gold['cases']['tri_poisson_8_k2']['n_nonzero_blocks']


# ------------------------------------------------- Neumann (traction) faces
def _box_workload(phys, k, u, qf, f, g, M, perturb):
    """(0,2) x (0,1) x (0,1), 4 x 2 x 2 hexahedra (interior vertices moved by
    up to perturb * h: the mapped Q^k space then still holds the linear
    fields, not the quadratic ones); Dirichlet faces at x = 0 only,
    prescribed outward flux g on the five other sides."""
    from hdg_inputs import mesh as meshmod
    m = meshmod.box_hex_mesh((4, 2, 2), (2.0, 1.0, 1.0), perturb=perturb, seed=8)
    ref = blk.reference_element(m, k, k + 4)
    return W.Workload('box', m, ref, blk.face_permutations(m, ref), phys, 1, 'function', f, u, qf, k=k,
                      dirichlet=W.boundary_faces_at(m, 0, 0.0), neumann_flux=g)


def test_neumann_patch_poisson_exact():
    """A quadratic u with Dirichlet data on one face and its outward flux
    g = -grad u . n on the other five is reproduced exactly by Q^2 (HDG
    consistency with flux boundary conditions)."""
    w0 = _patch(W.hex_poisson(n=2, k=2), 2)
    g = lambda x, n: -np.einsum('...d,...d->...', w0.q_exact(x)[..., 0, :], n)[..., None]
    w = _box_workload(blk.poisson(3), 2, w0.u_exact, w0.q_exact, w0.f_exact, g, 1, 0.0)
    assert w.face_neumann.sum() == 2 * 2 + 2 * (4 * 2) + 2 * (4 * 2) and w.face_dirichlet.sum() == 2 * 2
    _, _, _, (eu, eq) = _solve_errors(w)
    assert eu < 1e-11 and eq < 1e-10


@pytest.mark.parametrize('k', [1, 2])
def test_neumann_patch_elasticity_exact(k):
    """Linear elasticity (lambda = 0.7, mu = 1.3) with u_a = c_a + G_ab x_b
    (+ Q_abc x_b x_c for k = 2): body force f = -div sigma (constant), traction
    data g = -sigma n on five sides, Dirichlet data on x = 0; Q^k reproduces u
    and q = grad u exactly (k = 1 on a perturbed mesh)."""
    lam, mu = 0.7, 1.3
    rng = np.random.default_rng(12)
    c0 = rng.standard_normal(3)
    G = rng.standard_normal((3, 3))
    Q = rng.standard_normal((3, 3, 3)) * (k >= 2)
    Q = 0.5 * (Q + np.transpose(Q, (0, 2, 1)))              # symmetric in the two x indices

    def u(x):
        return c0 + x @ G.T + np.einsum('abc,...b,...c->...a', Q, x, x)

    def qf(x):                                               # q[a, d] = du_a/dx_d
        return G + 2.0 * np.einsum('adc,...c->...ad', Q, x)

    def sigma(x):
        q = qf(x)
        tr = np.einsum('...aa->...', q)
        return lam * tr[..., None, None] * np.eye(3) + mu * (q + np.swapaxes(q, -1, -2))

    # div sigma_a = lam d_a(tr q) + mu (lap u_a + d_a div u) = 2 lam Q_bba + mu (2 Q_add + 2 Q_dad)
    divs = 2 * lam * np.einsum('bba->a', Q) + mu * (2 * np.einsum('add->a', Q) + 2 * np.einsum('dad->a', Q))
    f = lambda x: np.broadcast_to(-divs, x.shape[:-1] + (3,)).copy()
    g = lambda x, n: -np.einsum('...ad,...d->...a', sigma(x), n)
    w = _box_workload(blk.elasticity(3, lam, mu, 1.0), k, u, qf, f, g, 3, 0.15 if k == 1 else 0.0)
    _, _, _, (eu, eq) = _solve_errors(w)
    assert eu < 1e-10 and eq < 1e-9


def test_beam_tip_deflection_timoshenko():
    """Sec. 6.2 beam, 20 x 4 x 4 hexahedra, Q^2, lambda = mu = 1: the mean
    tip deflection under unit traction t = (0, 0, -1) equals the compliance
    r . uhat = <g, uhat> and agrees within 2% with Timoshenko beam theory,
    delta = F L^3 / (3 E I) + F L / (kappa G A) = 200 + 6 (E = mu (3 lam +
    2 mu) / (lam + mu) = 2.5, I = 1/12, G = mu = 1, kappa = 5/6, A = 1)."""
    w = W.hex_beam(n=4, k=2)
    assert w.face_dirichlet.sum() == 16 and w.n_elem == 320
    s = OracleSystem(w)
    uh = s.direct()
    compliance = float(np.ravel(s.r) @ np.ravel(uh))
    delta = 125.0 / (3 * 2.5 / 12.0) + 5.0 / (5.0 / 6.0)
    assert compliance < 0.0                                  # deflects along the traction
    assert abs(-compliance - delta) < 0.02 * delta


# ------------------------------------------------------------ tetrahedra
@pytest.mark.parametrize('k,ns,lo', [(1, (4, 8), 1.85), (2, (2, 4), 2.7)])
def test_tet_mms_rates(k, ns, lo):
    """P^k on Kuhn tetrahedra: L2 errors of u and q decrease at about k+1."""
    errs = [_solve_errors(W.tet_poisson(n=n, k=k))[3] for n in ns]
    (eu0, eq0), (eu1, eq1) = errs
    assert np.log2(eu0 / eu1) > lo and np.log2(eq0 / eq1) > lo


def test_tet_patch_and_flux_exact():
    """A quadratic u on P^2 tetrahedra is reproduced exactly, with Dirichlet
    data on x = 0 and its outward flux g = -grad u . n on the five other
    sides (the faces' nodes are matched across elements by position, so the
    permuted face bases are exercised)."""
    from hdg_inputs import mesh as meshmod

    def u(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return (0.5 + 0.3 * X - 0.2 * Y + 0.4 * Z + X * X - 0.5 * X * Y + 0.7 * Y * Z - 0.3 * Z * Z)[..., None]

    def qf(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return np.stack([0.3 + 2 * X - 0.5 * Y, -0.2 - 0.5 * X + 0.7 * Z, 0.4 + 0.7 * Y - 0.6 * Z], -1)[..., None, :]
    f = lambda x: np.full(x.shape[:-1] + (1,), -(2.0 - 0.6))          # -lap u
    m = meshmod.tet_mesh(3)
    ref = blk.reference_element(m, 2)
    g = lambda x, n: -np.einsum('...d,...d->...', qf(x)[..., 0, :], n)[..., None]
    w = W.Workload('tet_patch', m, ref, blk.face_permutations(m, ref), blk.poisson(3), 1, 'function', f,
                   u, qf, k=2, dirichlet=W.boundary_faces_at(m, 0, 0.0), neumann_flux=g)
    assert (w.perm != np.arange(w.PF)).any()
    _, _, _, (eu, eq) = _solve_errors(w)
    assert eu < 1e-11 and eq < 1e-10


def test_class_blocks_equal_per_element_blocks():
    """The blocks gathered from one representative per element class (same
    shape up to translation, same face-node permutations) equal the blocks
    generated element by element; the traction loads stay per element."""
    w = W.tet_obstacle(n=6, k=2, hole=0.34)
    rb, cls, ruh = W.class_blocks(w)
    assert len(np.unique(cls)) < w.n_elem // 50
    full = w.blocks()
    for k in ('Me', 'Bd', 'Cd', 'D', 'E', 'F', 'G', 'H', 'J'):
        assert np.abs(rb[k][cls] - full[k]).max() <= 1e-14 * np.abs(full[k]).max(), k
    assert np.array_equal(ruh, full['ruh']) and not full['ru'].any()


@pytest.mark.parametrize('k,lo', [(1, 1.7), (2, 2.75)])
def test_quad_mms_rates(k, lo):
    """Q^k quadrilaterals (the Burgers workload's elements): Poisson with
    u = sin(pi x) sin(pi y), errors of u and q fall at about order k + 1."""
    from hdg_inputs import mesh as meshmod
    errs = []
    for n in (4, 8):
        m = meshmod.quad_mesh(n)
        ref = blk.reference_element(m, k)
        u, f, q = W._sin_product(2)
        w = W.Workload('quad_poisson', m, ref, blk.face_permutations(m, ref), blk.poisson(2), 1, 'function', f, u,
                       q, k=k)
        errs.append(_solve_errors(w)[3])
    (eu0, eq0), (eu1, eq1) = errs
    assert np.log2(eu0 / eu1) > lo and np.log2(eq0 / eq1) > lo


def test_beam_preconditioner_ordering():
    """Sec. 6.2's ordering on the 10 x 2 x 2 Q^1 beam, GMRES(50)-CGS to 1e-6:
    ASM-PP(10) < BJ-PP(10) < ASM < BJ in iterations (Tables 5-6), with the
    polynomials cutting the counts at least fivefold (here 6403 -> 19 for BJ,
    146 -> 16 for ASM)."""
    from oracle import precond, krylov
    w = W.hex_beam(n=2, k=1)
    s = OracleSystem(w)
    b = s.r[:, 0]
    K = s.K.tocsr()
    Binv = precond.bj_setup(K, s.bsz)
    subs = precond.asm_setup(K, s.elem_dofs)
    its = {}
    for name, M in (('BJ', lambda v: precond.bj_apply(Binv, v)), ('ASM', lambda v: precond.asm_apply(subs, v))):
        _, it = krylov.gmres(lambda v: K @ v, M, b, m=50, rtol=1e-6, maxit=20000)
        its[name] = it['iters']
        A = lambda v, M=M: M(K @ v)
        th = precond.pp_setup(A, w.random_vector(11), 10)
        _, it = krylov.gmres(lambda v: K @ v, lambda v: precond.pp_apply(A, th, M(v)), b, m=50, rtol=1e-6,
                             maxit=20000)
        its[name + '-PP'] = it['iters']
    assert its['ASM-PP'] < its['BJ-PP'] < its['ASM'] < its['BJ']
    assert its['BJ-PP'] * 5 < its['BJ'] and its['ASM-PP'] * 5 < its['ASM']


@pytest.mark.parametrize('name', ['elasticity_perturbed', 'poisson', 'beam', 'tets'])
def test_load_vectors_equal_block_load_vectors(name):
    """The load vectors computed without the element matrices (for the
    device-generated blocks) equal those of the full block generation."""
    w = {'elasticity_perturbed': lambda: W.hex_elasticity(n=3, k=2, R=3),
         'poisson': lambda: W.hex_poisson(n=3, k=2),
         'beam': lambda: W.hex_beam(n=2, k=1),
         'tets': lambda: W.tet_poisson(n=2, k=2)}[name]()
    full = w.blocks()
    ru, ruh = w.load_vectors()
    assert np.abs(ru - full['ru']).max() <= 1e-14 * max(np.abs(full['ru']).max(), 1e-300)
    assert np.array_equal(ruh, full['ruh'])
    part = w.load_vectors(5, 9)
    assert np.array_equal(part[0], ru[5:9])
