"""Pins of the oracle's GMRES and preconditioners against the mathematics
(Welter & Nguyen, Sec. 3.1-3.4, 4.4-4.7)."""
import numpy as np
import pytest
import scipy.sparse as sp

from hdg_inputs import workloads as W
from oracle import krylov, precond
from tests.oracle_helpers import OracleSystem


@pytest.fixture(scope='module')
def tri_sys():
    return OracleSystem(W.tri_poisson(8, 2))


@pytest.fixture(scope='module')
def hex_el_sys():
    return OracleSystem(W.hex_elasticity(n=3, k=1, R=1))


def test_gmres_bj_matches_direct(tri_sys):
    s = tri_sys
    Binv = precond.bj_setup(s.K, s.bsz)
    b = s.r[:, 0]
    x, info = krylov.gmres(lambda v: s.K @ v, lambda v: precond.bj_apply(Binv, v), b, m=30, rtol=1e-10)
    xd = s.direct()[:, 0] if s.direct().ndim == 2 else s.direct()
    assert info['converged'] and info['true_rel'] <= 1e-10
    cond = np.linalg.cond(s.K.toarray())
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < cond * 1e-10


@pytest.mark.parametrize('orth', ['cgs', 'mgs', 'cgs2'])
def test_gmres_full_space_converges_in_n_steps(orth):
    """With m >= n, GMRES is exact after at most n steps (here n = 12)."""
    rng = np.random.default_rng(0)
    n = 12
    A = rng.standard_normal((n, n)) + n * np.eye(n)
    b = rng.standard_normal(n)
    x, info = krylov.gmres(lambda v: A @ v, lambda v: v, b, m=n, rtol=1e-13, orth=orth)
    assert info['iters'] <= n
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


def test_gmres_ls_estimate_equals_true_preconditioned_residual(tri_sys):
    """Inside one cycle |g_{j+1}| equals ||P^{-1}(b - K x_j)|| (Givens LS),
    and it does not increase."""
    s = tri_sys
    K = s.K.toarray()
    Binv = precond.bj_setup(s.K, s.bsz)
    P = lambda v: precond.bj_apply(Binv, v)
    b = s.r[:, 0]
    zb = np.linalg.norm(P(b))
    hist = []
    for j in range(1, 12):
        x, info = krylov.gmres(lambda v: K @ v, P, b, m=j, rtol=1e-30, maxit=j)
        true = np.linalg.norm(P(b - K @ x)) / zb
        hist.append((info['history'][-1], true))
    for est, true in hist:
        assert abs(est - true) <= 1e-10 * max(true, 1e-300) + 1e-14
    est = [h[0] for h in hist]
    assert all(e1 <= e0 * (1 + 1e-12) for e0, e1 in zip(est[:-1], est[1:]))


def test_block_diagonal_system_bj_one_iteration():
    """If K is block diagonal, block-Jacobi is exact: one GMRES step."""
    rng = np.random.default_rng(1)
    blocks = [rng.standard_normal((4, 4)) + 4 * np.eye(4) for _ in range(7)]
    K = sp.csr_matrix(sp.block_diag(blocks))
    Binv = precond.bj_setup(K, 4)
    for f in range(7):
        assert np.allclose(Binv[f] @ blocks[f], np.eye(4), atol=1e-12)
    b = rng.standard_normal(28)
    x, info = krylov.gmres(lambda v: K @ v, lambda v: precond.bj_apply(Binv, v), b, m=10, rtol=1e-12)
    assert info['iters'] == 1 and info['true_rel'] < 1e-12


def test_bj_inverse_identity(hex_el_sys):
    s = hex_el_sys
    Binv = precond.bj_setup(s.K, s.bsz)
    Kc = s.K.tocsr()
    for f in range(0, Binv.shape[0], 7):
        sl = slice(f * s.bsz, (f + 1) * s.bsz)
        assert np.abs(Binv[f] @ Kc[sl, sl].toarray() - np.eye(s.bsz)).max() < 1e-12


def test_asm_blocks_equal_paper_construction(hex_el_sys):
    """Sec. 4.6 builds P^e from Kbar^e, replacing the diagonal block of every
    interior face by Kbar^{e1}_{l1l1} + Kbar^{e2}_{l2l2}; this equals the
    definition R_e K R_e^T (Sec. 3.3) on the element's free faces."""
    s = hex_el_sys
    w = s.w
    b = s.bsz
    fe = w.mesh.face_elem
    fd = w.face_dirichlet
    locs = precond.asm_local_matrices(s.K, s.elem_dofs)
    for e in range(w.n_elem):
        P = s.Kbar[e].copy()
        for l in range(w.n_lfe):
            f = w.mesh.elem_face[e, l]
            if fe[f, 2] >= 0:
                e1, l1, e2, l2 = fe[f]
                P[l * b:(l + 1) * b, l * b:(l + 1) * b] = (s.Kbar[e1][l1 * b:(l1 + 1) * b, l1 * b:(l1 + 1) * b]
                                                         + s.Kbar[e2][l2 * b:(l2 + 1) * b, l2 * b:(l2 + 1) * b])
        free = np.concatenate([np.arange(l * b, (l + 1) * b) for l in range(w.n_lfe)
                               if fd[w.mesh.elem_face[e, l]] == 0])
        assert np.abs(P[np.ix_(free, free)] - locs[e]).max() < 1e-12 * np.abs(locs[e]).max()


def test_asm_beats_bj(hex_el_sys):
    """ASM needs fewer iterations than BJ (Sec. 5, Tables 1, 5)."""
    s = hex_el_sys
    b = s.r[:, 0]
    Binv = precond.bj_setup(s.K, s.bsz)
    subs = precond.asm_setup(s.K, s.elem_dofs)
    _, i_bj = krylov.gmres(lambda v: s.K @ v, lambda v: precond.bj_apply(Binv, v), b, m=50, rtol=1e-8)
    _, i_asm = krylov.gmres(lambda v: s.K @ v, lambda v: precond.asm_apply(subs, v), b, m=50, rtol=1e-8)
    assert i_asm['converged'] and i_bj['converged']
    assert i_asm['iters'] < i_bj['iters']


def _few_eigs_matrix(seed=2):
    """A = S T S^{-1}, T block diagonal with five 2x2 rotation blocks
    (eigenvalues 1 +- 0.5i) and the values 2, 3, 5 repeated: five distinct
    eigenvalues in all."""
    rng = np.random.default_rng(seed)
    rot = np.array([[1.0, 0.5], [-0.5, 1.0]])
    T = sp.block_diag([rot] * 5 + [np.diag([2.0] * 7 + [3.0] * 7 + [5.0] * 6)]).toarray()
    n = T.shape[0]
    S = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    return S @ T @ np.linalg.inv(S)


def test_pp_exact_on_few_eigenvalues():
    """With exact Arnoldi on A with 5 distinct eigenvalues (one conjugate
    pair), the harmonic Ritz values are the eigenvalues and p(A) = A^{-1}."""
    A = _few_eigs_matrix()
    rng = np.random.default_rng(3)
    y = rng.standard_normal(A.shape[0])
    theta = precond.pp_setup(lambda v: A @ v, rng.standard_normal(A.shape[0]), 5)
    expect = np.array([2, 3, 5, 1 + 0.5j, 1 - 0.5j])
    assert np.allclose(np.sort_complex(theta), np.sort_complex(expect), atol=1e-9)
    z = precond.pp_apply(lambda v: A @ v, theta, y)
    assert np.linalg.norm(z - np.linalg.solve(A, y)) < 1e-9 * np.linalg.norm(z)


def test_pp_recurrence_equals_complex_product_form():
    """The real recurrence equals sum_j prod_{i<j}(I - A/theta_i) y/theta_j
    evaluated directly in complex arithmetic."""
    rng = np.random.default_rng(4)
    n = 16
    A = rng.standard_normal((n, n)) + 4 * np.eye(n)
    y = rng.standard_normal(n)
    theta = precond.pp_setup(lambda v: A @ v, rng.standard_normal(n), 6)
    assert np.any(theta.imag != 0)
    z = precond.pp_apply(lambda v: A @ v, theta, y)
    acc = np.zeros(n, complex)
    prod = np.eye(n, dtype=complex)
    for t in theta:
        acc += prod @ y / t
        prod = prod @ (np.eye(n) - A / t)
    assert np.abs(acc.imag).max() < 1e-10 * np.abs(acc).max()
    assert np.abs(z - acc.real).max() < 1e-10 * np.abs(acc).max()


def test_harmonic_ritz_defining_pencil():
    """theta is a harmonic Ritz value iff H_{P+1,P}^T H_{P+1,P} - theta H_PP^T
    is singular (the harmonic Ritz condition with respect to A K_P)."""
    rng = np.random.default_rng(5)
    n = 40
    A = rng.standard_normal((n, n)) / np.sqrt(n) + 2 * np.eye(n)
    P = 8
    H = precond.arnoldi_mgs(lambda v: A @ v, rng.standard_normal(n), P)
    th = precond.harmonic_ritz(H)
    G = H.T @ H
    for t in th:
        smin = np.linalg.svd(G - t * H[:P, :P].T, compute_uv=False)[-1]
        assert smin < 1e-10 * np.linalg.norm(G)


def test_leja_order_properties():
    th = np.array([1.0, 4.0, 2.0 + 1j, 2.0 - 1j, 0.5, 3.0])
    o = precond.leja_order(th)
    assert o[0] == 4.0
    for i, t in enumerate(o):
        if t.imag > 0:
            assert o[i + 1] == np.conj(t)
    # brute force of the greedy rule for the real values
    real = np.array([0.3, 1.7, 0.9, 2.5, 1.1])
    o = precond.leja_order(real).real
    chosen = [2.5]
    rest = [0.3, 1.7, 0.9, 1.1]
    while rest:
        nxt = max(rest, key=lambda v: np.sum(np.log(np.abs(v - np.array(chosen)))))
        chosen.append(nxt)
        rest.remove(nxt)
    assert np.allclose(o, chosen)


def test_chebyshev_residual_polynomial_closed_form():
    """For the Chebyshev iteration, 1 - lam p(lam) = T_{d+1}((c - lam)/h) /
    T_{d+1}(c/h) with c, h the centre and half-width of [alpha, beta]."""
    lam = np.linspace(0.2, 3.0, 9)
    alpha, beta, d = 0.15, 3.2, 4
    y = np.ones_like(lam)
    z = precond.chebyshev_apply(lambda v: lam * v, alpha, beta, d, y)
    c, h = (alpha + beta) / 2, (beta - alpha) / 2
    T = np.polynomial.chebyshev.Chebyshev.basis(d + 1)
    assert np.allclose(1 - lam * z, T((c - lam) / h) / T(c / h), atol=1e-12)


def test_hybrid_bj_pp_reduces_iterations(hex_el_sys):
    """BJ-PP(P) needs far fewer GMRES iterations than BJ (Sec. 5, Table 5)."""
    s = hex_el_sys
    b = s.r[:, 0]
    Binv = precond.bj_setup(s.K, s.bsz)
    M = lambda v: precond.bj_apply(Binv, v)
    A = lambda v: M(s.K @ v)
    theta = precond.pp_setup(A, np.random.default_rng(31).standard_normal(len(b)), 10)
    Pinv = lambda v: precond.pp_apply(A, theta, M(v))
    _, i_bj = krylov.gmres(lambda v: s.K @ v, M, b, m=50, rtol=1e-8)
    _, i_pp = krylov.gmres(lambda v: s.K @ v, Pinv, b, m=50, rtol=1e-8)
    assert i_pp['converged']
    assert i_pp['iters'] * 3 < i_bj['iters']


def test_chebyshev_bounds_from_exact_ritz_values():
    """With P = n Arnoldi steps on a symmetric matrix the Ritz values are the
    eigenvalues, so the bounds are [0.9 lambda_min, 1.1 lambda_max]."""
    rng = np.random.default_rng(6)
    lam = np.array([0.5, 0.8, 1.3, 2.0, 2.9, 4.0])
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    A = Q @ np.diag(lam) @ Q.T
    a, b = precond.chebyshev_bounds(lambda v: A @ v, rng.standard_normal(6), 6)
    assert abs(a - 0.45) < 1e-10 and abs(b - 4.4) < 1e-10


# ------------------------------------------------------------ ASM apply pins
def _asm_operator_checks(apply, s, subs):
    """Invariants of P = sum_e R_e^T (R_e K R_e^T)^{-1} R_e (Sec. 3.3) for a
    symmetric definite K: P is symmetric with K's sign of definiteness, and
    trace(P) = sum_e trace((R_e K R_e^T)^{-1}) because R_e R_e^T = I.  Returns
    (symmetry error, definiteness holds, relative trace error)."""
    rng = np.random.default_rng(12)
    n = s.K.shape[0]
    y1, y2 = rng.standard_normal(n), rng.standard_normal(n)
    p1, p2 = apply(subs, y1), apply(subs, y2)
    sym = abs(y1 @ p2 - y2 @ p1) / (np.linalg.norm(y1) * np.linalg.norm(p2))
    sign = np.sign((s.K @ y1) @ y1)
    definite = all(sign * (y @ apply(subs, y)) > 0 for y in rng.standard_normal((5, n)))
    tr = 0.0
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        tr += apply(subs, e)[i]
    tr_local = sum(np.sum(1.0 / np.linalg.eigvalsh(0.5 * (A + A.T)))
                   for A in precond.asm_local_matrices(s.K, s.elem_dofs))
    return sym, definite, abs(tr - tr_local) / abs(tr_local)


def test_asm_apply_symmetric_definite_and_trace(hex_el_sys):
    """The HDG elasticity K is symmetric and definite, so the ASM operator of
    Sec. 3.3 / 4.6 is symmetric, definite with the same sign, and its trace is
    the sum of the local inverses' traces.  Dropping or overwriting the
    contribution of one element on a shared face breaks all three."""
    s = hex_el_sys
    Kd = s.K.toarray()
    assert np.abs(Kd - Kd.T).max() < 1e-12 * np.abs(Kd).max()
    subs = precond.asm_setup(s.K, s.elem_dofs)
    sym, definite, tr = _asm_operator_checks(precond.asm_apply, s, subs)
    assert sym < 1e-12 and definite and tr < 1e-10


def test_asm_apply_planted_overwrite_is_caught(hex_el_sys):
    """Planted mistakes: z[d] = ... instead of z[d] += ... (each shared face
    keeps only the last element's contribution), and one element's
    contribution left out.  The invariants above must reject both."""
    s = hex_el_sys
    subs = precond.asm_setup(s.K, s.elem_dofs)

    def overwrite(subs_, y):
        z = np.zeros_like(y)
        for d, inv in subs_:
            z[d] = inv @ y[d]
        return z

    def drop_one(subs_, y):
        z = np.zeros_like(y)
        for d, inv in subs_[1:]:
            z[d] += inv @ y[d]
        return z
    for wrong in (overwrite, drop_one):
        sym, definite, tr = _asm_operator_checks(wrong, s, subs)
        assert sym > 1e-6 or not definite or tr > 1e-6


def test_asm_apply_exact_on_disjoint_subdomains():
    """Subdomains that partition the unknowns of a block-diagonal K (no face
    shared by two elements): the ASM operator is K^{-1} exactly."""
    rng = np.random.default_rng(13)
    sizes = [5, 3, 7, 4]
    blocks = []
    for m in sizes:
        G = rng.standard_normal((m, m))
        blocks.append(G @ G.T + m * np.eye(m))
    K = sp.csr_matrix(sp.block_diag(blocks))
    n = K.shape[0]
    perm = rng.permutation(n)                       # scatter each subdomain's unknowns
    Kp = sp.csr_matrix(K.toarray()[np.ix_(np.argsort(perm), np.argsort(perm))])
    offs = np.cumsum([0] + sizes)
    dofs = [perm[offs[i]:offs[i + 1]] for i in range(len(sizes))]
    # pad with -1 entries (Dirichlet faces are skipped)
    elem_dofs = [np.concatenate([d, [-1, -1]]) for d in dofs]
    subs = precond.asm_setup(Kp, elem_dofs)
    y = rng.standard_normal(n)
    z = precond.asm_apply(subs, y)
    assert np.abs(z - np.linalg.solve(Kp.toarray(), y)).max() < 1e-12 * np.abs(z).max()
