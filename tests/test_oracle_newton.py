"""Pins of the damped Newton outer loop and of the Burgers residual and
Jacobian blocks (Welter & Nguyen, Sec. 2.3 and Sec. 6.1's steady viscous
Burgers problem)."""
import numpy as np
import pytest

from hdg_inputs import burgers as BG
from oracle.newton import newton


def test_burgers_jacobian_matches_finite_differences():
    """The blocks D, E, F, G, H, J applied to an increment that satisfies the
    linear q-equation equal the centred difference of the residuals R_u and
    R_uhat along it (relative 1e-8): the Jacobian is the residual's."""
    P = BG.Burgers(n=3, k=2)
    q, u, uh = P.initial_state()
    rng = np.random.default_rng(0)
    free = (P.face_dirichlet == 0)[:, None]
    u = u + 0.1 * rng.standard_normal(u.shape)
    uh = uh + 0.1 * rng.standard_normal(uh.shape) * free
    q = P.q_from(u, uh)
    b = P.jacobian_blocks(q, u, uh)
    du, duh = rng.standard_normal(u.shape), rng.standard_normal(uh.shape) * free
    dq = P.q_from(du, duh)
    eps = 1e-6
    Rp = P.residual(q + eps * dq, u + eps * du, uh + eps * duh)
    Rm = P.residual(q - eps * dq, u - eps * du, uh - eps * duh)
    E = P.n_elem
    dqf, due = dq.reshape(E, -1), P.element_traces(duh).reshape(E, -1)
    Ju = np.einsum('eij,ej->ei', b['D'], dqf) + np.einsum('eij,ej->ei', b['E'], du) + \
        np.einsum('eij,ej->ei', b['F'], due)
    Juh = np.einsum('eij,ej->ei', b['G'], dqf) + np.einsum('eij,ej->ei', b['H'], du) + \
        np.einsum('eij,ej->ei', b['J'], due)
    fu, fuh = (Rp[0] - Rm[0]) / (2 * eps), ((Rp[1] - Rm[1]) / (2 * eps)).reshape(E, -1)
    assert np.abs(Ju - fu).max() <= 1e-8 * np.abs(fu).max()
    assert np.abs(Juh - fuh).max() <= 1e-8 * np.abs(fuh).max()


def test_newton_manufactured_rate_and_quadratic_convergence():
    """With f = u_y + u u_x - nu lap u for a smooth u and its Dirichlet data on
    every side, Newton converges quadratically (each residual at most a
    bounded multiple of the square of the previous one once below 1e-2) and
    the Q^2 errors fall at about order k + 1 = 3."""
    u_ex, _, f = BG.manufactured()
    errs = []
    for n in (4, 8):
        P = BG.Burgers(n=n, k=2, f=f, u_dirichlet=u_ex, outflow=False)
        (q, u, uh), hist = newton(P, P.initial_state(), tol=1e-11)
        r = [h for h, _ in hist]
        assert r[-1] <= 1e-11 and len(r) <= 6
        for a, b in zip(r[:-1], r[1:]):
            if a < 1e-2 and b > 1e-13:
                assert b <= 1e3 * a * a
        uq = np.einsum('qi,ei->eq', P.Q.phi, u)
        errs.append(np.sqrt((P.Q.wJ * (uq - u_ex(P.Q.xq)) ** 2).sum()))
    assert 2.7 < np.log2(errs[0] / errs[1]) < 3.3


def test_newton_paper_burgers_converges():
    """Sec. 6.1's problem (nu = 1/200, u = 1 - 2x on three sides, outflow at
    y = 1) on 8 x 8 Q^2 quadrilaterals: the damped Newton iteration from
    u = 1 - 2x reaches a residual of 1e-8 in at most 10 steps, with full
    steps at the end; the solution is antisymmetric about x = 1/2 to the
    tolerance (the problem is)."""
    P = BG.Burgers(n=8, k=2)
    (q, u, uh), hist = newton(P, P.initial_state(), tol=1e-8)
    assert hist[-1][0] <= 1e-8 and len(hist) <= 11 and hist[-1][1] == 1.0
    # u(1 - x, y) = -u(x, y): compare element values at mirrored quadrature points
    X = P.Q.xq
    uq = np.einsum('qi,ei->eq', P.Q.phi, u)
    key = lambda x: (np.round(x[..., 0], 9), np.round(x[..., 1], 9))
    pts = {key(x): v for x, v in zip(X.reshape(-1, 2), uq.ravel())}
    diffs = [abs(v + pts[key(np.array([1 - x[0], x[1]]))]) for x, v in zip(X.reshape(-1, 2), uq.ravel())]
    assert max(diffs) < 1e-6
