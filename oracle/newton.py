"""Damped Newton-Raphson outer loop (Welter & Nguyen, Sec. 2.3: linearise the
HDG system at the current iterate, condense, solve for the trace increment,
recover the element increments, update with a step alpha chosen by line
search so that the residual norm decreases; stop when the residual norm is
below a tolerance).  Test infrastructure: see oracle/__init__.py.

Each step here condenses with `condense_local` (Eqs. w15-w22), assembles K
by its definition and solves K dx = r with a sparse direct solver: the
exact linear solve the GPU path's preconditioned GMRES approximates.  The
problem object supplies the residual and the Jacobian blocks at a state
(hdg_inputs.burgers)."""
import numpy as np
import scipy.sparse.linalg as spl

from .condense import condense_local
from .assemble import assemble, element_traces, recover


def newton(P, state, tol=1e-8, max_steps=30, max_halvings=12):
    """Newton iterations from `state` = (q, u, uhat) (q consistent with the
    q-equation).  Returns (state, history) with history a list of
    (residual norm, alpha) per step, the first entry the initial norm."""
    q, u, uh = state
    E, PF, nl = P.n_elem, P.PF, P.n_lfe
    fd = P.face_dirichlet
    zD = np.zeros((P.mesh.n_face, PF, 1))
    hist = [(P.residual_norm(q, u, uh), None)]
    for _ in range(max_steps):
        if hist[-1][0] <= tol:
            break
        blk = P.jacobian_blocks(q, u, uh)
        Kbar, rbar, rec = condense_local(blk, 1, nl)
        K, r = assemble(Kbar, rbar, P.mesh.elem_face, fd, zD, 1, PF)
        dx = spl.spsolve(K.tocsc(), r[:, 0])
        due = element_traces(dx[:, None], P.mesh.elem_face, fd, zD, 1, PF)
        du, dq = recover(rec, due, 1, nl)
        duh = np.zeros_like(uh)
        duh[fd == 0] = dx.reshape(-1, PF)
        du = du[:, :, 0]
        dq = dq[:, :, 0].reshape(E, 2, -1)
        alpha, r0 = 1.0, hist[-1][0]
        for _ in range(max_halvings):
            rn = P.residual_norm(q + alpha * dq, u + alpha * du, uh + alpha * duh)
            if rn < r0:
                break
            alpha *= 0.5
        q, u, uh = q + alpha * dq, u + alpha * du, uh + alpha * duh
        hist.append((rn, alpha))
    return (q, u, uh), hist
