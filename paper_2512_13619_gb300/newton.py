"""Damped Newton-Raphson outer loop around the GPU trace solver (Welter &
Nguyen, Sec. 2.3): at each iterate the problem object supplies the
Jacobian blocks of Eq. matrixform and the residuals (as the right-hand
sides ru = -R_u, ruh = -R_uhat with r_q = 0); the library condenses them,
assembles the face-block trace matrix, sets up the preconditioner and solves
for the trace increment with preconditioned GMRES; recovery gives the
element increments; the step alpha halves until the residual norm
decreases.

The problem object (e.g. hdg_inputs.burgers.Burgers) provides mesh,
face_dirichlet, n_lfe, PE, PF, jacobian_blocks(q, u, uhat) and
residual_norm(q, u, uhat); states are (q (E, D, P_E), u (E, P_E),
uhat (N_F, P_F)) of a scalar equation.
"""
import time

import numpy as np

from . import driver


def newton_solve(P, o, v0=None, tol=1e-8, max_steps=30, max_halvings=12, device=0):
    """Newton iterations from P.initial_state(); o: hdg_solver_opts of the
    linear solves; v0: start vector of the polynomial preconditioner's
    Arnoldi cycle (over the free trace unknowns) when o uses one.  Returns
    (state, info) with info = {'history': [(norm, alpha)], 'gmres': total
    linear iterations, 'gmres_per_step': [...], 'linear_s': seconds in the
    condense/assemble/set-up/solve/recover calls, 'host_s': seconds in the
    residual and Jacobian evaluations}."""
    import torch
    m = P.mesh
    dim = m.dim
    p = driver.Problem(dim, P.n_lfe, 1, P.PE, P.PF, m.elem_face, m.face_elem, P.face_dirichlet, 1, device)
    q, u, uh = P.initial_state()
    E = m.n_elem
    zeros = np.zeros((m.n_face, P.PF, 1))
    hist = [(P.residual_norm(q, u, uh), None)]
    per_step, t_lin, t_host = [], 0.0, 0.0
    try:
        for _ in range(max_steps):
            if hist[-1][0] <= tol:
                break
            t0 = time.perf_counter()
            blk = P.jacobian_blocks(q, u, uh)
            t1 = time.perf_counter()
            p.condense(blk)
            p.set_dirichlet(zeros)
            p.assemble(o)
            p.setup_precond(o, v0)
            st, info = p.solve(o)
            if st != 0:
                raise RuntimeError('linear solve in Newton step %d: %s' % (len(hist), driver.L.hdg_status_str(st)))
            per_step.append(int(info.iters))
            duh = p.trace()[:, :, 0]
            du, dq = p.recover()
            torch.cuda.synchronize(device)
            t2 = time.perf_counter()
            du = du[:, :, 0]
            dq = dq[:, :, 0].reshape(E, dim, -1)
            alpha, r0 = 1.0, hist[-1][0]
            for _ in range(max_halvings):
                rn = P.residual_norm(q + alpha * dq, u + alpha * du, uh + alpha * duh)
                if rn < r0:
                    break
                alpha *= 0.5
            q, u, uh = q + alpha * dq, u + alpha * du, uh + alpha * duh
            hist.append((rn, alpha))
            t_lin += t2 - t1
            t_host += (t1 - t0) + (time.perf_counter() - t2)
    finally:
        p.close()
    return (q, u, uh), {'history': hist, 'gmres': int(sum(per_step)), 'gmres_per_step': per_step,
                        'linear_s': t_lin, 'host_s': t_host}
