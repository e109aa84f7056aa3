"""HDG local postprocessing u* (oracle only).  Not in Welter & Nguyen; it is
the standard element-wise postprocessing of Cockburn, Gopalakrishnan and Sayas
(2010): u* in P^{k+1}(K) with
    (grad u*, grad w)_K = (q_h, grad w)_K   for all w in P^{k+1}(K),
    (u*, 1)_K = (u_h, 1)_K,
where q_h approximates grad u (Eq. HDGa).  Triangles only.
Test infrastructure: see oracle/__init__.py."""
import numpy as np

from hdg_inputs import basis as B


def postprocess_tri(mesh, k, u, q, nquad=None):
    """u (E, PE) and q (E, D*PE) coefficients of the P^k nodal basis.
    Returns (phi_star at the quadrature points, coefficients (E, P_{k+1}),
    quadrature points (E, nq, 2), weights*|detJ| (E, nq))."""
    nquad = nquad or (k + 4)
    pts, wts = B.tri_rule(nquad)
    phi_k, _ = B.tri_basis(k, pts)
    phi_s, dphi_s = B.tri_basis(k + 1, pts)
    E = mesh.n_elem
    X3 = mesh.verts[mesh.elems]
    v0 = X3[:, 0, :]
    Jm = np.stack([X3[:, 1, :] - v0, X3[:, 2, :] - v0], axis=2)
    det = np.abs(np.linalg.det(Jm))
    Jinv = np.linalg.inv(Jm)
    PE = phi_k.shape[1]
    Ps = phi_s.shape[1]
    coef = np.empty((E, Ps))
    for e in range(E):
        g = np.einsum('qib,ba->qia', dphi_s, Jinv[e])                # physical gradients
        w = wts * det[e]
        S = np.einsum('q,qia,qja->ij', w, g, g)
        qh = np.einsum('qi,di->qd', phi_k, q[e].reshape(2, PE))
        rhs = np.einsum('q,qd,qid->i', w, qh, g)
        uh = phi_k @ u[e]
        # replace one (redundant) equation by the mean-value constraint
        mean_row = np.einsum('q,qi->i', w, phi_s)
        S[0] = mean_row
        rhs[0] = np.sum(w * uh)
        coef[e] = np.linalg.solve(S, rhs)
    xq = v0[:, None, :] + np.einsum('eab,nb->ena', Jm, pts)
    return phi_s, coef, xq, wts[None, :] * det[:, None]
