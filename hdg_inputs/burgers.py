"""Steady two-dimensional viscous Burgers problem of Welter & Nguyen, Sec. 6.1
(after Moro et al.): u_y + (u^2/2)_x - nu (u_xx + u_yy) = f on the unit square,
nu = 1/200, discretised by HDG on Q^k quadrilaterals (Sec. 2):

  q = grad u                                   (q-equation, linear)
  -(F(u, q), grad v) + <Fhat . n, v> = (f, v)    F = c(u) - nu q, c(u) = (u^2/2, u)
  sum over elements <Fhat . n, mu> = 0           Fhat . n = c(uhat) . n - nu q . n + tau (u - uhat)

with Dirichlet data on x = 0, x = 1, y = 0 and an outflow face y = 1, on which
the trace equation keeps only the diffusive and stabilisation parts of the
numerical flux (<Fhat . n - c(uhat) . n, mu> = 0).

This module evaluates, at a state (q, u, uhat), the residuals R_u, R_uhat and
the Newton-Jacobian blocks of Eq. matrixform (Sec. 2.3: D, E, F, G, H, J at
the current iterate; A, B, C are those of the linear q-equation).  The
blocks are the inputs of each Newton step's static condensation and trace
solve; the Newton update and line search (Sec. 2.3) live with the solvers.
"""
from dataclasses import dataclass
import numpy as np

from . import mesh as meshmod
from . import blocks as blk


@dataclass
class BurgersQuad:
    """Quadrature data of every element (constant over the Newton steps)."""
    wJ: np.ndarray        # (E, nq) volume weights
    phi: np.ndarray       # (nq, PE)
    g: np.ndarray         # (E, nq, PE, 2) physical gradients
    xq: np.ndarray        # (E, nq, 2)
    fw: list              # per face l: (E, nfq) weights
    fn: list              # per face l: (E, nfq, 2) unit outward normals
    fph: list             # per face l: (nfq, PE) element basis at the face points
    fpsi: list            # per face l: (E, nfq, PF) face basis in the face's global node order
    fx: list              # per face l: (E, nfq, 2) points


def quadrature_data(mesh, ref, perm):
    E = mesh.n_elem
    elems = np.arange(E)
    x, Jac, det, Jinv = blk.geometry(mesh, elems, ref.vol_pts)
    wJ = ref.vol_wts[None, :] * np.abs(det)
    g = np.einsum('qib,eqba->eqia', ref.dphi, Jinv)
    fw, fn, fph, fpsi, fx = [], [], [], [], []
    for l in range(ref.n_lfe):
        xf, Jf, detf, Jinvf = blk.geometry(mesh, elems, ref.face_ref_pts[l])
        nv = detf[:, :, None] * np.einsum('eqba,b->eqa', Jinvf, ref.face_normal_ref[l])
        dA = np.linalg.norm(nv, axis=2)
        fw.append(ref.face_wts[None, :] * dA)
        fn.append(nv / dA[:, :, None])
        fph.append(ref.face_phi[l])
        fpsi.append(np.transpose(ref.face_psi[:, perm[elems, l, :]], (1, 0, 2)))
        fx.append(xf)
    return BurgersQuad(wJ, ref.phi, g, x, fw, fn, fph, fpsi, fx)


class Burgers:
    """The discrete problem: mesh, reference element, boundary flags,
    viscosity, stabilisation, source, and the evaluation of residuals and
    Jacobian blocks at a state."""

    def __init__(self, n, k, nu=1.0 / 200.0, tau=2.0, f=None, u_dirichlet=None, outflow=True, nquad=None):
        self.mesh = meshmod.quad_mesh(n)
        self.k = k
        self.ref = blk.reference_element(self.mesh, k, nquad or (2 * k + 1))
        self.perm = blk.face_permutations(self.mesh, self.ref)
        self.nu, self.tau = nu, tau
        self.f = f
        self.u_dirichlet = u_dirichlet or (lambda x: 1.0 - 2.0 * x[..., 0])
        m = self.mesh
        fb = m.face_boundary.astype(bool)
        top = np.zeros(m.n_face, bool)
        if outflow:
            from .workloads import boundary_faces_at
            top = boundary_faces_at(m, 1, 1.0).astype(bool)
        self.face_dirichlet = (fb & ~top).astype(np.uint8)
        self.face_outflow = top
        self.Q = quadrature_data(m, self.ref, self.perm)
        # linear q-equation blocks (Eq. w16): M^e, B_d, C_d
        mats = blk.element_matrices(m, self.ref, self.perm, np.arange(m.n_elem))
        qb = blk.hdg_blocks(mats, blk.poisson(2))
        self.Me, self.Bd, self.Cd = qb['Me'], qb['Bd'], qb['Cd']

    # sizes
    @property
    def n_elem(self): return self.mesh.n_elem

    @property
    def PE(self): return self.ref.PE

    @property
    def PF(self): return self.ref.PF

    @property
    def n_lfe(self): return self.ref.n_lfe

    @property
    def n_free(self): return int((self.face_dirichlet == 0).sum())

    def dirichlet_traces(self):
        """(NF, PF) traces: L2 projection of the Dirichlet data on Dirichlet
        faces, zero elsewhere."""
        v = blk.dirichlet_face_values(self.mesh, self.ref, self.perm,
                                      lambda x: self.u_dirichlet(x)[..., None], 1)
        v[self.face_dirichlet == 0] = 0.0
        return v

    def initial_state(self, u0=None):
        """u = u0 at the element nodes (default: the Dirichlet data's
        extension 1 - 2x), uhat = the Dirichlet traces and u0 on free faces,
        q from the q-equation (so that its residual is zero)."""
        u0 = u0 or self.u_dirichlet
        m = self.mesh
        X = blk.geometry(m, np.arange(m.n_elem), self.ref_nodes())[0]
        u = u0(X)                                                       # (E, PE)
        uh = blk.dirichlet_face_values(m, self.ref, self.perm, lambda x: u0(x)[..., None], 1)
        # interior faces: the same projection (face_values covers boundary faces only)
        for f in np.nonzero(m.face_boundary == 0)[0]:
            e, l = m.face_elem[f, 0], m.face_elem[f, 1]
            uh[f] = self._face_projection(e, l, u0)
        D = self.dirichlet_traces()
        uh[self.face_dirichlet == 1] = D[self.face_dirichlet == 1]
        q = self.q_from(u, uh)
        return q, u, uh

    def ref_nodes(self):
        from . import basis as B
        return B.quad_nodes(self.k)

    def _face_projection(self, e, l, fun):
        Q = self.Q
        w, psi, x = Q.fw[l][e], Q.fpsi[l][e], Q.fx[l][e]
        FF = np.einsum('q,qi,qj->ij', w, psi, psi)
        rhs = np.einsum('q,q,qj->j', w, fun(x), psi)
        return np.linalg.solve(FF, rhs)

    def element_traces(self, uh):
        """(E, n_lfe, PF) traces of every element's faces (global node order)."""
        return uh[self.mesh.elem_face]

    def q_from(self, u, uh):
        """q solving the q-equation: M^e q_d = -(B_d u + C_d uhat^e)."""
        ue = self.element_traces(uh).reshape(self.n_elem, -1)
        rhs = -(np.einsum('edij,ej->edi', self.Bd, u) + np.einsum('edij,ej->edi', self.Cd, ue))
        return np.linalg.solve(self.Me[:, None], rhs[..., None])[..., 0]          # (E, 2, PE)

    # ----------------------------------------------------------- residuals
    def _face_fields(self, l, q, u, ue):
        Q = self.Q
        ph, psi, nrm = Q.fph[l], Q.fpsi[l], Q.fn[l]
        uf = u @ ph.T                                                             # (E, nfq)
        qn = (q[:, 0] @ ph.T) * nrm[..., 0] + (q[:, 1] @ ph.T) * nrm[..., 1]
        uhf = np.matmul(psi, ue[:, l][:, :, None])[..., 0]
        return uf, qn, uhf

    def residual(self, q, u, uh):
        """R_u (E, PE) and the element-side trace residuals R_uhat (E, n_lfe, PF)."""
        Q, nu, tau = self.Q, self.nu, self.tau
        uq = u @ Q.phi.T                                                          # (E, nq)
        Fx = 0.5 * uq * uq - nu * (q[:, 0] @ Q.phi.T)
        Fy = uq - nu * (q[:, 1] @ Q.phi.T)
        Ru = -(np.matmul((Q.wJ * Fx)[:, None, :], Q.g[..., 0]) + np.matmul((Q.wJ * Fy)[:, None, :], Q.g[..., 1]))[:, 0]
        if self.f is not None:
            Ru -= (Q.wJ * self.f(Q.xq)) @ Q.phi
        ue = self.element_traces(uh)
        Ruh = np.zeros((self.n_elem, self.n_lfe, self.PF))
        out = self.face_outflow[self.mesh.elem_face]                                # (E, n_lfe)
        for l in range(self.n_lfe):
            uf, qn, uhf = self._face_fields(l, q, u, ue)
            nrm, w = Q.fn[l], Q.fw[l]
            cn = 0.5 * uhf * uhf * nrm[..., 0] + uhf * nrm[..., 1]
            Fn = cn - nu * qn + tau * (uf - uhf)
            Ru += (w * Fn) @ Q.fph[l]
            Fn_tr = Fn - out[:, l][:, None] * cn
            Ruh[:, l] = np.matmul((w * Fn_tr)[:, None, :], Q.fpsi[l])[:, 0]
        return Ru, Ruh

    def residual_norm(self, q, u, uh):
        """sqrt(|R_u|^2 + |R_uhat|^2) with R_uhat summed over the two sides of
        every free face (the q-equation residual is zero by construction)."""
        Ru, Ruh = self.residual(q, u, uh)
        m = self.mesh
        Rf = np.zeros((m.n_face, self.PF))
        np.add.at(Rf, m.elem_face.ravel(), Ruh.reshape(-1, self.PF))
        Rf = Rf[self.face_dirichlet == 0]
        return float(np.sqrt((Ru ** 2).sum() + (Rf ** 2).sum()))

    # ------------------------------------------------------------ Jacobian
    def _constant_blocks(self):
        """The parts of D, E, F, G, H, J that do not depend on the state
        (computed once): D, G, H entirely; E without the u-dependent
        convection term; F and J without their uhat-dependent parts."""
        if getattr(self, '_const', None) is not None:
            return self._const
        Q, nu, tau = self.Q, self.nu, self.tau
        E, PE, PF, nl = self.n_elem, self.PE, self.PF, self.n_lfe
        wg = Q.wJ[:, :, None, None] * Q.g                                        # (E, nq, PE, 2)
        # D[i, (c, k)] = nu int d_c phi_i phi_k - nu <n_c phi_k, phi_i>
        Dm = nu * np.transpose(np.transpose(wg, (0, 2, 3, 1)) @ Q.phi, (0, 1, 2, 3))  # (E, PE, 2, PE)
        # E[i, k] = -int d_y phi_i phi_k + tau <phi_k, phi_i>   (+ the u d_x term per state)
        Em = -(np.transpose(wg[..., 1], (0, 2, 1)) @ Q.phi)
        Fm = np.zeros((E, PE, nl, PF))
        Gm = np.zeros((E, nl, PF, 2, PE))
        Hm = np.zeros((E, nl, PF, PE))
        Jm = np.zeros((E, nl, PF, PF))
        out = self.face_outflow[self.mesh.elem_face]
        for l in range(nl):
            ph, psi, nrm, w = Q.fph[l], Q.fpsi[l], Q.fn[l], Q.fw[l]
            phw = w[:, :, None] * ph[None]                                        # (E, nfq, PE)
            for c in range(2):
                Dm[:, :, c, :] -= nu * np.transpose(phw * nrm[:, :, c:c + 1], (0, 2, 1)) @ ph
                Gm[:, l, :, c, :] = -nu * np.transpose(psi, (0, 2, 1)) @ (phw * nrm[:, :, c:c + 1])
            Em += tau * (np.transpose(phw, (0, 2, 1)) @ ph)
            Fm[:, :, l] = np.transpose(phw * (nrm[:, :, 1:2] - tau), (0, 2, 1)) @ psi
            Hm[:, l] = tau * (np.transpose(psi, (0, 2, 1)) @ phw)
            cJ = (w * ((1.0 - out[:, l])[:, None] * nrm[..., 1] - tau))[:, :, None]
            Jm[:, l] = np.transpose(psi, (0, 2, 1)) @ (cJ * psi)
        self._const = dict(D=Dm.reshape(E, PE, 2 * PE), E=Em, F=Fm, G=Gm.reshape(E, nl * PF, 2 * PE),
                           H=Hm.reshape(E, nl * PF, PE), J=Jm)
        return self._const

    def jacobian_blocks(self, q, u, uh):
        """Blocks of Eq. matrixform at the state (M = 1, D = 2), in the
        condensation's input layout, with the right-hand sides ru = -R_u and
        ruh = -R_uhat (r_q = 0: q satisfies its linear equation):
          D[i,(c,k)]   = nu int d_c phi_i phi_k - nu <n_c phi_k, phi_i>
          E[i,k]       = -int (u, 1) . grad phi_i phi_k + tau <phi_k, phi_i>
          F[i,(l,j)]   = <(uhat n_x + n_y - tau) psi_j, phi_i>_l
          G[(l,j),(c,k)] = -nu <n_c phi_k, psi_j>_l
          H[(l,j),k]   = tau <phi_k, psi_j>_l
          J[(l,j),(l,j')] = <(uhat n_x + n_y - tau) psi_j', psi_j>_l, without
                         the convective part on outflow faces."""
        Q = self.Q
        E, PE, PF, nl = self.n_elem, self.PE, self.PF, self.n_lfe
        C = self._constant_blocks()
        uq = u @ Q.phi.T                                                          # (E, nq)
        Em = C['E'] - np.transpose((Q.wJ * uq)[:, :, None] * Q.g[..., 0], (0, 2, 1)) @ Q.phi
        Fm = C['F'].copy()
        Jd = C['J'].copy()
        ue = self.element_traces(uh)
        out = self.face_outflow[self.mesh.elem_face]
        for l in range(nl):
            ph, psi, nrm, w = Q.fph[l], Q.fpsi[l], Q.fn[l], Q.fw[l]
            uhf = np.matmul(psi, ue[:, l][:, :, None])[..., 0]
            cu = (w * uhf * nrm[..., 0])[:, :, None]                              # (E, nfq, 1)
            Fm[:, :, l] += np.transpose(cu * ph[None], (0, 2, 1)) @ psi
            Jd[:, l] += np.transpose(psi, (0, 2, 1)) @ ((1.0 - out[:, l])[:, None, None] * cu * psi)
        Jm = np.zeros((E, nl, PF, nl, PF))
        for l in range(nl):
            Jm[:, l, :, l, :] = Jd[:, l]
        Ru, Ruh = self.residual(q, u, uh)
        return {'Me': self.Me, 'Bd': self.Bd, 'Cd': self.Cd,
                'D': C['D'], 'E': Em, 'F': Fm.reshape(E, PE, nl * PF), 'G': C['G'], 'H': C['H'],
                'J': Jm.reshape(E, nl * PF, nl * PF),
                'ru': -Ru[:, :, None], 'ruh': -Ruh.reshape(E, nl * PF)[:, :, None]}


def manufactured(nu=1.0 / 200.0):
    """A smooth solution for convergence pins: u = sin(pi x) cos(pi y / 2) +
    (1 - 2x) / 2, with f = u_y + u u_x - nu lap u and its Dirichlet data on
    every side (use outflow=False)."""
    pi = np.pi

    def u(x):
        X, Y = x[..., 0], x[..., 1]
        return np.sin(pi * X) * np.cos(pi * Y / 2) + 0.5 * (1 - 2 * X)

    def grad(x):
        X, Y = x[..., 0], x[..., 1]
        ux = pi * np.cos(pi * X) * np.cos(pi * Y / 2) - 1.0
        uy = -0.5 * pi * np.sin(pi * X) * np.sin(pi * Y / 2)
        return ux, uy

    def f(x):
        X, Y = x[..., 0], x[..., 1]
        ux, uy = grad(x)
        lap = -(pi ** 2 + 0.25 * pi ** 2) * np.sin(pi * X) * np.cos(pi * Y / 2)
        return uy + u(x) * ux - nu * lap
    return u, grad, f
