"""Shared helpers for tests: build a workload's trace system with the oracle."""
import numpy as np
import scipy.sparse.linalg as spl

from oracle.condense import condense_local
from oracle.assemble import assemble, element_traces, recover, element_trace_maps


class OracleSystem:
    def __init__(self, w, blocks=None):
        self.w = w
        self.b = w.blocks() if blocks is None else blocks
        self.uD = w.uhat_dirichlet()
        self.Kbar, self.rbar, self.rec = condense_local(self.b, w.M, w.n_lfe)
        self.K, self.r = assemble(self.Kbar, self.rbar, w.mesh.elem_face, w.face_dirichlet,
                                  self.uD, w.M, w.PF)
        self.bsz = w.M * w.PF
        self.elem_dofs = element_trace_maps(w.mesh.elem_face, w.face_dirichlet, w.M, w.PF)

    def direct(self):
        return spl.spsolve(self.K.tocsc(), self.r)

    def recover(self, uhat_free):
        if uhat_free.ndim == 1:
            uhat_free = uhat_free[:, None]
        ue = element_traces(uhat_free, self.w.mesh.elem_face, self.w.face_dirichlet, self.uD,
                            self.w.M, self.w.PF)
        return recover(self.rec, ue, self.w.M, self.w.n_lfe)


def l2_errors(w, blocks, u, q):
    mats = blocks['_mats']
    phi = w.ref.phi
    uh = np.einsum('qi,eai->eqa', phi, u[:, :, 0].reshape(w.n_elem, w.M, w.PE))
    qh = np.einsum('qi,eadi->eqad', phi, q[:, :, 0].reshape(w.n_elem, w.M, w.D, w.PE))
    eu = np.sqrt(np.einsum('eq,eqa->', mats['wJ'], (uh - w.u_exact(mats['xq'])) ** 2))
    eq = np.sqrt(np.einsum('eq,eqad->', mats['wJ'], (qh - w.q_exact(mats['xq'])) ** 2))
    return eu, eq
