"""Host logic of the product's Newton driver (paper_2512_13619_gb300.newton,
Sec. 2.3) on the CPU: the library problem is replaced by a stand-in whose
linear algebra is the oracle's (condensation, assembly, a direct solve of the
trace system, recovery), so the driver's own steps -- right-hand sides,
increments of (q, u, uhat), line search, bookkeeping -- must reproduce the
oracle's Newton iteration exactly."""
import numpy as np
import pytest

from hdg_inputs import burgers as BG
from oracle.newton import newton
from oracle.condense import condense_local
from oracle.assemble import assemble, element_traces, recover
import scipy.sparse.linalg as spl


class _OracleProblem:
    """The calls newton_solve makes on driver.Problem, computed by the oracle."""

    def __init__(self, dim, n_lfe, M, PE, PF, elem_face, face_elem, face_dirichlet, nrhs=1, device=0):
        self.n_lfe, self.M, self.PE, self.PF, self.dim = n_lfe, M, PE, PF, dim
        self.ef, self.fd = elem_face, np.asarray(face_dirichlet)
        self.n_face = len(self.fd)

    def condense(self, blk):
        self.blk = blk
        self.Kbar, self.rbar, self.rec = condense_local(blk, self.M, self.n_lfe)

    def set_dirichlet(self, uD):
        self.uD = uD

    def assemble(self, o):
        self.K, self.r = assemble(self.Kbar, self.rbar, self.ef, self.fd, self.uD, self.M, self.PF)

    def setup_precond(self, o, v0=None):
        pass

    def solve(self, o):
        self.x = spl.spsolve(self.K.tocsc(), self.r[:, 0])

        class Info:
            iters = 1
        return 0, Info()

    def trace(self):
        full = np.zeros((self.n_face, self.PF, 1))
        full[self.fd == 0, :, 0] = self.x.reshape(-1, self.PF)
        return full

    def recover(self):
        ue = element_traces(self.x[:, None], self.ef, self.fd, self.uD, self.M, self.PF)
        return recover(self.rec, ue, self.M, self.n_lfe)

    def close(self):
        pass


def test_newton_driver_reproduces_the_oracle_newton(monkeypatch):
    import torch
    from paper_2512_13619_gb300 import newton as N, driver
    monkeypatch.setattr(N.driver, 'Problem', _OracleProblem)
    monkeypatch.setattr(torch.cuda, 'synchronize', lambda *a, **k: None)
    P = BG.Burgers(n=6, k=2)
    (qo, uo, uho), ho = newton(P, P.initial_state(), tol=1e-9)
    (q, u, uh), info = N.newton_solve(P, driver.opts(), None, tol=1e-9)
    h = info['history']
    assert [a for _, a in h] == [a for _, a in ho]
    assert np.allclose([r for r, _ in h], [r for r, _ in ho], rtol=1e-6, atol=1e-14)
    assert np.abs(u - uo).max() <= 1e-12 * np.abs(uo).max()
    assert np.abs(uh - uho).max() <= 1e-12 * np.abs(uho).max()
    assert info['gmres'] == len(h) - 1 and h[-1][0] <= 1e-9
