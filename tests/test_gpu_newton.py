"""Damped Newton-GMRES on the GPU trace solver (Welter & Nguyen, Sec. 2.3)
against the oracle's Newton with exact linear solves, on Sec. 6.1's steady
viscous Burgers problem."""
import numpy as np
import pytest

from hdg_inputs import burgers as BG
from oracle.newton import newton
from tests.gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize('pc', ['bj', 'asm'])
def test_newton_gmres_matches_oracle_newton(pc):
    """8 x 8 Q^2 quadrilaterals; each linear solve is GMRES(50) with the
    PP(10) polynomial on BJ or ASM to 1e-10: the same Newton steps and
    line-search factors as the oracle's direct solves, the same final
    residual level, and u within 1e-7 of the oracle's."""
    need_gpu()
    from paper_2512_13619_gb300 import driver
    from paper_2512_13619_gb300.newton import newton_solve
    P = BG.Burgers(n=8, k=2)
    (qo, uo, uho), ho = newton(P, P.initial_state(), tol=1e-8)
    o = driver.opts(restart=50, rtol=1e-10, pc=pc, poly='gmres', degree=10, max_iters=5000)
    v0 = np.random.default_rng(11).standard_normal(P.n_free * P.PF)
    (q, u, uh), info = newton_solve(P, o, v0, tol=1e-8)
    h = info['history']
    assert len(h) == len(ho)
    assert [a for _, a in h] == [a for _, a in ho]
    assert h[-1][0] <= 1e-8
    assert np.abs(u - uo).max() <= 1e-7 * np.abs(uo).max()
    assert info['gmres'] > 0 and len(info['gmres_per_step']) == len(h) - 1
