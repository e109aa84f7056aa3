"""Many small systems in one persistent launch (hdg_solve_batch): systems of
different meshes, polynomial orders, block sizes and right-hand-side counts
solved together by one cooperative kernel (restarted block-Jacobi GMRES,
Sec. 3.1 / 4.4 / 4.5).  Each system's trace is bitwise the same solved
alone and in the batch, and meets the tolerance against the oracle's
direct solve, in FP64 and in the restarted mixed mode (FP32 blocks, FP64
residual at every restart)."""
import numpy as np
import pytest

from hdg_inputs import workloads as W
from tests.gpu_helpers import need_gpu, sparse_mv
from tests.oracle_helpers import OracleSystem

pytestmark = pytest.mark.gpu


def _systems():
    # (workload, label): convection-diffusion of the serving stream at three
    # orders and two mesh sizes, and a two-RHS elasticity system
    return [(W.hex_convdiff(3, 1, 0.05, (1.0, 0.0, 0.0)), 'cd n3 k1'),
            (W.hex_convdiff(4, 2, 0.5, (0.0, 0.6, 0.8)), 'cd n4 k2'),
            (W.hex_convdiff(3, 3, 0.01, (0.6, 0.0, -0.8)), 'cd n3 k3'),
            (W.hex_convdiff(5, 1, 1.0, (0.0, 0.0, 1.0)), 'cd n5 k1'),
            (W.hex_elasticity(n=2, k=1, R=2), 'elast n2 k1 R2'),
            # several 2048-entry reduction chunks with a ragged tail, many face groups
            (W.hex_convdiff(8, 2, 0.2, (0.8, 0.6, 0.0)), 'cd n8 k2')]


@pytest.fixture(scope='module')
def setup():
    need_gpu()
    from paper_2512_13619_gb300 import driver
    out = []
    for w, label in _systems():
        s = OracleSystem(w)
        o = driver.opts(restart=30, rtol=1e-10, pc='bj')
        p = driver.Problem.from_workload(w)
        p.condense(w.blocks())
        p.set_dirichlet(w.uhat_dirichlet())
        p.assemble(o)
        p.setup_precond(o)
        out.append((w, label, s, p))
    yield out
    for _, _, _, p in out:
        p.close()


@pytest.mark.parametrize('mode', ['fp64', 'mixed'])
def test_batch_alone_equals_batched_and_meets_oracle(setup, mode):
    from paper_2512_13619_gb300 import driver, _lib as L
    rtol = 1e-10 if mode == 'fp64' else 1e-8
    o = driver.opts(restart=30, rtol=rtol, pc='bj', max_iters=3000,
                    inner='fp64' if mode == 'fp64' else 'fp32', max_outer=20 if mode == 'fp64' else -1)
    alone = []
    for w, label, s, p in setup:
        st, infos = L.hdg_solve_batch([p.h], o)
        assert st == L.HDG_OK and infos[0].converged == 1, (label, L.hdg_status_str(st))
        alone.append((p.free_trace(), infos[0].iters))
    st, infos = L.hdg_solve_batch([p.h for _, _, _, p in setup], o)
    assert st == L.HDG_OK
    for (w, label, s, p), (xa, ita), inf in zip(setup, alone, infos):
        xb = p.free_trace()
        assert np.array_equal(xa, xb), label               # bitwise: alone == in the batch
        assert inf.iters == ita and inf.converged == 1, label
        # against the oracle: true FP64 residual with the oracle's K, error vs its direct solve
        res = s.r - sparse_mv(s.K, xb)
        for r in range(w.R):
            assert np.linalg.norm(res[:, r]) / np.linalg.norm(s.r[:, r]) <= rtol, (label, r)
        if s.K.shape[0] > 4000:
            continue                                       # the dense condition number is too slow
        xd = s.direct()
        xd = xd[:, None] if xd.ndim == 1 else xd
        cond = np.linalg.cond(s.K.toarray())
        for r in range(w.R):
            assert np.linalg.norm(xb[:, r] - xd[:, r]) / np.linalg.norm(xd[:, r]) <= cond * rtol, (label, r)


def test_batch_order_does_not_matter(setup):
    """The same systems in reverse order give bitwise the same traces."""
    from paper_2512_13619_gb300 import driver, _lib as L
    o = driver.opts(restart=30, rtol=1e-10, pc='bj', max_iters=3000)
    st, _ = L.hdg_solve_batch([p.h for _, _, _, p in setup], o)
    assert st == L.HDG_OK
    first = [p.free_trace() for _, _, _, p in setup]
    st, _ = L.hdg_solve_batch([p.h for _, _, _, p in reversed(setup)], o)
    assert st == L.HDG_OK
    for (_, label, _, p), x in zip(setup, first):
        assert np.array_equal(p.free_trace(), x), label
