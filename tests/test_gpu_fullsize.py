"""Parity at the full size of the bench workload (HDG Poisson, 16^3 hex, Q3,
184,320 trace unknowns) in the launch configuration bench.py times: the
oracle condenses and assembles the whole problem (a few seconds on the host)
and the GPU results are compared element by element."""
import numpy as np
import pytest

from hdg_inputs import workloads as W
from oracle.condense import condense_local
from oracle.assemble import assemble
from tests.gpu_helpers import need_gpu, sparse_mv

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope='module')
def full():
    need_gpu()
    from paper_2512_13619_gb300 import driver
    w = W.hex_poisson(n=16, k=3)
    blk = w.blocks()
    uD = w.uhat_dirichlet()
    Kb, rb, rec = condense_local(blk, w.M, w.n_lfe)
    K, r = assemble(Kb, rb, w.mesh.elem_face, w.face_dirichlet, uD, w.M, w.PF)
    p = driver.Problem.from_workload(w)
    p.condense(blk)
    p.set_dirichlet(uD)
    return dict(w=w, blk=blk, uD=uD, Kb=Kb, rb=rb, rec=rec, K=K, r=r, p=p)


def test_fullsize_condensation_sampled(full):
    """Kbar^e, rbar^e of 64 sampled elements (incl. corner and edge elements)."""
    w, p = full['w'], full['p']
    idx = np.unique(np.concatenate([[0, w.n_elem - 1, 15, 255],
                                    np.random.default_rng(1).integers(0, w.n_elem, 60)]))
    for e in idx:
        Kg, rg = p.condensed(int(e), 1)
        assert np.abs(Kg[0] - full['Kb'][e]).max() <= 1e-12 * np.abs(full['Kb'][e]).max()
        assert np.abs(rg[0] - full['rb'][e]).max() <= 1e-12 * max(np.abs(full['rb'][e]).max(), 1e-300)


def test_fullsize_matvec_all_rows(full):
    """y = K x on all 184,320 rows, FP64 and FP32 blocks, with the bench's kernels."""
    from paper_2512_13619_gb300 import driver
    w, p, K = full['w'], full['p'], full['K']
    p.assemble(driver.opts(pc='bj'))
    x = np.random.default_rng(2).standard_normal((p.n_dof, 1))
    y_ref = sparse_mv(K, x)
    bound = sparse_mv(abs(K), np.abs(x))
    y64 = p.apply_K(x, 'fp64')
    assert np.abs(y64 - y_ref).max() <= 1e-13 * bound.max()
    nterm = (2 * w.n_lfe - 1) * w.M * w.PF
    y32 = p.apply_K(x, 'fp32')
    assert np.all(np.abs(y32 - y_ref) <= (U32 + (nterm + 1) * U32) * bound + 1e-300)


@pytest.mark.parametrize('inner,rtol', [('fp64', 1e-10), ('fp32', 1e-8)])
def test_fullsize_solve_and_recover(full, inner, rtol):
    """BJ-GMRES(50) FP64 to 1e-10 and mixed to 1e-8: the true residual of the
    GPU trace with the oracle's K meets rtol, and the recovered (q, u) of 64
    sampled elements satisfy the element equations of Eq. matrixform,
    [A B; D E][q; u] = [r_q; r_u] - [C; F] uhat^e, with the GPU's trace."""
    from paper_2512_13619_gb300 import driver
    from oracle.condense import q_blocks_dense
    from oracle.assemble import dirichlet_element_values, element_trace_maps
    w, p, K, r, blk = full['w'], full['p'], full['K'], full['r'], full['blk']
    o = driver.opts(restart=50, rtol=rtol, pc='bj', inner=inner, max_iters=5000)
    p.assemble(o)
    p.setup_precond(o)
    st, info = p.solve(o)
    assert st == 0 and info.converged == 1
    x = p.free_trace()
    b = r[:, 0]
    assert np.linalg.norm(b - K @ x[:, 0]) / np.linalg.norm(b) <= rtol
    u, q = p.recover()
    full_trace = p.trace()                                   # n_face x b x R, Dirichlet rows = u_D
    idx = np.unique(np.concatenate([[0, w.n_elem - 1], np.random.default_rng(3).integers(0, w.n_elem, 62)]))
    sub = {k: blk[k][idx] for k in ('Me', 'Bd', 'Cd')}
    A, B, C = q_blocks_dense(sub['Me'], sub['Bd'], sub['Cd'], w.M, w.n_lfe)
    for n, e in enumerate(idx):
        uh = full_trace[w.mesh.elem_face[e]].reshape(-1)       # (l, a, j) order of the element
        res_q = A[n] @ q[e, :, 0] + B[n] @ u[e, :, 0] + C[n] @ uh
        res_u = blk['D'][e] @ q[e, :, 0] + blk['E'][e] @ u[e, :, 0] + blk['F'][e] @ uh - blk['ru'][e, :, 0]
        scale_q = np.abs(A[n]).max() * np.abs(q[e]).max() + np.abs(C[n]).max() * np.abs(uh).max()
        scale_u = np.abs(blk['E'][e]).max() * np.abs(u[e]).max() + np.abs(blk['F'][e]).max() * np.abs(uh).max()
        assert np.abs(res_q).max() <= 1e-11 * scale_q
        assert np.abs(res_u).max() <= 1e-11 * scale_u


def test_fullsize_recover_host_outputs_match_device(full):
    """Host outputs of the trace and the recovery, both ways the library
    writes them, equal the device outputs bit for bit on every element:
    pageable buffers (recovery in 4 pieces of 1024 elements, each piece's
    copies overlapping the next piece's kernel) and pinned buffers (written
    by the kernels directly).  The Dirichlet values set from host memory on
    the copy stream reach the trace: its Dirichlet rows equal u_D."""
    import torch
    from paper_2512_13619_gb300 import driver, _lib as L
    w, p = full['w'], full['p']
    o = driver.opts(restart=50, rtol=1e-10, pc='bj', inner='fp64', max_iters=5000)
    p.set_dirichlet(full['uD'])
    p.assemble(o)
    p.setup_precond(o)
    st, info = p.solve(o)
    assert st == 0
    u_h, q_h = p.recover()
    u_d = torch.empty(u_h.shape, dtype=torch.float64, device='cuda')
    q_d = torch.empty(q_h.shape, dtype=torch.float64, device='cuda')
    driver.check(L.hdg_recover(p.h, u_d, q_d, 1, None), 'hdg_recover')
    torch.cuda.synchronize()
    assert np.array_equal(u_h, u_d.cpu().numpy())
    assert np.array_equal(q_h, q_d.cpu().numpy())
    u_p = torch.full(u_h.shape, np.nan, dtype=torch.float64).pin_memory()
    q_p = torch.full(q_h.shape, np.nan, dtype=torch.float64).pin_memory()
    driver.check(L.hdg_recover(p.h, u_p, q_p, 0, None), 'hdg_recover')
    assert np.array_equal(u_h, u_p.numpy()) and np.array_equal(q_h, q_p.numpy())
    tr = p.trace()
    tr_p = torch.full(tr.shape, np.nan, dtype=torch.float64).pin_memory()
    tr_d = torch.empty(tr.shape, dtype=torch.float64, device='cuda')
    driver.check(L.hdg_get_trace(p.h, tr_p, 0, None), 'hdg_get_trace')
    driver.check(L.hdg_get_trace(p.h, tr_d, 1, None), 'hdg_get_trace')
    torch.cuda.synchronize()
    assert np.array_equal(tr, tr_p.numpy()) and np.array_equal(tr, tr_d.cpu().numpy())
    dir_rows = w.face_dirichlet.astype(bool)
    assert np.array_equal(tr[dir_rows], np.asarray(full['uD']).reshape(tr.shape)[dir_rows])
