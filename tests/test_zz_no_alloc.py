"""The allocation-free matvec entry point (hdg_apply_K_noalloc) against the
regular one (hdg_apply_K).  It is for callers that cannot allocate device
memory when they need y = K x (inside a stream capture, under a foreign pool
allocator, in latency-critical loops); its scratch is a static device array.
This file is collected last so that a run stopping at its first failure has
run every other test already; it also passes on its own."""
import numpy as np
import pytest

from hdg_inputs import workloads as W
from tests.gpu_helpers import need_gpu, sparse_mv
from tests.oracle_helpers import OracleSystem

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U16 = 2.0 ** -8     # unit roundoff of BF16 storage


@pytest.mark.parametrize('prec', ['fp32', 'bf16'])
def test_apply_K_noalloc_matches_apply_K_twice(prec):
    need_gpu()
    import torch
    from paper_2512_13619_gb300 import driver, _lib as L
    w = W.hex_elasticity(n=2, k=1, R=2)
    s = OracleSystem(w)
    # BF16 blocks are built when the options ask for them
    o = driver.opts(inner=prec)
    p = driver.Problem.from_workload(w)
    p.condense(w.blocks())
    p.set_dirichlet(w.uhat_dirichlet())
    p.assemble(o)
    code = L.HDG_FP32 if prec == 'fp32' else L.HDG_BF16
    u_store = U32 if prec == 'fp32' else U16
    nterm = (2 * w.n_lfe - 1) * s.bsz
    tol = u_store + (nterm + 1) * U32          # storage rounding + FP32 dot product of nterm terms
    rng = np.random.default_rng(11)
    for call in range(2):      # two calls in a row share (and reuse) the static scratch
        x = rng.standard_normal((p.n_dof, w.R))
        xd = torch.from_numpy(x).cuda()
        y_ref = torch.empty_like(xd)
        y_new = torch.empty_like(xd)
        assert L.hdg_apply_K(p.h, code, xd, y_ref) == L.HDG_OK
        assert L.hdg_apply_K_noalloc(p.h, code, xd, y_new) == L.HDG_OK
        torch.cuda.synchronize()
        a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
        bound = sparse_mv(abs(s.K), np.abs(x))
        # the storage tolerance of the matvec tests, between the two entry points
        assert np.all(np.abs(a - b) <= 2 * tol * bound + 1e-300)
        # and against the oracle's FP64 product
        assert np.all(np.abs(a - sparse_mv(s.K, x)) <= tol * bound + 1e-300)
    xd = torch.zeros((p.n_dof, w.R), dtype=torch.float64, device='cuda')
    assert L.hdg_apply_K_noalloc(p.h, L.HDG_FP64, xd, xd) == L.HDG_ERR_ARG
    p.close()
