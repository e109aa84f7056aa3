"""Element blocks of hexahedral Q^k elements generated on the device (the
element integrals of Sec. 4.1 as batched products of basis tables with
quadrature weights, then the blocks of Eq. matrixform), through the C ABI,
against the host generator of the same blocks, and their condensation
against the oracle."""
import numpy as np
import pytest

from hdg_inputs import workloads as W
from oracle.condense import condense_local
from tests.gpu_helpers import need_gpu, rel

pytestmark = pytest.mark.gpu

NAMES9 = ('Me', 'Bd', 'Cd', 'D', 'E', 'F', 'G', 'H', 'J')

CASES = {
    'poisson_q3': lambda: W.hex_poisson(n=3, k=3),
    'elast_pert_q2_R2': lambda: W.hex_elasticity(n=2, k=2, R=2),      # perturbed: nquad 6, K = 216 > 192
    'cdr_M5_q1_R4': lambda: W.hex_cdr(n=2, k=1, R=4),                  # convection, reaction, P_E = 8 < 16
    'beam_q2': lambda: W.hex_beam(n=2, k=2),                           # 5 x 1 x 1 box, traction faces
    'elast_q3': lambda: W.hex_elasticity(n=2, k=3, R=1, perturb=0.0),  # Ebar 192 x 192 (block inverse)
}


def _gen_blocks(w, on_device, sf=1):
    import torch
    from paper_2512_13619_gb300 import driver, _lib as L
    p = driver.Problem.from_workload(w)
    assert L.hdg_set_hex_generation(p.h, sf) == 0
    verts, perm, nquad = driver.hex_geometry_inputs(w)
    ph, keep = L.physics(w.phys.Cq, w.phys.Cu, w.phys.Rr, w.phys.tau)
    ref = w.blocks()
    out = [torch.empty(ref[k].shape, dtype=torch.float64, device='cuda') for k in NAMES9]
    if on_device:
        verts, perm = torch.from_numpy(verts).cuda(), torch.from_numpy(perm).cuda()
    st = L.hdg_hex_blocks(p.h, w.n_elem, nquad, verts, perm, ph, out, int(on_device))
    p.close()
    return st, {k: o.cpu().numpy() for k, o in zip(NAMES9, out)}, ref


@pytest.mark.parametrize('sf', [1, 0])
@pytest.mark.parametrize('name', sorted(CASES))
def test_generated_blocks_match_host_generator(name, sf):
    """Every block of every element equals the host generator's within 1e-13
    of the block's largest entry (the reference tables are built
    independently in C++: Gauss and GLL nodes by Newton's method, Lagrange
    polynomials in product form), with M^e and B_d by sum factorisation
    (sf = 1) and by dense products (sf = 0)."""
    need_gpu()
    w = CASES[name]()
    st, gen, ref = _gen_blocks(w, on_device=(name == 'poisson_q3'), sf=sf)
    assert st == 0
    for k in NAMES9:
        assert rel(gen[k], ref[k]) < 1e-13, (k, rel(gen[k], ref[k]))


@pytest.mark.parametrize('name', ['poisson_q3', 'elast_pert_q2_R2', 'beam_q2'])
def test_condense_hex_matches_oracle(name):
    """hdg_condense_hex (blocks generated on the device, chunked) gives Kbar
    and rbar of the oracle's condensation of the host blocks within 1e-12,
    and a BJ-PP(10) solve on them the same iteration count as the host-block
    path (a fast-converging solver: plain BJ on the beam takes thousands of
    iterations, whose count moves with rounding)."""
    need_gpu()
    from paper_2512_13619_gb300 import driver, _lib as L
    w = CASES[name]()
    p = driver.Problem.from_workload(w)
    assert L.hdg_set_condense_chunk(p.h, 5) == 0            # several chunks
    p.condense_hex(w)
    Kg, rg = p.condensed()
    Ko, ro, _ = condense_local(w.blocks(), w.M, w.n_lfe)
    assert rel(Kg, Ko) < 1e-12 and rel(rg, ro) < 1e-12
    o = driver.opts(restart=50, rtol=1e-8, pc='bj', poly='gmres', degree=10, max_iters=20000)
    v0 = w.random_vector(11)
    p.set_dirichlet(w.uhat_dirichlet())
    p.assemble(o)
    p.setup_precond(o, v0)
    st, info = p.solve(o)
    q = driver.Problem.from_workload(w)
    q.condense(w.blocks())
    q.set_dirichlet(w.uhat_dirichlet())
    q.assemble(o)
    q.setup_precond(o, v0)
    st2, info2 = q.solve(o)
    assert st == 0 and st2 == 0
    assert abs(info.iters - info2.iters) <= max(2, 0.05 * info2.iters)
    assert rel(p.free_trace(), q.free_trace()) < 1e-6
    p.close()
    q.close()


def test_hex_generation_rejects_other_shapes():
    """Triangles (N_lfe = 3), nquad outside 1..12 and face permutation
    entries outside 0..P_F-1 are refused with HDG_ERR_ARG."""
    need_gpu()
    import torch
    from paper_2512_13619_gb300 import driver, _lib as L
    w = W.tri_poisson(n=2, k=1)
    p = driver.Problem.from_workload(w)
    ph, keep = L.physics(np.zeros((1, 3, 1, 3)))
    z = np.zeros(1)
    assert L.hdg_condense_hex(p.h, 0, 1, 3, z, np.zeros(1, np.int32), ph, z, z, 0) == L.HDG_ERR_ARG
    p.close()
    w = W.hex_poisson(n=2, k=1)
    p = driver.Problem.from_workload(w)
    verts, perm, nquad = driver.hex_geometry_inputs(w)
    ph, keep = L.physics(w.phys.Cq, w.phys.Cu, w.phys.Rr, w.phys.tau)
    out = [torch.empty(v.shape, dtype=torch.float64, device='cuda') for k, v in w.blocks().items() if k in NAMES9]
    assert L.hdg_hex_blocks(p.h, w.n_elem, 0, verts, perm, ph, out, 0) == L.HDG_ERR_ARG
    assert L.hdg_hex_blocks(p.h, w.n_elem, 13, verts, perm, ph, out, 0) == L.HDG_ERR_ARG
    bad = perm.copy()
    bad[3, 2, 1] = w.PF
    assert L.hdg_hex_blocks(p.h, w.n_elem, nquad, verts, bad, ph, out, 0) == L.HDG_ERR_ARG
    p.close()
