"""Batched FP64 GEMM of the condensation (Sec. 4.1, Eqs. w16-w22) on the FP64
cores and on the BF16 tensor cores with exact operand splitting, through the
C ABI, against numpy's FP64 product of the same inputs."""
import numpy as np
import pytest

from tests.gpu_helpers import need_gpu, rel

pytestmark = pytest.mark.gpu

# (M, N, K): condensation shapes (64/96 for Q3 Poisson, 81/162 for Q2
# elasticity, 135/270 for the 5-component Q2 system) and ragged edges
SHAPES = [(64, 64, 64), (96, 96, 192), (64, 96, 192), (135, 48, 81), (270, 70, 135), (17, 16, 1),
          (128, 64, 32), (162, 162, 81), (3, 200, 150), (125, 150, 375), (64, 64, 193)]


def _inputs(M, N, K, cnt, seed):
    rng = np.random.default_rng(seed)
    # entries over 13 binades with exact zeros, so that the per-row and
    # per-column scalings and the digit split are exercised
    A = rng.standard_normal((cnt, M, K)) * np.exp2(rng.integers(-6, 7, (cnt, M, K)))
    B = rng.standard_normal((cnt, K, N)) * np.exp2(rng.integers(-6, 7, (cnt, K, N)))
    A[rng.random(A.shape) < 0.1] = 0.0
    B[rng.random(B.shape) < 0.1] = 0.0
    C0 = rng.standard_normal((cnt, M, N))
    return A, B, C0


def _run(mode, A, B, C0, alpha, beta):
    import torch
    from paper_2512_13619_gb300 import _lib as L
    cnt, M, K = A.shape
    N = B.shape[2]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.from_numpy(np.ascontiguousarray(C0)).cuda()
    st = L.hdg_gemm_f64(mode, M, N, K, dA, K, M * K, dB, N, K * N, dC, N, M * N, alpha, beta, cnt)
    return st, dC.cpu().numpy()


@pytest.mark.parametrize('shape', SHAPES)
@pytest.mark.parametrize('mode', [0, 1, 2, 3])
def test_gemm_matches_fp64_product(shape, mode):
    """|C - (alpha A B + beta C0)| <= 2^-50 K |alpha| max_k|A_ik| max_k|B_kj|
    + 2^-50 (|beta C0| + |alpha| (|A||B|)): FP64-level accuracy (the
    splitting keeps 56 bits per operand; FP64 rounding of a K-term dot product
    is bounded by K 2^-53 (|A||B|))."""
    need_gpu()
    M, N, K = shape
    if mode >= 1 and (N < 16 or (mode >= 2 and K > 192)):
        pytest.skip('outside the tensor-core shapes')
    A, B, C0 = _inputs(M, N, K, 3, M * 7919 + N * 31 + K)
    amax = np.abs(A).max(axis=2)[:, :, None]
    bmax = np.abs(B).max(axis=1)[:, None, :]
    absAB = np.abs(A) @ np.abs(B)
    worst = 0.0
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0), (0.5, -2.0)):
        st, C = _run(mode, A, B, C0, alpha, beta)
        assert st == 0
        ref = alpha * (A @ B) + beta * C0
        bound = 2.0 ** -50 * (K * abs(alpha) * amax * bmax + np.abs(beta * C0) + abs(alpha) * absAB)
        err = np.abs(C - ref)
        assert np.all(err <= bound + 1e-300), (alpha, beta, float((err / (bound + 1e-300)).max()))
        worst = max(worst, float((err / (K * amax * bmax * 2.0 ** -53 + 1e-300)).max()))
    print('shape', shape, 'mode', mode, 'max |err| / (K 2^-53 maxA maxB) =', worst)


@pytest.mark.parametrize('mode', [1, 2, 3])
def test_gemm_tensor_exact_on_integers(mode):
    """Small integers are represented exactly by the digits, and their
    products and sums (< 2^53) are exact: the tensor-core result equals the
    integer product."""
    need_gpu()
    rng = np.random.default_rng(3)
    A = rng.integers(-1000, 1001, (2, 96, 192)).astype(float)
    B = rng.integers(-1000, 1001, (2, 192, 64)).astype(float)
    C0 = np.zeros((2, 96, 64))
    st, C = _run(mode, A, B, C0, 1.0, 0.0)
    assert st == 0
    assert np.array_equal(C, A @ B)


@pytest.mark.parametrize('mode', [1, 2, 3])
def test_gemm_tensor_zero_rows_and_nan(mode):
    """An all-zero row gives an exact zero row; an Inf/NaN input is reported
    (HDG_ERR_NAN); N < 16 is rejected on the tensor path, and K > 192 by the
    variants that do not slice K."""
    need_gpu()
    from paper_2512_13619_gb300 import _lib as L
    A, B, C0 = _inputs(64, 32, 64, 1, 5)
    A[0, 7, :] = 0.0
    st, C = _run(mode, A, B, C0, 1.0, 0.0)
    assert st == 0 and np.all(C[0, 7] == 0.0)
    assert rel(C, A @ B) < 1e-14
    A[0, 3, 5] = np.nan
    st, _ = _run(mode, A, B, C0, 1.0, 0.0)
    assert st == L.HDG_ERR_NAN
    A2, B2, C2 = _inputs(64, 32, 193, 1, 6)
    st, _ = _run(mode, A2, B2, C2, 1.0, 0.0)
    assert st == (L.HDG_OK if mode == 1 else L.HDG_ERR_ARG)     # mode 1 slices K > 192
    A3, B3, C3 = _inputs(64, 8, 64, 1, 7)
    st, _ = _run(mode, A3, B3, C3, 1.0, 0.0)
    assert st == L.HDG_ERR_ARG


def test_condensation_tensor_equals_fp64_cores():
    """Condensation (Eqs. w16-w22) with the tensor-core products (digits per
    tile, or digit planes) equals the one on the FP64 cores to 1e-13 (all
    against the same inputs)."""
    need_gpu()
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver, _lib as L
    w = W.hex_poisson(n=3, k=3)
    blk = w.blocks()
    out = []
    for mode in (0, 1, 2, 3):
        p = driver.Problem.from_workload(w)
        assert L.hdg_set_condense_mode(p.h, mode) == 0
        p.condense(blk)
        out.append(p.condensed())
        p.close()
    for m in (1, 2, 3):
        assert rel(out[m][0], out[0][0]) < 1e-13
        assert rel(out[m][1], out[0][1]) < 1e-13


def test_condensation_chunks_from_host_overlap_copies():
    """Host inputs condensed in many small chunks (the copies of chunk c+1
    overlap the condensation of chunk c through two staging buffers) give
    bitwise the results of one chunk."""
    need_gpu()
    import torch
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver, _lib as L
    w = W.hex_poisson(n=3, k=3)
    blk = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in w.blocks().items()
           if k in driver.BLOCK_NAMES}
    out = []
    for chunk in (None, 2, 5):
        p = driver.Problem.from_workload(w)
        if chunk:
            assert L.hdg_set_condense_chunk(p.h, chunk) == 0
        assert L.hdg_condense(p.h, 0, w.n_elem, *[blk[k] for k in driver.BLOCK_NAMES], 0, None) == 0
        out.append(p.condensed())
        assert L.hdg_set_condense_chunk(p.h, 0) == L.HDG_ERR_ARG
        p.close()
    for m in (1, 2):
        assert np.array_equal(out[m][0], out[0][0]) and np.array_equal(out[m][1], out[0][1])
