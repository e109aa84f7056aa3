"""Helpers shared by the GPU tests."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    from paper_2512_13619_gb300 import build
    build.build()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def sparse_mv(K, x):
    """oracle K (csr) times x (n, R)."""
    return np.column_stack([K @ x[:, r] for r in range(x.shape[1])])
