"""Complex GEMM kernels through ss_zgemm: the FP64 kernel, the split-BF16
tcgen05 kernel and the digit-sliced (exact-accumulation) tcgen05 kernel
against numpy's complex128 product.

Bars: FP64 1e-13 (relative Frobenius); the 3-product split carries ~17
significant bits (bar 5e-5); the 6-product split is limited by the FP32
accumulation over K' = 6*2k terms (about 2^-24 sqrt(K'), measured 5e-6:
bar 5e-5); the digit-sliced mode accumulates exactly and must match FP64
(bar 1e-13).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BARS = {0: 1e-13, 1: 5e-5, 2: 5e-5, 3: 1e-13}


@pytest.fixture(scope="module")
def ss():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1812_01396_gb300 as mod
    return mod


def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("m,n,k,ta,tb", [(256, 256, 256, 0, 0), (130, 70, 200, 0, 0), (64, 300, 96, 1, 0),
                                         (200, 128, 512, 0, 1), (17, 5, 33, 1, 1), (96, 40, 16, 0, 0),
                                         (128, 128, 2048, 0, 0)])
def test_zgemm_modes(ss, mode, m, n, k, ta, tb):
    import torch
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = cplx(rng, (k, m) if ta else (m, k))
    B = cplx(rng, (n, k) if tb else (k, n))
    ref = (A.conj().T if ta else A) @ (B.conj().T if tb else B)
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    tC = torch.full((m, n), complex("nan"), dtype=torch.complex128, device="cuda")
    ss.ss_zgemm(tA, tB, tC, precision=mode, transA=bool(ta), transB=bool(tb))
    C = tC.cpu().numpy()
    err = np.linalg.norm(C - ref) / np.linalg.norm(ref)
    print(f"mode {mode} {m}x{n}x{k} ta={ta} tb={tb}: rel err {err:.3e}")
    assert err < BARS[mode]


def test_exact_mode_on_wide_dynamic_range(ss):
    """Rows and columns scaled over 1e-12..1e12: per-row/column power-of-two
    scales keep every entry at full relative precision of its own row."""
    import torch
    rng = np.random.default_rng(5)
    m, n, k = 96, 80, 300
    A = cplx(rng, (m, k)) * (10.0 ** rng.uniform(-12, 12, (m, 1)))
    B = cplx(rng, (k, n)) * (10.0 ** rng.uniform(-12, 12, (1, n)))
    ref = A @ B
    tC = torch.zeros((m, n), dtype=torch.complex128, device="cuda")
    ss.ss_zgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), tC, precision=3)
    C = tC.cpu().numpy()
    scale = np.abs(A).max(1, keepdims=True) * np.abs(B).max(0, keepdims=True) * k
    assert np.max(np.abs(C - ref) / scale) < 1e-15
