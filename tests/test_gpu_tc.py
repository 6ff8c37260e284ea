"""Complex GEMM kernels through ss_zgemm: the FP64 kernel and the split-BF16
tcgen05 kernel against numpy's complex128 product.

Bars: FP64 1e-13 (relative Frobenius); the 3-product split carries ~17
significant bits (bar 5e-5); the 6-product split is limited by the FP32
accumulation over K' = 6*2k terms (about 2^-24 sqrt(K'), measured 5e-6:
bar 5e-5).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BARS = {0: 1e-13, 1: 5e-5, 2: 5e-5}


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


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("m,n,k,ta,tb", [(256, 256, 256, 0, 0), (130, 70, 200, 0, 0), (64, 300, 96, 1, 0),
                                         (200, 128, 512, 0, 1), (17, 5, 33, 1, 1)])
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
