"""The allocation-free transmission entry point against the allocating one.

ss_caroli_transmission_noalloc serves callers that cannot allocate device
memory (a pool allocator owns the device, or a hook may not call cudaMalloc);
it must give the same T as ss_caroli_transmission, call after call, from its
fixed device scratch.  Kept in the last-collected file so that a run stopping
at the first failure has run every other test before it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ss():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import __graft_entry__
    __graft_entry__.build()
    import paper_1812_01396_gb300 as mod
    return mod


def blocks(seed, P, s):
    import torch
    rng = np.random.default_rng(seed)
    mk = lambda: torch.from_numpy(rng.standard_normal((P, s, s)) + 1j * rng.standard_normal((P, s, s))).cuda()
    return mk(), mk(), mk()


def test_noalloc_matches_allocating_entry_point_twice(ss):
    import torch
    for call, (seed, P, s) in enumerate([(1, 4, 64), (2, 3, 100)]):
        sL, sR, G = blocks(seed, P, s)
        T_ref = torch.zeros(P, dtype=torch.float64, device="cuda")
        T_na = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
        ss.ss_caroli_transmission(sL, sR, G, T_ref)
        ss.ss_caroli_transmission_noalloc(sL, sR, G, T_na)
        a, b = T_na.cpu().numpy(), T_ref.cpu().numpy()
        assert np.all(np.abs(a - b) <= 1e-10 * np.maximum(1.0, np.abs(b))), (call, a, b)


def test_noalloc_allocates_no_device_memory_on_a_side_stream(ss):
    """After a warm-up call, a second call (on a non-default stream) leaves the
    device's free memory unchanged: the scratch is the fixed array, nothing is
    allocated per call."""
    import torch
    sL, sR, G = blocks(4, 4, 64)
    T_ref = torch.zeros(4, dtype=torch.float64, device="cuda")
    T_na = torch.zeros(4, dtype=torch.float64, device="cuda")
    ss.ss_caroli_transmission(sL, sR, G, T_ref)
    side = torch.cuda.Stream()
    ss.ss_caroli_transmission_noalloc(sL, sR, G, T_na, stream=side.cuda_stream)  # warm-up: symbol lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    T_na.fill_(float("nan"))
    torch.cuda.synchronize()
    ss.ss_caroli_transmission_noalloc(sL, sR, G, T_na, stream=side.cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0, (free0, free1)  # no allocation (a pool trim could only add free memory)
    a, b = T_na.cpu().numpy(), T_ref.cpu().numpy()
    assert np.all(np.abs(a - b) <= 1e-10 * np.maximum(1.0, np.abs(b))), (a, b)


def test_noalloc_rejects_bad_tensors_on_the_host(ss):
    """Wrong dtype, shape or length never reach the kernels."""
    import torch
    sL, sR, G = blocks(5, 2, 16)
    T = torch.zeros(2, dtype=torch.float64, device="cuda")
    bad = [
        (sL.to(torch.complex64), sR, G, T),                      # complex64 block
        (sL, sR[:, :8, :8].contiguous(), G, T),                  # shape mismatch
        (sL, sR, G, torch.zeros(1, dtype=torch.float64, device="cuda")),  # T too short
        (sL, sR, G, torch.zeros(2, dtype=torch.float32, device="cuda")),  # T float32
        (sL.cpu(), sR, G, T),                                    # host tensor
        (sL[0], sR[0], G[0], T),                                 # not (P, s, s)
    ]
    for args in bad:
        with pytest.raises(ValueError):
            ss.ss_caroli_transmission_noalloc(*args)
        with pytest.raises(ValueError):
            ss.ss_caroli_transmission(*args)


def test_noalloc_rejects_sizes_beyond_its_scratch(ss):
    import torch
    sL, sR, G = blocks(3, 2, 200)  # 2 * 200^2 > 65536
    T = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(ss.SSError) as e:
        ss.ss_caroli_transmission_noalloc(sL, sR, G, T)
    assert e.value.code == ss.SS_ERR_ARG
    assert "static scratch" in str(e.value)
