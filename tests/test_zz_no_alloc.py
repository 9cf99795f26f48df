"""amm_circulant_spectrum_noalloc against amm_decompose (GPU).

The allocation-free entry point serves callers that cannot call cudaMalloc (allocation is
forbidden while their framework captures a CUDA graph, or their device memory belongs to
another allocator).  Its scratch is a fixed device array shared by all calls, so this test
calls it twice in a row on different inputs and checks each result against the allocating
path: the Parseval norm, the residual norm and the top-k selection that amm_decompose reports
must follow from the returned keys, and the returned spectrum must match the FP64 oracle.
This file is collected last and also passes alone in a fresh process (first call sets up).
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _noalloc(torch, lib, A):
    n = A.shape[0]
    R = torch.empty((n // 2 + 1, n), dtype=torch.complex64, device="cuda")
    keys = torch.empty(n, dtype=torch.float64, device="cuda")
    st = lib.amm_circulant_spectrum_noalloc(A.data_ptr(), n, A.stride(0), R.data_ptr(), keys.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.amm_last_error()
    torch.cuda.synchronize()
    return R, keys.cpu().numpy()


def test_noalloc_spectrum_matches_decompose_on_two_calls():
    """Three calls in a row (the shared scratch keeps the previous call's contents): the keys are
    the same doubles amm_decompose ranks, so the top-k taken from them is amm_decompose's selection
    in its order; k is odd, so the boundary splits an exactly tied conjugate pair (t, n - t) and the
    lower index must win on both paths (checked: at least one of the calls splits a pair)."""
    torch, amm = torch_cuda()
    lib = amm.load_library()
    splits = 0
    for seed, n, k in [(1, 512, 9), (2, 4096, 33), (3, 512, 4)]:
        a, _ = S.exp32_pair(n, seed=seed) if n <= 512 else S.powerlaw_pair(n, seed=seed)
        A = dev32(torch, a)
        R, keys = _noalloc(torch, lib, A)
        h = amm.decompose(A, "circulant", k, "left")
        info, sel = h.info(), h.selection()
        assert np.array_equal(keys.view(np.uint64), h.keys().view(np.uint64))
        fro2 = n * float(np.sum(keys * keys))
        assert fro2 == pytest.approx(info["fro2"], rel=1e-12)
        assert fro2 - n * float(np.sum(keys[sel] ** 2)) == pytest.approx(info["resid_fro2"], rel=1e-9,
                                                                          abs=1e-12 * fro2)
        order = np.lexsort((np.arange(n), -keys))[:k]
        assert order.tolist() == sel.tolist()
        assert all(keys[t] == keys[n - t] for t in range(1, n // 2))
        splits += any((n - int(t)) % n not in set(sel.tolist()) for t in sel)
        ref = O.circulant_spectrum(as64(A))[: n // 2 + 1]
        assert rel(R.cpu().numpy().astype(np.complex128), ref) <= TOL
        h.close()
    assert splits >= 1


def test_noalloc_call_leaves_free_device_memory_unchanged():
    """After a first call on the device (kernels loaded, scratch address looked up), a call changes
    the device's free memory by nothing: it allocates no device memory."""
    torch, amm = torch_cuda()
    lib = amm.load_library()
    n = 1024
    a, _ = S.exp32_pair(n, seed=4)
    A = dev32(torch, a)
    R, keys = _noalloc(torch, lib, A)
    R2 = torch.empty_like(R)
    K2 = torch.empty(n, dtype=torch.float64, device="cuda")
    A.mul_(0.5)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = lib.amm_circulant_spectrum_noalloc(A.data_ptr(), n, A.stride(0), R2.data_ptr(), K2.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == 0, lib.amm_last_error()
    assert torch.cuda.mem_get_info()[0] == free0
    assert rel(R2.cpu().numpy().astype(np.complex128), O.circulant_spectrum(as64(A))[: n // 2 + 1]) <= TOL


def test_noalloc_rejects_sizes_beyond_the_scratch():
    torch, amm = torch_cuda()
    lib = amm.load_library()
    n = 8192
    A = torch.zeros((n, n), device="cuda")
    R = torch.empty((2, 2), dtype=torch.complex64, device="cuda")
    keys = torch.empty(2, dtype=torch.float64, device="cuda")
    st = lib.amm_circulant_spectrum_noalloc(A.data_ptr(), n, n, R.data_ptr(), keys.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    assert st == 2 and b"4096" in lib.amm_last_error()
