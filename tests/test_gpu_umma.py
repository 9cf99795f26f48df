"""The tcgen05 tensor-core GEMM (TMA + mbarrier pipeline, TMEM accumulator) against FP64 products."""
import numpy as np
import pytest

from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _gemm(torch, amm, mode, a, b, c0=None, alpha=1.0, beta=0.0):
    lib = amm.load_library()
    M, K = a.shape
    N = b.shape[0]
    C = torch.zeros((M, N), dtype=torch.float32, device="cuda") if c0 is None else c0.clone()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.amm_debug_gemm_tn(mode, M, N, K, alpha, a.data_ptr(), a.stride(0), b.data_ptr(), b.stride(0), beta,
                               C.data_ptr(), C.stride(0), err.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.amm_last_error()
    torch.cuda.synchronize()
    assert int(err.item()) == 0, "a bounded wait gave up"
    return C


def _padded(torch, x, dtype, mult):
    """Copy x into a tensor whose row stride is a multiple of `mult` elements (16-byte rows)."""
    M, K = x.shape
    ld = (K + mult - 1) // mult * mult
    buf = torch.zeros((M, ld), dtype=dtype, device="cuda")
    buf[:, :K] = x.to(dtype)
    return buf[:, :K]


SHAPES = [(128, 128, 64), (128, 128, 32), (256, 384, 1024), (200, 130, 100), (4096, 128, 4096),
          (128, 4096, 512), (1000, 777, 333),
          # thin N: the 16 / 32 / 64-wide tiles, ragged N and M, K splits
          (4096, 16, 4096), (4096, 32, 512), (1000, 17, 333), (256, 64, 1024), (300, 8, 96), (512, 40, 256),
          (128, 1, 64), (2048, 48, 4096),
          # thin M, wide N: computed as C^T = B A^T and stored transposed
          (16, 4096, 4096), (32, 777, 333), (48, 256, 1024), (1, 300, 64),
          # short K with a wide output: 64-column tiles on the two-CTA short ring (ragged K and N too)
          (4096, 4096, 64), (4096, 4096, 32), (2048, 3000, 100), (1200, 4100, 120)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_umma_bf16(M, N, K):
    torch, amm = torch_cuda()
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    a = _padded(torch, torch.randn((M, K), device="cuda", generator=g), torch.bfloat16, 8)
    b = _padded(torch, torch.randn((N, K), device="cuda", generator=g), torch.bfloat16, 8)
    C = _gemm(torch, amm, 1, a, b)
    ref = a.double() @ b.double().T
    err = float(torch.linalg.norm(C.double() - ref) / torch.linalg.norm(ref))
    assert err <= 1e-5, err


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_umma_tf32x3_fp32_accuracy(M, N, K):
    torch, amm = torch_cuda()
    g = torch.Generator(device="cuda").manual_seed(7 * M + N + K)
    a = _padded(torch, torch.randn((M, K), device="cuda", generator=g), torch.float32, 4)
    b = _padded(torch, torch.randn((N, K), device="cuda", generator=g), torch.float32, 4)
    C = _gemm(torch, amm, 0, a, b)
    ref = a.double() @ b.double().T
    err = float(torch.linalg.norm(C.double() - ref) / torch.linalg.norm(ref))
    # FP32 level: a length-K FP32 dot product carries ~sqrt(K) * 2^-24 relative rounding error;
    # a TF32-only product would be ~1e-3
    assert err <= 4 * np.sqrt(K) * 2.0 ** -24, err


def test_umma_short_ring_alpha_beta():
    """The short ring with beta != 0 (C read back) and alpha != 1."""
    torch, amm = torch_cuda()
    M, N, K = 4096, 2048, 96
    a = torch.randn((M, K), device="cuda")
    b = torch.randn((N, K), device="cuda")
    c0 = torch.randn((M, N), device="cuda")
    C = _gemm(torch, amm, 0, a, b, c0=c0, alpha=1.5, beta=-0.25)
    ref = 1.5 * (a.double() @ b.double().T) - 0.25 * c0.double()
    assert float(torch.linalg.norm(C.double() - ref) / torch.linalg.norm(ref)) <= 4 * np.sqrt(K) * 2.0 ** -24


def test_umma_alpha_beta():
    torch, amm = torch_cuda()
    M, N, K = 256, 256, 256
    a = torch.randn((M, K), device="cuda")
    b = torch.randn((N, K), device="cuda")
    c0 = torch.randn((M, N), device="cuda")
    C = _gemm(torch, amm, 0, a, b, c0=c0, alpha=-0.5, beta=2.0)
    ref = -0.5 * (a.double() @ b.double().T) + 2.0 * c0.double()
    assert float(torch.linalg.norm(C.double() - ref) / torch.linalg.norm(ref)) <= 4 * np.sqrt(K) * 2.0 ** -24
