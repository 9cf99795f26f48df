"""GPU parity of the randomized-SVD first-order product (Alg. 1, Section 2.2) and its backward."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _sketches(torch, n, p, k, seed):
    pa = S.sketch(n, k, seed, 0).astype(np.float32)
    pb = S.sketch(p, k, seed, 1).astype(np.float32)
    return pa, pb, dev32(torch, pa), dev32(torch, pb)


def _svd_case(torch, amm, a, b, k, seed=0, grad=False):
    A, B = dev32(torch, a), dev32(torch, b)
    pa, pb, PA, PB = _sketches(torch, a.shape[1], b.shape[1], k, seed)
    hA = amm.decompose(A, "svd", k, "left", sketch=PA)
    hB = amm.decompose(B, "svd", k, "right", sketch=PB)
    C = amm.approx_matmul(hA, hB)
    a64, b64 = as64(A), as64(B)
    ref, _, ta, tb = O.svd_matmul(a64, b64, k, pa.astype(np.float64), pb.astype(np.float64), full=True)
    err = rel(C.double().cpu().numpy(), ref)
    out = {"err": err}
    if grad:
        g = S.upstream_grad(a.shape[0], b.shape[1], seed)
        G = dev32(torch, g)
        dA, dB = amm.approx_matmul_backward(hA, hB, G)
        rda, rdb = O.svd_backward(ta, tb, as64(G))
        out["dA"] = rel(dA.double().cpu().numpy(), rda)
        out["dB"] = rel(dB.double().cpu().numpy(), rdb)
    return out


@pytest.mark.parametrize("k", [32, 64, 128, 256])
def test_svd_exp32_n512(k):
    """n = 512, sigma_i = e^{-i/32} + 1e-3 noise, the small FP32 case, rSVD rank sweep."""
    torch, amm = torch_cuda()
    a, b = S.exp32_pair(512, seed=0)
    assert _svd_case(torch, amm, a, b, k)["err"] <= TOL


@pytest.mark.parametrize("m,n,p,k", [(200, 300, 150, 17), (96, 64, 40, 8), (1000, 777, 333, 64)])
def test_svd_rectangular_ragged(m, n, p, k):
    """Rectangular operands with sizes that leave ragged GEMM tiles."""
    torch, amm = torch_cuda()
    g = S.rng(3, 0)
    a = S.spectrum_matrix(np.exp(-np.arange(n) / 10.0), g)[:m] if m <= n else g.standard_normal((m, n))
    b = g.standard_normal((n, p))
    r = _svd_case(torch, amm, a, b, k, grad=True)
    assert r["err"] <= TOL and r["dA"] <= TOL and r["dB"] <= TOL, r


@pytest.mark.parametrize("k", [32, 128])
def test_svd_powerlaw_n4096(k):
    torch, amm = torch_cuda()
    a, b = S.powerlaw_pair(4096, seed=0)
    assert _svd_case(torch, amm, a, b, k)["err"] <= TOL


def test_svd_backward_n512():
    torch, amm = torch_cuda()
    a, b = S.exp32_pair(512, seed=1)
    r = _svd_case(torch, amm, a, b, 32, seed=1, grad=True)
    assert r["err"] <= TOL and r["dA"] <= TOL and r["dB"] <= TOL, r


def test_svd_rank_deficient_is_exact():
    """Rank-r operands with k >= r: A~ = A, so the product is A B."""
    torch, amm = torch_cuda()
    n, r, k = 256, 6, 12
    g = S.rng(4, 0)
    a = g.standard_normal((n, r)) @ g.standard_normal((r, n))
    b = g.standard_normal((n, r)) @ g.standard_normal((r, n))
    A, B = dev32(torch, a), dev32(torch, b)
    _, _, PA, PB = _sketches(torch, n, n, k, 4)
    C = amm.approx_matmul(amm.decompose(A, "svd", k, "left", sketch=PA), amm.decompose(B, "svd", k, "right", sketch=PB))
    assert rel(C.double().cpu().numpy(), as64(A) @ as64(B)) <= 1e-5


def test_svd_generated_sketch_exported():
    """Without a caller sketch the library draws phi (Philox4x32-10 + Box-Muller); exporting it
    lets the oracle reproduce the product."""
    torch, amm = torch_cuda()
    n, k = 256, 16
    a, b = S.exp32_pair(n, seed=3)
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "svd", k, "left", seed=123)
    hB = amm.decompose(B, "svd", k, "right", seed=456)
    C = amm.approx_matmul(hA, hB)
    pa, pb = hA.sketch().astype(np.float64), hB.sketch().astype(np.float64)
    assert abs(pa.mean()) < 0.05 and abs(pa.std() - 1) < 0.05
    assert not np.array_equal(pa, pb)
    ref = O.svd_matmul(as64(A), as64(B), k, pa, pb)
    assert rel(C.double().cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("k", [32, 128])
def test_svd_bf16_tensor_core_mode(k):
    """BF16 precision mode: operands, sketch and every low-rank GEMM in BF16 on tcgen05 with FP32
    accumulation.  The error against the FP64 oracle is the BF16 rounding of the operands and
    intermediates (~2^-8 per element), far above the FP32 mode's 1e-5; it is bounded and reported."""
    torch, amm = torch_cuda()
    a, b = S.exp32_pair(512, seed=2)
    A, B = dev32(torch, a), dev32(torch, b)
    pa, pb, PA, PB = _sketches(torch, 512, 512, k, 2)
    hA = amm.decompose(A, "svd", k, "left", sketch=PA, compute="bf16")
    hB = amm.decompose(B, "svd", k, "right", sketch=PB, compute="bf16")
    C = amm.approx_matmul(hA, hB)
    ref, _, ta, tb = O.svd_matmul(as64(A), as64(B), k, pa.astype(np.float64), pb.astype(np.float64), full=True)
    err = rel(C.double().cpu().numpy(), ref)
    assert err <= 3e-2, err
    g = S.upstream_grad(512, 512, 2)
    dA, dB = amm.approx_matmul_backward(hA, hB, dev32(torch, g))
    rda, rdb = O.svd_backward(ta, tb, g.astype(np.float32).astype(np.float64))
    assert rel(dA.double().cpu().numpy(), rda) <= 3e-2
    assert rel(dB.double().cpu().numpy(), rdb) <= 3e-2
    # BF16 operands given directly
    hA2 = amm.decompose(A.bfloat16(), "svd", k, "left", sketch=PA, compute="bf16")
    hB2 = amm.decompose(B.bfloat16(), "svd", k, "right", sketch=PB, compute="bf16")
    C2 = amm.approx_matmul(hA2, hB2)
    ref2 = O.svd_matmul(as64(A.bfloat16()), as64(B.bfloat16()), k, pa.astype(np.float64), pb.astype(np.float64))
    assert rel(C2.double().cpu().numpy(), ref2) <= 3e-2
    assert hA.info()["resid_fro2"] > 0
