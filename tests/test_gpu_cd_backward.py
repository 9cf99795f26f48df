"""GPU parity of the circulant backward (frozen selections) against the oracle's gradients."""
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _case(torch, amm, a, b, g, ka, kb):
    A, B, Gt = dev32(torch, a), dev32(torch, b), dev32(torch, g)
    hA = amm.decompose(A, "circulant", ka, "left")
    hB = amm.decompose(B, "circulant", kb, "right")
    dA, dB = amm.approx_matmul_backward(hA, hB, Gt)
    a64, b64, g64 = as64(A), as64(B), as64(Gt)
    ta = O.truncate_circulant(a64, ka, hA.selection())
    tb = O.truncate_circulant(b64, kb, hB.selection())
    rda, rdb = O.cd_backward(ta, tb, g64)
    return rel(dA.double().cpu().numpy(), rda), rel(dB.double().cpu().numpy(), rdb), hA.info(), hB.info()


@pytest.mark.parametrize("n", [16, 64, 256])
@pytest.mark.parametrize("ka,kb", [(1, 1), (2, 3), (4, 4), (5, 8)])
def test_cd_backward_small(n, ka, kb):
    torch, amm = torch_cuda()
    g = S.rng(n + ka, 0)
    a = g.standard_normal((n, n)) + 1.0   # dominant component 0: odd k splits conjugate pairs
    b = S.toeplitz_uniform(n, g)
    gr = g.standard_normal((n, n))
    ea, eb, ia, ib = _case(torch, amm, a, b, gr, ka, kb)
    assert ea <= TOL and eb <= TOL, (ea, eb, ia["n_unpaired"], ib["n_unpaired"])


def test_cd_backward_unpaired_on_both_sides():
    torch, amm = torch_cuda()
    n = 128
    g = S.rng(3, 0)
    a = g.standard_normal((n, n)) + 1.0
    b = g.standard_normal((n, n)) + 1.0
    gr = g.standard_normal((n, n))
    ea, eb, ia, ib = _case(torch, amm, a, b, gr, 2, 4)
    assert ia["n_unpaired"] >= 1 and ib["n_unpaired"] >= 1
    assert ea <= TOL and eb <= TOL, (ea, eb)


@pytest.mark.parametrize("k", [16, 64, 256])
def test_cd_backward_powerlaw_n4096(k):
    torch, amm = torch_cuda()
    a, b = S.powerlaw_pair(4096, seed=0)
    gr = S.upstream_grad(4096, 4096, 0)
    ea, eb, _, _ = _case(torch, amm, a, b, gr, k, k)
    assert ea <= TOL and eb <= TOL, (ea, eb)


def test_cd_autograd_layer():
    """The autograd Function routes backward through the circulant adjoint kernels."""
    torch, amm = torch_cuda()
    n, k = 64, 5
    a, b = S.exp32_pair(n, seed=4)
    A = dev32(torch, a).requires_grad_(True)
    B = dev32(torch, b).requires_grad_(True)
    C = amm.approx_matmul_autograd(A, B, "circulant", k)
    gr = torch.randn_like(C)
    C.backward(gr)
    hA = amm.decompose(A.detach(), "circulant", k, "left")
    hB = amm.decompose(B.detach(), "circulant", k, "right")
    ta = O.truncate_circulant(as64(A), k, hA.selection())
    tb = O.truncate_circulant(as64(B), k, hB.selection())
    rda, rdb = O.cd_backward(ta, tb, as64(gr))
    assert rel(A.grad.double().cpu().numpy(), rda) <= TOL
    assert rel(B.grad.double().cpu().numpy(), rdb) <= TOL


@pytest.mark.parametrize("ka,kb", [(48, 45), (5, 60), (101, 3)])
def test_cd_backward_n1024_dense_and_sparse_selections(ka, kb):
    """n = 1024 with selections dense enough for the staged (tiled) SDDMM on one or both sides,
    odd k splitting conjugate pairs (unpaired terms on), and a sparse side on the warp kernel."""
    torch, amm = torch_cuda()
    n = 1024
    g = S.rng(n + ka + kb, 0)
    a = g.standard_normal((n, n)) + 1.0
    b = S.toeplitz_uniform(n, g) + 0.2 * g.standard_normal((n, n))
    gr = g.standard_normal((n, n))
    ea, eb, ia, ib = _case(torch, amm, a, b, gr, ka, kb)
    assert ea <= TOL and eb <= TOL, (ea, eb, ia["n_unpaired"], ib["n_unpaired"])
