"""GPU parity of the circulant method at lengths that are neither 2^a nor 3 * 2^a (chirp-z DFTs,
Thm 2.1 at any n) against the FP64 oracle: selections, products, norms and frozen-selection
gradients, also at odd and prime n, with BF16 operands, beside another method and in blocks."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, check_selection, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu

LENGTHS = [17, 100, 257, 700, 1000, 1531]


def _product(torch, amm, a, b, k, kb=None, dtype=None):
    A, B = dev32(torch, a), dev32(torch, b)
    if dtype is not None:
        A, B = A.to(dtype), B.to(dtype)
    hA = amm.decompose(A, "circulant", k, "left")
    hB = amm.decompose(B, "circulant", kb or k, "right")
    C = amm.approx_matmul(hA, hB)
    a64, b64 = as64(A), as64(B)
    check_selection(hA.selection(), O.component_keys(O.circulant_spectrum(a64)), k, "A")
    check_selection(hB.selection(), O.component_keys(O.circulant_spectrum(b64)), kb or k, "B")
    ref, _, ta, _ = O.cd_matmul(a64, b64, k, kb, sel_a=hA.selection(), sel_b=hB.selection(), full=True)
    return rel(C.double().cpu().numpy(), ref), hA, ta, a64


@pytest.mark.parametrize("n", LENGTHS)
@pytest.mark.parametrize("k", [1, 5, 9])
def test_circulant_any_length_product(n, k):
    torch, amm = torch_cuda()
    g = S.rng(n + k, 21)
    a = g.uniform(0, 1, (n, n))
    b = S.toeplitz_uniform(n, g) + 0.01 * g.standard_normal((n, n))
    err, hA, ta, a64 = _product(torch, amm, a, b, k)
    assert err <= TOL, (n, k, err)
    info = hA.info()
    assert info["fro2"] == pytest.approx(float(np.sum(a64 * a64)), rel=1e-5)
    assert info["resid_fro2"] == pytest.approx(float(np.linalg.norm(ta.resid) ** 2), rel=1e-4,
                                               abs=1e-6 * info["fro2"])


def test_circulant_any_length_longest_chirp():
    """n = 3000 > 2048: the chirp-z convolutions run at the longest power-of-two length, 8192."""
    torch, amm = torch_cuda()
    n, k = 3000, 3
    g = S.rng(n, 29)
    a = g.uniform(0, 1, (n, n))
    b = S.toeplitz_uniform(n, g)
    err, *_ = _product(torch, amm, a, b, k)
    assert err <= TOL, err


@pytest.mark.parametrize("n,k", [(300, 37), (1000, 125), (999, 64)])
def test_circulant_any_length_dense_selection(n, k):
    """Many components (k up to n/8): the spectral MAC runs over a long coefficient list."""
    torch, amm = torch_cuda()
    g = S.rng(n, 22)
    a, b = g.standard_normal((n, n)) + 0.5, g.standard_normal((n, n))
    err, *_ = _product(torch, amm, a, b, k, kb=k // 2 + 1)
    assert err <= TOL, (n, k, err)


def test_circulant_any_length_untruncated_is_exact():
    """k = n keeps every component: the product is AB (Thm 2.1 at n = 100)."""
    torch, amm = torch_cuda()
    n = 100
    g = S.rng(23, 0)
    a, b = g.standard_normal((n, n)), g.standard_normal((n, n))
    A, B = dev32(torch, a), dev32(torch, b)
    C = amm.approx_matmul(amm.decompose(A, "circulant", n, "left"), amm.decompose(B, "circulant", n, "right"))
    assert rel(C.double().cpu().numpy(), as64(A) @ as64(B)) <= 1e-5


@pytest.mark.parametrize("n", [100, 257, 700])
@pytest.mark.parametrize("ka,kb", [(1, 2), (5, 4), (9, 33)])
def test_circulant_any_length_backward(n, ka, kb):
    torch, amm = torch_cuda()
    g = S.rng(n + ka, 24)
    a = g.standard_normal((n, n)) + 1.0  # a dominant component 0: odd k splits conjugate pairs
    b = S.toeplitz_uniform(n, g)
    gr = g.standard_normal((n, n))
    A, B, G = dev32(torch, a), dev32(torch, b), dev32(torch, gr)
    hA = amm.decompose(A, "circulant", ka, "left")
    hB = amm.decompose(B, "circulant", kb, "right")
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    ta = O.truncate_circulant(as64(A), ka, hA.selection())
    tb = O.truncate_circulant(as64(B), kb, hB.selection())
    rda, rdb = O.cd_backward(ta, tb, as64(G))
    ea, eb = rel(dA.double().cpu().numpy(), rda), rel(dB.double().cpu().numpy(), rdb)
    assert ea <= TOL and eb <= TOL, (n, ka, kb, ea, eb)


def test_circulant_any_length_bf16_operands():
    torch, amm = torch_cuda()
    n = 300
    g = S.rng(25, 0)
    a, b = g.uniform(0, 1, (n, n)), S.toeplitz_uniform(n, g)
    err, *_ = _product(torch, amm, a, b, 7, dtype=torch.bfloat16)
    assert err <= TOL, err


def test_circulant_any_length_mixed_with_svd():
    """Circulant at n = 300 beside an rSVD operand: product and gradients."""
    torch, amm = torch_cuda()
    n, k = 300, 6
    g = S.rng(26, 0)
    a, b, gr = g.standard_normal((n, n)) + 0.5, S.toeplitz_uniform(n, g), g.standard_normal((n, n))
    A, B, G = dev32(torch, a), dev32(torch, b), dev32(torch, gr)
    phi = S.sketch(n, k, 26, 1).astype(np.float32)
    hA = amm.decompose(A, "circulant", k, "left")
    hB = amm.decompose(B, "svd", k, "right", sketch=dev32(torch, phi))
    ta = O.truncate_circulant(as64(A), k, hA.selection())
    tb = O.truncate_rsvd(as64(B), k, phi.astype(np.float64))
    C = amm.approx_matmul(hA, hB)
    assert rel(C.double().cpu().numpy(), O.mixed_product(ta, tb)) <= TOL
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    rda, rdb = O.mixed_backward(ta, tb, as64(G))
    assert rel(dA.double().cpu().numpy(), rda) <= TOL and rel(dB.double().cpu().numpy(), rdb) <= TOL


def test_circulant_any_length_blocks():
    """Square blocks of a length that is neither 2^a nor 3 * 2^a (b = 100) on ragged operands."""
    torch, amm = torch_cuda()
    m, n, p, bs, k = 250, 230, 180, 100, 5
    g = S.rng(27, 0)
    a, b = g.standard_normal((m, n)) + 0.3, g.uniform(0, 1, (n, p))
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "circulant", k, "left", block=bs)
    hB = amm.decompose(B, "circulant", k, "right", block=bs)
    ta = O.truncate_circulant_blocked(as64(A), bs, k, selections=hA.selection())
    tb = O.truncate_circulant_blocked(as64(B), bs, k, selections=hB.selection())
    C = amm.approx_matmul(hA, hB)
    assert rel(C.double().cpu().numpy(), O.blocked_first_order(ta, tb)) <= TOL


@pytest.mark.parametrize("tol", [0.3, 0.1, 0.03])
def test_choose_k_any_length(tol):
    """The smallest k whose truncation error (from the oracle's keys) is within tol, at n = 500;
    near-ties of the error curve at the tolerance are allowed either way by 1e-4."""
    torch, amm = torch_cuda()
    n = 500
    g = S.rng(28, 0)
    A = dev32(torch, S.toeplitz_uniform(n, g) + 0.05 * g.standard_normal((n, n)))
    k = amm.choose_k(A, "circulant", tol)
    a64 = as64(A)
    keys2 = O.component_keys(O.circulant_spectrum(a64)) ** 2 * n
    order = O.top_k(np.sqrt(keys2), n)
    total = np.sum(a64 ** 2)
    resid = lambda kk: (total - np.sum(keys2[order[:kk]])) / total
    assert resid(k) <= tol ** 2 * (1 + 1e-4)
    assert k == 1 or resid(k - 1) >= tol ** 2 * (1 - 1e-4)
