"""GPU parity of products whose operands are truncated by different methods (Eq. (2.3) with
each side's own truncation; the two decompositions may differ, Section 1)."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu

METHODS = ("circulant", "svd", "fourier", "cycle")
PAIRS = [(x, y) for x in METHODS for y in METHODS if x != y]


def _handle(torch, amm, X, method, k, side, seed):
    """GPU handle and the oracle truncation of the same operand (GPU selection / sketch)."""
    x64 = as64(X)
    if method == "svd":
        phi = S.sketch(X.shape[1], k, seed, 0 if side == "left" else 1).astype(np.float32)
        h = amm.decompose(X, method, k, side, sketch=dev32(torch, phi))
        return h, O.truncate_rsvd(x64, k, phi.astype(np.float64))
    h = amm.decompose(X, method, k, side)
    sel = h.selection()
    if method == "circulant":
        return h, O.truncate_circulant(x64, k, sel)
    if method == "cycle":
        return h, O.truncate_cycles(x64, k, sel)
    if side == "left":
        return h, O.truncate_fourier_left(x64, k, forced=sel)
    return h, O.truncate_fourier_right(x64, k, forced=sel)


def _case(ma, mb, a, b, k, seed):
    torch, amm = torch_cuda()
    A, B = dev32(torch, a), dev32(torch, b)
    hA, ta = _handle(torch, amm, A, ma, k, "left", seed)
    hB, tb = _handle(torch, amm, B, mb, k, "right", seed)
    C = amm.approx_matmul(hA, hB)
    return rel(C.double().cpu().numpy(), O.mixed_product(ta, tb))


@pytest.mark.parametrize("ma,mb", PAIRS)
@pytest.mark.parametrize("n,k", [(64, 5), (256, 9), (96, 7)])
def test_mixed_square(ma, mb, n, k):
    g = S.rng(n + k, 7)
    a = g.standard_normal((n, n)) + 0.5          # a dominant zero component: odd k splits a pair
    b = S.toeplitz_uniform(n, g) + 0.1 * g.standard_normal((n, n))
    err = _case(ma, mb, a, b, k, n)
    assert err <= TOL, (ma, mb, n, k, err)


@pytest.mark.parametrize("ma,mb,m,n,p", [("svd", "fourier", 100, 128, 37), ("fourier", "svd", 77, 64, 130),
                                         ("svd", "cycle", 90, 64, 64), ("fourier", "circulant", 50, 128, 128),
                                         ("cycle", "svd", 64, 64, 33), ("circulant", "fourier", 128, 128, 40),
                                         ("svd", "circulant", 33, 256, 256), ("circulant", "svd", 256, 256, 7)])
def test_mixed_rectangular_ragged(ma, mb, m, n, p):
    """Rectangular outer sizes, including ragged column / row counts for the spectral applies."""
    g = S.rng(m + n + p, 8)
    a = g.standard_normal((m, n)) + 0.3
    b = g.uniform(0, 1, (n, p))
    err = _case(ma, mb, a, b, 6, m + p)
    assert err <= TOL, (ma, mb, m, n, p, err)


def test_mixed_untruncated_reproduces_product():
    """k = n on both sides of an SVD x circulant product: the exact product."""
    torch, amm = torch_cuda()
    n = 64
    g = S.rng(9, 0)
    a, b = g.standard_normal((n, n)), g.standard_normal((n, n))
    A, B = dev32(torch, a), dev32(torch, b)
    phi = dev32(torch, S.sketch(n, n, 9, 0))
    C = amm.approx_matmul(amm.decompose(A, "svd", n, "left", sketch=phi), amm.decompose(B, "circulant", n, "right"))
    assert rel(C.double().cpu().numpy(), as64(A) @ as64(B)) <= 1e-5


@pytest.mark.parametrize("ma,mb", PAIRS)
@pytest.mark.parametrize("n,k", [(64, 5), (96, 7), (256, 9)])
def test_mixed_backward(ma, mb, n, k):
    """dA = Re[G B~^T + P_A'(G dB^T)], dB = Re[A~^T G + P_B'(dA^T G)] with each operand's own
    adjoint projector (frozen), against the oracle on the GPU's selections / sketches."""
    torch, amm = torch_cuda()
    g = S.rng(n + k, 12)
    a = g.standard_normal((n, n)) + 0.5
    b = S.toeplitz_uniform(n, g) + 0.1 * g.standard_normal((n, n))
    gr = g.standard_normal((n, n))
    A, B, G = dev32(torch, a), dev32(torch, b), dev32(torch, gr)
    hA, ta = _handle(torch, amm, A, ma, k, "left", n)
    hB, tb = _handle(torch, amm, B, mb, k, "right", n)
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    rda, rdb = O.mixed_backward(ta, tb, as64(G))
    ea, eb = rel(dA.double().cpu().numpy(), rda), rel(dB.double().cpu().numpy(), rdb)
    assert ea <= TOL and eb <= TOL, (ma, mb, n, ea, eb)


def _split_selection(n):
    """k = 5 circulant components with two split conjugate pairs (1 without n - 1, 3 without n - 3)."""
    return [0, 1, 5, n - 5, 3]


@pytest.mark.parametrize("circ_left", [True, False])
@pytest.mark.parametrize("n", [64, 96])
def test_mixed_backward_split_pair_with_fourier(circ_left, n):
    """Circulant x Fourier with a split conjugate pair: both truncations are complex, so the
    imaginary parts Im A~, Im B~ enter the adjoint projections; also one gradient at a time."""
    torch, amm = torch_cuda()
    g = S.rng(n, 13)
    a = g.standard_normal((n, n)) + 0.5
    b = S.toeplitz_uniform(n, g) + 0.1 * g.standard_normal((n, n))
    gr = g.standard_normal((n, n))
    A, B, G = dev32(torch, a), dev32(torch, b), dev32(torch, gr)
    sel = _split_selection(n)
    if circ_left:
        hA = amm.decompose(A, "circulant", 5, "left", forced_selection=sel)
        ta = O.truncate_circulant(as64(A), 5, sel)
        hB, tb = _handle(torch, amm, B, "fourier", 6, "right", n)
    else:
        hA, ta = _handle(torch, amm, A, "fourier", 6, "left", n)
        hB = amm.decompose(B, "circulant", 5, "right", forced_selection=sel)
        tb = O.truncate_circulant(as64(B), 5, sel)
    assert np.abs(np.imag(ta.approx)).max() > 1e-3 and np.abs(np.imag(tb.approx)).max() > 1e-3
    rda, rdb = O.mixed_backward(ta, tb, as64(G))
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    ea, eb = rel(dA.double().cpu().numpy(), rda), rel(dB.double().cpu().numpy(), rdb)
    assert ea <= TOL and eb <= TOL, (circ_left, n, ea, eb)
    dA1, none_b = amm.approx_matmul_backward(hA, hB, G, need_dB=False)
    none_a, dB1 = amm.approx_matmul_backward(hA, hB, G, need_dA=False)
    assert none_b is None and none_a is None
    assert rel(dA1.double().cpu().numpy(), rda) <= TOL and rel(dB1.double().cpu().numpy(), rdb) <= TOL


def test_mixed_backward_reports_what_is_not_built():
    torch, amm = torch_cuda()
    n = 32
    g = S.rng(10, 0)
    B = dev32(torch, g.standard_normal((n, n)))
    # rectangular operands: the circulant / cycle projections of the mixed backward are square
    A2 = dev32(torch, g.standard_normal((48, n)))
    phi = dev32(torch, S.sketch(n, 3, 10, 0))
    hA2 = amm.decompose(A2, "svd", 3, "left", sketch=phi)
    hB2 = amm.decompose(B, "cycle", 3, "right")
    with pytest.raises(RuntimeError, match="square"):
        amm.approx_matmul_backward(hA2, hB2, dev32(torch, g.standard_normal((48, n))))
