"""GPU parity of rectangular circulant operands in square blocks (Section 2.3: the cycle
decomposition is square; a rectangular operand is taken in b x b blocks, ragged edge zero-padded,
top-k per block, Eq. (2.3) on the padded operands, padded rows / columns dropped)."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, check_selection, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [(100, 200, 70, 64, 5), (256, 128, 300, 128, 9), (64, 64, 64, 32, 4), (33, 16, 17, 16, 3),
          (128, 384, 256, 128, 16)]


def _pair(m, n, p, seed):
    g = S.rng(m * n + p, seed)
    a = g.standard_normal((m, n)) + 0.5       # dominant zero components; odd k splits pairs
    b = g.uniform(0, 1, (n, p))
    return a, b


def _oracle_trunc(h, x64, bs, k):
    return O.truncate_circulant_blocked(x64, bs, k, selections=h.selection())


@pytest.mark.parametrize("m,n,p,bs,k", SHAPES)
def test_blocked_product(m, n, p, bs, k):
    torch, amm = torch_cuda()
    a, b = _pair(m, n, p, 60)
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "circulant", k, "left", block=bs)
    hB = amm.decompose(B, "circulant", k, "right", block=bs)
    C = amm.approx_matmul(hA, hB)
    a64, b64 = as64(A), as64(B)
    # every block's selection is the oracle's top-k of that block outside near-ties
    ta_top = O.truncate_circulant_blocked(a64, bs, k)
    sel = hA.selection()
    assert sel.shape == (len(ta_top.sel), k)
    for i, row in enumerate(ta_top.blocks):
        for j, t in enumerate(row):
            check_selection(sel[i * len(row) + j], t.keys, k, ("A", i, j))
    ta, tb = _oracle_trunc(hA, a64, bs, k), _oracle_trunc(hB, b64, bs, k)
    err = rel(C.double().cpu().numpy(), O.blocked_first_order(ta, tb))
    assert err <= TOL, (m, n, p, bs, k, err)
    info = hA.info()
    assert abs(info["fro2"] - np.sum(a64 ** 2)) <= 1e-5 * np.sum(a64 ** 2)
    assert abs(info["resid_fro2"] - np.linalg.norm(ta.resid) ** 2) <= 1e-4 * np.sum(a64 ** 2)


def test_blocked_untruncated_is_exact():
    """k = b keeps every component of every padded block: the product is AB."""
    torch, amm = torch_cuda()
    a, b = _pair(50, 40, 30, 61)
    A, B = dev32(torch, a), dev32(torch, b)
    C = amm.approx_matmul(amm.decompose(A, "circulant", 16, "left", block=16),
                          amm.decompose(B, "circulant", 16, "right", block=16))
    assert rel(C.double().cpu().numpy(), as64(A) @ as64(B)) <= 1e-5


def test_blocked_bf16_operands():
    torch, amm = torch_cuda()
    a, b = _pair(200, 256, 90, 62)
    A = torch.from_numpy(a.astype(np.float32)).cuda().bfloat16()
    B = torch.from_numpy(b.astype(np.float32)).cuda().bfloat16()
    hA = amm.decompose(A, "circulant", 7, "left", block=64)
    hB = amm.decompose(B, "circulant", 7, "right", block=64)
    C = amm.approx_matmul(hA, hB)
    ta, tb = _oracle_trunc(hA, as64(A), 64, 7), _oracle_trunc(hB, as64(B), 64, 7)
    assert rel(C.double().cpu().numpy(), O.blocked_first_order(ta, tb)) <= TOL


@pytest.mark.parametrize("m,n,p,bs,k", [(100, 200, 70, 64, 5), (64, 64, 64, 32, 4), (96, 128, 160, 64, 8)])
def test_blocked_backward(m, n, p, bs, k):
    torch, amm = torch_cuda()
    a, b = _pair(m, n, p, 63)
    gr = S.rng(m + n + p, 64).standard_normal((m, p))
    A, B, G = dev32(torch, a), dev32(torch, b), dev32(torch, gr)
    hA = amm.decompose(A, "circulant", k, "left", block=bs)
    hB = amm.decompose(B, "circulant", k, "right", block=bs)
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    ta, tb = _oracle_trunc(hA, as64(A), bs, k), _oracle_trunc(hB, as64(B), bs, k)
    rda, rdb = O.cd_backward_blocked(ta, tb, as64(G))
    assert rel(dA.double().cpu().numpy(), rda) <= TOL
    assert rel(dB.double().cpu().numpy(), rdb) <= TOL


def _other(torch, amm, X, method, k, side, seed):
    x64 = as64(X)
    if method == "svd":
        phi = S.sketch(X.shape[1], k, seed, 0 if side == "left" else 1).astype(np.float32)
        return amm.decompose(X, method, k, side, sketch=dev32(torch, phi)), O.truncate_rsvd(x64, k, phi.astype(np.float64))
    h = amm.decompose(X, method, k, side)
    if method == "cycle":
        return h, O.truncate_cycles(x64, k, h.selection())
    f = O.truncate_fourier_left if side == "left" else O.truncate_fourier_right
    return h, f(x64, k, forced=h.selection())


@pytest.mark.parametrize("other", ["svd", "fourier", "cycle"])
@pytest.mark.parametrize("blocked_side", ["left", "right"])
def test_blocked_mixed(other, blocked_side):
    """A blocked circulant operand against another method (e.g. activations by rSVD, a weight in
    circulant blocks); the other operand is padded with zeros along the shared dimension."""
    torch, amm = torch_cuda()
    if other == "svd":
        m, n, p = (90, 128, 200) if blocked_side == "right" else (200, 100, 128)
    else:  # the cycle and Fourier sparsifiers need a power-of-two inner dimension; cycle is square
        m, n, p = (128, 128, 128) if other == "cycle" else ((70, 128, 200) if blocked_side == "right" else (200, 128, 50))
    a, b = _pair(m, n, p, 65)
    A, B = dev32(torch, a), dev32(torch, b)
    k, bs = 6, 64
    if blocked_side == "left":
        hA = amm.decompose(A, "circulant", k, "left", block=bs)
        ta = _oracle_trunc(hA, as64(A), bs, k)
        hB, tb = _other(torch, amm, B, other, k, "right", 65)
    else:
        hA, ta = _other(torch, amm, A, other, k, "left", 65)
        hB = amm.decompose(B, "circulant", k, "right", block=bs)
        tb = _oracle_trunc(hB, as64(B), bs, k)
    C = amm.approx_matmul(hA, hB)
    err = rel(C.double().cpu().numpy(), O.blocked_first_order(ta, tb))
    assert err <= TOL, (other, blocked_side, err)


def _mixed_shapes(other, blocked_side):
    if other == "svd":
        return (90, 128, 200) if blocked_side == "right" else (200, 100, 128)
    if other == "cycle":  # square, in 2 x 2 blocks
        return 128, 128, 128
    return (70, 128, 200) if blocked_side == "right" else (200, 128, 50)


@pytest.mark.parametrize("other", ["svd", "fourier", "cycle"])
@pytest.mark.parametrize("blocked_side", ["left", "right"])
def test_blocked_mixed_backward(other, blocked_side):
    """Gradients of the blocked x other-method product with the projectors frozen: G padded with
    zeros, each block's adjoint on b-wide pieces of the inner sums, the gradients cropped; k = 6
    splits conjugate pairs in some blocks, so beside the Fourier sparsifier the imaginary parts
    enter as well.  Also one gradient at a time."""
    torch, amm = torch_cuda()
    m, n, p = _mixed_shapes(other, blocked_side)
    a, b = _pair(m, n, p, 66)
    gr = S.rng(66, 1).standard_normal((m, p))
    A, B, G = dev32(torch, a), dev32(torch, b), dev32(torch, gr)
    k, bs = 6, 64
    if blocked_side == "left":
        hA = amm.decompose(A, "circulant", k, "left", block=bs)
        ta = _oracle_trunc(hA, as64(A), bs, k)
        hB, tb = _other(torch, amm, B, other, k, "right", 66)
    else:
        hA, ta = _other(torch, amm, A, other, k, "left", 66)
        hB = amm.decompose(B, "circulant", k, "right", block=bs)
        tb = _oracle_trunc(hB, as64(B), bs, k)
    rda, rdb = O.blocked_mixed_backward(ta, tb, as64(G))
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    ea, eb = rel(dA.double().cpu().numpy(), rda), rel(dB.double().cpu().numpy(), rdb)
    assert ea <= TOL and eb <= TOL, (other, blocked_side, ea, eb)
    dA1, _ = amm.approx_matmul_backward(hA, hB, G, need_dB=False)
    _, dB1 = amm.approx_matmul_backward(hA, hB, G, need_dA=False)
    assert rel(dA1.double().cpu().numpy(), rda) <= TOL and rel(dB1.double().cpu().numpy(), rdb) <= TOL


def test_blocked_cycle_backward_needs_square():
    torch, amm = torch_cuda()
    a, b = _pair(96, 128, 128, 67)
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "circulant", 4, "left", block=64)
    hB = amm.decompose(B, "cycle", 4, "right")
    with pytest.raises(RuntimeError, match="square"):
        amm.approx_matmul_backward(hA, hB, dev32(torch, np.ones((96, 128))))


def test_blocked_argument_errors():
    torch, amm = torch_cuda()
    a, b = _pair(64, 128, 64, 66)
    A, B = dev32(torch, a), dev32(torch, b)
    with pytest.raises(RuntimeError, match="block=5000"):  # above 4096 and not 2^a
        amm.decompose(A, "circulant", 3, "left", block=5000)
    with pytest.raises(RuntimeError, match="block"):
        amm.decompose(A, "svd", 3, "left", block=64)
    with pytest.raises(RuntimeError, match="k="):
        amm.decompose(A, "circulant", 33, "left", block=32)
    with pytest.raises(ValueError, match="entries"):
        amm.decompose(A, "circulant", 2, "left", block=64, forced_selection=[0, 1])
    hA = amm.decompose(A, "circulant", 3, "left", block=64)
    hB = amm.decompose(B, "circulant", 3, "right", block=32)
    with pytest.raises(RuntimeError, match="blocks differ"):
        amm.approx_matmul(hA, hB)


def test_blocked_forced_selection_roundtrip():
    """A selection exported from one handle and forced on another reproduces the same product."""
    torch, amm = torch_cuda()
    a, b = _pair(100, 96, 40, 67)
    A, B = dev32(torch, a), dev32(torch, b)
    h1 = amm.decompose(A, "circulant", 4, "left", block=32)
    sel = h1.selection()
    h2 = amm.decompose(A, "circulant", 4, "left", block=32, forced_selection=sel[::-1].copy())
    assert np.array_equal(h2.selection(), sel[::-1])
    hB = amm.decompose(B, "circulant", 4, "right", block=32)
    ta = O.truncate_circulant_blocked(as64(A), 32, 4, selections=sel[::-1])
    tb = _oracle_trunc(hB, as64(B), 32, 4)
    C = amm.approx_matmul(h2, hB)
    assert rel(C.double().cpu().numpy(), O.blocked_first_order(ta, tb)) <= TOL
