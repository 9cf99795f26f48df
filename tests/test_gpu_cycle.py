"""GPU parity of the cycle-sparsified first-order product (Section 1.2.2, Eq. (2.4)-(2.5))."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, check_selection, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _check(torch, amm, a, b, ka, kb=None):
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "cycle", ka, "left")
    hB = amm.decompose(B, "cycle", kb or ka, "right")
    C = amm.approx_matmul(hA, hB)
    a64, b64 = as64(A), as64(B)
    # cycles are real and have no conjugate partners: the plain near-tie rule applies
    check_selection(hA.selection(), O.cycle_keys(a64), ka, "A")
    check_selection(hB.selection(), O.cycle_keys(b64), kb or ka, "B")
    ref, _, ta, _ = O.cycle_matmul(a64, b64, ka, kb, sel_a=hA.selection(), sel_b=hB.selection(), full=True)
    err = rel(C.double().cpu().numpy(), ref.real)
    assert err <= TOL, (a.shape, ka, err)
    info = hA.info()
    assert info["fro2"] == pytest.approx(float(np.sum(a64 * a64)), rel=1e-5)
    assert info["resid_fro2"] == pytest.approx(float(np.sum(ta.resid ** 2)), rel=1e-4, abs=1e-6 * info["fro2"])
    return err


@pytest.mark.parametrize("n", [16, 64, 256, 1024])
@pytest.mark.parametrize("k", [1, 3, 10])
def test_cycle_small(n, k):
    torch, amm = torch_cuda()
    g = S.rng(n + k, 0)
    a = g.standard_normal((n, n)) + np.diag(np.full(n, 3.0))   # the main cycle dominates
    b = S.toeplitz_uniform(n, g)
    _check(torch, amm, a, b, k, k + 1 if k < n else k)


@pytest.mark.parametrize("k", [41, 128])
def test_cycle_powerlaw_n4096(k):
    """k = ceil(0.01 n) = 41 cycles (1% of the entries) on the n = 4096 power-law pair."""
    torch, amm = torch_cuda()
    a, b = S.powerlaw_pair(4096, seed=0)
    _check(torch, amm, a, b, k)


def test_cycle_untruncated_exact():
    torch, amm = torch_cuda()
    n = 64
    a, b = S.exp32_pair(n, seed=2)
    A, B = dev32(torch, a), dev32(torch, b)
    C = amm.approx_matmul(amm.decompose(A, "cycle", n, "left"), amm.decompose(B, "cycle", n, "right"))
    assert rel(C.double().cpu().numpy(), as64(A) @ as64(B)) <= TOL


def test_cycle_banded_is_exact():
    """A banded matrix with k nonzero cycles is reproduced exactly: A_s = A, dA = 0."""
    torch, amm = torch_cuda()
    n = 128
    g = S.rng(3, 0)
    a = np.zeros((n, n))
    for j in (0, 1, n - 1):
        for l in range(n):
            a[(l + j) % n, l] = g.standard_normal()
    b = g.standard_normal((n, n))
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "cycle", 3, "left")
    assert sorted(hA.selection().tolist()) == [0, 1, n - 1]
    C = amm.approx_matmul(hA, amm.decompose(B, "cycle", 5, "right"))
    assert rel(C.double().cpu().numpy(), as64(A) @ as64(B)) <= TOL


@pytest.mark.parametrize("n,ka,kb", [(16, 1, 2), (64, 3, 5), (256, 10, 7), (1024, 11, 11)])
def test_cycle_backward(n, ka, kb):
    """Frozen-selection gradients of the cycle-sparsified product against the oracle."""
    torch, amm = torch_cuda()
    g = S.rng(n + ka + kb, 0)
    a = g.standard_normal((n, n)) + np.diag(np.full(n, 3.0))
    b = S.toeplitz_uniform(n, g)
    gr = g.standard_normal((n, n))
    A, B, Gt = dev32(torch, a), dev32(torch, b), dev32(torch, gr)
    hA = amm.decompose(A, "cycle", ka, "left")
    hB = amm.decompose(B, "cycle", kb, "right")
    dA, dB = amm.approx_matmul_backward(hA, hB, Gt)
    ta = O.truncate_cycles(as64(A), ka, hA.selection())
    tb = O.truncate_cycles(as64(B), kb, hB.selection())
    rda, rdb = O.cycle_backward(ta, tb, as64(Gt))
    assert rel(dA.double().cpu().numpy(), rda) <= TOL
    assert rel(dB.double().cpu().numpy(), rdb) <= TOL


@pytest.mark.parametrize("n,ka,kb", [(64, 4, 3), (2048, 21, 21)])
def test_cycle_backward_strided_gradient(n, ka, kb):
    """Upstream gradient with an odd leading dimension (rows not 16-byte aligned) and outputs with
    padded leading dimensions."""
    torch, amm = torch_cuda()
    lib = amm.load_library()
    g = S.rng(n + ka + kb, 1)
    a = g.standard_normal((n, n)) + np.diag(np.full(n, 3.0))
    b = S.toeplitz_uniform(n, g)
    gr = g.standard_normal((n, n))
    A, B = dev32(torch, a), dev32(torch, b)
    Gw = dev32(torch, np.concatenate([gr, np.zeros((n, 1))], axis=1))   # ldg = n + 1
    dAw = torch.zeros((n, n + 3), device="cuda")
    dBw = torch.zeros((n, n + 5), device="cuda")
    hA = amm.decompose(A, "cycle", ka, "left")
    hB = amm.decompose(B, "cycle", kb, "right")
    st = torch.cuda.current_stream().cuda_stream
    assert lib.amm_approx_matmul_backward(hA.ptr, hB.ptr, Gw.data_ptr(), n + 1, dAw.data_ptr(), n + 3,
                                          dBw.data_ptr(), n + 5, st) == 0
    ta = O.truncate_cycles(as64(A), ka, hA.selection())
    tb = O.truncate_cycles(as64(B), kb, hB.selection())
    rda, rdb = O.cycle_backward(ta, tb, gr.astype(np.float32).astype(np.float64))
    assert rel(dAw[:, :n].double().cpu().numpy(), rda) <= TOL
    assert rel(dBw[:, :n].double().cpu().numpy(), rdb) <= TOL


def test_cycle_bf16_operands():
    """BF16 operands of the cycle sparsifier (widened to FP32 once by the handle)."""
    torch, amm = torch_cuda()
    n, k = 256, 9
    a, b = S.general_times_toeplitz(n, seed=12)
    A = torch.from_numpy(a.astype(np.float32)).cuda().bfloat16()
    B = torch.from_numpy(b.astype(np.float32)).cuda().bfloat16()
    hA = amm.decompose(A, "cycle", k, "left")
    hB = amm.decompose(B, "cycle", k, "right")
    C = amm.approx_matmul(hA, hB)
    ref = O.cycle_matmul(as64(A), as64(B), k, sel_a=hA.selection(), sel_b=hB.selection())
    assert rel(C.double().cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("n,k", [(48, 3), (100, 5), (700, 7), (1000, 10), (3072, 31)])
def test_cycle_general_n(n, k):
    """Lengths that are not powers of two (multiples of 4), e.g. the paper's n = 700 experiments."""
    torch, amm = torch_cuda()
    a, b = S.general_times_toeplitz(n, seed=n)
    _check(torch, amm, a, b, k, k + 1)


@pytest.mark.parametrize("n,ka,kb", [(100, 3, 4), (700, 7, 7), (1000, 12, 9)])
def test_cycle_backward_general_n(n, ka, kb):
    torch, amm = torch_cuda()
    g = S.rng(n + ka + kb, 2)
    a = g.standard_normal((n, n)) + np.diag(np.full(n, 3.0))
    b = S.toeplitz_uniform(n, g)
    gr = g.standard_normal((n, n))
    A, B, Gt = dev32(torch, a), dev32(torch, b), dev32(torch, gr)
    hA = amm.decompose(A, "cycle", ka, "left")
    hB = amm.decompose(B, "cycle", kb, "right")
    dA, dB = amm.approx_matmul_backward(hA, hB, Gt)
    ta = O.truncate_cycles(as64(A), ka, hA.selection())
    tb = O.truncate_cycles(as64(B), kb, hB.selection())
    rda, rdb = O.cycle_backward(ta, tb, as64(Gt))
    assert rel(dA.double().cpu().numpy(), rda) <= TOL
    assert rel(dB.double().cpu().numpy(), rdb) <= TOL


@pytest.mark.parametrize("ma,mb,n", [("circulant", "cycle", 96), ("cycle", "circulant", 96), ("svd", "cycle", 100),
                                     ("cycle", "svd", 100)])
def test_mixed_general_n(ma, mb, n):
    """Mixed products at lengths the Fourier sparsifier does not take (3 * 2^a, 4 x odd)."""
    torch, amm = torch_cuda()
    g = S.rng(n, 3)
    a, b = g.standard_normal((n, n)) + 0.5, S.toeplitz_uniform(n, g)
    A, B = dev32(torch, a), dev32(torch, b)

    def side(method, X, role):
        x64 = as64(X)
        if method == "svd":
            phi = S.sketch(n, 6, n, 0 if role == "left" else 1).astype(np.float32)
            return amm.decompose(X, "svd", 6, role, sketch=dev32(torch, phi)), O.truncate_rsvd(x64, 6, phi.astype(np.float64))
        h = amm.decompose(X, method, 6, role)
        t = O.truncate_circulant(x64, 6, h.selection()) if method == "circulant" else O.truncate_cycles(x64, 6, h.selection())
        return h, t

    hA, ta = side(ma, A, "left")
    hB, tb = side(mb, B, "right")
    C = amm.approx_matmul(hA, hB)
    assert rel(C.double().cpu().numpy(), O.mixed_product(ta, tb)) <= TOL
