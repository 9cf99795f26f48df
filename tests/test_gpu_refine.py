"""GPU parity of the refinement of Section 2.5 (reading R16): the dense residue Re dA of each method
against the oracle's, and C + Re M2 - Im(A~) Im(B~) against the oracle's refine, where M2 is the
first-order product of decompositions of the residues."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, check_selection, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _decomp(torch, amm, X, method, k, role, seed):
    """Handle of X and the matching oracle truncation of its FP32 values (the GPU's selection, the
    same seeded sketch)."""
    x64 = as64(X)
    if method == "svd":
        phi = S.sketch(X.shape[1], k, seed, 0 if role == "left" else 1).astype(np.float32)
        return amm.decompose(X, "svd", k, role, sketch=dev32(torch, phi)), phi.astype(np.float64)
    return amm.decompose(X, method, k, role), None


def _oracle_trunc(h, x64, method, k, role, phi):
    if method == "svd":
        return O.truncate_rsvd(x64, k, phi)
    if method == "fourier":
        f = O.truncate_fourier_left if role == "left" else O.truncate_fourier_right
        return f(x64, k, forced=h.selection())
    return O.truncate(method, x64, k, selection=h.selection())


@pytest.mark.parametrize("method,role,k", [("svd", "left", 8), ("svd", "right", 8), ("circulant", "left", 4),
                                           ("circulant", "right", 4), ("cycle", "left", 5), ("cycle", "right", 5),
                                           ("fourier", "left", 5), ("fourier", "right", 5)])
def test_residual_matches_oracle(method, role, k):
    torch, amm = torch_cuda()
    n = 256
    a, b = S.general_times_toeplitz(n, seed=1)
    X = dev32(torch, a if role == "left" else b)
    h, phi = _decomp(torch, amm, X, method, k, role, 70)
    t = _oracle_trunc(h, as64(X), method, k, role, phi)
    D = amm.residual(h)
    assert D.shape == X.shape
    assert rel(D.double().cpu().numpy(), t.resid.real) <= TOL, method


PAIRS = [("circulant", "circulant", 4, 3), ("svd", "svd", 8, 4), ("cycle", "cycle", 5, 3),
         ("svd", "circulant", 6, 3), ("fourier", "circulant", 5, 4), ("circulant", "cycle", 4, 2),
         ("fourier", "svd", 5, 6), ("circulant", "fourier", 4, 5)]


@pytest.mark.parametrize("ma,mb,k,k2", PAIRS)
def test_refine_matches_oracle(ma, mb, k, k2):
    torch, amm = torch_cuda()
    n = 256
    a, b = S.general_times_toeplitz(n, seed=2)
    A, B = dev32(torch, a), dev32(torch, b)
    hA, pa = _decomp(torch, amm, A, ma, k, "left", 71)
    hB, pb = _decomp(torch, amm, B, mb, k, "right", 71)
    ta = _oracle_trunc(hA, as64(A), ma, k, "left", pa)
    tb = _oracle_trunc(hB, as64(B), mb, k, "right", pb)
    C = amm.approx_matmul(hA, hB)
    hA2, pa2 = _decomp(torch, amm, amm.residual(hA), ma, k2, "left", 72)
    hB2, pb2 = _decomp(torch, amm, amm.residual(hB), mb, k2, "right", 72)
    # the oracle decomposes its own residues (FP64), with the GPU's selections where it selects
    ta2 = _oracle_trunc(hA2, ta.resid.real, ma, k2, "left", pa2)
    tb2 = _oracle_trunc(hB2, tb.resid.real, mb, k2, "right", pb2)
    for h2, t, m, k_ in ((hA2, ta, ma, k2), (hB2, tb, mb, k2)):
        if m == "circulant":
            check_selection(h2.selection(), O.component_keys(O.circulant_spectrum(t.resid.real)), k_, m)
        elif m == "cycle":
            check_selection(h2.selection(), O.cycle_keys(t.resid.real), k_, m)
    amm.refine_product(hA, hB, hA2, hB2, C)
    ref = O.refine(ta, tb, ta2, tb2)
    assert rel(C.double().cpu().numpy(), ref) <= TOL, (ma, mb)


def test_refined_circulant_equals_the_larger_truncation():
    """Nested circulant selections: refining k = 1 by k2 = 4 gives the first-order product at k = 5
    (the top-4 components of the real residue are the operand's next four)."""
    torch, amm = torch_cuda()
    n = 256
    a, b = S.general_times_toeplitz(n, seed=0)
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "circulant", 1, "left")
    hB = amm.decompose(B, "circulant", 1, "right")
    C = amm.approx_matmul(hA, hB)
    C, hA2, hB2 = amm.refine(hA, hB, C, 4)
    C5 = amm.approx_matmul(amm.decompose(A, "circulant", 5, "left"), amm.decompose(B, "circulant", 5, "right"))
    assert rel(C.double().cpu().numpy(), C5.double().cpu().numpy()) <= TOL
    a64, b64 = as64(A), as64(B)
    exact = a64 @ b64
    assert rel(C.double().cpu().numpy(), exact) < rel(amm.approx_matmul(hA, hB).double().cpu().numpy(), exact)


def test_refine_argument_errors():
    torch, amm = torch_cuda()
    n = 64
    a, b = S.general_times_toeplitz(n, seed=3)
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "circulant", 3, "left")
    hB = amm.decompose(B, "circulant", 3, "right")
    C = amm.approx_matmul(hA, hB)
    small = dev32(torch, a[:32, :32])
    with pytest.raises(RuntimeError, match="shapes"):
        amm.refine_product(hA, hB, amm.decompose(small, "circulant", 2, "left"),
                           amm.decompose(small, "circulant", 2, "right"), C[:32, :32])
    Ab = A.bfloat16()
    hAb = amm.decompose(Ab, "circulant", 3, "left")
    with pytest.raises(RuntimeError, match="BF16"):
        amm.residual(hAb)
