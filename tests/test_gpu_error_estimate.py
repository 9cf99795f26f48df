"""Section 2.5 on the GPU: the posterior estimate (Corollary 3.7) and the a priori estimate against
the oracle's on the same truncations, k from a tolerance, and the choice of the most suitable
decomposition per operand."""
import math

import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method,k", [("circulant", 3), ("cycle", 9), ("fourier", 45), ("svd", 9)])
def test_error_estimate_matches_oracle(method, k):
    torch, amm = torch_cuda()
    n = 512
    a, b = S.general_times_toeplitz(n, seed=0)
    A, B = dev32(torch, a), dev32(torch, b)
    sa = dev32(torch, S.sketch(n, k, 0, 0)) if method == "svd" else None
    sb = dev32(torch, S.sketch(n, k, 0, 1)) if method == "svd" else None
    hA = amm.decompose(A, method, k, "left", sketch=sa)
    hB = amm.decompose(B, method, k, "right", sketch=sb)
    C = amm.approx_matmul(hA, hB)
    est = amm.error_estimate(hA, hB, C)
    a64, b64 = as64(A), as64(B)
    if method == "svd":
        ta = O.truncate_rsvd(a64, k, S.sketch(n, k, 0, 0).astype(np.float32).astype(np.float64))
        tb = O.truncate_rsvd(b64, k, S.sketch(n, k, 0, 1).astype(np.float32).astype(np.float64))
    elif method == "fourier":
        ta = O.truncate_fourier_left(a64, k, forced=hA.selection())
        tb = O.truncate_fourier_right(b64, k, forced=hB.selection())
    else:
        ta = O.truncate(method, a64, k, selection=hA.selection())
        tb = O.truncate(method, b64, k, selection=hB.selection())
    ref = O.posterior_estimate(np.linalg.norm(ta.resid), np.linalg.norm(tb.resid),
                               np.linalg.norm(O.first_order(ta, tb).real), n)
    # the truncation errors come from FP32 keys / norms: a relative difference of ~1e-4 at most
    assert abs(est - ref) <= 1e-3 * ref, (est, ref)
    actual = np.linalg.norm(ta.resid @ tb.resid) / np.linalg.norm(a64 @ b64)
    assert 0.5 < est / actual < 2.0, (est, actual)


@pytest.mark.parametrize("method", ["circulant", "cycle"])
@pytest.mark.parametrize("tol", [0.3, 0.1, 0.03])
def test_choose_k_is_minimal(method, tol):
    """amm_choose_k returns the smallest k whose truncation error (from the oracle's keys) is within
    tol; near-ties of the error curve at the tolerance are allowed either way by 1e-4."""
    torch, amm = torch_cuda()
    n = 256
    g = S.rng(13, 0)
    a = S.toeplitz_uniform(n, g) + 0.05 * g.standard_normal((n, n))
    A = dev32(torch, a)
    k = amm.choose_k(A, method, tol)
    a64 = as64(A)
    if method == "circulant":
        keys2 = O.component_keys(O.circulant_spectrum(a64)) ** 2 * n
    else:
        keys2 = O.cycle_keys(a64) ** 2
    order = O.top_k(np.sqrt(keys2), n)
    total = np.sum(a64 ** 2)
    resid = lambda kk: (total - np.sum(keys2[order[:kk]])) / total
    assert resid(k) <= tol ** 2 * (1 + 1e-4)
    assert k == 1 or resid(k - 1) >= tol ** 2 * (1 - 1e-4)
    h = amm.decompose_to_tolerance(A, method, tol)
    assert h.k == k


@pytest.mark.parametrize("method,role", [("svd", "left"), ("svd", "right"), ("fourier", "left"), ("fourier", "right")])
@pytest.mark.parametrize("tol", [0.5, 0.2])
def test_decompose_to_tolerance_grows_k(method, role, tol):
    """rSVD / Fourier sparsifier: k grows (doubling, then bisection) until the handle's truncation
    error meets tol; the trial at k - 1 (same seed) does not, and the error the handle reports is
    the oracle's for that truncation."""
    torch, amm = torch_cuda()
    n = 256
    g = S.rng(14, 0)
    sigma = np.exp(-np.arange(n) / 24.0)
    a = S.spectrum_matrix(sigma, g) + 0.002 * g.standard_normal((n, n))
    if method == "fourier":
        a = a + S.toeplitz_uniform(n, g)
    A = dev32(torch, a)
    h = amm.decompose_to_tolerance(A, method, tol, role)
    info = h.info()
    assert info["resid_fro2"] <= tol ** 2 * info["fro2"] * (1 + 1e-5)
    if h.k > 1:
        h1 = amm.decompose(A, method, h.k - 1, role)
        i1 = h1.info()
        assert i1["resid_fro2"] > tol ** 2 * i1["fro2"]
    a64 = as64(A)
    if method == "svd":
        t = O.truncate_rsvd(a64, h.k, h.sketch().astype(np.float64))
    else:
        f = O.truncate_fourier_left if role == "left" else O.truncate_fourier_right
        t = f(a64, h.k, forced=h.selection())
    assert info["resid_fro2"] == pytest.approx(float(np.linalg.norm(t.resid) ** 2), rel=1e-3, abs=1e-6 * info["fro2"])


def test_apriori_estimate_matches_oracle():
    """a priori estimate from the handles' norms with the U(0,1) front constant 3/4 for the operands
    and 1/sqrt(n) for the zero-mean residues: equal to the oracle's, and close to the error the
    product then has (General x Toeplitz, circulant)."""
    torch, amm = torch_cuda()
    n, k = 512, 3
    a, b = S.general_times_toeplitz(n, seed=0)
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "circulant", k, "left")
    hB = amm.decompose(B, "circulant", k, "right")
    c_ab, c_resid = 0.75, 1 / math.sqrt(n)
    est = amm.apriori_estimate(hA, hB, c_ab, c_resid)
    a64, b64 = as64(A), as64(B)
    ta = O.truncate("circulant", a64, k, selection=hA.selection())
    tb = O.truncate("circulant", b64, k, selection=hB.selection())
    ref = O.apriori_estimate(np.linalg.norm(ta.resid), np.linalg.norm(tb.resid), np.linalg.norm(a64),
                             np.linalg.norm(b64), c_ab, c_resid)
    assert abs(est - ref) <= 1e-3 * ref, (est, ref)
    actual = np.linalg.norm(ta.resid @ tb.resid) / np.linalg.norm(a64 @ b64)
    assert 0.9 < est / actual < 1.1, (est, actual)
    with pytest.raises(RuntimeError, match="constants"):
        amm.apriori_estimate(hA, hB, 0.0, c_resid)


@pytest.mark.parametrize("want", ["circulant", "svd", "cycle", "fourier"])
def test_best_method_picks_the_exact_structure(want):
    """An input that one decomposition represents exactly with k = 2 components selects it, whatever
    the order of the candidates; the kept handle has (numerically) zero truncation error."""
    torch, amm = torch_cuda()
    n = 64
    A = dev32(torch, S.two_structure_cases(n, S.rng(42, 0))[want])
    order = ["circulant", "svd", "cycle", "fourier"]
    for methods in (order, order[::-1]):
        h, got = amm.decompose_best_method(A, methods, 2)
        assert got == want and h.method == want, (methods, got)
        info = h.info()
        # rSVD and Fourier errors are ||A||^2 - ||A~||^2 of FP32 sums (cancellation near 1e-7);
        # every other candidate leaves more than 0.7 ||A||^2 on these inputs
        assert info["resid_fro2"] <= 1e-5 * info["fro2"], (want, info)


def test_best_method_matches_oracle_choice():
    """General x Toeplitz, k = 5: the general U(0,1) operand keeps the Fourier sparsifier and the
    Toeplitz operand the circulant decomposition, as in the oracle (the candidates' relative errors
    differ by 3% or more), and the mixed product of the two kept handles matches the oracle's."""
    torch, amm = torch_cuda()
    n, k = 256, 5
    a, b = S.general_times_toeplitz(n, seed=0)
    A, B = dev32(torch, a), dev32(torch, b)
    methods = ["circulant", "svd", "cycle", "fourier"]
    hA, ma = amm.decompose_best_method(A, methods, k, "left")
    hB, mb = amm.decompose_best_method(B, methods, k, "right")
    a64, b64 = as64(A), as64(B)
    oa, _ = O.best_method(a64, k, methods, phi=S.sketch(n, k, 0, 0), side="left")
    ob, _ = O.best_method(b64, k, methods, phi=S.sketch(n, k, 0, 1), side="right")
    assert (ma, mb) == (oa, ob) == ("fourier", "circulant")
    C = amm.approx_matmul(hA, hB)
    ta = O.truncate_fourier_left(a64, k, forced=hA.selection())
    tb = O.truncate_circulant(b64, k, hB.selection())
    assert rel(C.double().cpu().numpy(), O.mixed_product(ta, tb)) <= TOL


def test_best_method_skips_candidates_that_do_not_take_the_shape():
    torch, amm = torch_cuda()
    g = S.rng(43, 0)
    # not square (no circulant without blocks) and an inner dimension of 100 (neither 2^a nor
    # 3 * 2^a: no Fourier sparsifier)
    A = dev32(torch, g.uniform(0.0, 1.0, (96, 100)))
    h, got = amm.decompose_best_method(A, ["circulant", "fourier", "svd"], 4)
    assert got == "svd"
    # a square 100 x 100 takes the circulant method (any n up to 4096), still not the sparsifier
    A2 = dev32(torch, g.uniform(0.0, 1.0, (100, 100)))
    h, got = amm.decompose_best_method(A2, ["fourier", "circulant"], 4)
    assert got == "circulant"
    R = dev32(torch, g.uniform(0.0, 1.0, (96, 200)))    # the cycle sparsifier needs a square
    h, got = amm.decompose_best_method(R, ["cycle", "svd"], 4)
    assert got == "svd"
    h, got = amm.decompose_best_method(R, ["cycle", "circulant"], 4, block=64)
    assert got == "circulant" and h.blocks == (2, 4)
    with pytest.raises(RuntimeError, match="inner dimension 100"):
        amm.decompose_best_method(A, ["circulant", "fourier"], 4)
