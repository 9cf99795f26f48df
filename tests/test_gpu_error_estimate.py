"""amm_error_estimate (Corollary 3.7) against the oracle's estimate on the same truncations."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import as64, dev32, torch_cuda

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
