"""GPU parity of the circulant first-order product (Alg. 2, Alg. 3) against the FP64 oracle.

The oracle is evaluated on the FP32-rounded inputs the GPU sees.  Selections are compared
under the near-tie rule (gpu_util.check_selection); the product is compared with the oracle
re-run on the GPU's exported selection, element by element, at relative Frobenius <= 1e-5.
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, check_selection, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _run(torch, amm, a, b, k, kb=None, dtype=None):
    A, B = dev32(torch, a), dev32(torch, b)
    if dtype is not None:
        A, B = A.to(dtype), B.to(dtype)
    hA = amm.decompose(A, "circulant", k, "left")
    hB = amm.decompose(B, "circulant", kb or k, "right")
    C = amm.approx_matmul(hA, hB)
    torch.cuda.synchronize()
    return A, B, hA, hB, C


def _check(torch, amm, a, b, k, kb=None, tol=TOL):
    A, B, hA, hB, C = _run(torch, amm, a, b, k, kb)
    a64, b64 = as64(A), as64(B)
    ra, rb = O.circulant_spectrum(a64), O.circulant_spectrum(b64)
    check_selection(hA.selection(), O.component_keys(ra), k, "A")
    check_selection(hB.selection(), O.component_keys(rb), kb or k, "B")
    ref, mc, ta, tb = O.cd_matmul(a64, b64, k, kb, sel_a=hA.selection(), sel_b=hB.selection(), full=True)
    got = C.double().cpu().numpy()
    err = rel(got, ref)
    assert err <= tol, (a.shape, k, err)
    # norms reported by the handle (Parseval / orthogonality)
    ia = hA.info()
    assert ia["fro2"] == pytest.approx(float(np.sum(a64 * a64)), rel=1e-5)
    assert ia["resid_fro2"] == pytest.approx(float(np.linalg.norm(ta.resid) ** 2), rel=1e-4, abs=1e-6 * ia["fro2"])
    return err, ref, got


@pytest.mark.parametrize("n", [16, 32, 64, 128, 256, 512])
@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_circulant_small(n, k):
    torch, amm = torch_cuda()
    a, b = S.exp32_pair(n, seed=n + k)
    _check(torch, amm, a, b, k)


@pytest.mark.parametrize("pair,n,k", [(p, n, k) for p in ("general_toeplitz", "toeplitz_general", "gauss")
                                      for n, k in ((1024, 10), (1024, 33), (2048, 64))] + [("gauss", 8192, 13)])
def test_circulant_structured(pair, n, k):
    torch, amm = torch_cuda()
    if pair == "gauss":
        g = S.rng(5, 0)
        a, b = g.standard_normal((n, n)), g.standard_normal((n, n)) + 0.5
    elif pair == "general_toeplitz":
        a, b = S.general_times_toeplitz(n, seed=3)
    else:
        b, a = S.general_times_toeplitz(n, seed=4)
    _check(torch, amm, a, b, k)


@pytest.mark.parametrize("k", [16, 64, 256])
def test_circulant_powerlaw_n4096(k):
    """The n = 4096 power-law workload (sigma_i = i^-1.5 plus N(0, 1e-4) noise) at full size."""
    torch, amm = torch_cuda()
    a, b = S.powerlaw_pair(4096, seed=0)
    _check(torch, amm, a, b, k)


def test_circulant_untruncated_is_exact():
    """k = n keeps every component: the product equals A B (Thm 2.1)."""
    torch, amm = torch_cuda()
    n = 64
    a, b = S.exp32_pair(n, seed=1)
    A, B, hA, hB, C = _run(torch, amm, a, b, n)
    ex = as64(A) @ as64(B)
    assert rel(C.double().cpu().numpy(), ex) <= TOL


def test_circulant_mixed_k_and_unpaired_both_sides():
    """Unequal k on the two sides, and both selections with unpaired conjugates (Y V term)."""
    torch, amm = torch_cuda()
    n = 256
    g = S.rng(11, 0)
    a = g.standard_normal((n, n)) + 1.0   # component 0 dominates -> odd k leaves a pair split
    b = g.standard_normal((n, n)) + 1.0
    for ka, kb in [(2, 4), (4, 2), (2, 2), (7, 10)]:
        _, _, hA, hB, _ = _run(torch, amm, a, b, ka, kb)
        err, _, _ = _check(torch, amm, a, b, ka, kb)
        assert err <= TOL


def test_circulant_forced_selection_roundtrip():
    """A forced selection is applied verbatim (amm_opts.forced_selection)."""
    torch, amm = torch_cuda()
    n, k = 128, 5
    a, b = S.exp32_pair(n, seed=2)
    A, B = dev32(torch, a), dev32(torch, b)
    sel = [3, 0, 125, 64, 17]
    hA = amm.decompose(A, "circulant", k, "left", forced_selection=sel)
    hB = amm.decompose(B, "circulant", k, "right", forced_selection=sel[::-1])
    assert hA.selection().tolist() == sel
    C = amm.approx_matmul(hA, hB)
    ref = O.cd_matmul(as64(A), as64(B), k, sel_a=sel, sel_b=sel[::-1])
    assert rel(C.double().cpu().numpy(), ref) <= TOL


def test_circulant_strided_and_bf16_inputs():
    """A with a leading dimension larger than n, and BF16 operands (widened to FP32 in the FFT load)."""
    torch, amm = torch_cuda()
    n, k = 256, 9
    a, b = S.exp32_pair(n, seed=6)
    wide = torch.zeros((n, n + 40), dtype=torch.float32, device="cuda")
    wide[:, 8:8 + n] = dev32(torch, a)
    A = wide[:, 8:8 + n]
    B = dev32(torch, b)
    hA = amm.decompose(A, "circulant", k, "left")
    hB = amm.decompose(B, "circulant", k, "right")
    C = amm.approx_matmul(hA, hB)
    ref = O.cd_matmul(as64(A), as64(B), k, sel_a=hA.selection(), sel_b=hB.selection())
    assert rel(C.double().cpu().numpy(), ref) <= TOL
    # BF16
    Ab, Bb = dev32(torch, a).bfloat16(), dev32(torch, b).bfloat16()
    hA = amm.decompose(Ab, "circulant", k, "left")
    hB = amm.decompose(Bb, "circulant", k, "right")
    Cb = amm.approx_matmul(hA, hB)
    ref = O.cd_matmul(as64(Ab), as64(Bb), k, sel_a=hA.selection(), sel_b=hB.selection())
    assert rel(Cb.double().cpu().numpy(), ref) <= TOL


def test_circulant_deterministic():
    torch, amm = torch_cuda()
    n, k = 512, 17
    a, b = S.exp32_pair(n, seed=7)
    C1 = _run(torch, amm, a, b, k)[4].clone()
    C2 = _run(torch, amm, a, b, k)[4]
    assert torch.equal(C1, C2)


def test_circulant_flat_spectrum_ties():
    """A single nonzero entry has a flat spectrum (all keys tied): lowest indices are selected."""
    torch, amm = torch_cuda()
    n, k = 64, 5
    a = np.zeros((n, n))
    a[0, 0] = 1.0
    b = S.exp32_pair(n, seed=8)[1]
    A, B, hA, hB, C = _run(torch, amm, a, b, k)
    assert hA.selection().tolist() == [0, 1, 2, 3, 4]
    ref = O.cd_matmul(as64(A), as64(B), k, sel_a=hA.selection(), sel_b=hB.selection())
    assert rel(C.double().cpu().numpy(), ref) <= TOL


def test_circulant_errors_do_not_launch():
    torch, amm = torch_cuda()
    A = torch.zeros((4100, 4100), device="cuda")  # above 4096 and neither 2^a nor 3 * 2^a
    with pytest.raises(amm.AmmError) as e:
        amm.decompose(A, "circulant", 4)
    assert e.value.status == 2  # AMM_ERR_UNSUPPORTED_SIZE
    with pytest.raises(amm.AmmError) as e:
        amm.decompose(torch.zeros((12, 12), device="cuda"), "circulant", 4)
    assert e.value.status == 2
    A = torch.zeros((64, 64), device="cuda")
    with pytest.raises(amm.AmmError):
        amm.decompose(A, "circulant", 0)
    hA = amm.decompose(A, "circulant", 4, "left")
    hB = amm.decompose(A, "circulant", 4, "left")
    with pytest.raises(amm.AmmError) as e:
        amm.approx_matmul(hA, hB)
    assert e.value.status == 6  # AMM_ERR_STATE: hB is not a right operand


def test_injected_allocation_failure():
    torch, amm = torch_cuda()
    from paper_2504_19308_gb300.amm import debug_fail_alloc_after
    A = torch.randn((64, 64), device="cuda")
    for nth in (1, 3, 7):
        debug_fail_alloc_after(nth)
        with pytest.raises(amm.AmmError) as e:
            amm.decompose(A, "circulant", 4, "right")
        assert e.value.status == 3  # AMM_ERR_OOM
    debug_fail_alloc_after(0)
    h = amm.decompose(A, "circulant", 4, "right")
    assert h.selection().size == 4


@pytest.mark.parametrize("n,k", [(64, 5), (256, 9), (1024, 33)])
def test_circulant_pair_closed_selection(n, k):
    """pair_closed: the selection is closed under t -> n - t, A~ is real, no unpaired terms, and the
    product equals the oracle's with the closed set S u S-bar."""
    torch, amm = torch_cuda()
    g = S.rng(n + k, 5)
    a = g.standard_normal((n, n)) + 1.0   # odd k splits a pair without closure
    b = S.toeplitz_uniform(n, g)
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "circulant", k, "left", pair_closed=True)
    hB = amm.decompose(B, "circulant", k, "right", pair_closed=True)
    C = amm.approx_matmul(hA, hB)
    ia = hA.info()
    assert ia["n_unpaired"] == 0
    sa, sb = hA.selection(), hB.selection()
    closed = lambda sel: np.unique(np.concatenate([sel, (-np.asarray(sel)) % n]))
    ca, cb = closed(sa), closed(sb)
    assert ia["n_union"] == len(ca)
    a64, b64 = as64(A), as64(B)
    ta = O.truncate_circulant(a64, len(ca), ca)
    tb = O.truncate_circulant(b64, len(cb), cb)
    m = O.first_order(ta, tb)
    assert np.abs(m.imag).max() <= 1e-9 * np.abs(m.real).max()
    assert rel(C.double().cpu().numpy(), m.real) <= TOL
    # the truncation error reported is that of the closed set
    assert abs(ia["resid_fro2"] - np.linalg.norm(ta.resid) ** 2) <= 1e-4 * np.linalg.norm(a64) ** 2


@pytest.mark.parametrize("n", [1024, 4096])
def test_autotuned_apply_is_bit_identical(n):
    """The autotuner picks between spectral-apply variants that compute every output with the same
    operations: products with tuning off, during the timing call and after it are bit-identical."""
    torch, amm = torch_cuda()
    g = S.rng(n, 11)
    A, B = dev32(torch, g.standard_normal((n, n))), dev32(torch, g.standard_normal((n, n)) + 0.5)
    hA = amm.decompose(A, "circulant", 9, "left")
    hB = amm.decompose(B, "circulant", 9, "right")
    amm.set_autotune(False)
    C0 = amm.approx_matmul(hA, hB).clone()
    G = dev32(torch, g.standard_normal((n, n)))
    dA0, dB0 = [t.clone() for t in amm.approx_matmul_backward(hA, hB, G)]
    try:
        amm.set_autotune(True)
        C1 = amm.approx_matmul(hA, hB).clone()   # times the variants of these keys
        C2 = amm.approx_matmul(hA, hB).clone()   # uses the kept choice
        dA1, dB1 = amm.approx_matmul_backward(hA, hB, G)
    finally:
        amm.set_autotune(False)
    assert torch.equal(C0, C1) and torch.equal(C0, C2)
    assert torch.equal(dA0, dA1) and torch.equal(dB0, dB1)


def test_store_spectra_off_gives_identical_results_with_less_memory():
    """opts.store_spectra = 0 releases the half spectrum R after the decomposition: the product and
    the backward (which never read R) are bit-identical, the dense residual of a mixed product and
    the residual export recompute R from A and match too, and the handle holds at least R's
    (n/2+1) n complex values less device memory."""
    torch, amm = torch_cuda()
    n, k = 1024, 9
    a, b = S.general_times_toeplitz(n, seed=11)
    A, B = dev32(torch, a), dev32(torch, b)
    G = dev32(torch, S.upstream_grad(n, n, 11))
    keep = [amm.decompose(A, "circulant", k, "left"), amm.decompose(B, "circulant", k, "right")]
    drop = [amm.decompose(A, "circulant", k, "left", store_spectra=False),
            amm.decompose(B, "circulant", k, "right", store_spectra=False)]
    for hk, hd in zip(keep, drop):
        assert hd.device_bytes() <= hk.device_bytes() - (n // 2 + 1) * n * 8
        assert np.array_equal(hk.selection(), hd.selection())
    assert torch.equal(amm.approx_matmul(*keep), amm.approx_matmul(*drop))
    for gk, gd in zip(amm.approx_matmul_backward(*keep, G), amm.approx_matmul_backward(*drop, G)):
        assert torch.equal(gk, gd)
    sk = dev32(torch, S.sketch(n, 16, 11, 1))
    hs = amm.decompose(B, "svd", 16, "right", sketch=sk)
    assert torch.equal(amm.approx_matmul(keep[0], hs), amm.approx_matmul(drop[0], hs))
    assert torch.equal(amm.residual(keep[0]), amm.residual(drop[0]))
    ref = O.truncate_circulant(as64(A), k, keep[0].selection())
    assert rel(amm.residual(drop[0]).double().cpu().numpy(), ref.resid.real) <= TOL
    # blocked circulant LEFT operand of a mixed product: its dense residual needs every block's
    # spectrum, recomputed per block
    W = dev32(torch, S.rng(12, 1).standard_normal((384, 512)) + 0.5)
    hy = amm.decompose(dev32(torch, S.rng(12, 0).standard_normal((512, 256))), "svd", 16, "right",
                       sketch=dev32(torch, S.sketch(256, 16, 12, 1)))
    wk = amm.decompose(W, "circulant", 5, "left", block=128)
    wd = amm.decompose(W, "circulant", 5, "left", block=128, store_spectra=False)
    assert wd.device_bytes() < wk.device_bytes()
    assert torch.equal(amm.approx_matmul(wk, hy), amm.approx_matmul(wd, hy))
