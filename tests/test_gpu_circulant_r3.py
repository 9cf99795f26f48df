"""GPU parity of the circulant path at lengths n = 3 * 2^a (one radix-3 FFT pass before the
power-of-two passes): decomposition, product, backward, pair-closed and BF16 variants, blocks,
k from a tolerance.  The oracle is the same definition as for powers of two (it holds for any n)."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, check_selection, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu

R3 = [48, 96, 192, 384, 768, 1536, 3072]


def _pair(n, seed):
    g = S.rng(n, seed)
    a = g.standard_normal((n, n)) + 0.5                   # a dominant zero component
    b = S.toeplitz_uniform(n, g) + 0.1 * g.standard_normal((n, n))
    return a, b


@pytest.mark.parametrize("n", R3)
@pytest.mark.parametrize("k", [1, 4, 9])
def test_r3_product(n, k):
    torch, amm = torch_cuda()
    a, b = _pair(n, 80 + k)
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "circulant", k, "left")
    hB = amm.decompose(B, "circulant", k + 2, "right")
    C = amm.approx_matmul(hA, hB)
    a64, b64 = as64(A), as64(B)
    check_selection(hA.selection(), O.component_keys(O.circulant_spectrum(a64)), k, "A")
    check_selection(hB.selection(), O.component_keys(O.circulant_spectrum(b64)), k + 2, "B")
    ref, _, ta, _ = O.cd_matmul(a64, b64, k, k + 2, sel_a=hA.selection(), sel_b=hB.selection(), full=True)
    err = rel(C.double().cpu().numpy(), ref)
    assert err <= TOL, (n, k, err)
    info = hA.info()
    assert info["fro2"] == pytest.approx(float(np.sum(a64 * a64)), rel=1e-5)
    assert info["resid_fro2"] == pytest.approx(float(np.linalg.norm(ta.resid) ** 2), rel=1e-4,
                                               abs=1e-6 * info["fro2"])


@pytest.mark.parametrize("n", [48, 96])
def test_r3_untruncated_is_exact(n):
    torch, amm = torch_cuda()
    a, b = _pair(n, 81)
    A, B = dev32(torch, a), dev32(torch, b)
    C = amm.approx_matmul(amm.decompose(A, "circulant", n, "left"), amm.decompose(B, "circulant", n, "right"))
    assert rel(C.double().cpu().numpy(), as64(A) @ as64(B)) <= 1e-5


def test_r3_single_component_input():
    """A = circulant(c) D^t at n = 96 is the single component t (Thm 2.1): k = 1 finds it."""
    torch, amm = torch_cuda()
    n, t = 96, 48                                          # D^(n/2) is real: a real single component
    g = S.rng(82, 0)
    a = (O.circulant(g.standard_normal(n)) @ O.diag_D(n, t)).real
    hA = amm.decompose(dev32(torch, a), "circulant", 1, "left")
    assert hA.selection().tolist() == [t]
    assert hA.info()["resid_fro2"] <= 1e-9 * np.sum(a * a)


@pytest.mark.parametrize("n,ka,kb", [(48, 3, 2), (192, 7, 5), (768, 48, 40), (1536, 9, 100)])
def test_r3_backward(n, ka, kb):
    torch, amm = torch_cuda()
    a, b = _pair(n, 83)
    gr = S.rng(n, 84).standard_normal((n, n))
    A, B, G = dev32(torch, a), dev32(torch, b), dev32(torch, gr)
    hA = amm.decompose(A, "circulant", ka, "left")
    hB = amm.decompose(B, "circulant", kb, "right")
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    ta = O.truncate_circulant(as64(A), ka, hA.selection())
    tb = O.truncate_circulant(as64(B), kb, hB.selection())
    rda, rdb = O.cd_backward(ta, tb, as64(G))
    assert rel(dA.double().cpu().numpy(), rda) <= TOL
    assert rel(dB.double().cpu().numpy(), rdb) <= TOL


def test_r3_pair_closed_and_bf16():
    torch, amm = torch_cuda()
    n, k = 384, 7
    a, b = _pair(n, 85)
    A = torch.from_numpy(a.astype(np.float32)).cuda().bfloat16()
    B = torch.from_numpy(b.astype(np.float32)).cuda().bfloat16()
    hA = amm.decompose(A, "circulant", k, "left", pair_closed=True)
    hB = amm.decompose(B, "circulant", k, "right", pair_closed=True)
    C = amm.approx_matmul(hA, hB)
    closed = lambda sel: np.unique(np.concatenate([sel, (-np.asarray(sel)) % n]))
    ca, cb = closed(hA.selection()), closed(hB.selection())
    ta = O.truncate_circulant(as64(A), len(ca), ca)
    tb = O.truncate_circulant(as64(B), len(cb), cb)
    m = O.first_order(ta, tb)
    assert np.abs(m.imag).max() <= 1e-9 * np.abs(m.real).max()
    assert rel(C.double().cpu().numpy(), m.real) <= TOL


def test_r3_blocks():
    torch, amm = torch_cuda()
    g = S.rng(86, 0)
    a, b = g.standard_normal((150, 200)) + 0.5, g.uniform(0, 1, (200, 70))
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "circulant", 5, "left", block=96)
    hB = amm.decompose(B, "circulant", 5, "right", block=96)
    C = amm.approx_matmul(hA, hB)
    ta = O.truncate_circulant_blocked(as64(A), 96, 5, selections=hA.selection())
    tb = O.truncate_circulant_blocked(as64(B), 96, 5, selections=hB.selection())
    assert rel(C.double().cpu().numpy(), O.blocked_first_order(ta, tb)) <= TOL


def test_r3_choose_k():
    torch, amm = torch_cuda()
    n, tol = 192, 0.5
    a, _ = _pair(n, 87)
    A = dev32(torch, a)
    k = amm.choose_k(A, "circulant", tol)
    keys = O.component_keys(O.circulant_spectrum(as64(A)))
    order = O.top_k(keys, n)
    tot = np.sum(as64(A) ** 2)
    kept = n * np.cumsum(keys[order] ** 2)
    k_ref = int(np.argmax(tot - kept <= tol * tol * tot)) + 1
    assert k == k_ref


def test_r3_n6144_sampled_rows():
    """n = 6144 (largest radix-3 length), k = 64: rows of the product sampled against the oracle."""
    torch, amm = torch_cuda()
    n, k = 6144, 64
    g = S.rng(88, 0)
    a = g.standard_normal((n, n)) + 0.5
    b = g.standard_normal((n, n)) * 0.1 + 1.0
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "circulant", k, "left")
    hB = amm.decompose(B, "circulant", k, "right")
    C = amm.approx_matmul(hA, hB)
    a64, b64 = as64(A), as64(B)
    ta = O.truncate_circulant(a64, k, hA.selection())
    tb = O.truncate_circulant(b64, k, hB.selection())
    rows = np.sort(S.rng(89, 0).choice(n, 24, replace=False))
    ref = (ta.approx[rows] @ b64 + ta.resid[rows] @ tb.approx).real
    assert rel(C.double().cpu().numpy()[rows], ref) <= TOL
