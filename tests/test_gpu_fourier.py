"""GPU parity of the Fourier-sparsified first-order product (Alg. 4, Alg. 5)."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, check_selection, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu


def _check(torch, amm, a, b, k, check_rows=64):
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "fourier", k, "left")
    hB = amm.decompose(B, "fourier", k, "right")
    C = amm.approx_matmul(hA, hB)
    a64, b64 = as64(A), as64(B)
    sa, sb = hA.selection(), hB.selection()
    n = a.shape[1]
    # per-row / per-column selection against the oracle's magnitudes (near-tie rule per row)
    magA = O.magnitudes_mirrored_rows(a64 @ np.conj(O.unitary_W(n)).T)
    magB = O.magnitudes_mirrored_rows((O.unitary_W(n) @ b64).T)
    for i in np.linspace(0, a.shape[0] - 1, min(check_rows, a.shape[0])).astype(int):
        check_selection(sa[i], magA[i], k, "A row %d" % i)
    for c in np.linspace(0, b.shape[1] - 1, min(check_rows, b.shape[1])).astype(int):
        check_selection(sb[c], magB[c], k, "B col %d" % c)
    ref = O.fourier_matmul(a64, b64, k, forced_a=sa, forced_b=sb)
    err = rel(C.double().cpu().numpy(), ref)
    assert err <= TOL, (a.shape, b.shape, k, err)
    return err


@pytest.mark.parametrize("n", [16, 64, 256, 1024])
@pytest.mark.parametrize("k", [1, 2, 5, 16])
def test_fourier_small(n, k):
    torch, amm = torch_cuda()
    a, b = S.general_times_toeplitz(n, seed=n + k)
    _check(torch, amm, a, b, min(k, n))


@pytest.mark.parametrize("m,n,p,k", [(100, 64, 37, 3), (257, 128, 300, 7), (33, 512, 65, 6)])
def test_fourier_rectangular_ragged(m, n, p, k):
    torch, amm = torch_cuda()
    g = S.rng(m + p, 0)
    _check(torch, amm, g.standard_normal((m, n)), g.uniform(0, 1, (n, p)), k)


def test_fourier_powerlaw_n4096_top1pct():
    """Top 1% of the entries (k = ceil(0.01 n) = 41 per row / column) on the n = 4096 pair."""
    torch, amm = torch_cuda()
    a, b = S.powerlaw_pair(4096, seed=0)
    _check(torch, amm, a, b, 41, check_rows=128)


def test_fourier_untruncated_exact():
    torch, amm = torch_cuda()
    n = 32
    a, b = S.exp32_pair(n, seed=5)
    A, B = dev32(torch, a), dev32(torch, b)
    C = amm.approx_matmul(amm.decompose(A, "fourier", n, "left"), amm.decompose(B, "fourier", n, "right"))
    assert rel(C.double().cpu().numpy(), as64(A) @ as64(B)) <= TOL


def test_fourier_single_tone_rows_exact():
    """Rows that are single real tones cos(2 pi f l / n) have two nonzero frequencies: k = 2 keeps them."""
    torch, amm = torch_cuda()
    n, m = 128, 64
    l = np.arange(n)
    g = S.rng(6, 0)
    a = np.stack([np.cos(2 * np.pi * (i % 17 + 1) * l / n) * (1 + i) for i in range(m)])
    b = g.standard_normal((n, 40))
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "fourier", 2, "left")
    sel = hA.selection()
    assert all(sorted(sel[i].tolist()) == [i % 17 + 1, n - (i % 17 + 1)] for i in range(m))
    C = amm.approx_matmul(hA, amm.decompose(B, "fourier", 3, "right"))
    assert rel(C.double().cpu().numpy(), as64(A) @ as64(B)) <= 1e-5


def _backward_case(torch, amm, a, b, ka, kb, seed):
    A, B = dev32(torch, a), dev32(torch, b)
    hA = amm.decompose(A, "fourier", ka, "left")
    hB = amm.decompose(B, "fourier", kb, "right")
    g = S.upstream_grad(a.shape[0], b.shape[1], seed)
    G = dev32(torch, g)
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    ta = O.truncate_fourier_left(as64(A), ka, forced=hA.selection())
    tb = O.truncate_fourier_right(as64(B), kb, forced=hB.selection())
    rda, rdb = O.fourier_backward(ta, tb, as64(G))
    return rel(dA.double().cpu().numpy(), rda), rel(dB.double().cpu().numpy(), rdb)


@pytest.mark.parametrize("m,n,p,ka,kb", [(16, 16, 16, 3, 2), (64, 64, 64, 5, 5), (256, 256, 256, 16, 9),
                                         (1024, 1024, 1024, 11, 11), (100, 64, 37, 3, 4), (257, 128, 300, 7, 2),
                                         (33, 512, 65, 6, 6)])
def test_fourier_backward(m, n, p, ka, kb):
    """dA = Re[(P_A(G dB~^T) + G B~_a^T) conj W], dB = Re[W (A~_a^T G + P_B(dA~^T G))] (masks frozen)."""
    torch, amm = torch_cuda()
    g = S.rng(m + n + p, 1)
    a = g.standard_normal((m, n)) @ S.toeplitz_uniform(n, g) if m == n else g.standard_normal((m, n))
    b = g.uniform(0, 1, (n, p))
    ea, eb = _backward_case(torch, amm, a, b, ka, kb, m + p)
    assert ea <= TOL and eb <= TOL, (ea, eb)


def test_fourier_backward_asymmetric_masks():
    """Single-tone rows with k = 1 keep frequency f but not n - f (equal magnitudes, lower index
    first), so the kept sets are not mirror-symmetric and the gradient needs the Hermitian part."""
    torch, amm = torch_cuda()
    n, m, p = 128, 64, 48
    l = np.arange(n)
    a = np.stack([np.cos(2 * np.pi * (i % 17 + 1) * l / n) * (1 + i) for i in range(m)])
    b = np.stack([np.sin(2 * np.pi * (c % 13 + 2) * l / n) for c in range(p)], axis=1) + 0.01 * S.rng(7, 0).standard_normal((n, p))
    ea, eb = _backward_case(torch, amm, a, b, 1, 1, 9)
    assert ea <= TOL and eb <= TOL, (ea, eb)


def test_fourier_backward_powerlaw_n4096_top1pct():
    torch, amm = torch_cuda()
    a, b = S.powerlaw_pair(4096, seed=0)
    ea, eb = _backward_case(torch, amm, a, b, 41, 41, 0)
    assert ea <= TOL and eb <= TOL, (ea, eb)


def test_fourier_bf16_operands():
    """BF16 operands: the handle widens them to FP32 once; the product matches the oracle on the
    BF16-rounded inputs at the FP32 tolerance."""
    torch, amm = torch_cuda()
    n, k = 256, 9
    a, b = S.general_times_toeplitz(n, seed=11)
    A = torch.from_numpy(a.astype(np.float32)).cuda().bfloat16()
    B = torch.from_numpy(b.astype(np.float32)).cuda().bfloat16()
    hA = amm.decompose(A, "fourier", k, "left")
    hB = amm.decompose(B, "fourier", k, "right")
    C = amm.approx_matmul(hA, hB)
    ref = O.fourier_matmul(as64(A), as64(B), k, forced_a=hA.selection(), forced_b=hB.selection())
    assert rel(C.double().cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("m,n,p,k", [(40, 48, 30, 3), (100, 96, 77, 5), (200, 384, 150, 9), (64, 1536, 96, 16),
                                     (48, 3072, 40, 31)])
def test_fourier_radix3_lengths(m, n, p, k):
    """Inner dimensions n = 3 * 2^a (a radix-3 pass in the row / column transforms)."""
    torch, amm = torch_cuda()
    g = S.rng(m + n + p, 1)
    _check(torch, amm, g.standard_normal((m, n)) + 0.3, g.uniform(0, 1, (n, p)), k)


@pytest.mark.parametrize("m,n,p,ka,kb", [(50, 192, 60, 4, 6), (96, 768, 80, 8, 8)])
def test_fourier_backward_radix3(m, n, p, ka, kb):
    torch, amm = torch_cuda()
    g = S.rng(m + n + p, 2)
    a, b, gr = g.standard_normal((m, n)), g.uniform(0, 1, (n, p)), g.standard_normal((m, p))
    A, B, G = dev32(torch, a), dev32(torch, b), dev32(torch, gr)
    hA = amm.decompose(A, "fourier", ka, "left")
    hB = amm.decompose(B, "fourier", kb, "right")
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    ta = O.truncate_fourier_left(as64(A), ka, forced=hA.selection())
    tb = O.truncate_fourier_right(as64(B), kb, forced=hB.selection())
    rda, rdb = O.fourier_backward(ta, tb, as64(G))
    assert rel(dA.double().cpu().numpy(), rda) <= TOL
    assert rel(dB.double().cpu().numpy(), rdb) <= TOL
