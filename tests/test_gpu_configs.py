"""Full-size parity of the two workloads beyond the n = 4096 pair: the autograd layer
(A 8192 x 8192 with sigma_i = e^{-i/256}, B 8192 x 4096, k = 128, forward and backward) and the
LLM-shaped product (activations 2048 x 4096, weight 4096 x 11008, rSVD k = 256) in the FP32 mode
and in the BF16 tensor-core mode."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, check_selection, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu


def test_autograd_layer_n8192_k128():
    torch, amm = torch_cuda()
    a, b, g = S.differentiation_case(seed=0)
    k = 128
    A = dev32(torch, a).requires_grad_(True)
    B = dev32(torch, b).requires_grad_(True)
    G = dev32(torch, g)
    pa, pb = S.sketch(8192, k, 0, 0).astype(np.float32), S.sketch(4096, k, 0, 1).astype(np.float32)
    C = amm.approx_matmul_autograd(A, B, "svd", k, sketch_a=dev32(torch, pa), sketch_b=dev32(torch, pb))
    C.backward(G)
    ref, _, ta, tb = O.svd_matmul(as64(A.detach()), as64(B.detach()), k, pa.astype(np.float64),
                                  pb.astype(np.float64), full=True)
    rda, rdb = O.svd_backward(ta, tb, as64(G))
    assert rel(C.detach().double().cpu().numpy(), ref) <= TOL
    assert rel(A.grad.double().cpu().numpy(), rda) <= TOL
    assert rel(B.grad.double().cpu().numpy(), rdb) <= TOL


@pytest.mark.parametrize("compute,tol", [("f32", TOL), ("bf16", 3e-2)])
def test_llm_shaped_rsvd_k256(compute, tol):
    """X W with X 2048 x 4096 N(0,1) and W 4096 x 11008 (N(0, 0.02^2), 0.1% heavy-tailed entries),
    BF16 inputs; both operands by rSVD k = 256.  FP32 mode: parity at 1e-5 on the BF16-rounded
    inputs; BF16 mode: the BF16 GEMM rounding bound."""
    torch, amm = torch_cuda()
    x, w = S.llm_shaped(seed=0)
    k = 256
    X = torch.from_numpy(x.astype(np.float32)).cuda().bfloat16()
    W = torch.from_numpy(w.astype(np.float32)).cuda().bfloat16()
    pa, pb = S.sketch(4096, k, 0, 0).astype(np.float32), S.sketch(11008, k, 0, 1).astype(np.float32)
    hX = amm.decompose(X, "svd", k, "left", sketch=dev32(torch, pa), compute=compute)
    hW = amm.decompose(W, "svd", k, "right", sketch=dev32(torch, pb), compute=compute)
    C = amm.approx_matmul(hX, hW)
    ref = O.svd_matmul(as64(X), as64(W), k, pa.astype(np.float64), pb.astype(np.float64))
    err = rel(C.double().cpu().numpy(), ref)
    assert err <= tol, err


def test_llm_shaped_mixed_rsvd_times_circulant_blocks():
    """X W with the activations X (2048 x 4096) by rSVD k = 256 and the weight W (4096 x 11008) in
    4096 x 4096 circulant blocks (zero-padded to 4096 x 12288), k = 128 per block.  Parity on
    sampled output rows (the oracle evaluates only those rows of Eq. (2.3)); the selection of
    every weight block is the oracle's top-k outside near-ties."""
    torch, amm = torch_cuda()
    x, w = S.llm_shaped(seed=0)
    X = torch.from_numpy(x.astype(np.float32)).cuda().bfloat16().float()
    W = torch.from_numpy(w.astype(np.float32)).cuda().bfloat16().float()
    k, kc, bs = 256, 128, 4096
    pa = S.sketch(4096, k, 0, 0).astype(np.float32)
    hX = amm.decompose(X, "svd", k, "left", sketch=dev32(torch, pa))
    hW = amm.decompose(W, "circulant", kc, "right", block=bs)
    C = amm.approx_matmul(hX, hW)
    x64, w64 = as64(X), as64(W)
    tw = O.truncate_circulant_blocked(w64, bs, kc, selections=hW.selection())
    top = O.truncate_circulant_blocked(w64, bs, kc)
    for j, t in enumerate(top.blocks[0]):
        check_selection(hW.selection()[j], t.keys, kc, ("W block", j))
    tx = O.truncate_rsvd(x64, k, pa.astype(np.float64))
    rows = np.sort(S.rng(1, 70).choice(2048, 48, replace=False))
    tx_rows = O.Truncation("svd", tx.a[rows], tx.approx[rows])
    ref = O.blocked_first_order(tx_rows, tw)
    got = C.double().cpu().numpy()[rows]
    assert rel(got, ref) <= TOL


def test_circulant_n16384_k512():
    """The largest circulant length (one packed signal per CTA).  (1) k = 512 selection of an
    N(0,1) + 0.5 matrix against the oracle's FP64 keys (near-tie rule).  (2) Operands that are one
    real component each (circulant(c) D^(n/2), Thm 2.1): the truncation at k = 1 is exact, so the
    product and both gradients equal AB, G B^T and A^T G, checked on sampled rows / columns."""
    torch, amm = torch_cuda()
    n = 16384
    g = S.rng(90, 0)
    a = g.standard_normal((n, n)).astype(np.float32) + np.float32(0.5)
    A = torch.from_numpy(a).cuda()
    h = amm.decompose(A, "circulant", 512, "left")
    keys = O.component_keys(O.circulant_spectrum(a.astype(np.float64)))
    check_selection(h.selection(), keys, 512, "A")
    h.close()
    del A, a, keys
    sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)            # D^(n/2) = diag((-1)^q)
    a = O.circulant(g.standard_normal(n)) * sign[None, :]
    b = O.circulant(g.uniform(0, 1, n)) * sign[None, :]
    A, B = dev32(torch, a), dev32(torch, b)
    a64, b64 = as64(A), as64(B)
    del a, b
    hA = amm.decompose(A, "circulant", 1, "left")
    hB = amm.decompose(B, "circulant", 1, "right")
    assert hA.selection().tolist() == [n // 2] and hB.selection().tolist() == [n // 2]
    C = amm.approx_matmul(hA, hB)
    G = dev32(torch, g.standard_normal((n, n)))
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    rows = np.sort(S.rng(91, 0).choice(n, 16, replace=False))
    g64 = as64(G)
    assert rel(C.double().cpu().numpy()[rows], a64[rows] @ b64) <= TOL
    assert rel(dA.double().cpu().numpy()[rows], g64[rows] @ b64.T) <= TOL
    assert rel(dB.double().cpu().numpy()[:, rows], a64.T @ g64[:, rows]) <= TOL



@pytest.mark.parametrize("method", ["circulant", "svd", "fourier", "cycle"])
def test_zero_operand_gives_zero_product_and_gradient(method):
    """The degenerate operand A = 0 (every key of A ties at zero; the rSVD sketch Y = A phi is zero):
    the product and dB are exactly zero and nothing is NaN.  For the selection methods the tied
    selection of A follows the key order (index ascending) and dA matches the oracle's frozen
    gradient; for the rSVD, orth(0) spans nothing, so A~ = 0 and dA = G B~^T."""
    torch, amm = torch_cuda()
    n, k = 64, 4
    g = S.rng(44, 0)
    b, gr = g.standard_normal((n, n)), g.standard_normal((n, n))
    A = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    B, G = dev32(torch, b), dev32(torch, gr)
    svd = method == "svd"
    phi = dev32(torch, S.sketch(n, k, 44, 0).astype(np.float32)) if svd else None
    psi = S.sketch(n, k, 44, 1).astype(np.float32) if svd else None
    hA = amm.decompose(A, method, k, "left", sketch=phi)
    hB = amm.decompose(B, method, k, "right", sketch=None if psi is None else dev32(torch, psi))
    C = amm.approx_matmul(hA, hB)
    dA, dB = amm.approx_matmul_backward(hA, hB, G)
    for t in (C, dA, dB):
        assert bool(torch.isfinite(t).all())
    assert float(C.abs().max()) == 0.0 and float(dB.abs().max()) == 0.0
    a64, b64, g64 = np.zeros((n, n)), as64(B), as64(G)
    if svd:
        tb = O.truncate_rsvd(b64, k, psi.astype(np.float64))
        assert rel(dA.double().cpu().numpy(), g64 @ tb.approx.T) <= TOL
        return
    if method != "fourier":
        assert sorted(hA.selection().tolist()) == list(range(k))
    ta = O.truncate(method, a64, k, selection=hA.selection(), side="left")
    tb = O.truncate(method, b64, k, selection=hB.selection(), side="right")
    rda, _ = O.backward(method, ta, tb, g64)
    assert rel(dA.double().cpu().numpy(), rda) <= TOL
