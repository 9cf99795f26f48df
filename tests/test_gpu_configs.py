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
