"""Batched products of uneven sizes: eager run, graph capture and graph replay all reproduce the
individually computed products bit for bit."""
import pytest

import synth as S
from gpu_util import dev32, torch_cuda

pytestmark = pytest.mark.gpu


def test_batch_uneven_sizes_graph_replay():
    torch, amm = torch_cuda()
    sizes = [64, 128, 1024, 256, 512, 128, 2048, 64, 256, 512, 1024, 128]
    methods = ["circulant", "svd", "cycle", "fourier"]
    items = []
    for i, n in enumerate(sizes):
        method = methods[i % 4]
        k = max(2, n // 32)
        a, b = S.exp32_pair(n, seed=100 + i)
        A, B = dev32(torch, a), dev32(torch, b)
        C = torch.full((n, n), float("nan"), device="cuda")
        sa = dev32(torch, S.sketch(n, k, i, 0)) if method == "svd" else None
        sb = dev32(torch, S.sketch(n, k, i, 1)) if method == "svd" else None
        items.append((A, B, C, method, k, sa, sb))
    refs = []
    for A, B, C, method, k, sa, sb in items:
        hA = amm.decompose(A, method, k, "left", sketch=sa)
        hB = amm.decompose(B, method, k, "right", sketch=sb)
        refs.append(amm.approx_matmul(hA, hB).clone())
    batch = amm.Batch()
    for it in items:
        batch.add(*it[:3], it[3], it[4], sketch_a=it[5], sketch_b=it[6])
    batch.run(use_graph=False)
    torch.cuda.synchronize()
    for (A, B, C, *_), ref in zip(items, refs):
        assert torch.equal(C, ref)
    for _ in range(2):  # capture + launch, then replay
        for it in items:
            it[2].fill_(float("nan"))
        batch.run(use_graph=True)
        torch.cuda.synchronize()
        for (A, B, C, *_), ref in zip(items, refs):
            assert torch.equal(C, ref)
    # new input values flow through the same graph
    A0, B0, C0, method0, k0 = items[0][:5]
    A0.mul_(2.0)
    batch.run(use_graph=True)
    torch.cuda.synchronize()
    hA = amm.decompose(A0, method0, k0, "left")
    hB = amm.decompose(B0, method0, k0, "right")
    assert torch.equal(C0, amm.approx_matmul(hA, hB))
    batch.close()
