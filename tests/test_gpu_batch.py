"""Batched products of uneven sizes: eager run, graph capture and graph replay reproduce the
individually computed products bit for bit, and every item matches the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, check_selection, dev32, rel, torch_cuda

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


def _oracle_item(amm, A, B, method, k, sa, sb, compute):
    """The oracle's Re M for one batch item, on the values the GPU sees, with the selections and
    sketches of the same decompositions made one at a time (the batch makes identical ones)."""
    a64, b64 = as64(A), as64(B)
    hA = amm.decompose(A, method, k, "left", sketch=sa, compute=compute)
    hB = amm.decompose(B, method, k, "right", sketch=sb, compute=compute)
    if method == "circulant":
        check_selection(hA.selection(), O.component_keys(O.circulant_spectrum(a64)), k, "A")
        ta = O.truncate_circulant(a64, k, hA.selection())
        tb = O.truncate_circulant(b64, k, hB.selection())
    elif method == "cycle":
        check_selection(hA.selection(), O.cycle_keys(a64), k, "A")
        ta = O.truncate_cycles(a64, k, hA.selection())
        tb = O.truncate_cycles(b64, k, hB.selection())
    elif method == "svd":
        ta = O.truncate_rsvd(a64, k, hA.sketch().astype(np.float64))
        tb = O.truncate_rsvd(b64, k, hB.sketch().astype(np.float64))
    else:
        ta = O.truncate_fourier_left(a64, k, hA.selection())
        tb = O.truncate_fourier_right(b64, k, hB.selection())
    hA.close()
    hB.close()
    return O.product(method, ta, tb)


def test_batch_items_match_oracle():
    """Every item of a batch of uneven products (FP32 and BF16 operands, lengths 2^a and 3 * 2^a,
    one n = 4096 product) against the FP64 oracle: 1e-5 for FP32 arithmetic (BF16 operands of the
    circulant / sparsifier paths are read as BF16 and computed in FP32), 3e-2 for the rSVD in the
    BF16 tensor-core mode (operands, sketch and GEMM intermediates rounded to BF16).  Checked after
    the eager run and after a graph replay."""
    torch, amm = torch_cuda()
    spec = [(96, "circulant", "f32"), (192, "svd", "f32"), (384, "cycle", "f32"), (768, "fourier", "f32"),
            (4096, "circulant", "f32"), (1536, "svd", "bf16"), (256, "circulant", "bf16"),
            (3072, "cycle", "bf16"), (512, "fourier", "bf16"), (128, "svd", "f32"), (48, "circulant", "f32")]
    items, refs, tols = [], [], []
    for i, (n, method, dt) in enumerate(spec):
        k = max(2, -(-n // 32))
        a, b = S.exp32_pair(n, seed=200 + i) if n <= 1536 else S.general_times_toeplitz(n, seed=200 + i)
        A, B = dev32(torch, a), dev32(torch, b)
        if dt == "bf16":
            A, B = A.bfloat16(), B.bfloat16()
        compute = "bf16" if (dt == "bf16" and method == "svd") else "f32"
        own = method == "svd" and (i // 4) % 2 == 0     # caller sketch; else the library's Philox draw
        sa = dev32(torch, S.sketch(n, k, 200 + i, 0)) if own else None
        sb = dev32(torch, S.sketch(n, k, 200 + i, 1)) if own else None
        C = torch.full((n, n), float("nan"), device="cuda")
        items.append((A, B, C, method, k, sa, sb, compute))
        refs.append(_oracle_item(amm, A, B, method, k, sa, sb, compute))
        tols.append(3e-2 if compute == "bf16" else TOL)
    batch = amm.Batch()
    for A, B, C, method, k, sa, sb, compute in items:
        batch.add(A, B, C, method, k, sketch_a=sa, sketch_b=sb, compute=compute)
    for use_graph in (False, True, True):
        for it in items:
            it[2].fill_(float("nan"))
        batch.run(use_graph=use_graph)
        torch.cuda.synchronize()
        for (A, B, C, method, k, *_), ref, tol in zip(items, refs, tols):
            err = rel(C.double().cpu().numpy(), ref)
            assert err <= tol, (A.shape[0], method, str(A.dtype), use_graph, err)
    batch.close()


def test_batch_backward_items_match_single_calls_and_oracle():
    """Items added with their backward (amm_batch_add_grad) write the gradients of the frozen map:
    bit for bit those of amm_approx_matmul_backward on the same decompositions, and the oracle's
    gradients within 1e-5, eager and replayed from the graph."""
    torch, amm = torch_cuda()
    spec = [(128, "circulant"), (96, "svd"), (256, "cycle"), (192, "fourier"), (512, "circulant")]
    items, refs = [], []
    for i, (n, method) in enumerate(spec):
        k = max(2, n // 32)
        a, b = S.exp32_pair(n, seed=300 + i)
        A, B = dev32(torch, a), dev32(torch, b)
        G = dev32(torch, S.upstream_grad(n, n, 300 + i))
        sa = dev32(torch, S.sketch(n, k, 300 + i, 0)) if method == "svd" else None
        sb = dev32(torch, S.sketch(n, k, 300 + i, 1)) if method == "svd" else None
        hA = amm.decompose(A, method, k, "left", sketch=sa)
        hB = amm.decompose(B, method, k, "right", sketch=sb)
        C1 = amm.approx_matmul(hA, hB).clone()
        dA1, dB1 = amm.approx_matmul_backward(hA, hB, G)
        a64, b64, g64 = as64(A), as64(B), as64(G)
        if method == "svd":
            ta, tb = O.truncate_rsvd(a64, k, as64(sa)), O.truncate_rsvd(b64, k, as64(sb))
        elif method == "fourier":
            ta = O.truncate_fourier_left(a64, k, hA.selection())
            tb = O.truncate_fourier_right(b64, k, hB.selection())
        else:
            ta = O.truncate(method, a64, k, selection=hA.selection())
            tb = O.truncate(method, b64, k, selection=hB.selection())
        rda, rdb = O.backward(method, ta, tb, g64)
        assert rel(dA1.double().cpu().numpy(), rda) <= TOL and rel(dB1.double().cpu().numpy(), rdb) <= TOL
        refs.append((C1, dA1.clone(), dB1.clone()))
        items.append((A, B, torch.empty_like(A), method, k, sa, sb, G, torch.empty_like(A), torch.empty_like(B)))
        hA.close()
        hB.close()
    batch = amm.Batch()
    for A, B, C, method, k, sa, sb, G, dA, dB in items:
        batch.add(A, B, C, method, k, sketch_a=sa, sketch_b=sb, dC=G, dA=dA, dB=dB)
    for use_graph in (False, True, True):
        for it in items:
            for t in (it[2], it[8], it[9]):
                t.fill_(float("nan"))
        batch.run(use_graph=use_graph)
        torch.cuda.synchronize()
        for it, (C1, dA1, dB1) in zip(items, refs):
            assert torch.equal(it[2], C1) and torch.equal(it[8], dA1) and torch.equal(it[9], dB1), (it[3], use_graph)
    batch.close()


def test_batch_persistent_cycle_items_bit_identical_and_oracle():
    """The cycle-sparsifier items of a batch run in the persistent work-queue launch: lengths 2^a and
    others divisible by 4 (the paper's n = 700 among them), k from 1 to n, beside items of the other
    methods.  Their products equal the stream-pool run and single calls bit for bit, eager and as a
    replayed graph, and match the FP64 oracle; the launch reports no timeout."""
    torch, amm = torch_cuda()
    spec = [(16, 1, "cycle"), (700, 22, "cycle"), (4096, 128, "cycle"), (100, 100, "cycle"), (1020, 33, "cycle"),
            (256, 8, "circulant"), (64, 64, "cycle"), (512, 16, "svd"), (2048, 7, "cycle"), (1536, 48, "cycle")]
    items = []
    for i, (n, k, method) in enumerate(spec):
        a, b = S.exp32_pair(n, seed=300 + i) if n <= 1536 else S.general_times_toeplitz(n, seed=300 + i)
        A, B = dev32(torch, a), dev32(torch, b)
        sa = dev32(torch, S.sketch(n, k, 300 + i, 0)) if method == "svd" else None
        sb = dev32(torch, S.sketch(n, k, 300 + i, 1)) if method == "svd" else None
        items.append([A, B, torch.full((n, n), float("nan"), device="cuda"), method, k, sa, sb])
    singles = []
    for A, B, C, method, k, sa, sb in items:
        hA = amm.decompose(A, method, k, "left", sketch=sa)
        hB = amm.decompose(B, method, k, "right", sketch=sb)
        singles.append(amm.approx_matmul(hA, hB).clone())
    pool = amm.Batch()
    pool.set_persistent(False)
    pers = amm.Batch()
    pool_c = []
    for A, B, C, method, k, sa, sb in items:
        Cp = torch.full_like(C, float("nan"))
        pool_c.append(Cp)
        pool.add(A, B, Cp, method, k, sketch_a=sa, sketch_b=sb)
        pers.add(A, B, C, method, k, sketch_a=sa, sketch_b=sb)
    pool.run(use_graph=False)
    for use_graph in (False, True, True):
        for it in items:
            it[2].fill_(float("nan"))
        pers.run(use_graph=use_graph)
        status, item, stage, npq = pers.status()
        assert (status, item, stage) == (0, -1, -1)
        assert npq == sum(1 for s in spec if s[2] == "cycle")
        torch.cuda.synchronize()
        for (A, B, C, method, k, *_), Cp, ref in zip(items, pool_c, singles):
            assert torch.equal(C, ref), (A.shape[0], method, k, use_graph)
            assert torch.equal(Cp, ref), (A.shape[0], method, k)
    assert pool.status()[3] == 0
    for (A, B, C, method, k, sa, sb), (n, *_) in zip(items, spec):
        if method == "cycle" and n <= 1536:
            ref = _oracle_item(amm, A, B, method, k, sa, sb, "f32")
            assert rel(C.double().cpu().numpy(), ref) <= TOL, (n, k)
    pool.close()
    pers.close()


def test_batch_persistent_wait_runs_out_and_reports_timeout():
    """A task whose dependency never completes: the executor's bounded wait gives up after the
    limit, the launch returns with AMM_ERR_TIMEOUT and the stage it waited for (4, the column
    panels), and the device keeps working (a product afterwards is exact)."""
    import ctypes
    import time
    torch, amm = torch_cuda()
    lib = amm.load_library()
    st, stage = ctypes.c_int32(-1), ctypes.c_int32(-1)
    t0 = time.perf_counter()
    assert lib.amm_debug_persistent_wait_timeout(20_000_000, torch.cuda.current_stream().cuda_stream,
                                                 ctypes.byref(st), ctypes.byref(stage)) == 0
    waited = time.perf_counter() - t0
    assert st.value == 5 and stage.value == 4
    assert 0.015 <= waited < 5.0
    n = 64
    a, b = S.exp32_pair(n, seed=9)
    A, B = dev32(torch, a), dev32(torch, b)
    C = amm.approx_matmul(amm.decompose(A, "cycle", n, "left"), amm.decompose(B, "cycle", n, "right"))
    assert rel(C.double().cpu().numpy(), as64(A) @ as64(B)) <= TOL
