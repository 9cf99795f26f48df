"""Helpers for the GPU parity tests: device tensors from the shared generators and the
oracle evaluated on exactly the FP32 values the GPU sees."""
import numpy as np
import pytest

import oracle as O

TOL = 1e-5      # relative Frobenius tolerance of the FP32 path against the FP64 oracle
TAU = 1e-5      # keys closer than this (relative) to the k-th key are treated as near-ties


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2504_19308_gb300 as amm
    amm.load_library()
    return torch, amm


def dev32(torch, x):
    return torch.tensor(np.asarray(x, dtype=np.float32), device="cuda")


def as64(t):
    return t.detach().double().cpu().numpy()


def rel(x, ref):
    """Relative Frobenius error; complex arrays stay complex."""
    x = np.asarray(x)
    x = x.astype(np.complex128) if np.iscomplexobj(x) else x.astype(np.float64)
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def check_selection(gpu_sel, keys, k, what=""):
    """GPU selection == oracle top-k outside near-ties; inside, GPU picks come from the tied band."""
    must, maybe = O.near_tie_sets(keys, k, TAU)
    got = set(int(v) for v in gpu_sel)
    assert len(got) == k, (what, "repeated indices", gpu_sel)
    n = len(keys)
    # conjugate partners tie bit-exactly on both sides and are ordered by index on both:
    # a band made of one partner pair only is not ambiguous
    classes = {min(t, (n - t) % n) for t in maybe}
    if not maybe or len(classes) == 1:
        assert got == set(O.top_k(keys, k).tolist()), (what, sorted(got), sorted(O.top_k(keys, k).tolist()))
    else:
        assert must <= got, (what, "missing certain picks", sorted(must - got))
        assert got <= (must | maybe), (what, "picked outside the tied band", sorted(got - must - maybe))
