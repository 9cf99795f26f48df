"""Run one decomposition + first-order product (+ backward) for a profiler.

    python -m paper_2504_19308_gb300.profile_case --method circulant --k 256 --n 4096 [--backward] [--repeat 2]

Inputs are the seeded power-law pair of the bench (sigma_i = i^-1.5 + N(0, 1e-4)), drawn as
Gaussian-plus-spectrum matrices without QR when --fast is given (same sizes, cheaper to make).
Each repeat is wrapped in an NVTX range "case" so that a profiler can select it.
"""
import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synth  # noqa: E402
import paper_2504_19308_gb300 as amm  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--method", default="circulant")
    ap.add_argument("--k", type=int, default=256)
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--backward", action="store_true")
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--fast", action="store_true")
    a = ap.parse_args()
    n, k = a.n, a.k
    if a.fast:
        g = synth.rng(0, 0)
        x, y = g.standard_normal((n, n)) * 1e-2, g.standard_normal((n, n)) * 1e-2
    else:
        x, y = synth.powerlaw_pair(n, seed=0)
    dev = torch.device("cuda")
    A = torch.tensor(x, dtype=torch.float32, device=dev)
    B = torch.tensor(y, dtype=torch.float32, device=dev)
    sa = torch.tensor(synth.sketch(n, k, 0, 0), dtype=torch.float32, device=dev) if a.method == "svd" else None
    sb = torch.tensor(synth.sketch(n, k, 0, 1), dtype=torch.float32, device=dev) if a.method == "svd" else None
    G = torch.randn((n, n), device=dev)
    for _ in range(a.repeat):
        torch.cuda.nvtx.range_push("case")
        hA = amm.decompose(A, a.method, k, "left", sketch=sa)
        hB = amm.decompose(B, a.method, k, "right", sketch=sb)
        C = amm.approx_matmul(hA, hB)
        if a.backward:
            amm.approx_matmul_backward(hA, hB, G)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        hA.close()
        hB.close()
    print("ok", a.method, n, k, float(C.abs().sum()))


if __name__ == "__main__":
    main()
