"""Run one decomposition + first-order product (+ backward) for a profiler.

    python -m paper_2504_19308_gb300.profile_case --method circulant --k 256 --n 4096 [--backward] [--repeat 2]
    python -m paper_2504_19308_gb300.profile_case --step [--repeat 2] [--trace]

--step runs the sweep of the n = 4096 power-law step instead (circulant k = 16/64/256, rSVD
k = 32/128, Fourier and cycle sparsifiers k = 41, each decomposed, multiplied and differentiated).
--le1pct runs the products of the n = 4096 General U(0,1) x Toeplitz U(0,1) step that reach <= 1%
error (circulant k = 1/5/9, Fourier sparsifier k = 60), each decomposed, multiplied, differentiated.
--headline runs the throughput step of the bench: those four, the randomized SVD at k = 16 and 32 on
the same pair, and the randomized SVD at k = 256 on the n = 512 pair Q1 diag(e^{-i/32}) Q2^T +
1e-3 N(0,1), each decomposed, multiplied and differentiated.

Inputs are the seeded power-law pair of the bench (sigma_i = i^-1.5 + N(0, 1e-4)), drawn as
Gaussian-plus-spectrum matrices without QR when --fast is given (same sizes, cheaper to make).
The autotuner is on (as in the bench), so the first repeat times the kernel variants; it is
wrapped in an NVTX range "warmup", every later repeat in a range "case" that a profiler can
select (ncu --nvtx --nvtx-include "case/").  --trace times
every library launch of the repeats after the first with CUDA events on its own stream (the
library's launch trace) and prints one JSON object {kernel: [launches, total ms, ...]} per run.
"""
import argparse
import os
import sys

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
    ap.add_argument("--step", action="store_true")
    ap.add_argument("--trace", action="store_true")
    ap.add_argument("--le1pct", action="store_true")
    ap.add_argument("--headline", action="store_true")
    a = ap.parse_args()
    n, k = a.n, a.k
    if a.le1pct or a.headline:
        x, y = synth.general_times_toeplitz(n, seed=0)
    elif a.fast:
        g = synth.rng(0, 0)
        x, y = g.standard_normal((n, n)) * 1e-2, g.standard_normal((n, n)) * 1e-2
    else:
        x, y = synth.powerlaw_pair(n, seed=0)
    dev = torch.device("cuda")
    amm.load_library()
    amm.set_autotune(True)
    A = torch.tensor(x, dtype=torch.float32, device=dev)
    B = torch.tensor(y, dtype=torch.float32, device=dev)
    G = torch.randn((n, n), device=dev)
    ks = -(-n // 100)
    small = None
    if a.headline:
        cases = [("circulant", 1, True), ("circulant", 5, True), ("circulant", 9, True), ("svd", 16, True),
                 ("svd", 32, True), ("fourier", 60, True)]
        x5, y5 = synth.exp32_pair(512, seed=0)
        small = (torch.tensor(x5, dtype=torch.float32, device=dev), torch.tensor(y5, dtype=torch.float32, device=dev),
                 torch.randn((512, 512), device=dev))
    elif a.le1pct:
        cases = [("circulant", 1, True), ("circulant", 5, True), ("circulant", 9, True), ("fourier", 60, True)]
    elif a.step:
        cases = [("circulant", 16, True), ("circulant", 64, True), ("circulant", 256, True), ("svd", 32, True),
                 ("svd", 128, True), ("fourier", ks, True), ("cycle", ks, True)]
    else:
        cases = [(a.method, k, a.backward)]
    sk = {}
    for method, kk, _ in cases:
        if method == "svd":
            sk[kk] = tuple(torch.tensor(synth.sketch(n, kk, 0, side), dtype=torch.float32, device=dev)
                           for side in (0, 1))
    sk_small = tuple(torch.tensor(synth.sketch(512, 256, 0, side), dtype=torch.float32, device=dev) for side in (0, 1))
    for rep in range(a.repeat):
        if a.trace and rep == 1:  # the first repeat warms up (autotuning, allocations)
            torch.cuda.synchronize()
            amm.trace_enable(True)
        torch.cuda.nvtx.range_push("warmup" if rep == 0 and a.repeat > 1 else "case")
        for method, kk, bwd in cases:
            sa, sb = sk.get(kk, (None, None)) if method == "svd" else (None, None)
            hA = amm.decompose(A, method, kk, "left", sketch=sa)
            hB = amm.decompose(B, method, kk, "right", sketch=sb)
            C = amm.approx_matmul(hA, hB)
            if bwd:
                amm.approx_matmul_backward(hA, hB, G)
            hA.close()
            hB.close()
        if small is not None:  # rSVD k = 256 on the n = 512 pair
            hA = amm.decompose(small[0], "svd", 256, "left", sketch=sk_small[0])
            hB = amm.decompose(small[1], "svd", 256, "right", sketch=sk_small[1])
            amm.approx_matmul(hA, hB)
            amm.approx_matmul_backward(hA, hB, small[2])
            hA.close()
            hB.close()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    if a.trace and a.repeat > 1:
        import json
        kernels, launches = amm.trace_collect()
        amm.trace_enable(False)
        per = a.repeat - 1
        print(json.dumps({"repeats": per, "launches": launches,
                          "ms_per_repeat": {name: round(v[1] / per, 4) for name, v in sorted(kernels.items())}}))
    print("ok", "headline" if a.headline else "le1pct" if a.le1pct else ("step" if a.step else a.method), n, k,
          float(C.abs().sum()))


if __name__ == "__main__":
    main()
