"""FP64 CPU oracle for the first-order approximate product (test infrastructure only).

This package is the executable statement of what the GPU path computes.  It is slow and
plain on purpose: dense complex matrices, explicit DFT matrices at small sizes, library
matmul / FFT / QR / SVD / sort as single steps, and no blocking or fusion.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it;
the product path (``paper_2504_19308_gb300``) never does, and the two share no code.

Every function cites the passage of arXiv 2504.19308 it follows.  Conventions (fixed by
Thm 2.1 and Alg. 2; see ``oracle.amm``):
  * C is the full-cycle permutation with (C x)_i = x_{i-1}; row r of C^j has its 1 at (r-j) mod n.
  * omega = e^{+2 pi i / n}, D = diag(omega^q).
  * "FFT" is the unnormalised forward DFT F(p,q) = e^{-2 pi i pq/n}; "IFFT" is F^{-1} (1/n).
  * Right cycle form A = sum_j C^j Lambda_j with Lambda_j(l,l) = A((l+j) mod n, l).
"""
from .amm import *  # noqa: F401,F403
