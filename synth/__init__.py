"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and the bench.

This module only *draws* matrices. It contains none of the approximate-multiplication
arithmetic (no decomposition, no selection, no product): both the FP64 oracle and the
CUDA path consume what it returns, and neither imports the other.

Streams: every array is drawn from ``numpy.random.Generator(PCG64(SeedSequence([seed, stream])))``
so an input is a pure function of ``(seed, stream)``.  By convention A is stream 0,
B is stream 1, the sketch of the left operand stream 2, of the right operand stream 3,
and the upstream gradient stream 4.

Matrix families follow the paper's generators:
  * ``haar_orthogonal`` / ``spectrum_matrix``: Appendix C (QR of an i.i.d. N(0,1) matrix,
    columns sign-fixed by diag(R) so that Q is Haar distributed), then Q1 diag(S) Q2^T.
  * Type-1 (S_i = e^{-i/10}), Type-2 (Type-1 plus 0.5 ||T||/||U|| U, U ~ U(0,1)) and
    Type-3 (S_i = (n-i)/n): Appendix C.
  * General U(0,1), Toeplitz / Hankel from U(0,1) entries, symmetric, and the
    "Kappa" matrix K_ij = K_ji = e^{-0.5|i-j|} sin(i+1): Section 4 / Appendix A.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

STREAM_A, STREAM_B, STREAM_PHI_A, STREAM_PHI_B, STREAM_G = 0, 1, 2, 3, 4


def rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


def haar_orthogonal(n: int, g: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal n x n matrix (Appendix C: QR of N(0,1), sign fix)."""
    m = g.standard_normal((n, n))
    q, r = np.linalg.qr(m)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def spectrum_matrix(sigma: np.ndarray, g: np.random.Generator) -> np.ndarray:
    """Q1 diag(sigma) Q2^T with Haar Q1, Q2 (Appendix C)."""
    n = len(sigma)
    q1 = haar_orthogonal(n, g)
    q2 = haar_orthogonal(n, g)
    return (q1 * np.asarray(sigma, dtype=np.float64)[None, :]) @ q2.T


def type1(n, g):
    return spectrum_matrix(np.exp(-np.arange(n) / 10.0), g)


def type3(n, g):
    return spectrum_matrix((n - np.arange(n)) / n, g)


def type2(n, g):
    t = type1(n, g)
    u = g.uniform(0.0, 1.0, (n, n))
    return t + 0.5 * np.linalg.norm(t) / np.linalg.norm(u) * u


def general_uniform(n, g, m=None):
    return g.uniform(0.0, 1.0, (m or n, n))


def toeplitz_uniform(n, g):
    """T[i, j] = c[i - j] with the 2n-1 defining entries drawn from U(0,1)."""
    c = g.uniform(0.0, 1.0, 2 * n - 1)
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return c[(i - j) + (n - 1)]


def hankel_uniform(n, g):
    c = g.uniform(0.0, 1.0, 2 * n - 1)
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return c[i + j]


def symmetric_uniform(n, g):
    x = g.uniform(0.0, 1.0, (n, n))
    return np.triu(x) + np.triu(x, 1).T


def kappa(n):
    i = np.arange(n)[:, None].astype(np.float64)
    j = np.arange(n)[None, :].astype(np.float64)
    lo = np.minimum(i, j)
    return np.exp(-0.5 * np.abs(i - j)) * np.sin(lo + 1.0)


def circulant_from_column(c: np.ndarray) -> np.ndarray:
    """Circulant matrix whose first column is c: X[r, q] = c[(r - q) mod n]."""
    n = len(c)
    r = np.arange(n)[:, None]
    q = np.arange(n)[None, :]
    return np.asarray(c)[(r - q) % n]


def two_structure_cases(n: int, g) -> dict:
    """Four n x n inputs, each built from two pieces of one kind of structure: a circulant matrix,
    a rank-2 product of Gaussian factors, two wrapped diagonals with random entries
    (X[(l + j) mod n, l] for j = 0, 1), and rows that are single sinusoids
    X[r, q] = a_r cos(2 pi f_r q / n + p_r) with 0 < f_r < n/2."""
    circ = circulant_from_column(g.standard_normal(n))
    lowrank = g.standard_normal((n, 2)) @ g.standard_normal((2, n))
    band = np.zeros((n, n))
    l = np.arange(n)
    for j in (0, 1):
        band[(l + j) % n, l] = g.standard_normal(n)
    f = g.integers(1, n // 2, size=n)[:, None]
    amp = g.standard_normal(n)[:, None]
    ph = g.uniform(0.0, 2.0 * np.pi, n)[:, None]
    waves = amp * np.cos(2.0 * np.pi * f * l[None, :] / n + ph)
    return {"circulant": circ, "svd": lowrank, "cycle": band, "fourier": waves}


def gaussian(shape, g, sd=1.0):
    return sd * g.standard_normal(shape)


def sketch(n: int, k: int, seed: int, side: int) -> np.ndarray:
    """The rSVD test matrix phi (n x k, i.i.d. N(0,1)) for operand side 0 (A) or 1 (B)."""
    return rng(seed, STREAM_PHI_A + side).standard_normal((n, k))


# ---------------------------------------------------------------------------
# Workloads named by what they are.  Each returns float64 arrays; callers cast.
# ---------------------------------------------------------------------------

def decaying_plus_noise(n: int, sigma: np.ndarray, noise_sd: float, g) -> np.ndarray:
    x = spectrum_matrix(sigma, g)
    if noise_sd:
        x = x + noise_sd * g.standard_normal((n, n))
    return x


def exp32_pair(n: int = 512, seed: int = 0):
    """A, B = Q1 diag(e^{-i/32}) Q2^T + 1e-3 N(0,1), i = 0..n-1 (n=512 is the small FP32 case)."""
    sig = np.exp(-np.arange(n) / 32.0)
    a = decaying_plus_noise(n, sig, 1e-3, rng(seed, STREAM_A))
    b = decaying_plus_noise(n, sig, 1e-3, rng(seed, STREAM_B))
    return a, b


def powerlaw_pair(n: int = 4096, seed: int = 0, noise_sd: float = 1e-2):
    """A, B = Q1 diag(i^{-1.5}) Q2^T + N(0, 1e-4) noise (variance 1e-4 -> sd 1e-2), i = 1..n."""
    sig = np.arange(1, n + 1, dtype=np.float64) ** -1.5
    a = decaying_plus_noise(n, sig, noise_sd, rng(seed, STREAM_A))
    b = decaying_plus_noise(n, sig, noise_sd, rng(seed, STREAM_B))
    return a, b


def general_times_toeplitz(n: int, seed: int = 0):
    """General U(0,1) x Toeplitz U(0,1): the paper's structured pair that reaches ~1% error."""
    return general_uniform(n, rng(seed, STREAM_A)), toeplitz_uniform(n, rng(seed, STREAM_B))


def llm_shaped(seed: int = 0, m: int = 2048, d: int = 4096, f: int = 11008):
    """Activations m x d N(0,1); weight d x f N(0, 0.02^2) with 0.1% entries replaced by 20*0.02*t_3."""
    ga, gb = rng(seed, STREAM_A), rng(seed, STREAM_B)
    x = ga.standard_normal((m, d))
    w = 0.02 * gb.standard_normal((d, f))
    mask = gb.uniform(0.0, 1.0, (d, f)) < 1e-3
    w[mask] = 20 * 0.02 * gb.standard_t(3, int(mask.sum()))
    return x, w


def differentiation_case(seed: int = 0, n: int = 8192, p: int = 4096, decay: float = 256.0):
    """The autograd-layer workload: A n x n = Q1 diag(e^{-i/decay}) Q2^T (noise-free), B n x p and
    the upstream gradient m x p both N(0, 1)."""
    a = spectrum_matrix(np.exp(-np.arange(n) / decay), rng(seed, STREAM_A))
    b = rng(seed, STREAM_B).standard_normal((n, p))
    return a, b, upstream_grad(n, p, seed)


def upstream_grad(m: int, p: int, seed: int = 0) -> np.ndarray:
    return rng(seed, STREAM_G).standard_normal((m, p))


def batch_sizes(count: int = 256, seed: int = 0, lo: int = 128, hi: int = 4096, radix3: bool = False):
    """n_i = round(exp(U(ln lo, ln hi))) rounded to the nearest FFT size (in log distance): a power
    of two, or with radix3 the nearest of {2^a, 3 * 2^a}.  The same draws for both roundings."""
    g = rng(seed, 7)
    u = g.uniform(math.log(lo), math.log(hi), count)
    n = np.exp(u)
    if not radix3:
        return [int(2 ** round(math.log2(v))) for v in n]
    cands = sorted({2 ** a for a in range(4, 14)} | {3 * 2 ** a for a in range(4, 12)})
    return [int(min(cands, key=lambda c: abs(math.log(c) - math.log(v)))) for v in n]
