"""The seeded input generators against the recipes they state (the paper's matrix families and the
workloads' shapes, spectra and value distributions), on the CPU: a generator that drifted from its
recipe would silently change every parity case and bench line built on it."""
import math

import numpy as np
import pytest

import synth as S


def test_streams_are_pure_functions_of_seed_and_stream():
    x = S.rng(3, 1).standard_normal(8)
    assert np.array_equal(x, S.rng(3, 1).standard_normal(8))
    assert not np.array_equal(x, S.rng(3, 2).standard_normal(8))
    assert not np.array_equal(x, S.rng(4, 1).standard_normal(8))
    a1, b1 = S.general_times_toeplitz(32, seed=5)
    a2, b2 = S.general_times_toeplitz(32, seed=5)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)


def test_haar_orthogonal_and_prescribed_spectrum():
    g = S.rng(0, 0)
    q = S.haar_orthogonal(48, g)
    assert np.allclose(q.T @ q, np.eye(48), atol=1e-12)
    sig = np.exp(-np.arange(48) / 10.0)
    x = S.spectrum_matrix(sig, g)
    assert np.allclose(np.linalg.svd(x, compute_uv=False), sig, rtol=1e-10, atol=1e-14)
    assert np.allclose(np.linalg.svd(S.type3(40, g), compute_uv=False), (40 - np.arange(40)) / 40, atol=1e-12)


def test_noisy_spectra_within_the_noise_norm():
    """exp32: sigma_i = e^{-i/32} plus 1e-3 N(0,1) noise; power law: sigma_i = i^-1.5 plus N(0, 1e-4).
    By Weyl's inequality each singular value moves by at most ||noise||_2 <= ~2 sqrt(n) sd."""
    n = 64
    a, b = S.exp32_pair(n, seed=1)
    ref = np.exp(-np.arange(n) / 32.0)
    for x in (a, b):
        assert np.max(np.abs(np.linalg.svd(x, compute_uv=False) - ref)) <= 3 * math.sqrt(n) * 1e-3
    a, _ = S.powerlaw_pair(n, seed=1, noise_sd=0.0)
    assert np.allclose(np.linalg.svd(a, compute_uv=False), np.arange(1, n + 1) ** -1.5, rtol=1e-10)
    a, _ = S.powerlaw_pair(n, seed=1)
    assert np.max(np.abs(np.linalg.svd(a, compute_uv=False) - np.arange(1, n + 1) ** -1.5)) <= 3 * math.sqrt(n) * 1e-2


def test_structured_families():
    g = S.rng(2, 0)
    n = 24
    t, h, s = S.toeplitz_uniform(n, g), S.hankel_uniform(n, g), S.symmetric_uniform(n, g)
    for i in range(1, n):
        assert np.array_equal(t[i, 1:], t[i - 1, :-1])  # constant diagonals
        assert np.array_equal(h[i, :-1], h[i - 1, 1:])  # constant anti-diagonals
    assert np.array_equal(s, s.T)
    for x in (t, h, s, S.general_uniform(n, g)):
        assert x.min() >= 0.0 and x.max() < 1.0
    k = S.kappa(n)
    assert np.array_equal(k, k.T) and np.allclose(np.diag(k), np.sin(np.arange(n) + 1.0))
    assert k[3, 5] == pytest.approx(math.exp(-1.0) * math.sin(4.0))
    c = g.standard_normal(n)
    x = S.circulant_from_column(c)
    assert np.array_equal(x[:, 0], c) and all(np.array_equal(x[:, q], np.roll(c, q)) for q in range(n))


def test_type2_adds_a_scaled_uniform_matrix():
    n = 32
    g1, g2 = S.rng(9, 0), S.rng(9, 0)
    t = S.type1(n, g1)
    u = g1.uniform(0.0, 1.0, (n, n))
    x = S.type2(n, g2)  # the same draws in the same order
    assert np.allclose(x, t + 0.5 * np.linalg.norm(t) / np.linalg.norm(u) * u, rtol=1e-13, atol=1e-15)


def test_two_structure_cases_have_their_structure():
    n = 32
    cases = S.two_structure_cases(n, S.rng(6, 0))
    circ = cases["circulant"]
    assert all(np.array_equal(circ[:, q], np.roll(circ[:, 0], q)) for q in range(n))
    assert np.linalg.matrix_rank(cases["svd"]) == 2
    band = cases["cycle"]
    l = np.arange(n)
    kept = np.zeros((n, n), dtype=bool)
    for j in (0, 1):
        kept[(l + j) % n, l] = True
    assert np.all(band[~kept] == 0.0) and np.all(band[kept] != 0.0)
    spec = np.abs(np.fft.fft(cases["fourier"], axis=1))
    for r in range(n):  # one real sinusoid per row: two conjugate frequencies, 0 < f < n/2
        big = np.flatnonzero(spec[r] > 1e-9 * spec[r].max())
        assert len(big) == 2 and big[0] + big[1] == n and 0 < big[0] < n // 2


def test_sketches_and_gradients():
    phi0, phi1 = S.sketch(256, 8, 0, 0), S.sketch(256, 8, 0, 1)
    assert phi0.shape == (256, 8) and not np.array_equal(phi0, phi1)
    assert abs(phi0.mean()) < 0.1 and abs(phi0.std() - 1.0) < 0.1
    assert np.array_equal(S.upstream_grad(16, 8, 3), S.rng(3, S.STREAM_G).standard_normal((16, 8)))


def test_llm_shaped_weights():
    x, w = S.llm_shaped(seed=0, m=64, d=512, f=1024)
    assert x.shape == (64, 512) and w.shape == (512, 1024)
    out = np.abs(w) > 0.02 * 6  # beyond 6 sd of the Gaussian part: the t_3 outliers
    assert 2e-4 < out.mean() < 2e-3
    assert abs(w[~out].std() - 0.02) < 1e-3


def test_differentiation_case_spectrum_and_shapes():
    a, b, g = S.differentiation_case(seed=0, n=64, p=32, decay=16.0)
    assert b.shape == (64, 32) and g.shape == (64, 32)
    assert np.allclose(np.linalg.svd(a, compute_uv=False), np.exp(-np.arange(64) / 16.0), rtol=1e-10)


@pytest.mark.parametrize("radix3", [False, True])
def test_batch_sizes_are_log_uniform_fft_lengths(radix3):
    ns = S.batch_sizes(256, seed=0, radix3=radix3)
    assert ns == S.batch_sizes(256, seed=0, radix3=radix3) and len(ns) == 256
    allowed = {2 ** a for a in range(4, 14)} | ({3 * 2 ** a for a in range(4, 12)} if radix3 else set())
    assert set(ns) <= allowed and min(ns) >= 128 and max(ns) <= 4096
    logs = np.log(ns)
    # log-uniform on [ln 128, ln 4096]: median near the geometric mean 724, quartiles near 256 / 2048
    assert abs(np.median(logs) - math.log(724)) < 0.5
    assert len(set(ns)) >= (6 if not radix3 else 10)
