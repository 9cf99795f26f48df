"""Pins of the FP64 oracle to facts fixed by the paper or by mathematics (CPU only).

Each test names the passage it checks.  Together they are chosen so that a plausible
mistake in the oracle (a sign of omega, a transposed cycle layout, a dropped first-order
term, a wrong projector in the backward) fails at least one of them; test_planted_mistakes
demonstrates this by planting such mistakes into the oracle on the CPU.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
import oracle.amm as OA
import synth as S
from conftest import GOLDEN


def _rand(n, seed=0, m=None):
    return S.rng(seed, 9).standard_normal((m or n, n))


# --------------------------------------------------------------------------- cycles

def _read_example():
    grids, cur, cpow = {}, None, []
    with open(os.path.join(GOLDEN, "cycle_example_4x4.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line in ("right", "left", "Cpow"):
                cur = line
                grids.setdefault(cur, [])
                continue
            if cur == "Cpow":
                cpow.append(tuple(int(v) for v in line.split()))
            else:
                grids[cur].append(line.split())
    return grids, cpow


def test_cycle_layout_matches_worked_example():
    """Appendix 4x4 example: both printed cycle layouts, entry for entry."""
    grids, _ = _read_example()
    n = 4
    a = np.array([[100 + 10 * r + c for c in range(n)] for r in range(n)], dtype=np.float64)
    label = lambda v: "%d%d" % ((int(v) - 100) // 10, (int(v) - 100) % 10)
    right = [[label(v) for v in row] for row in O.cycle_layout(a)]
    left = [[label(v) for v in row] for row in O.cycle_layout_left(a)]
    assert right == grids["right"]
    assert left == grids["left"]


def test_cycle_power_nonzeros():
    """Appendix: row r of C^k has its nonzero in column (r - k) mod n."""
    _, cpow = _read_example()
    c = O.cycle_perm(4)
    for k, r, col in cpow:
        ck = np.linalg.matrix_power(c, k)
        assert ck[r, col] == 1.0 and ck[r].sum() == 1.0


@pytest.mark.parametrize("n", [3, 4, 7, 16])
def test_cycle_decomposition_sums_to_A(n):
    """Section 1.2.2 / Eq. rightdecomp: A = sum_j C^j Lambda_j with explicit C^j."""
    a = _rand(n)
    total = sum(cj @ lam for cj, lam in O.cycle_matrices(a))
    assert np.allclose(total, a, atol=1e-14, rtol=0)
    assert np.array_equal(O.from_cycle_layout(O.cycle_layout(a)), a)


# --------------------------------------------------------------------------- circulant decomposition

@pytest.mark.parametrize("n", [4, 5, 6, 7, 8, 9, 12, 15, 16])
def test_thm21_components_sum_to_A(n):
    """Thm 2.1: A = sum_k R_k D^k, with dense explicitly formed components."""
    a = _rand(n, 1)
    R = O.circulant_spectrum(a)
    assert np.abs(O.reconstruct_explicit(R, range(n)) - a).max() < 1e-13
    assert np.abs(O.reconstruct(R, range(n)) - a).max() < 1e-13


def test_components_frobenius_orthogonal():
    """Remark after Thm 2.1: <R_i D^i, R_j D^j>_F = 0 (i != j) and = ||R_i||_F^2."""
    n = 8
    R = O.circulant_spectrum(_rand(n, 2))
    comps = [O.component_dense(R, k) for k in range(n)]
    gram = np.array([[np.vdot(x, y) for y in comps] for x in comps])
    diag = np.array([np.linalg.norm(O.circulant(R[k])) ** 2 for k in range(n)])
    assert np.abs(gram - np.diag(diag)).max() < 1e-13


@pytest.mark.parametrize("n", [8, 9, 64, 128])
def test_parseval_keys(n):
    """||R_k D^k||_F^2 = n T[k]^2 and sum_k n T[k]^2 = ||A||_F^2 (Remark, Alg. 3's keys)."""
    a = _rand(n, 3)
    keys = O.component_keys(O.circulant_spectrum(a))
    assert abs(n * np.sum(keys ** 2) - np.sum(a * a)) < 1e-10 * np.sum(a * a)


def test_circulant_input_has_one_component():
    """A circulant matrix times D^t is the single component t: ||R_k|| = 0 for k != t."""
    n = 16
    col = S.rng(4, 1).standard_normal(n)
    for t in (0, 3, 8):
        R = O.circulant_spectrum(O.circulant(col) @ O.diag_D(n, t))
        norms = np.linalg.norm(R, axis=1)
        assert norms[t] > 0.1 and np.delete(norms, t).max() < 1e-14
        assert np.abs(R[t] - col).max() < 1e-14


def test_thm25_least_squares():
    """Thm 2.5: R_k minimises ||A - M D^k||_F over circulant M (basis C^j, lstsq)."""
    n = 6
    a = _rand(n, 5)
    R = O.circulant_spectrum(a)
    c = O.cycle_perm(n)
    for k in range(n):
        basis = [np.linalg.matrix_power(c, j) @ O.diag_D(n, k) for j in range(n)]
        mat = np.stack([b.ravel() for b in basis], axis=1)
        coef, *_ = np.linalg.lstsq(mat, a.ravel().astype(np.complex128), rcond=None)
        assert np.abs(coef - R[k]).max() < 1e-13


def test_eigen_spectrum_diagonalises_component():
    """Alg. 3: L_t = F R_A[t] are the eigenvalues of R_t: R_t = F^{-1} diag(L_t) F."""
    n = 16
    R = O.circulant_spectrum(_rand(n, 6))
    f = O.dft_matrix(n)
    for t in (0, 1, 5):
        lt = O.eigen_spectrum(R, t)
        assert np.abs(np.linalg.inv(f) @ np.diag(lt) @ f - O.circulant(R[t])).max() < 1e-13


def test_shift_identity():
    """Remark after Thm 2.1 / Section 2.3.2 (reading R2): W D^k W^* = C^k and F D^k b = C^k F b."""
    n = 8
    w = O.unitary_W(n)
    c = O.cycle_perm(n)
    for k in range(n):
        assert np.abs(w @ O.diag_D(n, k) @ w.conj().T - np.linalg.matrix_power(c, k)).max() < 1e-13


def test_library_fft_matches_dft_definition():
    n = 128
    x = S.rng(7, 0).standard_normal((n, 3))
    assert np.abs(O.fft_cols(x) - O.dft_matrix(n) @ x).max() < 1e-11


# --------------------------------------------------------------------------- selection

def test_topk_tie_rule():
    """Reading R6: (key descending, index ascending); conjugate partners tie exactly."""
    assert O.top_k(np.array([1.0, 3.0, 3.0, 2.0, 3.0]), 3).tolist() == [1, 2, 4]
    # a single nonzero entry has a flat spectrum: its cycle is a delta, every key is 1/n
    n = 8
    e00 = np.zeros((n, n))
    e00[0, 0] = 1.0
    keys = O.component_keys(O.circulant_spectrum(e00))
    assert np.allclose(keys, 1 / n, rtol=1e-14, atol=0)
    assert O.top_k(keys, 3).tolist() == [0, 1, 2]
    # real input: T[k] == T[n-k] bit for bit
    keys = O.component_keys(O.circulant_spectrum(_rand(12, 8)))
    assert all(keys[k] == keys[12 - k] for k in range(1, 12))


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_topk_minimises_residual_bruteforce(k):
    """Section 2.3 (orthogonality): the top-k components minimise ||dA||_F over all k-subsets."""
    n = 7
    a = _rand(n, 10)
    R = O.circulant_spectrum(a)
    best = min(np.linalg.norm(a - O.reconstruct_explicit(R, sub)) for sub in itertools.combinations(range(n), k))
    got = np.linalg.norm(O.truncate_circulant(a, k).resid)
    assert got <= best * (1 + 1e-12)


def test_truncation_error_from_keys():
    """||dA||_F^2 = ||A||_F^2 - n sum_{t in S} T[t]^2 (orthogonality)."""
    n = 32
    a = _rand(n, 11)
    tr = O.truncate_circulant(a, 5)
    pred = np.sum(a * a) - n * np.sum(tr.keys[tr.sel] ** 2)
    assert abs(np.linalg.norm(tr.resid) ** 2 - pred) < 1e-10 * np.sum(a * a)


# --------------------------------------------------------------------------- products

@pytest.mark.parametrize("n,k", [(16, 1), (16, 3), (16, 4), (16, 8), (32, 5), (32, 12), (15, 3), (17, 4), (21, 6)])
def test_alg3_fft_form_equals_explicit(n, k):
    """Alg. 3 (FFT form, shifts and conjugates as printed) equals the explicit dense A~B + dA B~."""
    a, b = _rand(n, 12), S.rng(12, 1).uniform(0, 1, (n, n))
    _, m, _, _ = O.cd_matmul(a, b, k, full=True)
    m3 = O.cd_matmul_alg3(a, b, k)
    assert np.abs(m - m3).max() < 1e-12 * np.abs(m).max()


@pytest.mark.parametrize("n,k", [(16, 2), (16, 5), (15, 4), (32, 7)])
def test_real_part_is_never_worse(n, k):
    """Reading R5: a selection that splits a conjugate pair makes M complex; AB is real, so
    ||AB - Re M||^2 = ||AB - M||^2 - ||Im M||^2 exactly, and the product returned (Re M) is never
    further from AB than M.  Random data ranks the components apart, so the pair split is forced
    through the selection argument."""
    a, b = _rand(n, 40 + k), S.rng(41 + k, 1).uniform(0, 1, (n, n))
    sel = np.array([0] + [1 + j for j in range(k - 1)], dtype=np.int64)  # 1..k-1 without partners
    re_m, m, _, _ = O.cd_matmul(a, b, k, sel_a=sel, sel_b=sel, full=True)
    exact = a @ b
    im = np.linalg.norm(m.imag)
    assert im > 1e-6 * np.linalg.norm(m)  # the split pairs leave an imaginary part
    e_re, e_c = np.linalg.norm(exact - re_m), np.linalg.norm(exact - m)
    assert e_re <= e_c
    assert abs(e_re ** 2 - (e_c ** 2 - im ** 2)) <= 1e-10 * e_c ** 2


def _truncs(method, a, b, k, seed=0):
    n = a.shape[1]
    if method == "svd":
        return O.truncate_rsvd(a, k, S.sketch(a.shape[1], k, seed, 0)), O.truncate_rsvd(b, k, S.sketch(b.shape[1], k, seed, 1))
    if method == "fourier":
        return O.truncate_fourier_left(a, k), O.truncate_fourier_right(b, k)
    return O.truncate(method, a, k), O.truncate(method, b, k)


@pytest.mark.parametrize("method", ["circulant", "svd", "fourier", "cycle"])
def test_untruncated_is_exact(method):
    """k = n keeps every component: M = AB for every decomposition."""
    n = 16
    a, b = _rand(n, 13), _rand(n, 14)
    ta, tb = _truncs(method, a, b, n)
    assert np.abs(O.product(method, ta, tb) - O.exact_product_loops(a, b)).max() < 1e-12 * np.abs(a @ b).max()


@pytest.mark.parametrize("method", ["circulant", "svd", "fourier", "cycle"])
@pytest.mark.parametrize("k", [1, 3, 6])
def test_first_order_identity(method, k):
    """Eq. (2.1)-(2.3): AB - M = dA dB exactly (the dropped second-order term)."""
    n = 12
    a, b = _rand(n, 15), S.rng(15, 1).uniform(0, 1, (n, n))
    ta, tb = _truncs(method, a, b, k)
    m = O.first_order(ta, tb)
    assert np.abs((a @ b - m) - ta.resid @ tb.resid).max() < 1e-12 * np.abs(a @ b).max()


_MIXED = [(x, y) for x in ("circulant", "svd", "fourier", "cycle") for y in ("circulant", "svd", "fourier", "cycle")
          if x != y]


def _trunc_side(method, x, k, side, seed):
    if method == "svd":
        return O.truncate_rsvd(x, k, S.sketch(x.shape[1], k, seed, 0 if side == "left" else 1))
    return O.truncate(method, x, k, side=side)


@pytest.mark.parametrize("ma,mb", _MIXED)
def test_mixed_untruncated_is_exact(ma, mb):
    """Mixed methods, k = n on both sides: M = AB."""
    n = 16
    a, b = _rand(n, 40), _rand(n, 41)
    ta, tb = _trunc_side(ma, a, n, "left", 40), _trunc_side(mb, b, n, "right", 40)
    assert np.abs(O.mixed_product(ta, tb) - O.exact_product_loops(a, b)).max() < 1e-12 * np.abs(a @ b).max()


@pytest.mark.parametrize("ma,mb", _MIXED)
def test_mixed_first_order_identity(ma, mb):
    """Mixed methods: AB - M = dA dB (Eq. (2.1)-(2.3)) with each side's own truncation, and the real
    part equals Re(A~) B + Re(dA) Re(B~) - Im(dA) Im(B~) term by term."""
    n, k = 16, 5
    a, b = _rand(n, 42), S.rng(42, 1).uniform(0, 1, (n, n))
    ta, tb = _trunc_side(ma, a, k, "left", 42), _trunc_side(mb, b, k, "right", 42)
    m = O.first_order(ta, tb)
    assert np.abs((a @ b - m) - ta.resid @ tb.resid).max() < 1e-12 * np.abs(a @ b).max()
    split = ta.approx.real @ b + ta.resid.real @ tb.approx.real - ta.resid.imag @ tb.approx.imag
    assert np.abs(O.mixed_product(ta, tb) - split).max() < 1e-12 * np.abs(a @ b).max()


def test_fourier_space_form_equals_transform_form():
    """Alg. 5's transform-domain product equals Eq. (2.3) with A_s = A~_a W and B_s = W^* B~_a."""
    n, k = 16, 3
    a, b = _rand(n, 43), _rand(n, 44)
    ta, tb = O.truncate_fourier_left(a, k), O.truncate_fourier_right(b, k)
    assert np.abs(O.product("fourier", ta, tb) - O.first_order(ta, tb).real).max() < 1e-12 * np.abs(a @ b).max()


def test_exact_product_loops():
    a, b = _rand(5, 16, m=3), _rand(4, 17, m=5)
    assert np.abs(O.exact_product_loops(a, b) - a @ b).max() < 1e-14


# --------------------------------------------------------------------------- SVD

def test_rsvd_rank_r_is_exact():
    """Alg. 1 on a rank-r matrix with k >= r reproduces it (range finder captures the range)."""
    n, r = 40, 5
    g = S.rng(18, 0)
    a = g.standard_normal((n, r)) @ g.standard_normal((r, n))
    tr = O.truncate_rsvd(a, 8, S.sketch(n, 8, 18, 0))
    assert np.abs(tr.resid).max() < 1e-11 * np.abs(a).max()


def test_exact_svd_eckart_young_tail():
    """Section 2.2: ||dA||_F = (||A||_F^2 - sum_{i<=k} sigma_i^2)^{1/2}, sigma known from the generator."""
    n = 60
    sig = np.exp(-np.arange(n) / 8.0)
    a = S.spectrum_matrix(sig, S.rng(19, 0))
    for k in (3, 10, 25):
        tr = O.truncate_svd_exact(a, k)
        assert abs(np.linalg.norm(tr.resid) - math.sqrt(np.sum(sig[k:] ** 2))) < 1e-12
        assert np.allclose(tr.S, sig, atol=1e-12)


def test_rsvd_sigma_interlacing():
    """Alg. 1: singular values of Q^T A never exceed those of A."""
    n = 64
    sig = np.exp(-np.arange(n) / 6.0)
    a = S.spectrum_matrix(sig, S.rng(20, 0))
    u, s, v, q = O.rsvd(a, 10, S.sketch(n, 10, 20, 0))
    assert np.all(s <= sig[:10] * (1 + 1e-12))
    assert np.abs(q.T @ q - np.eye(10)).max() < 1e-13


# --------------------------------------------------------------------------- bounds

def test_thm38_svd_residual_bound():
    """Thm 3.8: ||dA dB||_F^2 <= ||dA||_2 ||dB||_2 ||dA||_F ||dB||_F for best rank-k residuals."""
    n = 50
    a = S.type2(n, S.rng(21, 0))
    b = S.type2(n, S.rng(21, 1))
    for k in (2, 8, 20):
        ta, tb = O.truncate_svd_exact(a, k), O.truncate_svd_exact(b, k)
        lhs = np.linalg.norm(ta.resid @ tb.resid) ** 2
        rhs = (np.linalg.norm(ta.resid, 2) * np.linalg.norm(tb.resid, 2) *
               np.linalg.norm(ta.resid) * np.linalg.norm(tb.resid))
        assert lhs <= rhs * (1 + 1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_thm312_cd_residual_bound(seed):
    """Thm 3.12: ||dA dB||_F <= (mu_A mu_B)^{1/4} n^{-1/2} ||dA||_F ||dB||_F (Def. 3.11 for mu)."""
    n = 32
    g = S.rng(22 + seed, 0)
    a = g.standard_normal((n, n)) + 2.0
    b = S.toeplitz_uniform(n, g) + 0.1 * g.standard_normal((n, n))
    for k in (1, 4, 9):
        _, _, ta, tb = O.cd_matmul(a, b, k, full=True)
        na, nb = np.linalg.norm(ta.resid), np.linalg.norm(tb.resid)
        mua = O.mu_circulant(ta.R, ta.sel, na ** 2)
        mub = O.mu_circulant(tb.R, tb.sel, nb ** 2)
        assert np.linalg.norm(ta.resid @ tb.resid) <= (mua * mub) ** 0.25 / math.sqrt(n) * na * nb * (1 + 1e-12)


# --------------------------------------------------------------------------- sparsifiers

def test_fourier_unitary_parseval():
    """Thm 2.3 / Section 2.4: A W^* preserves the Frobenius norm (sum_k a_k^2 = ||A||_F^2)."""
    a = _rand(10, 23, m=7)
    assert abs(np.linalg.norm(a @ O.unitary_W(10).conj().T) - np.linalg.norm(a)) < 1e-13


def test_fourier_topk_rows_optimal():
    """Alg. 4: per row the kept k entries minimise the row residual (unitary W => ||dA|| = ||dA~||)."""
    n, k = 7, 3
    a = _rand(n, 24, m=4)
    tr = O.truncate_fourier_left(a, k)
    for i in range(4):
        row = tr.T[i]
        best = min(np.linalg.norm(np.delete(row, list(sub))) for sub in itertools.combinations(range(n), k))
        assert np.linalg.norm(row[~tr.mask[i]]) <= best * (1 + 1e-12)
        assert np.linalg.norm(tr.resid[i]) == pytest.approx(np.linalg.norm(row[~tr.mask[i]]), rel=1e-12)


def _fourier_columns_optimal(b, tr, k):
    """True when every column of the right Fourier truncation keeps exactly k entries of W B and
    those entries minimise the column's residual among all k-subsets (brute force), measured in
    the space domain through W^* (||(B - B_s) e_j|| = ||(W B - B~_a) e_j||, W unitary)."""
    n = b.shape[0]
    w = O.unitary_W(n)
    bt = w @ b
    for j in range(b.shape[1]):
        kept = np.nonzero(tr.mask[:, j])[0]
        if len(kept) != k:
            return False
        best = math.inf
        for sub in itertools.combinations(range(n), k):
            z = np.zeros(n, dtype=np.complex128)
            z[list(sub)] = bt[list(sub), j]
            best = min(best, float(np.linalg.norm(b[:, j] - np.conj(w).T @ z)))
        if np.linalg.norm(tr.resid[:, j]) > best * (1 + 1e-10) + 1e-14:
            return False
    return True


@pytest.mark.parametrize("n,p,k", [(7, 5, 2), (8, 6, 3), (6, 9, 1)])
def test_fourier_topk_columns_optimal(n, p, k):
    """Section 2.4 / Alg. 5 (reading R8): the right operand keeps the top k entries of every COLUMN
    of W B; per column these minimise the column residual (brute force over all k-subsets)."""
    b = _rand(n, 27, m=p).T.copy()       # n x p, p != n so a row / column mix-up changes shapes
    tr = O.truncate_fourier_right(b, k)
    assert _fourier_columns_optimal(b, tr, k)
    # ||dB||_F^2 is the sum of the dropped column energies of W B (Parseval per column)
    dropped = sum(float(np.sum(np.abs(tr.T[~tr.mask[:, j], j]) ** 2)) for j in range(p))
    assert np.linalg.norm(tr.resid) ** 2 == pytest.approx(dropped, rel=1e-12)


def test_fourier_conjugate_ties_mirrored():
    """Reading R8: |A~(i,q)| and |A~(i,n-q)| tie exactly; the lower index wins the tie."""
    n = 8
    a = _rand(n, 25, m=3)
    tr = O.truncate_fourier_left(a, 1)
    mag = O.magnitudes_mirrored_rows(tr.T)
    assert all(mag[i, q] == mag[i, n - q] for i in range(3) for q in range(1, n))
    for i in range(3):
        q = int(np.nonzero(tr.mask[i])[0][0])
        assert q <= n // 2


@pytest.mark.parametrize("k", [1, 2, 4])
def test_cycle_topk_optimal(k):
    """Cycles are orthogonal (disjoint supports): the k largest cycles minimise ||dA||_F."""
    n = 6
    a = _rand(n, 26)
    acyc = O.cycle_layout(a)
    best = min(np.linalg.norm(np.delete(acyc, list(sub), axis=1)) for sub in itertools.combinations(range(n), k))
    assert np.linalg.norm(O.truncate_cycles(a, k).resid) <= best * (1 + 1e-12)


def test_cycle_apply_is_shift_and_scale():
    """Section 1.2.2: C^j Lambda_j B = row shift of B by j, rows scaled by the cycle entries."""
    n = 9
    a, b = _rand(n, 27), _rand(n, 28)
    acyc = O.cycle_layout(a)
    j = 4
    direct = O.cycle_matrices(a)[j][0] @ O.cycle_matrices(a)[j][1] @ b
    shifted = np.zeros_like(b)
    for r in range(n):
        shifted[r] = acyc[(r - j) % n, j] * b[(r - j) % n]
    assert np.abs(direct - shifted).max() < 1e-14


# --------------------------------------------------------------------------- backward

@pytest.mark.parametrize("method", ["circulant", "svd", "fourier", "cycle"])
def test_backward_matches_bruteforce(method):
    """Reading R10: closed-form gradients equal <G, M(E_ij)> over every basis matrix E_ij."""
    n, k = 5, 2
    g = S.rng(29, 0)
    a, b, gr = g.standard_normal((n, n)), g.standard_normal((n, n)), g.standard_normal((n, n))
    ta, tb = _truncs(method, a, b, k, seed=29)
    da, db = O.backward(method, ta, tb, gr)
    bda, bdb = O.brute_force_gradient(method, ta, tb, gr)
    assert np.abs(da - bda).max() < 1e-12 and np.abs(db - bdb).max() < 1e-12


_MIX3 = [(x, y) for x in ("circulant", "svd", "cycle") for y in ("circulant", "svd", "cycle") if x != y]


@pytest.mark.parametrize("ma,mb", _MIXED)
def test_mixed_backward_matches_bruteforce(ma, mb):
    """Reading R10 for operands of different methods: the closed-form gradients (each operand's own
    adjoint projector) equal <G, M(E_ij)> of the frozen mixed map over every basis matrix, and the
    frozen map at the operands themselves is the mixed product."""
    n, k = 6, 2
    g = S.rng(57, 0)
    a, b, gr = g.standard_normal((n, n)) + 0.3, g.standard_normal((n, n)), g.standard_normal((n, n))
    ta, tb = _trunc_side(ma, a, k, "left", 57), _trunc_side(mb, b, k, "right", 57)
    da, db = O.mixed_backward(ta, tb, gr)
    f = lambda x, y: np.sum(gr * O.frozen_mixed_product(ta, tb, x, y))
    assert abs(f(a, b) - np.sum(gr * O.mixed_product(ta, tb))) < 1e-10
    bda, bdb = np.zeros_like(a), np.zeros_like(b)
    for i, j in itertools.product(range(n), range(n)):
        e = np.zeros_like(a)
        e[i, j] = 1.0
        bda[i, j] = f(e, b) - f(np.zeros_like(a), b)
        bdb[i, j] = f(a, e) - f(a, np.zeros_like(b))
    assert np.abs(da - bda).max() < 1e-12 and np.abs(db - bdb).max() < 1e-12


def test_fourier_projector_is_the_truncation():
    """Section 2.4 with the element masks frozen: P(A) = A~ on both sides, P is idempotent, and the
    adjoint satisfies <Y, P(X)> = <P'(Y), X> for the plain (bilinear) pairing, on rectangular shapes."""
    g = S.rng(62, 0)
    a, b = g.standard_normal((5, 8)), g.standard_normal((8, 7))
    ta, tb = O.truncate_fourier_left(a, 3), O.truncate_fourier_right(b, 2)
    for t, x0, shape in ((ta, a, a.shape), (tb, b, b.shape)):
        assert np.abs(O.project(t, x0) - t.approx).max() < 1e-13
        x, y = g.standard_normal(shape), g.standard_normal(shape)
        px = O.project(t, x)
        assert np.abs(O.project(t, px) - px).max() < 1e-13
        assert abs(np.sum(y * px) - np.sum(O.project(t, y, adjoint=True) * x)) < 1e-12


def test_mixed_backward_same_method_reduces():
    """With both operands truncated by one method the mixed formula is that method's backward."""
    g = S.rng(58, 0)
    n = 8
    a, b, gr = g.standard_normal((n, n)), g.standard_normal((n, n)), g.standard_normal((n, n))
    for method in ("circulant", "svd", "cycle", "fourier"):
        ta, tb = _truncs(method, a, b, 3, seed=58)
        da, db = O.mixed_backward(ta, tb, gr)
        ra, rb = O.backward(method, ta, tb, gr)
        assert np.abs(da - ra).max() < 1e-12 and np.abs(db - rb).max() < 1e-12


def test_fourier_backward_asymmetric_masks_bruteforce():
    """Single-tone rows keep f but not n - f at k = 1 (exact tie, lower index first): the kept
    set is not mirror-symmetric, M is complex, and the gradient of Re M still matches brute force."""
    n = 8
    l = np.arange(n)
    a = np.stack([np.cos(2 * np.pi * (i % 3 + 1) * l / n) * (1 + i) for i in range(5)])
    g = S.rng(31, 0)
    b, gr = g.standard_normal((n, 6)), g.standard_normal((5, 6))
    ta, tb = O.truncate_fourier_left(a, 1), O.truncate_fourier_right(b, 2)
    assert not np.array_equal(ta.mask, ta.mask[:, (-np.arange(n)) % n])
    da, db = O.fourier_backward(ta, tb, gr)
    bda, bdb = O.brute_force_gradient("fourier", ta, tb, gr)
    assert np.abs(da - bda).max() < 1e-12 and np.abs(db - bdb).max() < 1e-12


@pytest.mark.parametrize("method", ["circulant", "svd", "fourier", "cycle"])
def test_backward_finite_differences_n64(method):
    """Central finite differences of the frozen map at n = 64 (FP64) along random directions."""
    n, k = 64, 6
    g = S.rng(30, 0)
    a, b, gr = g.standard_normal((n, n)), g.standard_normal((n, n)), g.standard_normal((n, n))
    ta, tb = _truncs(method, a, b, k, seed=30)
    da, db = O.backward(method, ta, tb, gr)
    for _ in range(2):
        ea, eb = g.standard_normal((n, n)), g.standard_normal((n, n))
        h = 1e-3
        f = lambda x, y: np.sum(gr * O.frozen_product(method, ta, tb, x, y))
        fd_a = (f(a + h * ea, b) - f(a - h * ea, b)) / (2 * h)
        fd_b = (f(a, b + h * eb) - f(a, b - h * eb)) / (2 * h)
        assert fd_a == pytest.approx(np.sum(da * ea), rel=1e-9)
        assert fd_b == pytest.approx(np.sum(db * eb), rel=1e-9)


# --------------------------------------------------------------------------- square blocks (R13)

_RAGGED = [(10, 13, 7, 4), (8, 8, 12, 4), (5, 16, 9, 8), (16, 16, 16, 16)]


@pytest.mark.parametrize("m,n,p,bs", _RAGGED)
def test_blocked_untruncated_is_exact(m, n, p, bs):
    """k = bs keeps every component of every padded block: the cropped product is AB exactly."""
    g = S.rng(m * n + p, 50)
    a, b = g.standard_normal((m, n)), g.standard_normal((n, p))
    ta = O.truncate_circulant_blocked(a, bs, bs)
    tb = O.truncate_circulant_blocked(b, bs, bs)
    assert np.abs(O.blocked_first_order(ta, tb) - O.exact_product_loops(a, b)).max() < 1e-12 * np.abs(a @ b).max()


@pytest.mark.parametrize("m,n,p,bs", _RAGGED)
@pytest.mark.parametrize("k", [1, 3])
def test_blocked_first_order_identity(m, n, p, bs, k):
    """Eq. (2.1)-(2.3) on the padded operands: AB - Re M = Re(dA dB) cropped; the padding is zero
    in A and B but not in their truncations, so a product formed without it fails this."""
    g = S.rng(m * n + p + k, 51)
    a, b = g.standard_normal((m, n)) + 0.5, g.uniform(0, 1, (n, p))
    ta = O.truncate_circulant_blocked(a, bs, k)
    tb = O.truncate_circulant_blocked(b, bs, k)
    second = (ta.resid @ tb.resid)[:m, :p].real
    assert np.abs((a @ b - O.blocked_first_order(ta, tb)) - second).max() < 1e-12 * np.abs(a @ b).max()


def test_blocked_one_shift_per_block_is_exact():
    """Block (I, J) = Re(circulant(c_IJ) D^(t_IJ)) holds only the conjugate pair t_IJ, bs - t_IJ of
    that block (Thm 2.1): k = 2 selects that pair in every block, the truncation is exact and
    M = AB.  A block grid read in the wrong order picks the wrong pairs."""
    bs, nbr, nbc = 8, 2, 3
    g = S.rng(52, 0)
    shifts = [[1 + (i + 2 * j) % 3 for j in range(nbc)] for i in range(nbr)]
    a = np.block([[(O.circulant(g.standard_normal(bs)) @ O.diag_D(bs, shifts[i][j])).real for j in range(nbc)]
                  for i in range(nbr)])
    ta = O.truncate_circulant_blocked(a, bs, 2)
    assert [sorted(int(v) for v in t) for t in ta.sel] == [[shifts[i][j], bs - shifts[i][j]] for i in range(nbr)
                                                           for j in range(nbc)]
    assert np.abs(ta.resid).max() < 1e-12 * np.abs(a).max()
    b = g.standard_normal((nbc * bs, 5))
    tb = O.truncate_circulant_blocked(b, bs, 2)
    assert np.abs(O.blocked_first_order(ta, tb) - a @ b).max() < 1e-12 * np.abs(a @ b).max()


def test_blocked_truncation_error_is_parseval_per_block():
    """Section 2.3 per block: ||dA||^2 = sum over blocks of ||A_IJ||^2 - bs sum_{t in S_IJ} T_IJ[t]^2."""
    bs, k = 8, 3
    a = S.rng(53, 0).standard_normal((13, 21))
    ta = O.truncate_circulant_blocked(a, bs, k)
    total = 0.0
    for row in ta.blocks:
        for t in row:
            total += np.sum(t.a ** 2) - bs * np.sum(t.keys[t.sel] ** 2)
    assert abs(np.linalg.norm(ta.resid) ** 2 - total) < 1e-10 * np.sum(a * a)


def test_blocked_single_block_is_the_square_decomposition():
    """bs = n on a square operand: one block, the truncation of Alg. 3 itself."""
    n, k = 16, 5
    a = _rand(n, 54)
    tb, ts = O.truncate_circulant_blocked(a, n, k), O.truncate_circulant(a, k)
    assert np.array_equal(tb.sel[0], ts.sel) and np.abs(tb.approx - ts.approx).max() < 1e-14


@pytest.mark.parametrize("mb", ["svd", "fourier", "cycle"])
def test_blocked_mixed_identity(mb):
    """A blockwise circulant left operand times another method's right operand: AB - Re M =
    Re(dA dB) cropped, with the other operand zero-padded along the inner dimension."""
    m, n, p, bs, k = 11, 16, 16, 8, 3
    g = S.rng(55, 0)
    a, b = g.standard_normal((m, n)), g.uniform(0, 1, (n, p))
    ta = O.truncate_circulant_blocked(a, bs, k)
    tb = _trunc_side(mb, b, k, "right", 55)
    second = (ta.resid[:, :n] @ tb.resid)[:m, :].real
    assert np.abs((a @ b - O.blocked_first_order(ta, tb)) - second).max() < 1e-12 * np.abs(a @ b).max()


def test_blocked_backward_matches_bruteforce():
    """Reading R10 + R13: the blockwise gradients equal <G, M(E_ij)> over every basis matrix."""
    m, n, p, bs, k = 5, 7, 6, 4, 2
    g = S.rng(56, 0)
    a, b, gr = g.standard_normal((m, n)), g.standard_normal((n, p)), g.standard_normal((m, p))
    ta, tb = O.truncate_circulant_blocked(a, bs, k), O.truncate_circulant_blocked(b, bs, k)
    da, db = O.cd_backward_blocked(ta, tb, gr)
    f = lambda x, y: np.sum(gr * O.frozen_product_blocked(ta, tb, x, y))
    bda = np.zeros_like(a)
    bdb = np.zeros_like(b)
    for i, j in itertools.product(range(m), range(n)):
        e = np.zeros_like(a)
        e[i, j] = 1.0
        bda[i, j] = f(e, b) - f(np.zeros_like(a), b)
    for i, j in itertools.product(range(n), range(p)):
        e = np.zeros_like(b)
        e[i, j] = 1.0
        bdb[i, j] = f(a, e) - f(a, np.zeros_like(b))
    assert np.abs(da - bda).max() < 1e-12 and np.abs(db - bdb).max() < 1e-12
    # the frozen map at the operands themselves is the product
    assert np.abs(f(a, b) - np.sum(gr * O.blocked_first_order(ta, tb))) < 1e-10


@pytest.mark.parametrize("other", ["svd", "fourier", "cycle"])
@pytest.mark.parametrize("blocked_left", [True, False])
def test_blocked_mixed_backward_matches_bruteforce(other, blocked_left):
    """Readings R10 + R13 for a blockwise circulant operand beside another method: the gradients
    equal <G, M(E_ij)> of the frozen padded-and-cropped map over every basis matrix, and the frozen
    map at the operands themselves is the blocked mixed product (ragged blocks on both sides)."""
    bs, k = 4, 2
    m, n, p = (5, 6, 6) if other == "cycle" else (5, 6, 7)
    if other == "cycle" and not blocked_left:
        m = 6
    g = S.rng(58, int(blocked_left))
    a, b, gr = g.standard_normal((m, n)) + 0.3, g.standard_normal((n, p)), g.standard_normal((m, p))
    if blocked_left:
        ta, tb = O.truncate_circulant_blocked(a, bs, k), _trunc_side(other, b, k, "right", 58)
    else:
        ta, tb = _trunc_side(other, a, k, "left", 58), O.truncate_circulant_blocked(b, bs, k)
    da, db = O.blocked_mixed_backward(ta, tb, gr)
    assert da.shape == (m, n) and db.shape == (n, p)
    f = lambda x, y: np.sum(gr * O.frozen_blocked_mixed_product(ta, tb, x, y))
    assert abs(f(a, b) - np.sum(gr * O.blocked_first_order(ta, tb))) < 1e-10
    bda, bdb = np.zeros_like(a), np.zeros_like(b)
    for i, j in itertools.product(range(m), range(n)):
        e = np.zeros_like(a)
        e[i, j] = 1.0
        bda[i, j] = f(e, b) - f(np.zeros_like(a), b)
    for i, j in itertools.product(range(n), range(p)):
        e = np.zeros_like(b)
        e[i, j] = 1.0
        bdb[i, j] = f(a, e) - f(a, np.zeros_like(b))
    assert np.abs(da - bda).max() < 1e-12 and np.abs(db - bdb).max() < 1e-12


# --------------------------------------------------------------------------- printed tables

def _table_rows():
    rows = []
    with open(os.path.join(GOLDEN, "paper_tables_n700.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t, pair, method, order, tol, s, expect = line.split()
                rows.append((int(t), pair, method, order, float(tol), int(s), expect))
    return rows


_MAKERS = {"general": S.general_uniform, "toeplitz": S.toeplitz_uniform, "type1": S.type1}


@pytest.mark.slow
def test_paper_tables_n700():
    """Tables 1 and 2 (n = 700, k = ceil(s log2 n)): the printed error thresholds."""
    n = 700
    cache = {}
    for table, pair, method, order, tol, s, expect in _table_rows():
        if pair not in cache:
            x, y = pair.split(",")
            a, b = _MAKERS[x](n, S.rng(0, 0)), _MAKERS[y](n, S.rng(0, 1))
            cache[pair] = (a, b, a @ b)
        a, b, ex = cache[pair]
        k = math.ceil(s * math.log2(n))
        if method == "circulant":
            ta, tb = O.truncate_circulant(a, k), O.truncate_circulant(b, k)
        elif method == "rsvd":
            ta, tb = O.truncate_rsvd(a, k, S.sketch(n, k, 0, 0)), O.truncate_rsvd(b, k, S.sketch(n, k, 0, 1))
        else:
            ta, tb = O.truncate_svd_exact(a, k), O.truncate_svd_exact(b, k)
        m = O.first_order(ta, tb) if order == "first" else ta.approx @ tb.approx
        err = O.rel_fro(m.real, ex)
        ok = err <= tol if expect == "le" else err > tol
        assert ok, (table, pair, method, order, tol, s, expect, err)


# --------------------------------------------------------------------------- planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Plant plausible mistakes in the oracle (CPU) and check that a pin above fails for each."""
    n = 8
    a = _rand(n, 31)

    # 1) wrong sign of omega in D: Thm 2.1 reconstruction breaks
    good_D = OA.diag_D
    monkeypatch.setattr(OA, "diag_D", lambda nn, k=1: np.conj(good_D(nn, k)))
    R = O.circulant_spectrum(a)
    assert np.abs(O.reconstruct_explicit(R, range(n)) - a).max() > 1e-3
    monkeypatch.setattr(OA, "diag_D", good_D)

    # 2) cycle layout of the other form (Lambda_j C^j): the worked example pin breaks
    grids, _ = _read_example()
    aa = np.array([[100 + 10 * r + c for c in range(4)] for r in range(4)], dtype=np.float64)
    label = lambda v: "%d%d" % ((int(v) - 100) // 10, (int(v) - 100) % 10)
    assert [[label(v) for v in row] for row in O.cycle_layout_left(aa)] != grids["right"]

    # 3) dropped first-order term: the first-order identity breaks
    b = _rand(n, 32)
    ta, tb = O.truncate_circulant(a, 2), O.truncate_circulant(b, 2)
    zeroth = ta.approx @ tb.approx
    assert np.abs((a @ b - zeroth) - ta.resid @ tb.resid).max() > 1e-3

    # 4) backward projecting onto S instead of S-bar: brute force disagrees (unpaired selection)
    g = _rand(n, 33)
    k = next(k for k in range(1, n) if set(O.truncate_circulant(a, k).sel.tolist()) !=
             set(O.mirror(O.truncate_circulant(a, k).sel, n).tolist()))
    ta, tb = O.truncate_circulant(a, k), O.truncate_circulant(b, k)
    monkeypatch.setattr(OA, "mirror", lambda sel, nn: np.asarray(sel))
    da, _ = O.cd_backward(ta, tb, g)
    monkeypatch.undo()
    bda, _ = O.brute_force_gradient("circulant", ta, tb, g)
    assert np.abs(da - bda).max() > 1e-6

    # 5) blocked product that drops the padded part of the truncations (treats the padding of A~
    #    as zero): the first-order identity on a ragged shape breaks
    a5, b5 = S.rng(34, 0).standard_normal((10, 14)), S.rng(34, 1).uniform(0, 1, (14, 7))
    tab, tbb = O.truncate_circulant_blocked(a5, 4, 2), O.truncate_circulant_blocked(b5, 4, 2)
    cut = lambda t: O.Truncation(t.method, t.a, O.pad_to(t.approx[:t.shape0[0], :t.shape0[1]], *t.a.shape))
    ta5, tb5 = cut(tab), cut(tbb)
    ta5.shape0, tb5.shape0 = tab.shape0, tbb.shape0
    wrong = O.blocked_first_order(ta5, tb5)
    second = (tab.resid @ tbb.resid)[:10, :7].real
    assert np.abs((a5 @ b5 - wrong) - second).max() > 1e-3

    # 6) mixed backward projecting G B^T instead of G dB^T (the partner's operand in place of its
    #    residual): the brute-force gradient of the frozen mixed map disagrees.  (Projecting onto S
    #    instead of S-bar would not be a mistake here: the partner's residual is real, and on a real
    #    matrix the two projections have the same real part.)
    n6 = 6
    a6, b6, g6 = (S.rng(35, i).standard_normal((n6, n6)) for i in range(3))
    ta6 = O.truncate_circulant(a6, 3)
    tb6 = O.truncate_rsvd(b6, 2, S.sketch(n6, 2, 35, 1))
    tb_wrong = O.Truncation(tb6.method, tb6.a, tb6.approx, tb6.sel, Q=tb6.Q)
    tb_wrong.resid = tb6.a
    da6, _ = O.mixed_backward(ta6, tb_wrong, g6)
    f = lambda x: np.sum(g6 * O.frozen_mixed_product(ta6, tb6, x, b6))
    bda6 = np.zeros_like(a6)
    for i, j in itertools.product(range(n6), range(n6)):
        e = np.zeros_like(a6)
        e[i, j] = 1.0
        bda6[i, j] = f(e) - f(np.zeros_like(a6))
    assert np.abs(da6 - bda6).max() > 1e-6

    # 7) right Fourier truncation selecting per ROW of W B (per frequency, across columns) instead
    #    of per column: the brute-force column pin fails (Section 2.4, reading R8)
    b7 = _rand(8, 36, m=6).T.copy()
    good_right = OA.truncate_fourier_right

    def per_row(bb, kk, forced=None):
        bt = O.unitary_W(bb.shape[0]) @ bb
        mask = O.topk_mask_rows(np.abs(bt), kk)
        bt_a = np.where(mask, bt, 0)
        return O.Truncation("fourier", bb, np.conj(O.unitary_W(bb.shape[0])).T @ bt_a, None, T=bt, mask=mask,
                            T_a=bt_a)

    monkeypatch.setattr(OA, "truncate_fourier_right", per_row)
    assert not _fourier_columns_optimal(b7, OA.truncate_fourier_right(b7, 2), 2)
    monkeypatch.setattr(OA, "truncate_fourier_right", good_right)
    assert _fourier_columns_optimal(b7, OA.truncate_fourier_right(b7, 2), 2)

    # 8) spectral concentration mu (Def. 3.11) without the 1/n of the mean: the closed form
    #    mu(J) = n of the all-ones residue fails
    good_mu = OA.mu_circulant
    monkeypatch.setattr(OA, "mu_circulant", lambda R, sel, r2: good_mu(R, sel, r2) * R.shape[0])
    jn = np.ones((8, 8))
    assert OA.mu_circulant(O.circulant_spectrum(jn), [], 64.0) != pytest.approx(8.0)
    monkeypatch.setattr(OA, "mu_circulant", good_mu)
    assert OA.mu_circulant(O.circulant_spectrum(jn), [], 64.0) == pytest.approx(8.0)

    # 9) Fourier adjoint projector with the conjugations swapped ((M o (X W^*)) W instead of
    #    (M o (X W)) conj(W), i.e. the projector itself): the mixed backward leaves brute force once
    #    the partner's residual is complex (a circulant selection that splits a conjugate pair; on
    #    a real argument the two maps have the same real part)
    n9 = 6
    a9, b9, g9 = (S.rng(37, i).standard_normal((n9, n9)) for i in range(3))
    k9 = next(k for k in range(1, n9) if set(O.truncate_circulant(b9, k).sel.tolist()) !=
              set(O.mirror(O.truncate_circulant(b9, k).sel, n9).tolist()))
    ta9, tb9 = O.truncate_fourier_left(a9, 2), O.truncate_circulant(b9, k9)
    assert np.abs(tb9.resid.imag).max() > 1e-6
    good_project = OA.project
    monkeypatch.setattr(OA, "project", lambda t, x, adjoint=False: good_project(t, x, False)
                        if t.method == "fourier" else good_project(t, x, adjoint))
    da9, _ = OA.mixed_backward(ta9, tb9, g9)
    monkeypatch.setattr(OA, "project", good_project)
    f9 = lambda x: np.sum(g9 * O.frozen_mixed_product(ta9, tb9, x, b9))
    bda9 = np.zeros_like(a9)
    for i, j in itertools.product(range(n9), range(n9)):
        e = np.zeros_like(a9)
        e[i, j] = 1.0
        bda9[i, j] = f9(e) - f9(np.zeros_like(a9))
    assert np.abs(da9 - bda9).max() > 1e-6
    assert np.abs(OA.mixed_backward(ta9, tb9, g9)[0] - bda9).max() < 1e-12


# --------------------------------------------------------------------------- spectral concentration

@pytest.mark.parametrize("n", [8, 16, 33])
def test_mu_closed_forms(n):
    """Def. 3.11: mu = max_i X_i / mean_i X_i (the mean of X_i is ||dA||_F^2 / n by Parseval), so
    1 <= mu <= n.  Closed forms: a residue that is one cycle of ones (A = C^m, unit-modulus
    eigenvalues) has mu = 1; the all-ones residue J (eigenvalues n, 0, ..., 0) has mu = n; a
    residue alpha J + beta I has X_0 = (alpha n + beta)^2, X_i = beta^2 otherwise."""
    cm = np.linalg.matrix_power(O.cycle_perm(n), 3 % n)
    assert O.mu_circulant(O.circulant_spectrum(cm), [], float(n)) == pytest.approx(1.0, rel=1e-12)
    jn = np.ones((n, n))
    assert O.mu_circulant(O.circulant_spectrum(jn), [], float(n * n)) == pytest.approx(float(n), rel=1e-12)
    al, be = 0.7, 1.3
    x = al * jn + be * np.eye(n)
    x0, xi = (al * n + be) ** 2, be ** 2
    want = x0 / ((x0 + (n - 1) * xi) / n)
    assert O.mu_circulant(O.circulant_spectrum(x), [], float(np.linalg.norm(x) ** 2)) == pytest.approx(want, rel=1e-12)
    # a selection removes its components from X: Y = J + 2 C^3 D has component 0 = J and
    # component 1 = 2 C^3 (Thm 2.1); keeping 0 leaves 2 C^3 D (mu = 1), keeping 1 leaves J (mu = n)
    y = jn + 2.0 * (cm @ O.diag_D(n, 1))
    ry = O.circulant_spectrum(y)
    assert O.mu_circulant(ry, [0], 4.0 * n) == pytest.approx(1.0, rel=1e-12)
    assert O.mu_circulant(ry, [1], float(n * n)) == pytest.approx(float(n), rel=1e-12)
    g = S.rng(61, n)
    for k in (1, 3):
        a = g.standard_normal((n, n)) + 1.0
        t = O.truncate_circulant(a, k)
        mu = O.mu_circulant(t.R, t.sel, float(np.linalg.norm(t.resid) ** 2))
        assert 1.0 - 1e-12 <= mu <= n * (1 + 1e-12)


# --------------------------------------------------------------------------- error estimation

def test_posterior_estimate_tracks_observed_error():
    """Cor. 3.7: ||dA|| ||dB|| / (sqrt(n) ||M||) overlaps the observed relative error for the
    structured operands of Section 4 (General x Toeplitz with CD, Type-1 with rSVD)."""
    n = 512
    a, b = S.general_times_toeplitz(n, seed=0)
    for k in (1, 3, 5, 9):
        ta, tb = O.truncate("circulant", a, k), O.truncate("circulant", b, k)
        m = O.first_order(ta, tb)
        actual = np.linalg.norm(ta.resid @ tb.resid) / np.linalg.norm(a @ b)
        est = O.posterior_estimate(np.linalg.norm(ta.resid), np.linalg.norm(tb.resid), np.linalg.norm(m), n)
        assert 0.9 < est / actual < 1.1, (k, est, actual)
    a1, b1 = S.type1(n, S.rng(1, 0)), S.type1(n, S.rng(1, 1))
    for k in (8, 64):
        ta, tb = O.truncate_rsvd(a1, k, S.sketch(n, k, 0, 0)), O.truncate_rsvd(b1, k, S.sketch(n, k, 0, 1))
        m = O.first_order(ta, tb)
        actual = np.linalg.norm(ta.resid @ tb.resid) / np.linalg.norm(a1 @ b1)
        est = O.posterior_estimate(np.linalg.norm(ta.resid), np.linalg.norm(tb.resid), np.linalg.norm(m), n)
        assert 0.9 < est / actual < 1.2, (k, est, actual)


def test_posterior_constant_is_lemma31_by_monte_carlo():
    """Lemma 3.1: for A = Q1 D1 Q2 and B = Q3 D2 Q4 with Haar factors, E||AB||_F^2 equals
    ||D1||^2 ||D2||^2 / n, the square of the posterior estimate's constant (Cor. 3.7) applied to
    ||D1||, ||D2|| with ||M|| = 1.  Checked by Monte Carlo at n = 8 within four standard errors.
    The band uses the exact variance from the fourth moments of a real Haar orthogonal matrix
    (E q^4 = 3/(n(n+2)); two entries in one row or column 1/(n(n+2)); in neither
    (n+1)/((n-1)n(n+2))): the variance printed in the appendix assigns one value to every pair of
    distinct entries and is negative for D1 = D2 = I, where ||AB||^2 = n is deterministic."""
    n, trials = 8, 4000
    g = S.rng(7, 0)
    d1, d2 = np.exp(-np.arange(n) / 3.0), 1.0 + np.arange(n)
    s = np.empty(trials)
    for i in range(trials):
        q1, q2, q3, q4 = (S.haar_orthogonal(n, g) for _ in range(4))
        s[i] = np.sum((((q1 * d1) @ q2) @ ((q3 * d2) @ q4)) ** 2)
    al1, al2, be1, be2 = np.sum(d1 ** 2), np.sum(d2 ** 2), np.sum(d1 ** 4), np.sum(d2 ** 4)
    e4, erow, eoff = 3 / (n * (n + 2)), 1 / (n * (n + 2)), (n + 1) / ((n - 1) * n * (n + 2))
    es2 = (be1 * be2 * e4 + (be1 * (al2 ** 2 - be2) + (al1 ** 2 - be1) * be2) * erow
           + (al1 ** 2 - be1) * (al2 ** 2 - be2) * eoff)
    mean = al1 * al2 / n
    var = es2 - mean ** 2
    assert abs(s.var() / var - 1) < 0.1, (s.var(), var)
    assert abs(s.mean() - mean) <= 4 * math.sqrt(var / trials), (s.mean(), mean)
    est = O.posterior_estimate(math.sqrt(al1), math.sqrt(al2), 1.0, n)
    assert abs(est ** 2 - s.mean()) <= 4 * math.sqrt(var / trials)
    # the same moments at D1 = D2 = I give zero variance
    one = np.ones(n)
    a, b = np.sum(one), np.sum(one)
    v0 = b * b * e4 + 2 * b * (a * a - b) * erow + (a * a - b) ** 2 * eoff - (a * a / n) ** 2
    assert abs(v0) < 1e-12


# Mean and second moment of each distribution of the appendix's front-constant table.
_MOMENTS = {"uniform01": (0.5, 1 / 3), "rademacher": (0.0, 1.0), "normal01": (0.0, 1.0),
            "lognormal01": (math.exp(0.5), math.exp(2.0)), "student_t3": (0.0, 3.0)}


def _front_constant(mean, m2, n):
    """E||XY||^2 / (E||X||^2 E||Y||^2) for i.i.d. entries: each (XY)_ij sums n products with
    second moment m2^2 and n(n-1) cross terms with mean mean^4, so the ratio is
    1/n + (n-1) mean^4 / (n m2^2); c is its square root (the ratio concentrates as n grows)."""
    return math.sqrt(1 / n + (n - 1) * mean ** 4 / (n * m2 ** 2))


def test_front_constants_table():
    """The appendix's front constants agree with the closed form from the entry moments (within
    four printed sigmas at n = 5000) and with Monte Carlo at n = 400; for zero-mean entries the
    constant is the posterior estimate's 1/sqrt(n) (Cor. 3.7)."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "front_constants.txt")) if ln.strip() and not ln.startswith("#")]
    assert {r[0] for r in rows} == set(_MOMENTS)
    n = 5000
    for name, c, scaled, sigma in rows:
        c, sigma = float(c), float(sigma)
        closed = _front_constant(*_MOMENTS[name], n)
        printed = c / math.sqrt(n) if scaled == "1" else c
        assert abs(closed - printed) <= 4 * sigma, (name, closed, printed)
        if _MOMENTS[name][0] == 0.0:
            assert closed == pytest.approx(O.posterior_estimate(1.0, 1.0, 1.0, n), rel=1e-12)
    gens = {"uniform01": lambda g, s: g.uniform(0.0, 1.0, s),
            "rademacher": lambda g, s: g.choice([-1.0, 1.0], s),
            "normal01": lambda g, s: g.standard_normal(s),
            "lognormal01": lambda g, s: np.exp(g.standard_normal(s))}
    m, trials = 400, 5
    for name, gen in gens.items():
        g = S.rng(11, 0)
        r = np.empty(trials)
        for i in range(trials):
            x, y = gen(g, (m, m)), gen(g, (m, m))
            r[i] = np.linalg.norm(x @ y) / (np.linalg.norm(x) * np.linalg.norm(y))
        band = 4 * r.std(ddof=1) / math.sqrt(trials) + 1.0 / m ** 2
        assert abs(r.mean() - _front_constant(*_MOMENTS[name], m)) <= band, (name, r.mean())


def test_apriori_estimate_tracks_observed_error():
    """Section 2.5, before the product: with the front constants of the entries (3/4 for the U(0,1)
    operands; 1/sqrt(n) for the residues, zero-mean once the dominant component is kept) the a
    priori estimate predicts the observed error of General x Toeplitz within 5%; for Gaussian
    operands both constants are 1/sqrt(n) and the estimate is the ratio of the truncation errors."""
    n = 512
    a, b = S.general_times_toeplitz(n, seed=0)
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    for k in (1, 3, 5, 9):
        ta, tb = O.truncate("circulant", a, k), O.truncate("circulant", b, k)
        actual = np.linalg.norm(ta.resid @ tb.resid) / np.linalg.norm(a @ b)
        est = O.apriori_estimate(np.linalg.norm(ta.resid), np.linalg.norm(tb.resid), na, nb, 0.75, 1 / math.sqrt(n))
        assert 0.95 < est / actual < 1.05, (k, est, actual)
    n, k = 256, 32
    g = S.rng(n, 5)
    a, b = g.standard_normal((n, n)), g.standard_normal((n, n))
    for method in ("circulant", "cycle", "svd"):
        ta = O.truncate(method, a, k, phi=S.sketch(n, k, 5, 0))
        tb = O.truncate(method, b, k, phi=S.sketch(n, k, 5, 1))
        actual = np.linalg.norm(ta.resid @ tb.resid) / np.linalg.norm(a @ b)
        c = 1 / math.sqrt(n)
        est = O.apriori_estimate(np.linalg.norm(ta.resid), np.linalg.norm(tb.resid), np.linalg.norm(a),
                                 np.linalg.norm(b), c, c)
        assert 0.95 < est / actual < 1.05, (method, est, actual)


def test_best_method_special_cases():
    """Section 2.5: each input that one decomposition represents exactly with k = 2 components (a
    circulant matrix, rank 2, two cycles, one conjugate frequency pair per row) selects that
    decomposition: zero truncation error, every other method far from zero, in either order."""
    n = 32
    cases = S.two_structure_cases(n, S.rng(41, 0))
    order = ["circulant", "svd", "cycle", "fourier"]
    phi = S.sketch(n, 2, 41, 0)
    for want, a in cases.items():
        for methods in (order, order[::-1]):
            got, t = O.best_method(a, 2, methods, phi=phi)
            assert got == want, (want, methods, got)
            assert np.linalg.norm(t.resid) <= 1e-12 * np.linalg.norm(a)
        for other in order:
            if other != want:
                t = O.truncate(other, a, 2, phi=phi)
                assert np.linalg.norm(t.resid) > 1e-2 * np.linalg.norm(a), (want, other)


def test_refinement_identity():
    """Section 2.5 refinement (reading R16): AB - refine equals Re(dA2 dB2), the product of the
    second-level residues, for every pair of methods the library refines (complex first truncations
    included, where the exact Im dA Im dB term is needed); an untruncated second level gives AB."""
    n = 16
    g = S.rng(44, 0)
    a, b = g.standard_normal((n, n)) + 0.5, g.standard_normal((n, n)) + 0.5
    ab = a @ b
    scale = np.abs(ab).max()
    pairs = [("circulant", "circulant"), ("svd", "svd"), ("cycle", "cycle"), ("svd", "circulant"),
             ("fourier", "circulant"), ("circulant", "cycle"), ("fourier", "svd")]
    complex_seen = False
    for ma, mb in pairs:
        ta = O.truncate(ma, a, 3, phi=S.sketch(n, 3, 44, 0), side="left")
        tb = O.truncate(mb, b, 3, phi=S.sketch(n, 3, 44, 1), side="right")
        ta2 = O.truncate(ma, ta.resid.real, 2, phi=S.sketch(n, 2, 45, 0), side="left")
        tb2 = O.truncate(mb, tb.resid.real, 2, phi=S.sketch(n, 2, 45, 1), side="right")
        r = O.refine(ta, tb, ta2, tb2)
        assert np.abs((ab - r) - (ta2.resid @ tb2.resid).real).max() <= 1e-12 * scale, (ma, mb)
        if np.abs(ta.resid.imag).max() > 0.1 and np.abs(tb.resid.imag).max() > 0.1:
            complex_seen = True
            wrong = (O.first_order(ta, tb) + O.first_order(ta2, tb2)).real   # without Im dA Im dB
            assert np.abs((ab - wrong) - (ta2.resid @ tb2.resid).real).max() > 1e-3 * scale
        fa = O.truncate(ma, ta.resid.real, n, phi=S.sketch(n, n, 46, 0), side="left")
        fb = O.truncate(mb, tb.resid.real, n, phi=S.sketch(n, n, 46, 1), side="right")
        assert np.abs(O.refine(ta, tb, fa, fb) - ab).max() <= 1e-11 * scale, (ma, mb)
    assert complex_seen


def test_refinement_of_nested_truncations_is_the_larger_truncation():
    """For orthogonal components selected by magnitude (circulant, cycles, exact SVD) the top-k2 of
    a real residue are the next k2 components of the operand, so refining a k truncation by k2 has
    the error of the first-order product at k + k2: AB - refine = dA_{k+k2} dB_{k+k2}."""
    n = 64
    a, b = S.general_times_toeplitz(n, seed=3)
    ab = a @ b
    for method, k, k2 in (("circulant", 1, 4), ("cycle", 3, 5)):
        ta, tb = O.truncate(method, a, k), O.truncate(method, b, k)
        ta2, tb2 = O.truncate(method, ta.resid.real, k2), O.truncate(method, tb.resid.real, k2)
        big_a, big_b = O.truncate(method, a, k + k2), O.truncate(method, b, k + k2)
        err = ab - O.refine(ta, tb, ta2, tb2)
        assert np.abs(err - (big_a.resid @ big_b.resid).real).max() <= 1e-11 * np.abs(ab).max(), method
    ta, tb = O.truncate_svd_exact(a, 4), O.truncate_svd_exact(b, 4)
    ta2, tb2 = O.truncate_svd_exact(ta.resid, 3), O.truncate_svd_exact(tb.resid, 3)
    big_a, big_b = O.truncate_svd_exact(a, 7), O.truncate_svd_exact(b, 7)
    err = ab - O.refine(ta, tb, ta2, tb2)
    assert np.abs(err - big_a.resid @ big_b.resid).max() <= 1e-10 * np.abs(ab).max()


def test_product_wrappers_agree_with_the_pinned_forms():
    """The per-method product helpers the GPU tests call are the pinned first-order form on the
    truncations (transform-domain form for the Fourier sparsifier) and reproduce AB untruncated."""
    n, k = 32, 5
    g = S.rng(47, 0)
    a, b = g.standard_normal((n, n)) + 0.5, g.standard_normal((n, n)) + 0.5
    ab = a @ b
    tol = 1e-12 * np.abs(ab).max()
    pa, pb = S.sketch(n, k, 47, 0), S.sketch(n, k, 47, 1)
    got = {"circulant": O.cd_matmul(a, b, k).real, "svd": O.svd_matmul(a, b, k, pa, pb).real,
           "fourier": O.fourier_matmul(a, b, k), "cycle": O.cycle_matmul(a, b, k).real}
    for method, m in got.items():
        ta = O.truncate(method, a, k, phi=pa, side="left")
        tb = O.truncate(method, b, k, phi=pb, side="right")
        assert np.abs(m - O.product(method, ta, tb)).max() <= tol, method
    full = {"circulant": O.cd_matmul(a, b, n).real, "svd": O.svd_matmul(a, b, n, S.sketch(n, n, 1, 0),
                                                                          S.sketch(n, n, 1, 1)).real,
            "fourier": O.fourier_matmul(a, b, n), "cycle": O.cycle_matmul(a, b, n).real,
            "svd_exact": O.svd_matmul(a, b, n, None, None, exact=True).real}
    for method, m in full.items():
        assert np.abs(m - ab).max() <= 1e-11 * np.abs(ab).max(), method


def test_near_tie_protocol_sets():
    """The selection-parity protocol: keys within tau of the k-th key are ambiguous, the rest of the
    top k certain; an exact tie has boundary gap 0; k >= n has no boundary."""
    keys = np.array([5.0, 4.0, 3.0, 3.0, 2.0, 1.0])
    must, maybe = O.near_tie_sets(keys, 3, 1e-6)
    assert must == {0, 1} and maybe == {2, 3}
    assert O.boundary_gap(keys, 3) == 0.0
    assert O.boundary_gap(keys, 2) == pytest.approx(0.25)
    near = np.array([5.0, 4.0, 3.0, 3.0 * (1 - 1e-7), 2.0])
    must, maybe = O.near_tie_sets(near, 3, 1e-6)
    assert must == {0, 1} and maybe == {2, 3}
    must, maybe = O.near_tie_sets(near, 2, 1e-6)
    assert must == {0} and maybe == {1}
    assert O.near_tie_sets(keys, 6, 1e-6) == (set(range(6)), set())
    assert O.boundary_gap(keys, 6) == float("inf")
    # top_k: key descending, the lower index first among equal keys
    assert O.top_k(keys, 4).tolist() == [0, 1, 2, 3]
    assert O.top_k(np.array([1.0, 2.0, 2.0, 0.5]), 2).tolist() == [1, 2]


def test_cor39_flat_residue_svd_bound():
    """Cor. 3.9: when the singular values of dA and dB are all equal (a flat tail after the top k of
    the exact SVD), ||dA dB||_F <= ||dA||_F ||dB||_F / sqrt(n - k)."""
    n, k = 48, 6
    for t in range(5):
        g = S.rng(60, t)
        a = S.spectrum_matrix(np.concatenate([np.linspace(50, 10, k), np.ones(n - k)]), g)
        b = S.spectrum_matrix(np.concatenate([np.linspace(30, 5, k), np.full(n - k, 0.5)]), g)
        ta, tb = O.truncate_svd_exact(a, k), O.truncate_svd_exact(b, k)
        assert np.allclose(np.linalg.svd(ta.resid, compute_uv=False)[: n - k], 1.0)
        lhs = np.linalg.norm(ta.resid @ tb.resid)
        assert lhs <= np.linalg.norm(ta.resid) * np.linalg.norm(tb.resid) / math.sqrt(n - k) * (1 + 1e-12)


def test_cor314_circulant_residue_layout_bounds():
    """Cor. 3.14: ||dA dB||_F^2 <= ||dA_cyc||_2 ||dB_cyc||_2 ||dA||_F ||dB||_F and the 1 / infinity-norm
    form of it, with dA_cyc the cycle layout of the circulant residue, on every computed instance."""
    g = S.rng(50, 0)
    for trial in range(18):
        n = (16, 32, 64)[trial % 3]
        k = 1 + trial % (n // 4)
        if trial % 2:
            a, b = S.general_times_toeplitz(n, seed=trial)
        else:
            a, b = g.standard_normal((n, n)), g.uniform(0, 1, (n, n))
        da, db = O.truncate_circulant(a, k).resid, O.truncate_circulant(b, k).resid
        la, lb = O.cycle_layout(da), O.cycle_layout(db)
        fa, fb = np.linalg.norm(da), np.linalg.norm(db)
        lhs = np.linalg.norm(da @ db)
        assert lhs ** 2 <= np.linalg.norm(la, 2) * np.linalg.norm(lb, 2) * fa * fb * (1 + 1e-12)
        norms = [np.linalg.norm(x, o) for x in (la, lb) for o in (np.inf, 1)]
        assert lhs <= float(np.prod(norms)) ** 0.25 * math.sqrt(fa * fb) * (1 + 1e-12)


def test_posterior_estimate_bounds_gaussian_error():
    """Independent Gaussian operands: the estimate is an upper bound of the observed error."""
    n = 256
    g = S.rng(n, 0)
    a, b = g.standard_normal((n, n)), g.standard_normal((n, n))
    for method in ("circulant", "cycle"):
        ta, tb = O.truncate(method, a, n // 8), O.truncate(method, b, n // 8)
        m = O.first_order(ta, tb)
        actual = np.linalg.norm(ta.resid @ tb.resid) / np.linalg.norm(a @ b)
        est = O.posterior_estimate(np.linalg.norm(ta.resid), np.linalg.norm(tb.resid), np.linalg.norm(m), n)
        assert est >= actual
