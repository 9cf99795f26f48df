"""FP64 oracle: truncated decompositions and the first-order approximate product.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, __graft_entry__.smoke() and the CPU
baseline of bench.py; never by the product package.

Paper: Kar, Hariprasad, Sai Gowri, Venkatapathi, "Efficient approximations of matrix
multiplication using truncated decompositions" (arXiv 2504.19308).  Section numbers,
equations and algorithm numbers below are the paper's.

Readings taken where the paper is silent or inconsistent:
  R1  omega = e^{+2 pi i/n} as in Thm 2.1 (Lemma 3.10 uses the opposite sign).
  R2  The shift identity is W D^k W^* = C^k (Remark after Thm 2.1); the form printed in
      Section 2.3.2 with W^* and W swapped is taken as a typo.
  R3  Cycle form A = sum_j C^j Lambda_j (Eq. "rightdecomp", Alg. 7), not Lambda_j C^j.
  R4  FFT unnormalised forward, IFFT with 1/n; R = F A_cyc / n, L = F R (Alg. 2, Alg. 3).
  R5  For real A the components t and n-t are complex conjugates and tie exactly; top-k may
      split a pair, making M complex.  The product returned is Re(M); ||Im M|| is reported.
  R6  Top-k order is (key descending, index ascending).  Keys of conjugate partners are
      computed once (index <= n/2) and mirrored so the tie is exact.
  R7  rSVD: phi ~ N(0,1) supplied by the caller, no oversampling, no power iteration
      (Alg. 1 as printed).  Only A~ = Q Q^T A enters M, so QR/SVD signs do not matter.
  R8  Fourier sparsifier: top-k per ROW of A W^* and per COLUMN of W B (Section 2.4 text),
      constant k; magnitudes of conjugate partners mirrored as in R6.
  R9  Cycle sparsifier key: ||diag Lambda_j||_2 (by analogy with Alg. 3's component keys).
  R10 Backward: selections, Q factors and masks are frozen; the gradient is that of the
      resulting bilinear map.
  R13 Rectangular circulant operands: b x b blocks, ragged edge zero-padded, top-k per block,
      Eq. (2.3) on the padded operands, padded rows / columns of the product dropped.
  R16 Refinement of Section 2.5: the real parts of the residues are decomposed again and their
      first-order product added; the product of the imaginary parts is added exactly.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# ---------------------------------------------------------------------------
# Basic objects (Section 1.2.2, Thm 2.1)
# ---------------------------------------------------------------------------


def omega(n: int) -> complex:
    """omega = e^{+2 pi i / n} (Thm 2.1, reading R1)."""
    return np.exp(2j * np.pi / n)


def cycle_perm(n: int) -> np.ndarray:
    """C = [[0, 1], [I_{n-1}, 0]] (Eq. (1.1)): C[i, (i-1) mod n] = 1."""
    c = np.zeros((n, n))
    for i in range(n):
        c[i, (i - 1) % n] = 1.0
    return c


def diag_D(n: int, k: int = 1) -> np.ndarray:
    """D^k with D(q, q) = omega^q (Thm 2.1)."""
    q = np.arange(n)
    return np.diag(np.exp(2j * np.pi * ((k * q) % n) / n))


def dft_matrix(n: int) -> np.ndarray:
    """Unnormalised forward DFT F(p, q) = e^{-2 pi i pq / n} = sqrt(n) W (Section 2.3.1).

    The exponent is reduced mod n before the exponential so entries are exact to rounding.
    """
    p = np.arange(n)
    return np.exp(-2j * np.pi * ((p[:, None] * p[None, :]) % n) / n)


def unitary_W(n: int) -> np.ndarray:
    """W(p, q) = n^{-1/2} e^{-2 pi i pq/n} (Remark after Thm 2.1)."""
    return dft_matrix(n) / math.sqrt(n)


def fft_cols(x: np.ndarray) -> np.ndarray:
    """F x along axis 0.  Explicit DFT matrix for small n, library FFT otherwise."""
    n = x.shape[0]
    if n <= 64:
        return dft_matrix(n) @ x
    return np.fft.fft(x, axis=0)


def ifft_cols(x: np.ndarray) -> np.ndarray:
    """F^{-1} x along axis 0 (1/n scaling, MATLAB convention)."""
    n = x.shape[0]
    if n <= 64:
        return np.conj(dft_matrix(n)) @ x / n
    return np.fft.ifft(x, axis=0)


def circulant(col: np.ndarray) -> np.ndarray:
    """Circulant matrix sum_j col[j] C^j: X[r, q] = col[(r - q) mod n] (first column = col)."""
    n = len(col)
    r = np.arange(n)[:, None]
    q = np.arange(n)[None, :]
    return np.asarray(col)[(r - q) % n]


# ---------------------------------------------------------------------------
# Cycle decomposition (Section 1.2.2; Appendix, Alg. 7 and the 4x4 example)
# ---------------------------------------------------------------------------


def cycle_layout(a: np.ndarray) -> np.ndarray:
    """A_cyc[l, j] = A((l + j) mod n, l): column j holds the cycle Lambda_j of A = sum_j C^j Lambda_j.

    Appendix Alg. 7: A_cyc[i, j] = A^T[i, (i + j) mod n].  Written as the plain loop.
    """
    n = a.shape[0]
    assert a.shape == (n, n)
    if n > 64:  # same index map, written with index arrays for large n
        l = np.arange(n)[:, None]
        j = np.arange(n)[None, :]
        return a[(l + j) % n, l]
    out = np.zeros((n, n), dtype=a.dtype)
    for j in range(n):
        for l in range(n):
            out[l, j] = a[(l + j) % n, l]
    return out


def cycle_layout_left(a: np.ndarray) -> np.ndarray:
    """Cycles for the other form A = sum_j Lambda_j C^j (Appendix Eq. get_At1): [l, j] = A(l, (l-j) mod n)."""
    n = a.shape[0]
    out = np.zeros((n, n), dtype=a.dtype)
    for j in range(n):
        for l in range(n):
            out[l, j] = a[l, (l - j) % n]
    return out


def from_cycle_layout(acyc: np.ndarray) -> np.ndarray:
    """Inverse of cycle_layout: A((l + j) mod n, l) = A_cyc[l, j]."""
    n = acyc.shape[0]
    out = np.zeros((n, n), dtype=acyc.dtype)
    if n > 64:
        l = np.arange(n)[:, None]
        j = np.arange(n)[None, :]
        out[(l + j) % n, l] = acyc
        return out
    for j in range(n):
        for l in range(n):
            out[(l + j) % n, l] = acyc[l, j]
    return out


def cycle_matrices(a: np.ndarray):
    """[(C^j, Lambda_j)] with A = sum_j C^j Lambda_j (Eq. rightdecomp)."""
    n = a.shape[0]
    c = cycle_perm(n)
    acyc = cycle_layout(a)
    out = []
    cj = np.eye(n)
    for j in range(n):
        out.append((cj.copy(), np.diag(acyc[:, j])))
        cj = c @ cj
    return out


# ---------------------------------------------------------------------------
# Circulant decomposition (Thm 2.1, Thm 2.5, Alg. 2)
# ---------------------------------------------------------------------------


def circulant_spectrum(a: np.ndarray) -> np.ndarray:
    """R[k, j] = r_{j,k} = (1/n) sum_l e^{-2 pi i k l/n} Lambda_j(l, l)  (Thm 2.1 proof, Alg. 2).

    Column FFTs of the cycle layout divided by n.  Row k is R_A[k], the first column of R_k.
    Works for complex input as well (used by the backward projector).
    """
    n = a.shape[0]
    return fft_cols(cycle_layout(a).astype(np.complex128)) / n


def component_dense(R: np.ndarray, k: int) -> np.ndarray:
    """R_k D^k as a dense complex matrix, R_k = sum_j r_{j,k} C^j (Thm 2.1)."""
    n = R.shape[0]
    return circulant(R[k]) @ diag_D(n, k)


def reconstruct_explicit(R: np.ndarray, sel) -> np.ndarray:
    """sum_{t in sel} R_t D^t, summing explicitly formed dense components (Thm 2.1)."""
    n = R.shape[0]
    out = np.zeros((n, n), dtype=np.complex128)
    for t in sel:
        out += component_dense(R, int(t))
    return out


def reconstruct(R: np.ndarray, sel) -> np.ndarray:
    """sum_{t in sel} R_t D^t via the cycles: Lambda_j(c) = sum_{t in sel} r_{j,t} omega^{t c}.

    Same definition as reconstruct_explicit, evaluated cycle by cycle (a matrix product with
    the Vandermonde rows omega^{t c}); used where n is too large for dense components.
    """
    n = R.shape[0]
    sel = np.asarray(list(sel), dtype=np.int64)
    if sel.size == 0:
        return np.zeros((n, n), dtype=np.complex128)
    c = np.arange(n)
    vand = np.exp(2j * np.pi * ((sel[:, None] * c[None, :]) % n) / n)  # [t, c] = omega^{t c}
    lam = R[sel].T @ vand                                                 # [j, c] = Lambda_j(c)
    return from_cycle_layout(lam.T)                                       # cycle layout is [l=c, j]


def component_keys(R: np.ndarray) -> np.ndarray:
    """T[k] = ||R_A[k]||_2 (the keys of Alg. 3), evaluated for k <= n/2 and mirrored (reading R6)."""
    n = R.shape[0]
    t = np.zeros(n)
    for k in range(n // 2 + 1):
        t[k] = math.sqrt(float(np.sum(np.abs(R[k]) ** 2)))
    for k in range(n // 2 + 1, n):
        t[k] = t[n - k]
    return t


def eigen_spectrum(R: np.ndarray, t: int) -> np.ndarray:
    """L_t = sqrt(n) W R_A[t] = F R_A[t], the eigenvalues of R_t (Alg. 3)."""
    return fft_cols(R[t].reshape(-1, 1)).ravel()


# ---------------------------------------------------------------------------
# Selection (Alg. 3, Alg. 4) -- reading R6
# ---------------------------------------------------------------------------


def top_k(keys: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k largest keys, ordered by (key descending, index ascending)."""
    keys = np.asarray(keys, dtype=np.float64)
    idx = np.arange(len(keys))
    order = np.lexsort((idx, -keys))  # last key is primary
    return order[: min(k, len(keys))].astype(np.int64)


def boundary_gap(keys: np.ndarray, k: int) -> float:
    """Relative gap between the k-th and (k+1)-th largest keys (0 for an exact tie).

    A selection is only bit-reproducible across precisions when this gap exceeds the key
    error of the lower precision; the GPU parity tests use it to flag near-ties.
    """
    s = np.sort(np.asarray(keys, dtype=np.float64))[::-1]
    if k <= 0 or k >= len(s):
        return float("inf")
    top = max(s[k - 1], 1e-300)
    return float((s[k - 1] - s[k]) / top)


def near_tie_sets(keys: np.ndarray, k: int, tau: float):
    """(must, maybe): indices certainly selected, and the ambiguous set around the boundary.

    Keys within relative distance tau of the k-th largest key are 'maybe'.
    """
    keys = np.asarray(keys, dtype=np.float64)
    order = top_k(keys, len(keys))
    if k >= len(keys):
        return set(order.tolist()), set()
    kth = keys[order[k - 1]]
    band = np.abs(keys - kth) <= tau * max(abs(kth), 1e-300)
    maybe = set(np.nonzero(band)[0].tolist())
    must = set(i for i in order[:k].tolist() if i not in maybe)
    return must, maybe


# ---------------------------------------------------------------------------
# Truncations
# ---------------------------------------------------------------------------


class Truncation:
    """A = A~ + dA for one operand, with the data the product and backward need."""

    def __init__(self, method, a, approx, sel=None, **extra):
        self.method = method
        self.a = a
        self.approx = approx            # A~ (complex for circulant / Fourier)
        self.resid = a - approx         # dA
        self.sel = sel
        self.__dict__.update(extra)


def truncate_circulant(a: np.ndarray, k: int, selection=None) -> Truncation:
    """A~ = sum_{t in S} R_t D^t with S = top-k of T (Alg. 2, then Alg. 3's keys and selection)."""
    R = circulant_spectrum(a)
    keys = component_keys(R)
    sel = np.asarray(selection, dtype=np.int64) if selection is not None else top_k(keys, k)
    approx = reconstruct(R, sel) if a.shape[0] > 32 else reconstruct_explicit(R, sel)
    return Truncation("circulant", a, approx, sel, R=R, keys=keys)


def rsvd(a: np.ndarray, k: int, phi: np.ndarray):
    """Randomized partial SVD, Alg. 1: Y = A phi; Q R = qr(Y); X = Q^T A; U S V^T = svd(X); U <- Q U."""
    y = a @ phi
    q, _ = np.linalg.qr(y)
    x = q.T @ a
    ux, s, vt = np.linalg.svd(x, full_matrices=False)
    return q @ ux, s, vt.T, q


def truncate_rsvd(a: np.ndarray, k: int, phi: np.ndarray) -> Truncation:
    """A~ = U Sigma V^T from Alg. 1 (Section 2.2)."""
    u, s, v, q = rsvd(a, k, phi)
    approx = (u * s[None, :]) @ v.T
    return Truncation("svd", a, approx, None, U=u, S=s, V=v, Q=q)


def truncate_svd_exact(a: np.ndarray, k: int) -> Truncation:
    """Best rank-k approximation from the full SVD (Section 1.2.1, Eckart-Young)."""
    u, s, vt = np.linalg.svd(a)
    approx = (u[:, :k] * s[None, :k]) @ vt[:k]
    return Truncation("svd_exact", a, approx, None, U=u[:, :k], S=s, V=vt[:k].T, Q=u[:, :k])


def magnitudes_mirrored_rows(x: np.ndarray) -> np.ndarray:
    """|x[i, q]| with q > n/2 copied from n - q (conjugate partners of a real signal; R6/R8)."""
    n = x.shape[1]
    mag = np.abs(x)
    for q in range(n // 2 + 1, n):
        mag[:, q] = mag[:, n - q]
    return mag


def topk_mask_rows(mag: np.ndarray, k: int, forced=None) -> np.ndarray:
    """Alg. 4: keep the k largest entries of every row (ties: lower index first)."""
    m, n = mag.shape
    mask = np.zeros((m, n), dtype=bool)
    for i in range(m):
        sel = forced[i] if forced is not None else top_k(mag[i], k)
        mask[i, np.asarray(sel, dtype=np.int64)] = True
    return mask


def truncate_fourier_left(a: np.ndarray, k: int, forced=None) -> Truncation:
    """A~ = A W^* kept on its top-k entries per row (Alg. 5's row transforms and selection; Alg. 4)."""
    n = a.shape[1]
    at = a @ np.conj(unitary_W(n)).T
    mask = topk_mask_rows(magnitudes_mirrored_rows(at), k, forced)
    at_a = np.where(mask, at, 0)
    # space-domain form A_s = A~_a W, so that A_s B = A~_a (W B) (Alg. 5's first product)
    return Truncation("fourier", a, at_a @ unitary_W(n), None, T=at, mask=mask, T_a=at_a, side="left")


def truncate_fourier_right(b: np.ndarray, k: int, forced=None) -> Truncation:
    """B~ = W B kept on its top-k entries per column (Alg. 5's column transforms and selection; reading R8)."""
    n = b.shape[0]
    bt = unitary_W(n) @ b
    mask = topk_mask_rows(magnitudes_mirrored_rows(bt.T), k, forced).T
    bt_a = np.where(mask, bt, 0)
    # space-domain form B_s = W^* B~_a, so that dA B_s = (A~ - A~_a) B~_a (Alg. 5's second product)
    return Truncation("fourier", b, np.conj(unitary_W(n)).T @ bt_a, None, T=bt, mask=mask, T_a=bt_a, side="right")


def cycle_keys(a: np.ndarray) -> np.ndarray:
    """||diag Lambda_j||_2 for each cycle j (reading R9)."""
    acyc = cycle_layout(a)
    return np.sqrt(np.sum(np.abs(acyc) ** 2, axis=0))


def truncate_cycles(a: np.ndarray, k: int, selection=None) -> Truncation:
    """A_s = sum_{j in S} C^j Lambda_j, S = the k dominant cycles (Section 1.2.2, Section 4.3)."""
    n = a.shape[0]
    keys = cycle_keys(a)
    sel = np.asarray(selection, dtype=np.int64) if selection is not None else top_k(keys, k)
    acyc = cycle_layout(a)
    kept = np.zeros_like(acyc)
    kept[:, sel] = acyc[:, sel]
    return Truncation("cycle", a, from_cycle_layout(kept), sel, keys=keys)


# ---------------------------------------------------------------------------
# First-order products (Eq. (2.1)-(2.3); Section 2.2, Alg. 3, Alg. 5)
# ---------------------------------------------------------------------------


def exact_product_loops(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The triple loop A B (reference for the library matmul at small sizes)."""
    m, n = a.shape
    n2, p = b.shape
    assert n == n2
    out = np.zeros((m, p), dtype=np.result_type(a, b))
    for i in range(m):
        for j in range(p):
            s = 0.0
            for l in range(n):
                s += a[i, l] * b[l, j]
            out[i, j] = s
    return out


def first_order(ta: Truncation, tb: Truncation) -> np.ndarray:
    """M = A~ B + dA B~ (Eq. (2.3)); complex in general."""
    return ta.approx @ tb.a + ta.resid @ tb.approx


def cd_matmul(a, b, ka, kb=None, sel_a=None, sel_b=None, full=False):
    """Circulant first-order product (Alg. 3) evaluated with explicitly formed components.

    Returns Re(M) (reading R5), or (Re M, M, ta, tb) with full=True.
    """
    ta = truncate_circulant(a, ka, sel_a)
    tb = truncate_circulant(b, ka if kb is None else kb, sel_b)
    m = first_order(ta, tb)
    return (m.real, m, ta, tb) if full else m.real


def cd_matmul_alg3(a, b, ka, kb=None, sel_a=None, sel_b=None) -> np.ndarray:
    """Alg. 3 evaluated as printed (FFT form); returns the complex M.

    zeroth-order term:  M = IFFT( sum_t diag(L_A[t]) C^{In_A[t]} FFT(B) ),
    first-order term:   M += ( IFFT( sum_t (C^{In_B[t]})^* diag(conj L_B[t]) FFT(dA^*) ) )^*.
    (C^t Y)(p, :) = Y((p - t) mod n, :), i.e. np.roll(Y, t, axis=0).
    """
    n = a.shape[0]
    kb = ka if kb is None else kb
    ta = truncate_circulant(a, ka, sel_a)
    tb = truncate_circulant(b, kb, sel_b)
    fb = fft_cols(b.astype(np.complex128))
    acc = np.zeros((n, b.shape[1]), dtype=np.complex128)
    for t in ta.sel:
        la = eigen_spectrum(ta.R, int(t))
        acc += la[:, None] * np.roll(fb, int(t), axis=0)
    m = ifft_cols(acc)
    fda = fft_cols(np.conj(ta.resid).T)
    acc = np.zeros_like(fda)
    for t in tb.sel:
        lb = eigen_spectrum(tb.R, int(t))
        acc += np.roll(np.conj(lb)[:, None] * fda, -int(t), axis=0)
    m = m + np.conj(ifft_cols(acc)).T
    return m


def svd_matmul(a, b, k, phi_a, phi_b, full=False, exact=False):
    """SVD first-order product (Section 2.2): M = A~ B + dA B~ with Alg. 1 on A and on B."""
    if exact:
        ta, tb = truncate_svd_exact(a, k), truncate_svd_exact(b, k)
    else:
        ta, tb = truncate_rsvd(a, k, phi_a), truncate_rsvd(b, k, phi_b)
    m = first_order(ta, tb)
    return (m, m, ta, tb) if full else m


def fourier_matmul(a, b, k, forced_a=None, forced_b=None, full=False):
    """Alg. 5: M = A~_a B~ + (A~ - A~_a) B~_a with A~ = A W^*, B~ = W B; returns Re(M)."""
    ta = truncate_fourier_left(a, k, forced_a)
    tb = truncate_fourier_right(b, k, forced_b)
    m = ta.T_a @ tb.T + (ta.T - ta.T_a) @ tb.T_a
    return (m.real, m, ta, tb) if full else m.real


def cycle_matmul(a, b, ka, kb=None, sel_a=None, sel_b=None, full=False):
    """Cycle sparsification: M = A_s B + dA B_s (Eq. (2.4)-(2.5) with the cycles of Section 1.2.2)."""
    ta = truncate_cycles(a, ka, sel_a)
    tb = truncate_cycles(b, ka if kb is None else kb, sel_b)
    m = first_order(ta, tb)
    return (m, m, ta, tb) if full else m


# ---------------------------------------------------------------------------
# Error quantities (Section 2.1, Section 3)
# ---------------------------------------------------------------------------


def rel_fro(x, ref) -> float:
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def mu_circulant(R: np.ndarray, sel, resid_fro2: float) -> float:
    """Spectral concentration mu (Def. 3.11): max_i X_i / (||dA||_F^2 / n), X_i = sum_{j not in S} |lambda_i(R_j)|^2."""
    n = R.shape[0]
    keep = np.ones(n, dtype=bool)
    keep[np.asarray(sel, dtype=np.int64)] = False
    lam = fft_cols(R.T)  # [i, j] = lambda_i(R_j)
    x = np.sum(np.abs(lam[:, keep]) ** 2, axis=1)
    return float(x.max() / (resid_fro2 / n))


def posterior_estimate(resid_a_fro, resid_b_fro, m_fro, n) -> float:
    """Cor. 3.7: E[||dA dB|| / ||AB||] ~ ||dA|| ||dB|| / (sqrt(n) ||M||)."""
    return float(resid_a_fro * resid_b_fro / (math.sqrt(n) * m_fro))


def apriori_estimate(resid_a_fro, resid_b_fro, a_fro, b_fro, c_ab, c_resid) -> float:
    """Section 2.5, a priori (before the product): E||dA dB|| ~ c_resid ||dA|| ||dB|| and
    E||AB|| ~ c_ab ||A|| ||B||, with front constants for independent entries (Section 3, appendix
    table): 1/sqrt(n) for zero mean, 3/4 for U(0,1)."""
    return float(c_resid * resid_a_fro * resid_b_fro / (c_ab * a_fro * b_fro))


def best_method(a: np.ndarray, k: int, methods, phi=None, side: str = "left"):
    """Section 2.5: the suitability of a decomposition at k components is its relative truncation
    error ||dA||_F / ||A||_F.  Returns (method, truncation) of the smallest; ties keep the earlier
    method of the list."""
    best = None
    for m in methods:
        t = truncate(m, a, k, phi=phi, side=side)
        r = float(np.linalg.norm(t.resid) / np.linalg.norm(a))
        if best is None or r < best[0]:
            best = (r, m, t)
    return best[1], best[2]


# ---------------------------------------------------------------------------
# Backward of the frozen first-order map (reading R10)
# ---------------------------------------------------------------------------


def project_circulant(z: np.ndarray, sel) -> np.ndarray:
    """P_S(Z) = sum_{t in S} R_t(Z) D^t: orthogonal projection onto the selected components."""
    return reconstruct(circulant_spectrum(z), sel)


def mirror(sel, n):
    return np.array([(n - int(t)) % n for t in sel], dtype=np.int64)


def cd_backward(ta: Truncation, tb: Truncation, g: np.ndarray):
    """Gradients of <G, Re M> for M = A~ B + dA B~ with frozen selections S_A, S_B.

    dA = Re[ G B~^T + P_{S_A-bar}(G dB^T) ],  dB = Re[ A~^T G + P_{S_B-bar}(dA^T G) ],
    where S-bar = {n - t} (the bilinear adjoint of P_S) and ^T is the plain transpose.
    """
    n = ta.a.shape[0]
    da = g @ tb.approx.T + project_circulant(g @ tb.resid.T, mirror(ta.sel, n))
    db = ta.approx.T @ g + project_circulant(ta.resid.T @ g, mirror(tb.sel, n))
    return da.real, db.real


def svd_backward(ta: Truncation, tb: Truncation, g: np.ndarray):
    """Same map for the SVD truncation: P_A(X) = Q_A Q_A^T X, P_B(X) = Q_B Q_B^T X (real, self-adjoint)."""
    qa, qb = ta.Q, tb.Q
    da = g @ tb.approx.T + qa @ (qa.T @ (g @ tb.resid.T))
    db = ta.approx.T @ g + qb @ (qb.T @ (ta.resid.T @ g))
    return da, db


def project_cycles(z: np.ndarray, sel) -> np.ndarray:
    """Orthogonal projection onto the selected cycles."""
    zc = cycle_layout(z)
    kept = np.zeros_like(zc)
    kept[:, sel] = zc[:, sel]
    return from_cycle_layout(kept)


def cycle_backward(ta: Truncation, tb: Truncation, g: np.ndarray):
    da = g @ tb.approx.T + project_cycles(g @ tb.resid.T, ta.sel)
    db = ta.approx.T @ g + project_cycles(ta.resid.T @ g, tb.sel)
    return da, db


def fourier_backward(ta: Truncation, tb: Truncation, g: np.ndarray):
    """For M = P_A(A W^*) W B + (A W^* - P_A(A W^*)) P_B(W B) with frozen element masks.

    dA = Re[ (P_A(G dB~^T) + G B~_a^T) conj(W) ],  dB = Re[ W (A~_a^T G + P_B(dA~^T G)) ].
    """
    n = ta.a.shape[1]
    w = unitary_W(n)
    dbt = tb.T - tb.T_a
    dat = ta.T - ta.T_a
    da = (np.where(ta.mask, g @ dbt.T, 0) + g @ tb.T_a.T) @ np.conj(w)
    db = w @ (ta.T_a.T @ g + np.where(tb.mask, dat.T @ g, 0))
    return da.real, db.real


def frozen_product(method: str, ta: Truncation, tb: Truncation, a, b) -> np.ndarray:
    """Evaluate the frozen first-order map at new operands (a, b); real part.

    The projectors of ta/tb (selections, Q factors, masks) are kept; only the operands change.
    Used for finite differences and brute-force gradients.
    """
    n = a.shape[1]
    if method == "circulant":
        pa = project_circulant(a.astype(np.complex128), ta.sel)
        pb = project_circulant(b.astype(np.complex128), tb.sel)
    elif method == "svd":
        pa = ta.Q @ (ta.Q.T @ a)
        pb = tb.Q @ (tb.Q.T @ b)
    elif method == "cycle":
        pa = project_cycles(a, ta.sel)
        pb = project_cycles(b, tb.sel)
    elif method == "fourier":
        w = unitary_W(n)
        at = a @ np.conj(w).T
        bt = w @ b
        at_a = np.where(ta.mask, at, 0)
        bt_a = np.where(tb.mask, bt, 0)
        return (at_a @ bt + (at - at_a) @ bt_a).real
    else:
        raise ValueError(method)
    return (pa @ b + (a - pa) @ pb).real


def truncate(method: str, a, k, phi=None, selection=None, side="left"):
    if method == "circulant":
        return truncate_circulant(a, k, selection)
    if method == "svd":
        return truncate_rsvd(a, k, phi)
    if method == "cycle":
        return truncate_cycles(a, k, selection)
    if method == "fourier":
        return truncate_fourier_left(a, k, selection) if side == "left" else truncate_fourier_right(a, k, selection)
    raise ValueError(method)


def product(method: str, ta: Truncation, tb: Truncation) -> np.ndarray:
    """Re(M) for any method from its two truncations."""
    if method == "fourier":
        return (ta.T_a @ tb.T + (ta.T - ta.T_a) @ tb.T_a).real
    return first_order(ta, tb).real


def mixed_product(ta: Truncation, tb: Truncation) -> np.ndarray:
    """Re(M) when A and B are truncated by different methods (Section 1: the decompositions of the
    two operands may differ).  Eq. (2.3) with each side's space-domain truncation; for the
    Fourier sparsifier that is A_s = A~_a W (left) or B_s = W^* B~_a (right)."""
    return first_order(ta, tb).real


def refine(ta: Truncation, tb: Truncation, ta2: Truncation, tb2: Truncation) -> np.ndarray:
    """Section 2.5 (after the posterior estimate): when Re M is not accurate enough, the residue
    product dA dB is approximated by the same first-order approach and added.  For real A, B,
    Re(dA dB) = Re dA Re dB - Im dA Im dB.  Reading R16: ta2, tb2 truncate Re dA (m x n) and
    Re dB (n x p), their first-order product stands for the first term, and the second term
    (non-zero only when both first truncations are complex) is added exactly."""
    return first_order(ta, tb).real + first_order(ta2, tb2).real - ta.resid.imag @ tb.resid.imag


# ---------------------------------------------------------------------------
# Rectangular operands in square circulant blocks (Section 2.3: the cycle decomposition is
# defined for square matrices and a rectangular one is handled in square blocks).  Reading R13:
# both dimensions are cut into b x b blocks, the ragged edge is padded with zeros, every block
# keeps its own top-k components, Eq. (2.3) is evaluated on the padded operands and the padded
# rows / columns of the product are dropped.
# ---------------------------------------------------------------------------


def pad_to(a: np.ndarray, rows: int, cols: int) -> np.ndarray:
    """a in the top-left corner of a zero rows x cols matrix."""
    out = np.zeros((rows, cols), dtype=np.result_type(a, np.float64))
    out[: a.shape[0], : a.shape[1]] = a
    return out


def ceil_to(x: int, b: int) -> int:
    return -(-x // b) * b


def truncate_circulant_blocked(a: np.ndarray, bs: int, k: int, selections=None) -> Truncation:
    """Blockwise circulant truncation (reading R13).  Block (I, J) is rows I*bs.. and columns
    J*bs.. of the zero-padded operand; `selections[I * nbc + J]` replaces its top-k selection.
    The Truncation holds the PADDED operand and truncation; .shape0 is the original shape and
    .blocks[I][J] the per-block truncations."""
    ap = pad_to(a, ceil_to(a.shape[0], bs), ceil_to(a.shape[1], bs))
    nbr, nbc = ap.shape[0] // bs, ap.shape[1] // bs
    approx = np.zeros(ap.shape, dtype=np.complex128)
    blocks, sels = [], []
    for i in range(nbr):
        row = []
        for j in range(nbc):
            sel = None if selections is None else selections[i * nbc + j]
            t = truncate_circulant(ap[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs], k, sel)
            approx[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = t.approx
            row.append(t)
            sels.append(t.sel)
        blocks.append(row)
    return Truncation("circulant_blocked", ap, approx, np.array(sels), blocks=blocks, bs=bs, shape0=a.shape)


def padded(t: Truncation, rows: int, cols: int) -> Truncation:
    """The same truncation seen on the operand padded with zeros to rows x cols: the padding is
    zero in A, in A~ and in dA (true for every method: a zero row or column of A stays zero in
    Q Q^T A, A P, and in the sparsifier and cycle truncations of the padded square)."""
    out = Truncation(t.method, pad_to(t.a, rows, cols), pad_to(t.approx, rows, cols), t.sel)
    out.shape0 = getattr(t, "shape0", t.a.shape)
    return out


def blocked_first_order(ta: Truncation, tb: Truncation) -> np.ndarray:
    """Re M of Eq. (2.3) where either operand may be a blockwise circulant truncation (reading
    R13): both are brought to the common padded shape, M is formed there and cropped to m x p."""
    m0 = getattr(ta, "shape0", ta.a.shape)[0]
    p0 = getattr(tb, "shape0", tb.a.shape)[1]
    rows, inner, cols = ta.a.shape[0], max(ta.a.shape[1], tb.a.shape[0]), tb.a.shape[1]
    pa, pb = padded(ta, rows, inner), padded(tb, inner, cols)
    return first_order(pa, pb)[:m0, :p0].real


def project_circulant_blocked(z: np.ndarray, t: Truncation, adjoint: bool = False) -> np.ndarray:
    """Blockwise projection onto the selected components of every block (the adjoint keeps the
    mirrored components n - t of each block, as for one square block)."""
    bs = t.bs
    out = np.zeros(z.shape, dtype=np.complex128)
    for i, row in enumerate(t.blocks):
        for j, tt in enumerate(row):
            sel = mirror(tt.sel, bs) if adjoint else tt.sel
            out[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = project_circulant(
                z[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs], sel)
    return out


def cd_backward_blocked(ta: Truncation, tb: Truncation, g: np.ndarray):
    """Gradients of <G, Re M> for the blockwise circulant product with the selections frozen:
    the formulas of cd_backward on the padded operands with the blockwise adjoint projectors;
    G is padded with zeros (the padded part of M is dropped) and the gradients are cropped."""
    m0, n0 = ta.shape0
    p0 = tb.shape0[1]
    gp = pad_to(g, ta.a.shape[0], tb.a.shape[1])
    da = gp @ tb.approx.T + project_circulant_blocked(gp @ tb.resid.T, ta, adjoint=True)
    db = ta.approx.T @ gp + project_circulant_blocked(ta.resid.T @ gp, tb, adjoint=True)
    return da[:m0, :n0].real, db[:n0, :p0].real


def frozen_product_blocked(ta: Truncation, tb: Truncation, a, b) -> np.ndarray:
    """The blockwise circulant map with frozen selections evaluated at new operands (a, b)."""
    ap = pad_to(a, *ta.a.shape)
    bp = pad_to(b, *tb.a.shape)
    pa = project_circulant_blocked(ap.astype(np.complex128), ta)
    pb = project_circulant_blocked(bp.astype(np.complex128), tb)
    return (pa @ bp + (ap - pa) @ pb)[: ta.shape0[0], : tb.shape0[1]].real


def project(t: Truncation, x: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """The truncation's projector P (A~ = P(A)) applied to x, or its bilinear adjoint: circulant
    P_S / P_{S-bar}, SVD Q Q^T x (self-adjoint), cycles (self-adjoint), Fourier sparsifier with its
    element mask M frozen (Section 2.4): left P(X) = (M o (X W^*)) W, adjoint (M o (X W)) conj(W);
    right P(X) = W^* (M o (W X)), adjoint W (M o (conj(W) X)) (W is symmetric).  Reading R10."""
    if t.method == "fourier":
        w = unitary_W(x.shape[1] if t.side == "left" else x.shape[0])
        if t.side == "left":
            return np.where(t.mask, x @ (w if adjoint else np.conj(w).T), 0) @ (np.conj(w) if adjoint else w)
        return (w if adjoint else np.conj(w).T) @ np.where(t.mask, (np.conj(w) if adjoint else w) @ x, 0)
    if t.method == "circulant":
        n = x.shape[0]
        return project_circulant(x.astype(np.complex128), mirror(t.sel, n) if adjoint else t.sel)
    if t.method == "svd":
        return t.Q @ (t.Q.T @ x)
    if t.method == "cycle":
        return project_cycles(x, t.sel)
    raise ValueError(t.method)


def mixed_backward(ta: Truncation, tb: Truncation, g: np.ndarray):
    """Gradients of <G, Re M> for operands truncated by different methods (circulant, SVD, cycle,
    Fourier sparsifier), projectors frozen: the first-order map M = P_A(A) B + (A - P_A(A)) P_B(B) is bilinear, and
    dA = Re[G B~^T + P_A'(G dB^T)], dB = Re[A~^T G + P_B'(dA^T G)] with P' each operand's adjoint."""
    da = g @ tb.approx.T + project(ta, g @ tb.resid.T, adjoint=True)
    db = ta.approx.T @ g + project(tb, ta.resid.T @ g, adjoint=True)
    return np.real(da), np.real(db)


def _project_any(t: Truncation, x: np.ndarray, adjoint: bool = False) -> np.ndarray:
    if t.method == "circulant_blocked":
        return project_circulant_blocked(x.astype(np.complex128), t, adjoint)
    return project(t, x, adjoint)


def _adjoint_within(t: Truncation, y: np.ndarray) -> np.ndarray:
    """t's adjoint projector on the leading part of y that has t's operand shape (the padded shape
    of a blockwise circulant truncation), zero on the rest of y."""
    r, c = t.a.shape
    out = np.zeros(y.shape, dtype=np.complex128)
    out[:r, :c] = _project_any(t, y[:r, :c], adjoint=True)
    return out


def blocked_mixed_backward(ta: Truncation, tb: Truncation, g: np.ndarray):
    """Gradients of <G, Re M> when one operand is a blockwise circulant truncation and the other
    is truncated by another method (readings R10 and R13), projectors frozen.  M is formed on the
    common padded shape and cropped (blocked_first_order), so with G_p = G padded with zeros and
    both operands padded to that shape,
        dA = crop Re[G_p B~_p^T + P_A'(G_p dB_p^T)],   dB = crop Re[A~_p^T G_p + P_B'(dA_p^T G_p)],
    each adjoint acting on its own operand's shape (blockwise for the blocked one)."""
    m0, n0 = getattr(ta, "shape0", ta.a.shape)
    p0 = getattr(tb, "shape0", tb.a.shape)[1]
    rows, inner, cols = ta.a.shape[0], max(ta.a.shape[1], tb.a.shape[0]), tb.a.shape[1]
    pa, pb = padded(ta, rows, inner), padded(tb, inner, cols)
    gp = pad_to(g, rows, cols)
    da = gp @ pb.approx.T + _adjoint_within(ta, gp @ pb.resid.T)
    db = pa.approx.T @ gp + _adjoint_within(tb, pa.resid.T @ gp)
    return np.real(da)[:m0, :n0], np.real(db)[:n0, :p0]


def frozen_blocked_mixed_product(ta: Truncation, tb: Truncation, a, b) -> np.ndarray:
    """The mixed map with a blockwise circulant operand, projectors frozen, at new operands (a, b):
    each operand padded to its truncation's shape and projected, then both padded to the common
    shape, M formed there and cropped."""
    m0 = getattr(ta, "shape0", ta.a.shape)[0]
    p0 = getattr(tb, "shape0", tb.a.shape)[1]
    rows, inner, cols = ta.a.shape[0], max(ta.a.shape[1], tb.a.shape[0]), tb.a.shape[1]
    qa = pad_to(_project_any(ta, pad_to(a, *ta.a.shape)), rows, inner)
    qb = pad_to(_project_any(tb, pad_to(b, *tb.a.shape)), inner, cols)
    ap, bp = pad_to(a, rows, inner), pad_to(b, inner, cols)
    return np.real(qa @ bp + (ap - qa) @ qb)[:m0, :p0]


def frozen_mixed_product(ta: Truncation, tb: Truncation, a, b) -> np.ndarray:
    """The mixed first-order map with frozen projectors evaluated at new operands (a, b)."""
    pa, pb = project(ta, a), project(tb, b)
    return np.real(pa @ b + (a - pa) @ pb)


def backward(method: str, ta, tb, g):
    return {"circulant": cd_backward, "svd": svd_backward, "cycle": cycle_backward,
            "fourier": fourier_backward}[method](ta, tb, g)


def brute_force_gradient(method, ta, tb, g):
    """d<G, M>/dA and d/dB by evaluating the frozen map on every basis matrix (tiny n only)."""
    a, b = ta.a, tb.a
    da = np.zeros_like(a, dtype=np.float64)
    db = np.zeros_like(b, dtype=np.float64)
    zb = np.zeros_like(b)
    za = np.zeros_like(a)
    for i, j in itertools.product(range(a.shape[0]), range(a.shape[1])):
        e = np.zeros_like(a)
        e[i, j] = 1.0
        # the map is bilinear: M(a, b) = M1(a) b-terms; isolate the a-linear part at fixed b
        da[i, j] = np.sum(g * (frozen_product(method, ta, tb, e, b) - frozen_product(method, ta, tb, za, b)))
    for i, j in itertools.product(range(b.shape[0]), range(b.shape[1])):
        e = np.zeros_like(b)
        e[i, j] = 1.0
        db[i, j] = np.sum(g * (frozen_product(method, ta, tb, a, e) - frozen_product(method, ta, tb, a, zb)))
    return da, db
