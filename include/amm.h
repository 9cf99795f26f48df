/*
 * amm.h -- C ABI of libamm: approximate matrix multiplication from truncated
 * decompositions, evaluated in the first-order form
 *
 *        A B  ~=  M = A~ B + dA B~        (A = A~ + dA,  B = B~ + dB)
 *
 * of Kar, Hariprasad, Sai Gowri, Venkatapathi, "Efficient approximations of matrix
 * multiplication using truncated decompositions", arXiv 2504.19308, Eq. (2.1)-(2.3).
 * The dropped term is dA dB.  Implemented for one NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are row-major.  A "leading dimension" is the distance in elements
 *    between the starts of consecutive rows and must be >= the number of columns.
 *  - Every matrix pointer is a DEVICE pointer unless the argument name starts
 *    with host_.  The caller owns every matrix it passes in or out.
 *  - Calls are asynchronous on the CUDA stream passed as `stream` (a cudaStream_t;
 *    NULL is the legacy default stream).  Argument errors are detected on the host
 *    and returned before anything is launched; nothing is then modified.
 *  - No C++ exception crosses this boundary.  A non-OK status leaves a one-line
 *    reason readable with amm_last_error() (thread-local).
 *  - Device memory that a handle owns is allocated stream-ordered on the stream
 *    of amm_decompose() and released by amm_handle_destroy().
 *  - The product written to C (and the gradients) are real FP32.  Where a
 *    truncation keeps one of two complex-conjugate components but not the other,
 *    M is complex; the library returns Re(M) (real inputs make A B real, so the
 *    real part is never a worse approximation).
 *  - Devices: calls run on the calling thread's current CUDA device, and a handle
 *    must be used on the device it was made on.  Kernel attributes are set once per
 *    device; the SM count that sizes grids and K splits is read once per process
 *    (from the first device used), as are the autotuner's choices.
 */
#ifndef AMM_H
#define AMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMM_VERSION 7

typedef enum {
  AMM_OK = 0,
  AMM_ERR_INVALID_ARG = 1,      /* NULL pointer, bad enum, bad leading dimension, k out of range */
  AMM_ERR_UNSUPPORTED_SIZE = 2, /* size the kernels do not implement (e.g. non power-of-two FFT length) */
  AMM_ERR_OOM = 3,              /* a device allocation failed (or an injected failure fired) */
  AMM_ERR_CUDA = 4,             /* a CUDA runtime call or kernel launch failed */
  AMM_ERR_TIMEOUT = 5,          /* a bounded device-side wait gave up (batch scheduler) */
  AMM_ERR_STATE = 6,            /* handles do not fit together (role, shape, method) */
  AMM_ERR_NOT_IMPLEMENTED = 7   /* valid request for a feature the library does not provide */
} amm_status_t;

/* The truncated decompositions of the paper. */
typedef enum {
  AMM_SVD = 0,            /* randomized rank-k SVD, Alg. 1 (Section 2.2)                      */
  AMM_CIRCULANT = 1,      /* k leading circulant components R_t D^t, Thm 2.1, Alg. 2-3 (Sec. 2.3) */
  AMM_SPARSE_FOURIER = 2, /* top-k entries per row of A W^* / per column of W B, Alg. 4-5 (Sec. 2.4) */
  AMM_SPARSE_CYCLE = 3    /* k dominant cycles C^j Lambda_j (Section 1.2.2)                   */
} amm_method_t;

/* Element type of an input matrix, and arithmetic mode of the low-rank GEMMs. */
typedef enum { AMM_F32 = 0, AMM_BF16 = 1 } amm_dtype_t;

/* Which side of the product a handle stands for.  The first-order form is not
 * symmetric in A and B (A~ multiplies B; dA multiplies B~), so a decomposition
 * is made for one side. */
typedef enum { AMM_LEFT = 1, AMM_RIGHT = 2 } amm_role_t;

typedef struct amm_opts {
  uint32_t struct_size;           /* sizeof(amm_opts_t); set by amm_opts_init()             */
  int32_t role;                   /* amm_role_t; default AMM_LEFT                            */
  int32_t compute;                /* amm_dtype_t of the SVD GEMMs; default AMM_F32           */
  uint64_t seed;                  /* seed of the rSVD test matrix when `sketch` is NULL      */
  const float* sketch;            /* optional DEVICE pointer to phi (cols x k, row-major,
                                     N(0,1) entries) for AMM_SVD; copied at decompose time   */
  int32_t store_spectra;          /* AMM_CIRCULANT: 1 (default) keeps the half spectrum R
                                     ((n/2+1) x n complex; 64 MiB at n = 4096) and the key
                                     partials in the handle; 0 releases both when amm_decompose
                                     is done.  The product never reads R; the backward of
                                     the left operand's gradient dB, the dense residual of a
                                     mixed-method product, amm_handle_residual and
                                     amm_refine_product then compute R again from A, which the
                                     handle borrows (one more spectrum pass per call).  Results
                                     are identical either way.                                 */
  const int32_t* forced_selection;/* optional HOST array of k component indices that replaces
                                     the top-k selection (AMM_CIRCULANT, AMM_SPARSE_CYCLE);
                                     used to evaluate a selection exported elsewhere          */
  int32_t pair_closed;            /* AMM_CIRCULANT: 1 keeps the conjugate partner n - t of every
                                     selected component t as well (S u S-bar, at most 2k
                                     components; usually k or k + 1), which makes A~ real and
                                     M = Re M.  amm_handle_get_selection still returns the k
                                     ranked components; the truncation error of amm_handle_info
                                     is that of the closed set.  Default 0.                   */
  int32_t block;                  /* AMM_CIRCULANT: square block size b (a circulant length:
                                     2^a in [16, 16384] or 3 * 2^a in [48, 6144]) for a
                                     rectangular operand (Section 2.3: the
                                     cycle decomposition is defined for square matrices, larger
                                     or rectangular ones are taken in square blocks).  Both
                                     dimensions are cut into b x b blocks; a ragged edge is
                                     padded with zeros (a handle-owned copy); each block keeps
                                     its own top-k components; the product is Eq. (2.3) on the
                                     padded operands, padded rows / columns dropped.  forced_
                                     selection then holds k indices per block, blocks row-major,
                                     and amm_handle_get_selection returns them in that order.
                                     0 (default): one square decomposition.                   */
} amm_opts_t;

typedef struct amm_info {
  int32_t method, role, dtype;
  int64_t rows, cols, k;
  int64_t n_union;       /* circulant: |S u S-bar|, components applied with weights 1 or 1/2 */
  int64_t n_unpaired;    /* circulant: selected components whose conjugate partner was not   */
  double fro2;           /* ||A||_F^2 as seen by the decomposition (Parseval for circulant)  */
  double resid_fro2;     /* ||dA||_F^2 = ||A||_F^2 - ||A~||_F^2 (orthogonality, Sec. 2.3)    */
  double boundary_gap;   /* relative gap between the k-th and (k+1)-th keys (0 = exact tie)  */
} amm_info_t;

typedef struct amm_handle* amm_handle_t;

/* Human-readable name of a status.  Never NULL. */
const char* amm_status_string(amm_status_t status);

/* One-line reason for the last non-OK status returned on this thread ("" if none). */
const char* amm_last_error(void);

/* AMM_VERSION of the loaded library. */
int32_t amm_version(void);

/* Fill `opts` with defaults (role LEFT, F32, seed 0, no sketch, no forced selection). */
amm_status_t amm_opts_init(amm_opts_t* opts);

/*
 * Truncated decomposition of one operand (Section 2: A = sum_{i<k} A_i + dA).
 *
 *   A       device pointer, rows x cols row-major, leading dimension lda, element type
 *           `dtype`.  BORROWED: the handle keeps the pointer (the residual terms and the
 *           backward read A again), so A must stay allocated and unchanged until
 *           amm_handle_destroy().  (BF16 operands of AMM_SPARSE_FOURIER / AMM_SPARSE_CYCLE are
 *           read once: the handle keeps its own FP32 copy.)
 *   method  AMM_CIRCULANT and AMM_SPARSE_CYCLE need rows == cols (square, Section 2.3), except
 *           AMM_CIRCULANT with opts->block = b > 0, which takes any rows x cols in b x b blocks;
 *           lengths: circulant n (or b) any integer in [16, 4096], and above that 2^a up to
 *           16384 or 3 * 2^a up to 6144 (Thm 2.1 holds for every n: 2^a and 3 * 2^a run the fused
 *           Stockham kernels, every other length chirp-z (Bluestein) transforms with the steps
 *           between them as separate passes, slower); the Fourier sparsifier's inner dimension
 *           2^a in [16, 8192] or 3 * 2^a in [48, 6144]; cycle sparsifier n a multiple of 4 in
 *           [16, 8192].
 *   k       number of kept components (1 <= k <= min(rows, cols) for AMM_SVD; <= b per block
 *           for blocked AMM_CIRCULANT; <= n else).
 *   opts    may be NULL (defaults).
 *   stream  cudaStream_t for all work and allocations of this handle.
 *   out     receives the handle; unchanged on error.
 *
 * Circulant: computes the cycle spectrum R (Alg. 2) and then, following Alg. 3, the keys
 * T[t] = ||R_A[t]||_2, the top-k selection ordered by (key desc, index asc), the eigen-
 * spectra L_t = F R_A[t] of the selected components, and, for the RIGHT role, the dense
 * residual dB (for the other operand's first-order term).
 * SVD: Y = A phi, Q = orth(Y), X = Q^T A (Alg. 1, without the small SVD, which does not
 * change A~ = Q Q^T A).
 */
amm_status_t amm_decompose(const void* A, int64_t rows, int64_t cols, int64_t lda,
                           amm_dtype_t dtype, amm_method_t method, int64_t k,
                           const amm_opts_t* opts, void* stream, amm_handle_t* out);

/*
 * C = Re(M) = Re(A~ B + dA B~)  (Eq. (2.3); Alg. 3 for circulant; Section 2.2 for SVD).
 *
 *   hA      handle of A (role AMM_LEFT), hB handle of B (role AMM_RIGHT); A is m x n,
 *           B is n x p (inner dimensions must match).  The two methods may differ (the
 *           paper lets each operand use its own decomposition): C is then evaluated as
 *           Re(A~) B + (A - Re A~) Re(B~) + Im(A~) Im(B~), each term one operand's truncation
 *           applied to a dense matrix.  Mixed products need FP32 operands.  Blocked circulant
 *           operands (opts.block) need the same block size on both sides when both are
 *           circulant; the product is then the sum over inner blocks J of the square first-
 *           order products of blocks (I, J) and (J, L), and a non-circulant partner is padded
 *           with zeros along the shared dimension.
 *   C       device pointer, m x p FP32 row-major, leading dimension ldc >= p.  Overwritten.
 *   stream  stream of the call; must be ordered after the decompositions' streams.
 */
amm_status_t amm_approx_matmul(amm_handle_t hA, amm_handle_t hB, float* C, int64_t ldc,
                               void* stream);

/*
 * Gradients of L = <dC, Re M> with the truncation frozen (selections, Q factors and
 * masks held fixed; M is then bilinear in A and B):
 *     dA = Re[ dC B~^T + P_A'(dC dB^T) ],   dB = Re[ A~^T dC + P_B'(dA^T dC) ]
 * where P' is the adjoint projector onto the kept components.  Per method:
 *   AMM_SVD             P(X) = Q Q^T X; every term is a thin GEMM.
 *   AMM_CIRCULANT       P' keeps the components S-bar = {n - t : t in S} (the bilinear adjoint
 *                       of R_t D^t is R_{n-t} D^{n-t}); a component of dC dB^T or dA^T dC is
 *                       sampled from column / row spectra (an SDDMM over the kept t only).
 *   AMM_SPARSE_CYCLE    P' keeps the selected cycles (self-adjoint).
 *   AMM_SPARSE_FOURIER  dA = Re[(dC B~_a^T + P_A(dC dB~^T)) conj(W)],
 *                       dB = Re[W (A~_a^T dC + P_B(dA~^T dC))]  with the element masks P_A, P_B
 *                       (Alg. 5 differentiated with the masks frozen).
 *   Handles of different methods (any pair of SVD, circulant, cycle, Fourier; FP32):
 *                       the same formulas with each operand's own P' and the other operand's
 *                       residual dB = Re dB - i Im B~ (likewise dA), so beside the plain terms
 *                       Im P_A'(dC (Im B~)^T) and Im P_B'((Im A~)^T dC) enter when both
 *                       truncations can be complex (circulant with a split pair, Fourier).
 *                       Unblocked pairs need square operands (m = n = p).  With one operand in
 *                       circulant blocks (opts.block) M is formed on the zero-padded shape and
 *                       cropped: dC is padded with zeros, the blocked projection runs per block
 *                       on b-wide pieces of the inner sums and the gradients are cropped; any
 *                       m, n, p then, except a cycle partner (square).  Other shapes return
 *                       AMM_ERR_UNSUPPORTED_SIZE.
 *   dC  device m x p FP32 (lddc).  dA (m x n, ldda) and dB (n x p, lddb) are overwritten;
 *   either may be NULL to skip it.
 */
amm_status_t amm_approx_matmul_backward(amm_handle_t hA, amm_handle_t hB, const float* dC,
                                        int64_t lddc, float* dA, int64_t ldda, float* dB,
                                        int64_t lddb, void* stream);

/* Sizes, norms and selection statistics: ||A||_F^2 and the truncation error ||dA||_F^2 of
 * A = A~ + dA (Section 2, Eq. (2.1)), the gap at the top-k boundary (Alg. 3's selection).
 * Synchronises the handle's stream. */
amm_status_t amm_handle_info(amm_handle_t h, amm_info_t* info);

/*
 * Smallest k whose truncation meets a tolerance on the operand: ||dA||_F <= tol ||A||_F, with the
 * components kept in the order of amm_decompose (key desc, index asc).  The truncation error of
 * the top-k set follows from the keys alone because the components are orthogonal (circulant:
 * Thm 2.1 / Section 2.3, ||dA||^2 = ||A||^2 - n sum_{t in S} ||R_A[t]||^2; cycles: disjoint
 * supports).  Section 2.5 uses such truncation errors as the a-priori handle on the error of the
 * product (more components when the estimate is not satisfactory).
 *   A        DEVICE, n x n, lda, FP32 or BF16, n a length of the method (see amm_decompose)
 *   method   AMM_CIRCULANT or AMM_SPARSE_CYCLE (else AMM_ERR_NOT_IMPLEMENTED)
 *   tol      >= 0; *k_out in [1, n] (host)
 * Computes the spectrum / cycle norms into temporary device memory; synchronises `stream`.
 */
amm_status_t amm_choose_k(const void* A, int64_t rows, int64_t cols, int64_t lda, amm_dtype_t dtype,
                          amm_method_t method, double tol, void* stream, int64_t* k_out);

/*
 * Decompose A with the smallest k (up to k_max; k_max <= 0: no limit) whose truncation meets
 * ||dA||_F <= tol ||A||_F (Section 2.5: add components while the error estimate is not
 * satisfactory).  AMM_CIRCULANT / AMM_SPARSE_CYCLE: k from amm_choose_k (exact).  AMM_SVD /
 * AMM_SPARSE_FOURIER: k doubles from 8 until a trial decomposition meets the tolerance (its error
 * from amm_handle_info), then bisection inside the last bracket; each trial is a full
 * decomposition (with the same opts, so the same seed or sketch rule), and the returned handle is
 * the accepted trial.  When no k up to the cap meets tol, the handle at the cap is returned.
 * *out receives the handle and *k_out its k (host).  Synchronises `stream`.  Circulant blocks,
 * forced selections and caller sketches (opts->sketch, whose k is fixed) are rejected; the rSVD
 * cap is min(rows, cols, 1024).
 */
amm_status_t amm_decompose_to_tolerance(const void* A, int64_t rows, int64_t cols, int64_t lda, amm_dtype_t dtype,
                                        amm_method_t method, double tol, int64_t k_max, const amm_opts_t* opts,
                                        void* stream, amm_handle_t* out, int64_t* k_out);

/*
 * Posterior estimate of the relative error ||dA dB||_F / ||A B||_F of a computed product
 * (Corollary 3.7, Section 3): ||dA||_F ||dB||_F / (sqrt(n) ||C||_F), n the inner dimension,
 * with ||dA||_F, ||dB||_F the truncation errors of the two handles (amm_handle_info) and C the
 * product written by amm_approx_matmul (device, m x p, ldc).  For independent residue entries it
 * bounds the expected error; for structured operands it tracks the observed error.
 * Synchronises `stream` and both handles' streams; *estimate is a host double.
 */
amm_status_t amm_error_estimate(amm_handle_t hA, amm_handle_t hB, const float* C, int64_t ldc,
                                void* stream, double* estimate);

/*
 * A priori estimate of the relative error ||dA dB||_F / ||A B||_F before the product is formed
 * (Section 2.5; Lemma 3.1 and the statements after it for independent entries):
 *     c_resid ||dA||_F ||dB||_F / (c_ab ||A||_F ||B||_F),
 * with the truncation errors and norms of the two handles (amm_handle_info).  c_ab and c_resid
 * are the front constants of E||X Y||_F ~ c ||X||_F ||Y||_F for the operands and for the
 * residues: 1/sqrt(n) for zero-mean entries (n the inner dimension), 3/4 for U(0,1), 1/e for
 * exp(N(0,1)) (appendix table of front constants).  Both must be > 0.  A residue left after the
 * dominant component (the mean) is taken out has zero-mean entries, e.g. c_ab = 3/4 and
 * c_resid = 1/sqrt(n) for U(0,1) operands.  Synchronises both handles' streams; *estimate is a
 * host double.  AMM_ERR_STATE when ||A||_F ||B||_F = 0.
 */
amm_status_t amm_apriori_estimate(amm_handle_t hA, amm_handle_t hB, double c_ab, double c_resid,
                                  double* estimate);

/*
 * The most suitable decomposition of one operand at a given k (Section 2.5: the relative
 * truncation error ||dA||_F / ||A||_F of each decomposition at k components decides; A and B may
 * use different ones, Section 1 and Section 2.5).  Each method in host_methods[0 .. n_methods)
 * is decomposed with k and opts as by amm_decompose (opts->block is passed to AMM_CIRCULANT only),
 * its error read with amm_handle_info, and the handle with the smallest ||dA||_F^2 / ||A||_F^2
 * is kept (ties: the earlier candidate); the others are destroyed.  A candidate that rejects
 * this shape or k (AMM_ERR_UNSUPPORTED_SIZE / AMM_ERR_INVALID_ARG from amm_decompose, e.g. the
 * cycle sparsifier on a rectangular operand) is skipped; when every candidate is skipped, the
 * last one's status is returned.  Other errors end the call with nothing kept.  The truncation
 * error of a pair-closed circulant selection is that of the closed set, and that of a blocked
 * circulant operand includes its padding (the operand the product uses).
 *   host_methods  HOST array of amm_method_t values; n_methods >= 1
 *   opts          may be NULL; forced selections and caller sketches (per method) are rejected
 *   out           receives the kept handle; *method_out its method (host)
 * Synchronises `stream`.
 */
amm_status_t amm_decompose_best_method(const void* A, int64_t rows, int64_t cols, int64_t lda,
                                       amm_dtype_t dtype, const int32_t* host_methods,
                                       int32_t n_methods, int64_t k, const amm_opts_t* opts,
                                       void* stream, amm_handle_t* out, int32_t* method_out);

/*
 * Re dA = A - Re A~ of a handle (the residue of A = A~ + dA, Section 2, Eq. (2.1)) as a dense FP32
 * matrix (rows x cols, leading dimension ldd >=
 * cols, DEVICE, caller-owned, overwritten): the residue that amm_refine_product's second-level
 * decompositions take.  FP32 operands without circulant blocks (else AMM_ERR_NOT_IMPLEMENTED).
 * Asynchronous on `stream`, which must be ordered after the handle's stream.
 */
amm_status_t amm_handle_residual(amm_handle_t h, float* D, int64_t ldd, void* stream);

/*
 * Refinement of a computed product (Section 2.5: when the estimated error is not small enough,
 * approximate dA dB by the same approach and add it).  For real A and B,
 *     Re(dA dB) = Re dA Re dB - Im(A~) Im(B~),
 * and
 *     C += Re(A2~ Re dB + dA2 B2~) - Im(A~) Im(B~),
 * where hA2 (role LEFT, rows x cols of A) and hB2 (role RIGHT, the shape of B) are decompositions,
 * by any methods and k, of Re dA and Re dB as written by amm_handle_residual(hA) / (hB), and the
 * last term (zero unless both truncations can be complex: circulant with a split conjugate pair,
 * Fourier sparsifier) is exact.  Then A B - C = Re(dA2 dB2), the product of the second-level
 * residues.  C (m x p, ldc, DEVICE) must hold Re M of hA, hB (amm_approx_matmul) on entry.  hA and
 * hB: FP32, no circulant blocks (else AMM_ERR_NOT_IMPLEMENTED).  That hA2 / hB2 decompose the
 * residues is the caller's contract; shapes and roles are checked (AMM_ERR_STATE).  Asynchronous
 * on `stream`, which must be ordered after the four handles' streams.
 */
amm_status_t amm_refine_product(amm_handle_t hA, amm_handle_t hB, amm_handle_t hA2, amm_handle_t hB2,
                                float* C, int64_t ldc, void* stream);

/*
 * Copy the selection to host memory: circulant component indices / cycle indices in
 * selection order (k entries; Alg. 3, Section 1.2.2); for AMM_SPARSE_FOURIER the kept frequencies of every row
 * (left operand, rows x k) or column (right operand, cols x k), ascending within each (Alg. 4).
 * `cap` is the capacity of host_idx in elements; *count receives the number written.
 * Synchronises the handle's stream.
 */
amm_status_t amm_handle_get_selection(amm_handle_t h, int32_t* host_idx, int64_t cap,
                                      int64_t* count);

/*
 * Copy the component keys to host memory: for AMM_CIRCULANT T[t] = ||R_A[t]||_2, t = 0..n-1 (Alg. 3;
 * T[n-t] is the same double as T[t], computed once for t <= n/2), for AMM_SPARSE_CYCLE the
 * cycle norms ||diag Lambda_j||_2 (Section 1.2.2), the values the top-k selection ranks.  `cap` is
 * the capacity of host_keys in doubles (>= n); *count receives n.  Square handles only (blocked
 * circulant handles: AMM_ERR_NOT_IMPLEMENTED; other methods: AMM_ERR_STATE).  Synchronises the
 * handle's stream.
 */
amm_status_t amm_handle_get_keys(amm_handle_t h, double* host_keys, int64_t cap, int64_t* count);

/* Copy the rSVD test matrix phi of Alg. 1 (cols x k, row-major) to host memory.  Synchronises. */
amm_status_t amm_handle_get_sketch(amm_handle_t h, float* host_phi, int64_t cap);

/*
 * A decomposition carried to another process (Section 4: a trained weight is decomposed once,
 * ahead of the products that use it).  amm_handle_export writes the handle's device state -- every
 * factor, spectrum, selection and workspace its products and backward read, and how each refers to
 * the operand -- into a host byte string; amm_handle_import rebuilds a handle from it without
 * recomputing anything, so the imported handle's products and gradients are bit-identical to the
 * original's.
 *   export: host_buf (capacity cap bytes) receives the string and *len its length; when host_buf
 *           is NULL or cap is too small, *len is still set and AMM_ERR_INVALID_ARG returned (call
 *           once to size the buffer).  Synchronises the handle's stream.
 *   import: host_buf / len as exported by a library of the same AMM_VERSION; A the same operand
 *           (DEVICE, rows x cols, lda, dtype as at export -- the handle borrows it again, so it must
 *           stay allocated and unchanged until amm_handle_destroy; lda and dtype are checked only
 *           when the handle reads A, which a sparsifier handle of a BF16 operand does not).  Device
 *           memory is allocated stream-ordered on `stream`; *out receives the handle.  A string of
 *           another format or version, a truncated string or a shape mismatch returns an error with
 *           nothing allocated.
 */
amm_status_t amm_handle_export(amm_handle_t h, void* host_buf, int64_t cap, int64_t* len);
amm_status_t amm_handle_import(const void* host_buf, int64_t len, const void* A, int64_t rows, int64_t cols,
                               int64_t lda, amm_dtype_t dtype, void* stream, amm_handle_t* out);

/* Device memory the handle owns, in bytes (its factors, spectra, selections and workspaces; the
 * borrowed input not included; blocks of a blocked circulant handle summed).  Host only. */
amm_status_t amm_handle_device_bytes(amm_handle_t h, int64_t* bytes);

/* Release every device buffer the handle owns (stream-ordered) and the handle. */
amm_status_t amm_handle_destroy(amm_handle_t h);

/*
 * Cycle spectrum and component keys of one square FP32 matrix WITHOUT allocating device memory.
 * The paper has no counterpart: this is an interface for callers that cannot call cudaMalloc,
 * e.g. code running while a framework captures a CUDA graph and forbids allocation there, or a
 * process whose device memory is owned entirely by another allocator.  It computes the spectrum
 * and the keys that amm_decompose(..., AMM_CIRCULANT, ...) computes first, with the same kernels
 * and the same summation order, so the keys are the doubles amm_handle_get_keys returns:
 *   R     DEVICE output, (n/2+1) x n complex64 (interleaved float pairs), row k = R_A[k],
 *         16-byte aligned; caller-owned
 *   keys  DEVICE output, n doubles, keys[t] = ||R_A[t]||_2 (t and n-t bit-identical)
 *   A     DEVICE input, n x n FP32 row-major, leading dimension lda >= n
 *   n     power of two in [16, AMM_NOALLOC_MAX_N]; larger n returns AMM_ERR_UNSUPPORTED_SIZE
 * Its scratch (twiddles and per-block partial sums) is a fixed AMM_NOALLOC_SCRATCH_BYTES array
 * in device memory that every GPU loading the library holds until the process exits.  The
 * first call on a device looks up that array's address (cudaGetSymbolAddress) with the device
 * current: make that first call before any stream capture.  All calls share the array, so
 * calls that overlap on the GPU race; issue them in order on one stream.
 */
#define AMM_NOALLOC_MAX_N 4096
#define AMM_NOALLOC_SCRATCH_BYTES 4456448
amm_status_t amm_circulant_spectrum_noalloc(const float* A, int64_t n, int64_t lda, void* R,
                                            double* keys, void* stream);

/*
 * Batches of independent products of uneven sizes (e.g. the layers of an LLM-shaped stack).
 * amm_batch_add records one product C = Re(A~ B + dA B~) (A m x n, B n x p, device pointers,
 * caller-owned; the same method, k and element type for both operands; opts_a / opts_b may be
 * NULL, their role is set by the batch).  amm_batch_run executes every item -- decompose both
 * operands, product, release -- on a pool of 16 streams forked from `stream` and joined back into
 * it, the items in descending order of m n p, each on the stream with the least work so far (the
 * results do not depend on the order).  Forward products of the cycle sparsifier (AMM_SPARSE_CYCLE,
 * FP32, square n x n with n <= 4096) run instead in one persistent launch: its CTAs take
 * (product, stage, tile) tasks -- cycle keys, key reduction, selection, gather of the kept
 * cycles, the column panels of A_s B, the row panels of dA B_s -- from a device queue written stage
 * by stage (largest product first), each task waiting (bounded) for the product's previous stage;
 * that launch takes its place in the order above with the summed work of its products, and its
 * results are bit-identical to amm_decompose + amm_approx_matmul.  With use_graph != 0 the first
 * run executes the items once eagerly and then records the same work into one CUDA graph; that
 * run and every later run launch the graph.  Pointers and sizes are baked into the graph: rerun
 * with the same buffers (their contents may change).  After the first graph run no item can be
 * added.
 */
typedef struct amm_batch* amm_batch_t;
amm_status_t amm_batch_create(amm_batch_t* out);
amm_status_t amm_batch_add(amm_batch_t batch, const void* A, const void* B, float* C, int64_t m,
                           int64_t n, int64_t p, int64_t lda, int64_t ldb, int64_t ldc,
                           amm_dtype_t dtype, amm_method_t method, int64_t k,
                           const amm_opts_t* opts_a, const amm_opts_t* opts_b);
/*
 * amm_batch_add with the backward of the item: after the product, the run also writes the frozen-
 * truncation gradients of <dC, Re M> (as amm_approx_matmul_backward) to dA (m x n, ldda) and / or
 * dB (n x p, lddb) -- device, caller-owned, overwritten; one of them may be NULL -- from dC (m x p,
 * lddc).  Same mixed-method and shape limits as amm_approx_matmul_backward (checked when the batch
 * runs).
 */
amm_status_t amm_batch_add_grad(amm_batch_t batch, const void* A, const void* B, float* C, int64_t m,
                                int64_t n, int64_t p, int64_t lda, int64_t ldb, int64_t ldc,
                                amm_dtype_t dtype, amm_method_t method, int64_t k,
                                const amm_opts_t* opts_a, const amm_opts_t* opts_b, const float* dC,
                                int64_t lddc, float* dA, int64_t ldda, float* dB, int64_t lddb);
amm_status_t amm_batch_run(amm_batch_t batch, void* stream, int32_t use_graph);
amm_status_t amm_batch_destroy(amm_batch_t batch);
/*
 * The persistent executor of the cycle-sparsifier items: on != 0 (the default) runs them in the
 * persistent launch, 0 on the stream pool like every other item.  wait_limit_ns (> 0; default 2e9)
 * bounds each wait of a task for its product's previous stage: a wait that runs out stops the
 * launch and is reported by amm_batch_status.  Before the first graph run only
 * (AMM_ERR_STATE after).  Host only.
 */
amm_status_t amm_batch_set_persistent(amm_batch_t batch, int32_t on, int64_t wait_limit_ns);
/*
 * Waits for the last amm_batch_run's stream, then reports the persistent launch's control block:
 * *status = AMM_OK, or AMM_ERR_TIMEOUT when a task's wait ran out (the products' results are
 * then incomplete), with *item the batch index of the product and *stage the stage (0 keys,
 * 1 key reduction, 2 selection, 3 gather, 4 column panels, 5 row panels) whose completion it
 * waited for (-1 when none); *persistent_products = how many items the persistent launch runs.
 */
amm_status_t amm_batch_status(amm_batch_t batch, int32_t* status, int64_t* item, int32_t* stage,
                              int32_t* persistent_products);

/*
 * Launch tracing for measurement.  While enabled, every kernel launch the library makes is
 * bracketed by two CUDA events on the launch's own stream.  amm_trace_collect() waits for
 * the recorded launches, writes a JSON object {"kernel name": [launches, total_ms], ...} of
 * everything recorded since the previous collect into host_json (capacity `cap` bytes,
 * NUL-terminated) and the number of launches into *launches (may be NULL).
 */
amm_status_t amm_trace_enable(int32_t on);
amm_status_t amm_trace_collect(char* host_json, int64_t cap, int64_t* launches);

/*
 * Test hook for the tensor-core GEMM used by the SVD path: C = alpha A B^T + beta C with
 * A (M x K, lda) and B (N x K, ldb) row-major along K (device pointers), C (M x N, ldc) FP32.
 * mode 1: A, B are BF16 (tcgen05 kind::f16, FP32 accumulation).  mode 0: A, B are FP32, split
 * into TF32 hi/lo parts (three kind::tf32 products, FP32-level accuracy).  Rows of A and B
 * must start 16-byte aligned.  *dev_err (device int) is set to 1 if a bounded wait gave up.
 */
amm_status_t amm_debug_gemm_tn(int32_t mode, int64_t M, int64_t N, int64_t K, float alpha,
                               const void* A, int64_t lda, const void* B, int64_t ldb, float beta,
                               float* C, int64_t ldc, int32_t* dev_err, void* stream);

/*
 * Autotuning of kernel variants (off by default; an implementation choice with no counterpart in
 * the paper).  With on != 0, the first call of a kernel that has several compiled variants -- the
 * circulant spectral apply (per length, direction, coefficient pairing and element type), the
 * inverse cycle transform and the column and row half spectra of the backward (per length): a
 * full or a halved number of packed signals (and threads) per CTA -- times each variant on that
 * call's own operands (into scratch memory; the call's result is computed afterwards by the
 * fastest) and keeps the choice for the process.  The variants compute every output with the same
 * operations, so the choice never changes results.  Timing synchronises the stream once per new
 * key; calls made while their stream is being captured into a CUDA graph use the current choice
 * without timing.  Untuned keys use defaults measured on GB300.  When the environment variable
 * AMM_TUNE_CACHE names a file, the table is loaded from it at first use (a file that does not
 * parse is ignored) and written back, in the text form of amm_autotune_export, after every new
 * choice, so later processes start tuned.
 */
amm_status_t amm_set_autotune(int32_t on);

/*
 * The autotuner's choices as text, for reuse by another process of the same build (a serving
 * process can load the choices a tuning run made instead of timing again): a header line
 * "amm-autotune 1", then one "key variant" line per tuned (length, direction, element type), keys
 * ascending.  host_buf (capacity cap bytes) receives the NUL-terminated text and *len its length
 * without the NUL, also when cap is too small (then AMM_ERR_INVALID_ARG and host_buf untouched).
 * Host only: no device work.
 */
amm_status_t amm_autotune_export(char* host_buf, int64_t cap, int64_t* len);

/*
 * Install choices written by amm_autotune_export (they override entries for the same keys; a
 * choice in the table is used whether or not autotuning is on).  A key is kernel << 24 | length << 3
 * | flags (kernel 0: spectral apply, flags = 4 row + 2 reversed pairing + BF16; kernel 1: inverse
 * cycle transform, flag 1 = accumulating form; kernels 2, 3: column and row backward spectra,
 * flags 0).  Every line is checked
 * first: a wrong header, an unknown kernel, flags on a kernel without them, a length that is not a
 * circulant length the library supports, a variant other than 0 / 1 or trailing text returns
 * AMM_ERR_INVALID_ARG with nothing installed.  Host only.
 */
amm_status_t amm_autotune_import(const char* host_text);

/*
 * Test hook for the bounded waits of the batch's persistent executor: runs it (one CTA) on a queue
 * whose only task waits for a stage that no task completes, on `stream`, and synchronises.  The
 * wait gives up after limit_ns (in (0, 5e9]) and the launch returns; *status_out receives the
 * control block's status (AMM_ERR_TIMEOUT) and *stage_out the stage waited for (4).  No GPU
 * fault: the kernel returns normally.
 */
amm_status_t amm_debug_persistent_wait_timeout(int64_t limit_ns, void* stream, int32_t* status_out,
                                               int32_t* stage_out);

/*
 * Fault injection for tests: the n-th device allocation from now on (1-based) fails with
 * AMM_ERR_OOM; 0 disables.  Affects only this process.
 */
amm_status_t amm_debug_fail_alloc_after(int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* AMM_H */
