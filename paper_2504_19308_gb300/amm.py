"""Python binding of libamm (include/amm.h): argument marshalling only.

Every numerical step runs in the CUDA kernels behind the C ABI.  PyTorch supplies device
memory and the current CUDA stream.  There is no CPU fallback: if libamm.so is missing or a
call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamm.so")

METHODS = {"svd": 0, "circulant": 1, "fourier": 2, "cycle": 3}
DTYPES = {torch.float32: 0, torch.bfloat16: 1}
ROLES = {"left": 1, "right": 2}
STATUS = ["AMM_OK", "AMM_ERR_INVALID_ARG", "AMM_ERR_UNSUPPORTED_SIZE", "AMM_ERR_OOM", "AMM_ERR_CUDA",
          "AMM_ERR_TIMEOUT", "AMM_ERR_STATE", "AMM_ERR_NOT_IMPLEMENTED"]


class AmmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__("%s failed: %s (%s)" % (where, name, detail))


class Opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("role", ctypes.c_int32), ("compute", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("sketch", ctypes.c_void_p), ("store_spectra", ctypes.c_int32),
                ("forced_selection", ctypes.POINTER(ctypes.c_int32)), ("pair_closed", ctypes.c_int32),
                ("block", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("role", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("k", ctypes.c_int64),
                ("n_union", ctypes.c_int64), ("n_unpaired", ctypes.c_int64), ("fro2", ctypes.c_double),
                ("resid_fro2", ctypes.c_double), ("boundary_gap", ctypes.c_double)]


# every exported symbol of include/amm.h with its ctypes signature
SIGNATURES = {
    "amm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "amm_last_error": (ctypes.c_char_p, []),
    "amm_version": (ctypes.c_int32, []),
    "amm_set_autotune": (ctypes.c_int, [ctypes.c_int32]),
    "amm_autotune_export": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "amm_autotune_import": (ctypes.c_int, [ctypes.c_char_p]),
    "amm_decompose_to_tolerance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                                  ctypes.POINTER(Opts), ctypes.c_void_p,
                                                  ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64)]),
    "amm_opts_init": (ctypes.c_int, [ctypes.POINTER(Opts)]),
    "amm_decompose": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int64, ctypes.POINTER(Opts), ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_void_p)]),
    "amm_approx_matmul": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p]),
    "amm_choose_k": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "amm_error_estimate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "amm_apriori_estimate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_double)]),
    "amm_handle_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "amm_refine_product": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "amm_decompose_best_method": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                 ctypes.c_int64, ctypes.POINTER(Opts), ctypes.c_void_p,
                                                 ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int32)]),
    "amm_approx_matmul_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                                  ctypes.c_void_p]),
    "amm_handle_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Info)]),
    "amm_handle_get_selection": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64,
                                                ctypes.POINTER(ctypes.c_int64)]),
    "amm_handle_get_sketch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int64]),
    "amm_handle_get_keys": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                           ctypes.POINTER(ctypes.c_int64)]),
    "amm_handle_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "amm_handle_device_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "amm_handle_export": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64)]),
    "amm_handle_import": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "amm_debug_fail_alloc_after": (ctypes.c_int, [ctypes.c_int32]),
    "amm_circulant_spectrum_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "amm_debug_gemm_tn": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_float, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "amm_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p)]),
    "amm_batch_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                     ctypes.POINTER(Opts), ctypes.POINTER(Opts)]),
    "amm_batch_add_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                          ctypes.POINTER(Opts), ctypes.POINTER(Opts), ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_int64]),
    "amm_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "amm_batch_set_persistent": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    "amm_batch_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32)]),
    "amm_debug_persistent_wait_timeout": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p,
                                                         ctypes.POINTER(ctypes.c_int32),
                                                         ctypes.POINTER(ctypes.c_int32)]),
    "amm_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "amm_trace_enable": (ctypes.c_int, [ctypes.c_int32]),
    "amm_trace_collect": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libamm.so (built by paper_2504_19308_gb300.build).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libamm.so not found at %s: run __graft_entry__.build() (nvcc, sm_103a) first" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        raise AmmError(status, where, load_library().amm_last_error().decode(errors="replace"))


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _require_cuda(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor (the library has no CPU path)" % name)
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("%s must be a 2-D row-major tensor with unit column stride" % name)


class Handle:
    """Truncated decomposition of one operand; keeps the operand alive (the library borrows it)."""

    def __init__(self, ptr: int, source: torch.Tensor, method: str, role: str, k: int, extras=(), block: int = 0):
        self.ptr = ctypes.c_void_p(ptr)
        self.source = source
        self.method = method
        self.role = role
        self.k = k
        self.block = block
        self._extras = extras  # tensors that must outlive the launch (sketch)

    @property
    def blocks(self):
        """(block rows, block columns) of a blocked circulant handle; (1, 1) otherwise."""
        if not self.block:
            return 1, 1
        return -(-self.shape[0] // self.block), -(-self.shape[1] // self.block)

    @property
    def shape(self):
        return tuple(self.source.shape)

    def info(self) -> dict:
        info = Info()
        _check(load_library().amm_handle_info(self.ptr, ctypes.byref(info)), "amm_handle_info")
        return {f: getattr(info, f) for f, _ in Info._fields_}

    def selection(self) -> np.ndarray:
        """Selected components (k,), per-block components (blocks, k) of a blocked circulant handle
        (blocks row-major), or per-row / per-column kept frequencies (rows, k) for 'fourier'."""
        rows = 1
        if self.method == "fourier":
            rows = self.shape[0] if self.role == "left" else self.shape[1]
        elif self.block:
            rows = self.blocks[0] * self.blocks[1]
        cap = self.k * rows
        buf = (ctypes.c_int32 * cap)()
        cnt = ctypes.c_int64(0)
        _check(load_library().amm_handle_get_selection(self.ptr, buf, cap, ctypes.byref(cnt)),
               "amm_handle_get_selection")
        out = np.frombuffer(buf, dtype=np.int32, count=cnt.value).copy()
        return out.reshape(rows, self.k) if self.method == "fourier" or self.block else out

    def export(self) -> bytes:
        """amm_handle_export: the decomposition's device state as bytes (reusable in another process)."""
        lib = load_library()
        n = ctypes.c_int64(0)
        lib.amm_handle_export(self.ptr, None, 0, ctypes.byref(n))
        buf = ctypes.create_string_buffer(max(1, n.value))
        _check(lib.amm_handle_export(self.ptr, buf, n.value, ctypes.byref(n)), "amm_handle_export")
        return buf.raw[: n.value]

    def device_bytes(self) -> int:
        """Device memory the handle owns (amm_handle_device_bytes)."""
        b = ctypes.c_int64(0)
        _check(load_library().amm_handle_device_bytes(self.ptr, ctypes.byref(b)), "amm_handle_device_bytes")
        return b.value

    def keys(self) -> np.ndarray:
        """Component keys (circulant T[t] = ||R_A[t]||_2, or the cycle norms), length n."""
        n = self.shape[0]
        buf = (ctypes.c_double * n)()
        cnt = ctypes.c_int64(0)
        _check(load_library().amm_handle_get_keys(self.ptr, buf, n, ctypes.byref(cnt)), "amm_handle_get_keys")
        return np.frombuffer(buf, dtype=np.float64, count=cnt.value).copy()

    def sketch(self) -> np.ndarray:
        n = self.source.shape[1]
        buf = (ctypes.c_float * (n * self.k))()
        _check(load_library().amm_handle_get_sketch(self.ptr, buf, n * self.k), "amm_handle_get_sketch")
        return np.frombuffer(buf, dtype=np.float32).reshape(n, self.k).copy()

    def close(self):
        if self.ptr is not None and self.ptr.value:
            _check(load_library().amm_handle_destroy(self.ptr), "amm_handle_destroy")
        self.ptr = None

    def __del__(self):
        try:
            if self.ptr is not None and self.ptr.value and _lib is not None:
                _lib.amm_handle_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass


def decompose(A: torch.Tensor, method: str, k: int, role: str = "left", sketch: Optional[torch.Tensor] = None,
              seed: int = 0, forced_selection=None, compute: str = "f32", pair_closed: bool = False,
              block: int = 0, store_spectra: bool = True) -> Handle:
    """amm_decompose: truncated decomposition of A (method 'circulant' | 'svd' | 'fourier' | 'cycle').

    compute: arithmetic of the SVD GEMMs, 'f32' (FP32-accurate) or 'bf16' (BF16 tensor cores).
    pair_closed: circulant selections closed under t -> n - t (a real truncation).
    block: circulant operand of any shape in block x block squares (zero-padded edge, top-k per
    block); forced_selection then holds k indices per block, blocks row-major.
    store_spectra: False releases a circulant handle's half spectrum after the decomposition
    (recomputed from A where a mixed product or the residual export needs it).
    """
    lib = load_library()
    _require_cuda(A, "A")
    if A.dtype not in DTYPES:
        raise ValueError("A must be float32 or bfloat16")
    opts = Opts()
    _check(lib.amm_opts_init(ctypes.byref(opts)), "amm_opts_init")
    opts.role = ROLES[role]
    opts.seed = seed
    opts.compute = {"f32": 0, "bf16": 1}[compute]
    opts.pair_closed = 1 if pair_closed else 0
    opts.block = int(block)
    opts.store_spectra = 1 if store_spectra else 0
    extras = []
    if sketch is not None:
        _require_cuda(sketch, "sketch")
        sketch = sketch.to(torch.float32).contiguous()
        opts.sketch = sketch.data_ptr()
        extras.append(sketch)
    forced = None
    if forced_selection is not None:
        flat = np.asarray(forced_selection, dtype=np.int64).reshape(-1)
        nblk = (-(-A.shape[0] // block)) * (-(-A.shape[1] // block)) if block else 1
        if flat.size != nblk * k:
            raise ValueError("forced_selection needs %d entries (k per block), got %d" % (nblk * k, flat.size))
        forced = (ctypes.c_int32 * flat.size)(*[int(v) for v in flat])
        opts.forced_selection = ctypes.cast(forced, ctypes.POINTER(ctypes.c_int32))
    out = ctypes.c_void_p(0)
    _check(lib.amm_decompose(A.data_ptr(), A.shape[0], A.shape[1], A.stride(0), DTYPES[A.dtype], METHODS[method], k,
                             ctypes.byref(opts), _stream_ptr(A.device), ctypes.byref(out)), "amm_decompose")
    blocked = block and not (A.shape[0] == block and A.shape[1] == block)
    return Handle(out.value, A, method, role, k, tuple(extras), int(block) if blocked else 0)


def import_handle(blob: bytes, A: torch.Tensor, method: str, k: int, role: str = "left", block: int = 0) -> Handle:
    """amm_handle_import: a handle rebuilt from amm_handle_export's bytes, borrowing A (the same
    operand; method / k / role / block describe the exported handle for the binding's bookkeeping)."""
    lib = load_library()
    _require_cuda(A, "A")
    out = ctypes.c_void_p(0)
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    _check(lib.amm_handle_import(buf, len(blob), A.data_ptr(), A.shape[0], A.shape[1], A.stride(0), DTYPES[A.dtype],
                                 _stream_ptr(A.device), ctypes.byref(out)), "amm_handle_import")
    blocked = block and not (A.shape[0] == block and A.shape[1] == block)
    return Handle(out.value, A, method, role, k, (), int(block) if blocked else 0)


def approx_matmul(hA: Handle, hB: Handle, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """amm_approx_matmul: Re(A~ B + dA B~) as an FP32 tensor."""
    m, p = hA.shape[0], hB.shape[1]
    if out is None:
        out = torch.empty((m, p), dtype=torch.float32, device=hA.source.device)
    _require_cuda(out, "out")
    _check(load_library().amm_approx_matmul(hA.ptr, hB.ptr, out.data_ptr(), out.stride(0),
                                            _stream_ptr(out.device)), "amm_approx_matmul")
    return out


def set_autotune(on: bool = True):
    """amm_set_autotune: time the compiled variants of tunable kernels on first use and keep the
    fastest (results do not depend on the choice)."""
    _check(load_library().amm_set_autotune(1 if on else 0), "amm_set_autotune")


def autotune_export() -> str:
    """amm_autotune_export: the autotuner's choices as text (for autotune_import in another process)."""
    lib = load_library()
    n = ctypes.c_int64(0)
    buf = ctypes.create_string_buffer(1 << 12)
    if lib.amm_autotune_export(buf, len(buf), ctypes.byref(n)) != 0:
        buf = ctypes.create_string_buffer(n.value + 1)
        _check(lib.amm_autotune_export(buf, len(buf), ctypes.byref(n)), "amm_autotune_export")
    return buf.value.decode()


def autotune_import(text: str):
    """amm_autotune_import: install choices written by autotune_export (all or nothing)."""
    _check(load_library().amm_autotune_import(text.encode()), "amm_autotune_import")


def choose_k(A: torch.Tensor, method: str, tol: float) -> int:
    """amm_choose_k: smallest k with ||dA||_F <= tol ||A||_F (circulant or cycle truncation)."""
    _require_cuda(A, "A")
    k = ctypes.c_int64(0)
    _check(load_library().amm_choose_k(A.data_ptr(), A.shape[0], A.shape[1], A.stride(0), DTYPES[A.dtype],
                                       METHODS[method], float(tol), _stream_ptr(A.device), ctypes.byref(k)),
           "amm_choose_k")
    return k.value


def decompose_to_tolerance(A: torch.Tensor, method: str, tol: float, role: str = "left", k_max: int = 0,
                           seed: int = 0, compute: str = "f32", pair_closed: bool = False) -> Handle:
    """amm_decompose_to_tolerance: the smallest k with ||dA||_F <= tol ||A||_F (exact from the keys for
    'circulant' / 'cycle'; geometric growth and bisection over trial decompositions for 'svd' /
    'fourier')."""
    lib = load_library()
    _require_cuda(A, "A")
    opts = Opts()
    _check(lib.amm_opts_init(ctypes.byref(opts)), "amm_opts_init")
    opts.role = ROLES[role]
    opts.seed = seed
    opts.compute = {"f32": 0, "bf16": 1}[compute]
    opts.pair_closed = 1 if pair_closed else 0
    out, k = ctypes.c_void_p(0), ctypes.c_int64(0)
    _check(lib.amm_decompose_to_tolerance(A.data_ptr(), A.shape[0], A.shape[1], A.stride(0), DTYPES[A.dtype],
                                          METHODS[method], float(tol), int(k_max), ctypes.byref(opts),
                                          _stream_ptr(A.device), ctypes.byref(out), ctypes.byref(k)),
           "amm_decompose_to_tolerance")
    return Handle(out.value, A, method, role, k.value)


def error_estimate(hA: Handle, hB: Handle, C: torch.Tensor) -> float:
    """amm_error_estimate: ||dA|| ||dB|| / (sqrt(n) ||C||) (Corollary 3.7) for a computed product C."""
    _require_cuda(C, "C")
    est = ctypes.c_double(0.0)
    _check(load_library().amm_error_estimate(hA.ptr, hB.ptr, C.data_ptr(), C.stride(0), _stream_ptr(C.device),
                                             ctypes.byref(est)), "amm_error_estimate")
    return est.value


def apriori_estimate(hA: Handle, hB: Handle, c_ab: float, c_resid: float) -> float:
    """amm_apriori_estimate: c_resid ||dA|| ||dB|| / (c_ab ||A|| ||B||) before the product (Section 2.5),
    with the front constants of the operands (c_ab) and of the residues (c_resid)."""
    est = ctypes.c_double(0.0)
    _check(load_library().amm_apriori_estimate(hA.ptr, hB.ptr, float(c_ab), float(c_resid), ctypes.byref(est)),
           "amm_apriori_estimate")
    return est.value


def residual(h: Handle) -> torch.Tensor:
    """amm_handle_residual: Re dA = A - Re A~ as a dense FP32 tensor of the operand's shape."""
    out = torch.empty(h.shape, dtype=torch.float32, device=h.source.device)
    _check(load_library().amm_handle_residual(h.ptr, out.data_ptr(), out.stride(0), _stream_ptr(out.device)),
           "amm_handle_residual")
    return out


def refine_product(hA: Handle, hB: Handle, hA2: Handle, hB2: Handle, C: torch.Tensor) -> torch.Tensor:
    """amm_refine_product: C += Re M2 - Im(A~) Im(B~) in place, hA2 / hB2 decompositions of
    residual(hA) / residual(hB) (Section 2.5)."""
    _require_cuda(C, "C")
    if C.dtype != torch.float32:
        raise ValueError("C must be float32")
    _check(load_library().amm_refine_product(hA.ptr, hB.ptr, hA2.ptr, hB2.ptr, C.data_ptr(), C.stride(0),
                                             _stream_ptr(C.device)), "amm_refine_product")
    return C


def refine(hA: Handle, hB: Handle, C: torch.Tensor, k2: int, methods=None, sketch_a=None, sketch_b=None,
           seed: int = 0, compute: str = "f32"):
    """Section 2.5 refinement of C = Re M: decompose Re dA and Re dB with k2 components (by the first
    handles' methods unless `methods` = (method_a, method_b) is given) and add their first-order
    product and the exact Im dA Im dB term to C in place.  Returns (C, hA2, hB2)."""
    ma, mb = methods if methods is not None else (hA.method, hB.method)
    hA2 = decompose(residual(hA), ma, k2, "left", sketch=sketch_a, seed=seed, compute=compute)
    hB2 = decompose(residual(hB), mb, k2, "right", sketch=sketch_b, seed=seed, compute=compute)
    refine_product(hA, hB, hA2, hB2, C)
    return C, hA2, hB2


def decompose_best_method(A: torch.Tensor, methods, k: int, role: str = "left", seed: int = 0,
                          compute: str = "f32", pair_closed: bool = False, block: int = 0):
    """amm_decompose_best_method: decompose A with each of `methods` at k and keep the one with the
    smallest relative truncation error (Section 2.5).  Returns (handle, method name)."""
    lib = load_library()
    _require_cuda(A, "A")
    if A.dtype not in DTYPES:
        raise ValueError("A must be float32 or bfloat16")
    names = list(methods)
    if not names:
        raise ValueError("methods is empty")
    codes = (ctypes.c_int32 * len(names))(*[METHODS[m] for m in names])
    opts = Opts()
    _check(lib.amm_opts_init(ctypes.byref(opts)), "amm_opts_init")
    opts.role = ROLES[role]
    opts.seed = seed
    opts.compute = {"f32": 0, "bf16": 1}[compute]
    opts.pair_closed = 1 if pair_closed else 0
    opts.block = int(block)
    out, chosen = ctypes.c_void_p(0), ctypes.c_int32(-1)
    _check(lib.amm_decompose_best_method(A.data_ptr(), A.shape[0], A.shape[1], A.stride(0), DTYPES[A.dtype], codes,
                                         len(names), k, ctypes.byref(opts), _stream_ptr(A.device), ctypes.byref(out),
                                         ctypes.byref(chosen)), "amm_decompose_best_method")
    method = {v: n for n, v in METHODS.items()}[chosen.value]
    blocked = method == "circulant" and block and not (A.shape[0] == block and A.shape[1] == block)
    return Handle(out.value, A, method, role, k, (), int(block) if blocked else 0), method


def approx_matmul_backward(hA: Handle, hB: Handle, dC: torch.Tensor, need_dA: bool = True, need_dB: bool = True):
    """amm_approx_matmul_backward: gradients of <dC, Re M> with the truncation frozen."""
    _require_cuda(dC, "dC")
    dC = dC.to(torch.float32).contiguous()
    dev = dC.device
    dA = torch.empty(hA.shape, dtype=torch.float32, device=dev) if need_dA else None
    dB = torch.empty(hB.shape, dtype=torch.float32, device=dev) if need_dB else None
    _check(load_library().amm_approx_matmul_backward(
        hA.ptr, hB.ptr, dC.data_ptr(), dC.stride(0), dA.data_ptr() if dA is not None else None,
        dA.stride(0) if dA is not None else 0, dB.data_ptr() if dB is not None else None,
        dB.stride(0) if dB is not None else 0, _stream_ptr(dev)), "amm_approx_matmul_backward")
    return dA, dB


class ApproxMatmulFn(torch.autograd.Function):
    """Autograd layer: forward decomposes both operands and evaluates the first-order product;
    backward calls the hand-written adjoint kernels with the truncation frozen."""

    @staticmethod
    def forward(ctx, A, B, method: str, k: int, sketch_a=None, sketch_b=None):
        hA = decompose(A.detach(), method, k, "left", sketch=sketch_a)
        hB = decompose(B.detach(), method, k, "right", sketch=sketch_b)
        ctx.handles = (hA, hB)
        return approx_matmul(hA, hB)

    @staticmethod
    def backward(ctx, grad):
        hA, hB = ctx.handles
        dA, dB = approx_matmul_backward(hA, hB, grad, ctx.needs_input_grad[0], ctx.needs_input_grad[1])
        return dA, dB, None, None, None, None


def approx_matmul_autograd(A, B, method: str, k: int, sketch_a=None, sketch_b=None):
    return ApproxMatmulFn.apply(A, B, method, k, sketch_a, sketch_b)


class Batch:
    """amm_batch_*: many independent products run together, optionally as one CUDA graph."""

    def __init__(self):
        self.ptr = ctypes.c_void_p(0)
        _check(load_library().amm_batch_create(ctypes.byref(self.ptr)), "amm_batch_create")
        self.keep = []

    def add(self, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, method: str, k: int,
            sketch_a: Optional[torch.Tensor] = None, sketch_b: Optional[torch.Tensor] = None, compute: str = "f32",
            dC: Optional[torch.Tensor] = None, dA: Optional[torch.Tensor] = None, dB: Optional[torch.Tensor] = None):
        """One product C = Re M; with dC given, also its backward into dA and / or dB (amm_batch_add_grad)."""
        for t, nm in ((A, "A"), (B, "B"), (C, "C"), (dC, "dC"), (dA, "dA"), (dB, "dB")):
            if t is not None:
                _require_cuda(t, nm)
        oa, ob = Opts(), Opts()
        lib = load_library()
        _check(lib.amm_opts_init(ctypes.byref(oa)), "amm_opts_init")
        _check(lib.amm_opts_init(ctypes.byref(ob)), "amm_opts_init")
        oa.compute = ob.compute = {"f32": 0, "bf16": 1}[compute]
        if sketch_a is not None:
            oa.sketch = sketch_a.data_ptr()
        if sketch_b is not None:
            ob.sketch = sketch_b.data_ptr()
        self.keep += [A, B, C, sketch_a, sketch_b, dC, dA, dB]
        if dC is None:
            _check(lib.amm_batch_add(self.ptr, A.data_ptr(), B.data_ptr(), C.data_ptr(), A.shape[0], A.shape[1],
                                     B.shape[1], A.stride(0), B.stride(0), C.stride(0), DTYPES[A.dtype],
                                     METHODS[method], k, ctypes.byref(oa), ctypes.byref(ob)), "amm_batch_add")
            return
        _check(lib.amm_batch_add_grad(self.ptr, A.data_ptr(), B.data_ptr(), C.data_ptr(), A.shape[0], A.shape[1],
                                      B.shape[1], A.stride(0), B.stride(0), C.stride(0), DTYPES[A.dtype],
                                      METHODS[method], k, ctypes.byref(oa), ctypes.byref(ob), dC.data_ptr(),
                                      dC.stride(0), dA.data_ptr() if dA is not None else None,
                                      dA.stride(0) if dA is not None else 0,
                                      dB.data_ptr() if dB is not None else None,
                                      dB.stride(0) if dB is not None else 0), "amm_batch_add_grad")

    def run(self, use_graph: bool = True):
        dev = self.keep[0].device
        _check(load_library().amm_batch_run(self.ptr, _stream_ptr(dev), 1 if use_graph else 0), "amm_batch_run")

    def set_persistent(self, on: bool = True, wait_limit_ns: int = 2_000_000_000):
        """Cycle-sparsifier items in the persistent work-queue launch (default) or on the stream pool."""
        _check(load_library().amm_batch_set_persistent(self.ptr, 1 if on else 0, int(wait_limit_ns)),
               "amm_batch_set_persistent")

    def status(self):
        """(status, item, stage, persistent_products) of the last run's persistent launch (waits for it)."""
        st, it, sg, npq = ctypes.c_int32(0), ctypes.c_int64(-1), ctypes.c_int32(-1), ctypes.c_int32(0)
        _check(load_library().amm_batch_status(self.ptr, ctypes.byref(st), ctypes.byref(it), ctypes.byref(sg),
                                               ctypes.byref(npq)), "amm_batch_status")
        return st.value, it.value, sg.value, npq.value

    def close(self):
        if self.ptr is not None and self.ptr.value:
            _check(load_library().amm_batch_destroy(self.ptr), "amm_batch_destroy")
        self.ptr = None


def trace_enable(on: bool = True):
    _check(load_library().amm_trace_enable(1 if on else 0), "amm_trace_enable")


def trace_collect():
    """{kernel name: (launches, total_ms)} since the previous collect, and the launch count."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    n = ctypes.c_int64(0)
    _check(load_library().amm_trace_collect(buf, len(buf), ctypes.byref(n)), "amm_trace_collect")
    return {k: tuple(v) for k, v in json.loads(buf.value.decode()).items()}, n.value


def debug_fail_alloc_after(n: int):
    _check(load_library().amm_debug_fail_alloc_after(n), "amm_debug_fail_alloc_after")
