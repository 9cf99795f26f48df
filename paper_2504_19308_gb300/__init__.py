"""GB300-native first-order approximate matrix multiplication from truncated decompositions.

Python front end of libamm (include/amm.h): arXiv 2504.19308, M = A~ B + dA B~.
"""
from .amm import (AmmError, Batch, ApproxMatmulFn, Handle, approx_matmul, approx_matmul_autograd,  # noqa: F401
                  autotune_export, autotune_import,
                  approx_matmul_backward, apriori_estimate, choose_k, decompose, decompose_best_method,
                  decompose_to_tolerance, error_estimate, import_handle, load_library, refine, refine_product, residual,
                  set_autotune, trace_collect, trace_enable, LIB_PATH)
