"""The C ABI on the CPU: the library loads without a GPU and exports every declared symbol;
argument errors are reported before anything is launched."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "amm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_19308_gb300 import build as b
    b.build()
    import paper_2504_19308_gb300.amm as amm
    return amm.load_library()


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for s in ["amm_decompose", "amm_approx_matmul", "amm_approx_matmul_backward", "amm_handle_destroy",
              "amm_handle_info", "amm_handle_get_selection", "amm_status_string"]:
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    import paper_2504_19308_gb300.amm as amm
    for s in _declared_symbols():
        assert hasattr(lib, s), s
        assert s in amm.SIGNATURES, "binding lacks " + s


def test_library_resolves_every_symbol_at_load(lib):
    """Eager binding (RTLD_NOW): a symbol the library references but no object defines fails here
    on the CPU rather than at the first call on a machine with a GPU."""
    path = os.path.join(ROOT, "paper_2504_19308_gb300", "libamm.so")
    ctypes.CDLL(path, mode=os.RTLD_NOW | os.RTLD_LOCAL)


def test_status_strings(lib):
    assert lib.amm_status_string(0) == b"AMM_OK"
    assert lib.amm_status_string(5) == b"AMM_ERR_TIMEOUT"
    assert lib.amm_version() == 7


def test_argument_errors_without_gpu(lib):
    import paper_2504_19308_gb300.amm as amm
    opts = amm.Opts()
    assert lib.amm_opts_init(ctypes.byref(opts)) == 0
    out = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: every call below fails validation first
    # NULL A
    assert lib.amm_decompose(None, 64, 64, 64, 0, 1, 4, ctypes.byref(opts), None, ctypes.byref(out)) == 1
    # k = 0
    assert lib.amm_decompose(fake, 64, 64, 64, 0, 1, 0, ctypes.byref(opts), None, ctypes.byref(out)) == 1
    # empty operands, for every method
    for method in range(4):
        assert lib.amm_decompose(fake, 0, 64, 64, 0, method, 4, ctypes.byref(opts), None, ctypes.byref(out)) == 1
        assert lib.amm_decompose(fake, 64, 0, 64, 0, method, 4, ctypes.byref(opts), None, ctypes.byref(out)) == 1
        assert b"empty matrix" in lib.amm_last_error()
    # lda < cols
    assert lib.amm_decompose(fake, 64, 64, 32, 0, 1, 4, ctypes.byref(opts), None, ctypes.byref(out)) == 1
    # circulant needs a square of a supported length
    assert lib.amm_decompose(fake, 64, 32, 64, 0, 1, 4, ctypes.byref(opts), None, ctypes.byref(out)) == 2
    # circulant lengths: any n in [16, 4096], above that 2^a or 3 * 2^a only (4100 and 6000 are not)
    assert lib.amm_decompose(fake, 4100, 4100, 4100, 0, 1, 4, ctypes.byref(opts), None, ctypes.byref(out)) == 2
    assert lib.amm_decompose(fake, 6000, 6000, 6000, 0, 1, 4, ctypes.byref(opts), None, ctypes.byref(out)) == 2
    assert lib.amm_decompose(fake, 12, 12, 12, 0, 1, 4, ctypes.byref(opts), None, ctypes.byref(out)) == 2
    # k from a tolerance: outputs required, negative tolerance rejected, before any launch
    k_out = ctypes.c_int64(0)
    assert lib.amm_decompose_to_tolerance(fake, 64, 64, 64, 0, 1, 0.1, 0, None, None, None,
                                          ctypes.byref(k_out)) == 1
    assert lib.amm_decompose_to_tolerance(fake, 64, 64, 64, 0, 0, -1.0, 0, None, None, ctypes.byref(out),
                                          ctypes.byref(k_out)) == 1
    assert lib.amm_set_autotune(0) == 0
    # method choice: outputs, candidates and per-method options checked before any launch; a
    # candidate that does not take the shape is skipped, and with none left its status returns
    cand = (ctypes.c_int32 * 2)(1, 1)
    chosen = ctypes.c_int32(-1)
    assert lib.amm_decompose_best_method(fake, 64, 64, 64, 0, cand, 2, 4, None, None, None,
                                         ctypes.byref(chosen)) == 1
    assert lib.amm_decompose_best_method(None, 64, 64, 64, 0, cand, 2, 4, None, None, ctypes.byref(out),
                                         ctypes.byref(chosen)) == 1
    assert lib.amm_decompose_best_method(fake, 64, 64, 64, 0, None, 2, 4, None, None, ctypes.byref(out),
                                         ctypes.byref(chosen)) == 1
    assert lib.amm_decompose_best_method(fake, 64, 64, 64, 0, cand, 0, 4, None, None, ctypes.byref(out),
                                         ctypes.byref(chosen)) == 1
    bad = (ctypes.c_int32 * 1)(7)
    assert lib.amm_decompose_best_method(fake, 64, 64, 64, 0, bad, 1, 4, None, None, ctypes.byref(out),
                                         ctypes.byref(chosen)) == 1
    forced = (ctypes.c_int32 * 4)(0, 1, 2, 3)
    fo = amm.Opts()
    assert lib.amm_opts_init(ctypes.byref(fo)) == 0
    fo.forced_selection = ctypes.cast(forced, ctypes.POINTER(ctypes.c_int32))
    assert lib.amm_decompose_best_method(fake, 64, 64, 64, 0, cand, 2, 4, ctypes.byref(fo), None, ctypes.byref(out),
                                         ctypes.byref(chosen)) == 1
    assert lib.amm_decompose_best_method(fake, 4100, 4100, 4100, 0, cand, 2, 4, None, None, ctypes.byref(out),
                                         ctypes.byref(chosen)) == 2
    assert b"n=4100" in lib.amm_last_error()
    assert out.value in (None, 0) and chosen.value == -1
    # refinement: outputs and handles checked on the host
    assert lib.amm_handle_residual(None, fake, 64, None) == 1
    assert lib.amm_refine_product(None, None, None, None, None, 64, None) == 1
    assert lib.amm_refine_product(None, None, None, None, fake, 64, None) == 1
    # a priori estimate: output, constants and handles checked on the host
    est = ctypes.c_double(0.0)
    assert lib.amm_apriori_estimate(None, None, 1.0, 1.0, None) == 1
    assert lib.amm_apriori_estimate(None, None, 0.0, 1.0, ctypes.byref(est)) == 1
    assert lib.amm_apriori_estimate(None, None, 1.0, float("nan"), ctypes.byref(est)) == 1
    assert lib.amm_apriori_estimate(None, None, 1.0, 1.0, ctypes.byref(est)) == 1
    # bad struct size
    opts.struct_size = 3
    assert lib.amm_decompose(fake, 64, 64, 64, 0, 1, 4, ctypes.byref(opts), None, ctypes.byref(out)) == 1
    assert out.value in (0, None)
    assert b"struct_size" in lib.amm_last_error()
    # NULL handles
    assert lib.amm_approx_matmul(None, None, fake, 64, None) == 1
    assert lib.amm_handle_destroy(None) == 1


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: without the compiled library every entry point raises."""
    import paper_2504_19308_gb300.amm as amm
    monkeypatch.setattr(amm, "_lib", None)
    with pytest.raises(RuntimeError, match="libamm.so not found"):
        amm.load_library(os.path.join(ROOT, "no_such_dir", "libamm.so"))


def test_cpu_tensors_are_rejected(lib):
    """The binding only marshals device pointers: host tensors are refused before any call."""
    torch = pytest.importorskip("torch")
    import paper_2504_19308_gb300 as amm
    x = torch.zeros((64, 64))
    with pytest.raises(ValueError, match="CUDA tensor"):
        amm.decompose(x, "circulant", 4)
    with pytest.raises(ValueError, match="CUDA tensor"):
        amm.decompose_best_method(x, ["circulant", "svd"], 4)
    with pytest.raises(ValueError, match="CUDA tensor"):
        amm.decompose_to_tolerance(x, "svd", 0.1)
    with pytest.raises(ValueError, match="CUDA tensor"):
        amm.choose_k(x, "circulant", 0.1)


def test_autotune_table_round_trip(lib):
    """The autotuner's table survives export / import (host only); malformed text installs nothing."""
    import paper_2504_19308_gb300 as amm
    key = lambda n, row, rev, bf16: n * 8 + 4 * row + 2 * rev + bf16
    entries = {key(4096, 0, 0, 0): 1, key(4096, 1, 1, 0): 0, key(96, 0, 0, 1): 1, key(16384, 1, 1, 1): 0}
    text = "amm-autotune 1\n" + "".join("%d %d\n" % kv for kv in sorted(entries.items()))
    amm.autotune_import(text)
    got = amm.autotune_export()
    assert got.startswith("amm-autotune 1\n")
    table = dict(tuple(map(int, ln.split())) for ln in got.splitlines()[1:])
    assert all(table[k] == v for k, v in entries.items())
    assert [int(ln.split()[0]) for ln in got.splitlines()[1:]] == sorted(table)
    for bad in ("amm-autotune 2\n", "tune 1\n", "amm-autotune 1\n%d 2\n" % key(4096, 0, 0, 0),
                "amm-autotune 1\n%d 1\n" % key(40, 0, 0, 0), "amm-autotune 1\n%d 1\nx\n" % key(512, 0, 0, 0),
                "amm-autotune 1\n%d 0\n%d 1\n" % (key(1024, 0, 0, 0), key(80, 0, 0, 0)),
                "amm-autotune 1\n%d\n" % key(2048, 0, 0, 0), "amm-autotune 1\n%d 1.5\n" % key(2048, 0, 0, 0),
                "amm-autotune 1\n-8 1\n", ""):
        with pytest.raises(RuntimeError, match="malformed"):
            amm.autotune_import(bad)
    assert amm.autotune_export() == got                    # nothing from the rejected texts
    small = ctypes.create_string_buffer(4)
    n = ctypes.c_int64(0)
    assert lib.amm_autotune_export(small, 4, ctypes.byref(n)) == 1 and n.value == len(got)
    assert lib.amm_autotune_import(None) == 1


def test_autotune_keys_of_the_other_kernels(lib):
    """Keys carry a kernel id above bit 24 (1: inverse cycle transform, 2 / 3: column / row backward
    spectra, which have no flags); unknown ids and flags on those kernels are rejected."""
    import paper_2504_19308_gb300 as amm
    k = lambda kid, n, flags=0: (kid << 24) | (n << 3) | flags
    amm.autotune_import("amm-autotune 1\n%d 1\n%d 0\n%d 1\n" % (k(1, 4096), k(2, 3072), k(3, 1024)))
    table = dict(tuple(map(int, ln.split())) for ln in amm.autotune_export().splitlines()[1:])
    assert table[k(1, 4096)] == 1 and table[k(2, 3072)] == 0 and table[k(3, 1024)] == 1
    amm.autotune_import("amm-autotune 1\n%d 0\n" % k(1, 4096, 1))     # the accumulating residual form
    for bad in ("amm-autotune 1\n%d 1\n" % k(4, 4096), "amm-autotune 1\n%d 1\n" % k(1, 4096, 2),
                "amm-autotune 1\n%d 1\n" % k(2, 4096, 1), "amm-autotune 1\n%d 1\n" % k(2, 40)):
        with pytest.raises(RuntimeError, match="malformed"):
            amm.autotune_import(bad)


def _tune_child(env_path, code):
    import subprocess
    import sys
    env = dict(os.environ, AMM_TUNE_CACHE=env_path)
    r = subprocess.run([sys.executable, "-c", "import sys; sys.path.insert(0, %r)\n" % ROOT + code], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_autotune_cache_file_is_loaded_at_first_use(lib, tmp_path):
    """AMM_TUNE_CACHE names a text file of exported choices: a new process sees them before it tunes
    anything; a file that does not parse is ignored (an empty table), not an error."""
    path = str(tmp_path / "tune.txt")
    k = 4096 * 8 + 4
    with open(path, "w") as f:
        f.write("amm-autotune 1\n%d 1\n%d 0\n" % (k, (1 << 24) | (4096 << 3)))
    out = _tune_child(path, "import paper_2504_19308_gb300 as amm\nprint(amm.autotune_export())")
    table = dict(tuple(map(int, ln.split())) for ln in out.strip().splitlines()[1:])
    assert table == {k: 1, (1 << 24) | (4096 << 3): 0}
    with open(path, "w") as f:
        f.write("not a table\n")
    out = _tune_child(path, "import paper_2504_19308_gb300 as amm\nprint(amm.autotune_export())")
    assert out.strip() == "amm-autotune 1"


def test_batch_host_logic(lib):
    """Batches record items on the host: arguments are checked when an item is added (before any
    item of the batch launches); a batch that never ran is destroyed without device work."""
    import paper_2504_19308_gb300.amm as amm
    batch = ctypes.c_void_p(0)
    assert lib.amm_batch_create(None) == 1
    assert lib.amm_batch_create(ctypes.byref(batch)) == 0 and batch.value
    fake = ctypes.c_void_p(0x1000)            # recorded, never dereferenced: the batch is not run
    add = lambda *a: lib.amm_batch_add(batch, *a)
    assert add(None, fake, fake, 64, 64, 64, 64, 64, 64, 0, 1, 4, None, None) == 1
    assert add(fake, fake, fake, 64, 64, 64, 32, 64, 64, 0, 1, 4, None, None) == 1   # lda < n
    assert add(fake, fake, fake, 64, 64, 64, 64, 64, 64, 5, 1, 4, None, None) == 1   # dtype
    assert add(fake, fake, fake, 64, 64, 64, 64, 64, 64, 0, 9, 4, None, None) == 1   # method
    bad = amm.Opts()
    assert lib.amm_opts_init(ctypes.byref(bad)) == 0
    bad.struct_size = 8
    assert add(fake, fake, fake, 64, 64, 64, 64, 64, 64, 0, 1, 4, ctypes.byref(bad), None) == 1
    forced = (ctypes.c_int32 * 4)(0, 1, 2, 3)
    fo = amm.Opts()
    assert lib.amm_opts_init(ctypes.byref(fo)) == 0
    fo.forced_selection = ctypes.cast(forced, ctypes.POINTER(ctypes.c_int32))
    assert add(fake, fake, fake, 64, 64, 64, 64, 64, 64, 0, 1, 4, None, ctypes.byref(fo)) == 1
    assert add(fake, fake, fake, 64, 64, 64, 64, 64, 64, 0, 1, 4, None, None) == 0
    assert add(fake, fake, fake, 96, 96, 96, 96, 96, 96, 1, 0, 8, None, None) == 0
    # the persistent executor's switch and wait limit: checked on the host, no device work
    assert lib.amm_batch_set_persistent(None, 1, 10**9) == 1
    assert lib.amm_batch_set_persistent(batch, 1, 0) == 1
    assert lib.amm_batch_set_persistent(batch, 0, 10**9) == 0
    assert lib.amm_batch_set_persistent(batch, 1, 5 * 10**8) == 0
    st, it, sg, npq = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    assert lib.amm_batch_status(batch, None, ctypes.byref(it), ctypes.byref(sg), ctypes.byref(npq)) == 1
    assert lib.amm_batch_status(batch, ctypes.byref(st), ctypes.byref(it), ctypes.byref(sg), ctypes.byref(npq)) == 0
    assert (st.value, it.value, sg.value, npq.value) == (0, -1, -1, 0)   # never ran
    assert lib.amm_debug_persistent_wait_timeout(0, None, ctypes.byref(st), ctypes.byref(sg)) == 1
    assert lib.amm_debug_persistent_wait_timeout(10**6, None, None, ctypes.byref(sg)) == 1
    assert lib.amm_batch_destroy(batch) == 0
    assert lib.amm_batch_destroy(None) == 1


def test_last_error_is_per_thread(lib):
    """amm_last_error is thread-local: a failure on one thread leaves another thread's reason."""
    import threading
    assert lib.amm_decompose(None, 64, 64, 64, 0, 1, 4, None, None, ctypes.byref(ctypes.c_void_p(0))) == 1
    mine = lib.amm_last_error()
    assert b"A is NULL" in mine
    seen = {}

    def other():
        seen["before"] = lib.amm_last_error()
        lib.amm_batch_destroy(None)
        seen["after"] = lib.amm_last_error()

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["before"] == b"" and b"amm_batch_destroy" in seen["after"]
    assert lib.amm_last_error() == mine
