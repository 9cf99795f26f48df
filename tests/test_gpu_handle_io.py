"""Export / import of a decomposition's device state (an offline weight decomposition reused by
another process, Section 4): the imported handle's products and gradients equal the original's
bit for bit, in this process and in a fresh one, and malformed strings are rejected."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
import synth as S
from gpu_util import TOL, as64, dev32, rel, torch_cuda

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cases(torch, amm):
    n = 512
    a, b = S.general_times_toeplitz(n, seed=21)
    A, B = dev32(torch, a), dev32(torch, b)
    sk = dev32(torch, S.sketch(n, 16, 21, 1))
    W = dev32(torch, S.rng(21, 3).standard_normal((384, 640)) + 0.5)   # ragged blocks: padded copy
    return A, B, W, [("circulant", 9, {}), ("svd", 16, {"sketch": sk}), ("cycle", 8, {}), ("fourier", 12, {}),
                     ("circulant", 7, {"store_spectra": False}), ("svd", 16, {"sketch": sk, "compute": "bf16"})]


def test_export_import_same_process_bit_identical():
    torch, amm = torch_cuda()
    A, B, W, cases = _cases(torch, amm)
    G = dev32(torch, S.upstream_grad(512, 512, 21))
    for method, k, kw in cases:
        ka = dict(kw)
        if method == "svd":
            ka["sketch"] = dev32(torch, S.sketch(512, k, 21, 0))
        hA = amm.decompose(A, method, k, "left", **ka)
        hB = amm.decompose(B, method, k, "right", **kw)
        iA = amm.import_handle(hA.export(), A, method, k, "left")
        iB = amm.import_handle(hB.export(), B, method, k, "right")
        assert iA.device_bytes() <= hA.device_bytes() and iB.device_bytes() <= hB.device_bytes()
        assert torch.equal(amm.approx_matmul(hA, hB), amm.approx_matmul(iA, iB)), method
        for g0, g1 in zip(amm.approx_matmul_backward(hA, hB, G), amm.approx_matmul_backward(iA, iB, G)):
            assert torch.equal(g0, g1), method
        # the original may go away: the import owns its own buffers
        hA.close()
        hB.close()
        C = amm.approx_matmul(iA, iB)
        assert torch.isfinite(C).all()
    # blocked circulant weights: blocks of the operand itself (384 x 640 in 128-blocks) and of a
    # zero-padded copy (400 x 600 padded to 512 x 640)
    for Wb in (W, dev32(torch, S.rng(21, 5).standard_normal((400, 600)) + 0.5)):
        kx = Wb.shape[0]
        hx = amm.decompose(dev32(torch, S.rng(21, 4).standard_normal((256, kx))), "svd", 16, "left",
                           sketch=dev32(torch, S.sketch(kx, 16, 21, 0)))
        hw = amm.decompose(Wb, "circulant", 5, "right", block=128)
        iw = amm.import_handle(hw.export(), Wb, "circulant", 5, "right", block=128)
        assert torch.equal(amm.approx_matmul(hx, hw), amm.approx_matmul(hx, iw))
        assert np.array_equal(hw.selection(), iw.selection())


def test_import_rejects_malformed_strings_and_other_operands():
    torch, amm = torch_cuda()
    A, B, W, _ = _cases(torch, amm)
    blob = amm.decompose(A, "circulant", 9, "left").export()
    for bad in (blob[:-1], blob[:40], b"XXXX" + blob[4:], blob + b"\0"):
        with pytest.raises(amm.AmmError):
            amm.import_handle(bad, A, "circulant", 9)
    with pytest.raises(amm.AmmError):           # another shape
        amm.import_handle(blob, W, "circulant", 9)


def test_import_in_a_fresh_process(tmp_path):
    """The weight is decomposed here; a second process imports the string, multiplies with its
    own decomposition of the other operand and matches the product computed here and the oracle."""
    torch, amm = torch_cuda()
    n, k = 512, 9
    a, b = S.general_times_toeplitz(n, seed=22)
    A, B = dev32(torch, a), dev32(torch, b)
    hB = amm.decompose(B, "circulant", k, "right")
    (tmp_path / "w.bin").write_bytes(hB.export())
    C = amm.approx_matmul(amm.decompose(A, "circulant", k, "left"), hB)
    np.save(tmp_path / "c.npy", C.cpu().numpy())
    code = r'''
import sys, numpy as np, torch
sys.path.insert(0, %r)
sys.path.insert(0, %r)
import synth as S, paper_2504_19308_gb300 as amm
from gpu_util import dev32
a, b = S.general_times_toeplitz(%d, seed=22)
A, B = dev32(torch, a), dev32(torch, b)
hB = amm.import_handle(open(%r, "rb").read(), B, "circulant", %d, "right")
C = amm.approx_matmul(amm.decompose(A, "circulant", %d, "left"), hB)
assert np.array_equal(C.cpu().numpy(), np.load(%r)), "imported product differs"
print("ok")
''' % (ROOT, os.path.join(ROOT, "tests"), n, str(tmp_path / "w.bin"), k, k, str(tmp_path / "c.npy"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]
    hA = amm.decompose(A, "circulant", k, "left")
    ref = O.cd_matmul(as64(A), as64(B), k, sel_a=hA.selection(), sel_b=hB.selection())
    assert rel(C.double().cpu().numpy(), ref) <= TOL
