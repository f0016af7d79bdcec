"""The tcgen05 split-bf16 GEMM behind the complex64 Taylor powers.

Layout and descriptor pins are bit-exact: small-integer operands are exact in
bf16 and their products and sums are exact in fp32, so any swizzle, transpose
or K-offset mistake shows up as a mismatch.  Accuracy per slice count is
checked against a float64 product.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _run(hw, A, B, slices):
    import torch
    a = torch.from_numpy(A).cuda()
    b = torch.from_numpy(B).cuda()
    c = torch.full((A.shape[0], B.shape[0]), float("nan"), dtype=torch.float32, device="cuda")
    hw.hw_gemm_tc(a, b, c, slices)
    return c.cpu().numpy()


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (256, 384, 512), (300, 200, 100), (1, 130, 7),
                                   (513, 129, 1000)])
def test_small_integers_exact(hw, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.integers(-3, 4, size=(m, k)).astype(np.float32)
    B = rng.integers(-3, 4, size=(n, k)).astype(np.float32)
    C = _run(hw, A, B, 1)
    assert np.array_equal(C, (A.astype(np.float64) @ B.T.astype(np.float64)).astype(np.float32))


def test_small_integers_exact_fp16_scaled(hw):
    # fp16 mode scales each operand by a power of two (exact) and splits in two
    # slices: integers up to 2^10 are exact in the leading slice
    rng = np.random.default_rng(5)
    A = rng.integers(-1000, 1001, size=(256, 320)).astype(np.float32)
    B = rng.integers(-1000, 1001, size=(200, 320)).astype(np.float32)
    C = _run(hw, A, B, 4)
    ref = A.astype(np.float64) @ B.T.astype(np.float64)
    assert np.max(np.abs(C - ref)) <= 2.0 ** -22 * np.abs(ref).max() * 4


def test_identity_transposes(hw):
    n = 256
    B = synth.complex_gaussian(3, n * n).real.reshape(n, n).astype(np.float32)
    C = _run(hw, np.eye(n, dtype=np.float32), B, 3)
    assert np.array_equal(C, B.T)


@pytest.mark.parametrize("slices,rel", [(3, 2e-6), (2, 1e-4), (1, 2e-2), (4, 4e-6)])
def test_split_accuracy(hw, slices, rel):
    m, n, k = 384, 256, 1024
    A = synth.complex_gaussian(1, m * k).real.reshape(m, k).astype(np.float32)
    B = synth.complex_gaussian(2, n * k).real.reshape(n, k).astype(np.float32)
    C = _run(hw, A, B, slices)
    ref = A.astype(np.float64) @ B.T.astype(np.float64)
    bound = np.outer(np.linalg.norm(A, axis=1), np.linalg.norm(B, axis=1))
    assert np.max(np.abs(C - ref) / bound) < rel


def test_rejects_operands_not_on_the_device(hw):
    # the tensor-core GEMM takes device memory of the current device only
    import ctypes
    import torch
    m, n, k = 128, 128, 64
    host = np.zeros((m, k), dtype=np.float32)
    pinned = torch.zeros((m, k), dtype=torch.float32).pin_memory()
    dev_b = torch.zeros((n, k), dtype=torch.float32, device="cuda")
    dev_c = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    for a_ptr in (host.ctypes.data, pinned.data_ptr()):
        st = hw.lib().hw_gemm_tc(m, n, k, ctypes.c_void_p(a_ptr), ctypes.c_void_p(dev_b.data_ptr()),
                                 ctypes.c_void_p(dev_c.data_ptr()), 1, None)
        assert st == hw.HW_EINVAL
