"""The tensor-core building block (tcgen05.mma, K-major operands in shared
memory, FP32 accumulation in tensor memory) against a plain NumPy product of
the same rounded operands."""
import numpy as np
import pytest

from rounding import round_bf16, round_tf32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_5344_gb300 import build
    build.build()
    from paper_1404_5344_gb300 import fe as fe_mod
    return fe_mod


def _run(fe, prec, N, K, A, B):
    D = np.empty((128, N), np.float32)
    st = fe.lib.fe_tc_gemm_selftest(prec, N, K, A.ctypes.data, B.ctypes.data, D.ctypes.data)
    assert st == fe.FE_OK, fe.lib.fe_status_string(st)
    return D


@pytest.mark.parametrize("prec,K", [(2, 16), (2, 64), (2, 128), (1, 8), (1, 56), (1, 112)])
@pytest.mark.parametrize("N", [16, 48, 64])
def test_exact_integer_products(fe, prec, K, N):
    """Small integers are exact in both operand types and their dot products
    are exact in FP32: the result must match bit for bit, which pins the
    operand layout, the descriptors and the accumulation over K steps."""
    rng = np.random.default_rng(prec * 1000 + K * 10 + N)
    A = rng.integers(-8, 9, (128, K)).astype(np.float32)
    B = rng.integers(-8, 9, (N, K)).astype(np.float32)
    D = _run(fe, prec, N, K, A, B)
    np.testing.assert_array_equal(D, A.astype(np.float64) @ B.T.astype(np.float64))


@pytest.mark.parametrize("prec", [1, 2])
def test_rounded_real_operands(fe, prec):
    rng = np.random.default_rng(prec)
    K = 64
    A = rng.standard_normal((128, K)).astype(np.float32) * 50
    B = rng.standard_normal((48, K)).astype(np.float32) * 0.2
    rnd = round_bf16 if prec == 2 else round_tf32
    ref = rnd(A).astype(np.float64) @ rnd(B).T.astype(np.float64)
    D = _run(fe, prec, 48, K, A, B)
    scale = np.abs(rnd(A)).astype(np.float64) @ np.abs(rnd(B)).T
    assert np.max(np.abs(D - ref) / scale) < 1e-6


def test_bounded_wait_gives_up_and_the_context_stays_usable(fe):
    """An mbarrier wait that nothing completes gives up after its bound,
    frees its tensor memory and leaves the context usable: a tensor-core
    GEMM runs correctly right after it."""
    import ctypes as C
    t = C.c_int(-1)
    assert fe.lib.fe_tc_wait_selftest(2000, C.byref(t)) == fe.FE_ETIMEOUT
    assert t.value == 1
    rng = np.random.default_rng(0)
    A = rng.standard_normal((128, 32)).astype(np.float32)
    B = rng.standard_normal((16, 32)).astype(np.float32)
    D = np.empty((128, 16), np.float32)
    st = fe.lib.fe_tc_gemm_selftest(fe.FE_BF16, 16, 32, A.ctypes.data, B.ctypes.data, D.ctypes.data)
    assert st == fe.FE_OK
    ref = round_bf16(A).astype(np.float64) @ round_bf16(B).astype(np.float64).T
    np.testing.assert_allclose(D, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
