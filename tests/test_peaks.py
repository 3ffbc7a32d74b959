"""fe_peak: the measured roofline denominators (peak-rate microbenchmarks).

Each kind runs through the C ABI on the GPU; its rate must be positive and
within a plausible range of the device's unit counts (a kernel whose work the
compiler folded away would report an impossible rate).  Bounds use the SM
count from the device and a maximum clock of 2.1 GHz; the tensor-core bounds
use the nominal dense rates (2.25 PFLOP/s BF16, 1.1 TF32) with wide margins.
"""
import pytest

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


def test_peak_rates_are_plausible(fe):
    sms = fe.device_sms()
    assert sms > 0
    clk = 2.1e9
    r = {k: fe.peak(k, target_ms=5.0, reps=2)["rate"] for k in fe.PEAK_KINDS}
    ffma_max = sms * 128 * 2 * clk
    assert 0.3 * ffma_max < r["ffma"] <= ffma_max
    # the packed form does at least the scalar form's work per second
    assert 0.9 * r["ffma"] < r["ffma2"] <= 2.0 * ffma_max
    assert 0 < r["dfma"] < r["ffma"]
    for k in ("mufu_rcp", "mufu_lg2"):
        assert 0 < r[k] <= sms * 64 * clk, k
    assert 0.3 * 2.25e15 < r["tc_bf16"] < 1.3 * 2.25e15
    assert 0.3 * 1.1e15 < r["tc_tf32"] < 1.3 * 2.25e15


def test_peak_rejects_bad_arguments(fe):
    import ctypes as C
    d = C.c_double()
    assert fe.lib.fe_peak(7, 5.0, 1, C.byref(d), None, None) == fe.FE_EINVAL
    assert fe.lib.fe_peak(0, 5.0, 0, C.byref(d), None, None) == fe.FE_EINVAL
    assert fe.lib.fe_peak(0, 0.0, 1, C.byref(d), None, None) == fe.FE_EINVAL
    assert fe.lib.fe_peak(0, 5.0, 1, None, None, None) == fe.FE_EINVAL
