"""GPU quality measures (fe_ssim, fe_psnr) against the oracle's plain
definitions.  Both accumulate in FP64 on the GPU (the moments of SSIM, the
squared differences of PSNR) from FP32 images, so they agree with the FP64
oracle to rounding: 1e-9 relative."""
import numpy as np
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


@pytest.mark.parametrize("shape", [(11, 11), (64, 80), (131, 77), (300, 45)])
def test_ssim_and_psnr_parity(fe, shape):
    import torch
    from oracle import quality
    from paper_1404_5344_gb300 import synth
    H, W = shape
    clean = synth.textured_image(H, W, seed=H + W)
    noisy = synth.speckle(clean, L=4.0, seed=H * W)
    x, y = torch.from_numpy(noisy).cuda(), torch.from_numpy(clean).cuda()
    assert fe.ssim(x, y) == pytest.approx(quality.ssim(noisy, clean), rel=1e-9)
    assert fe.psnr(x, y) == pytest.approx(quality.psnr(noisy, clean), rel=1e-9)
    assert fe.ssim(y, y) == pytest.approx(1.0, abs=1e-12)
    assert fe.psnr(y, y) == float("inf")


def test_quality_invalid_arguments(fe):
    import torch
    x = torch.ones((10, 40), device="cuda")
    with pytest.raises(fe.FeError):
        fe.ssim(x, x)  # smaller than the window
    h = np.ones((20, 20), np.float32)
    with pytest.raises(fe.FeError):
        fe.ssim(h, h)  # host arrays
    y = torch.ones((20, 20), device="cuda")
    with pytest.raises(fe.FeError):
        fe.ssim(y, y, peak=0.0)
