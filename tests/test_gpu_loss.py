"""The training losses on the GPU against the float64 oracle (Sec. 3.4.1, Eq. 11).

gabsplat_loss (mean L1 / L2) rounds each difference to float32 once and sums with compensated
float32 per thread and float64 across threads, so its value must agree with the oracle to the
rounding of the differences (2^-24 relative, twice that for L2) and its L1 gradient bit for bit.

gabsplat_loss_l1_dssim computes in float32.  Its bars follow from that arithmetic: a local
variance w*x^2 - mx^2 carries an absolute error of about 1e-7, which the SSIM denominator
(>= C2 = 9e-4) magnifies to about 1e-4 relative in flat regions.  So the loss, a mean of values
in [0, 2], must agree to 5e-5.  The gradient combines terms up to 1/C2 ~ 1e3 times its size in
flat regions, so it must agree to 1e-3 relative L2, and to 1e-2 of the largest magnitude per
element.  The shapes cover several 32 x 32 tiles with ragged tails, images smaller than the
window, a single pixel and the full 3 x 1064 x 1600 training image with flat patches.
"""
import numpy as np
import pytest
import torch

from oracle import gabsplat_oracle as O
from tests.conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def images(shape, seed, flat=False):
    rng = np.random.default_rng(seed)
    x = rng.random(shape).astype(np.float32)
    y = rng.random(shape).astype(np.float32)
    if flat:                                   # smooth content and flat patches, like a render
        C, H, W = shape
        yy, xx = np.mgrid[0:H, 0:W] / max(H, W)
        x = (0.5 + 0.4 * np.sin(7 * xx + 3 * yy))[None].repeat(C, 0).astype(np.float32) * x ** 0.1
        x[:, : H // 3, : W // 4] = 0.0         # background
        x[:, H // 2:, W // 2:] = 0.25          # constant patch
        y[:, H // 2:, : W // 3] = 0.6
    return x, y


def gpu_l1_dssim(B, x, y, lam):
    X, Y = torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dL = torch.full_like(X, float("nan"))
    scratch = torch.empty(B.gabsplat_loss_l1_dssim_scratch_bytes(*x.shape), dtype=torch.uint8, device="cuda")
    B.gabsplat_loss_l1_dssim(X, Y, lam, loss, dL, scratch)
    torch.cuda.synchronize()
    return loss.item(), dL.cpu().numpy()


@pytest.mark.parametrize("shape,seed,flat,lam", [
    ((3, 37, 53), 1, False, 0.2),       # two tile columns and two tile rows, ragged
    ((1, 5, 7), 2, False, 0.2),         # smaller than the window
    ((2, 64, 96), 3, True, 0.2),        # whole tiles, flat patches
    ((3, 1, 1), 4, False, 0.2),         # one pixel
    ((3, 70, 41), 5, True, 0.0),        # lambda = 0: plain L1
    ((3, 33, 65), 6, True, 1.0),        # lambda = 1: D-SSIM alone
])
def test_l1_dssim_matches_oracle(shape, seed, flat, lam):
    from paper_2508_05343_b300 import binding as B
    x, y = images(shape, seed, flat)
    got_l, got_g = gpu_l1_dssim(B, x, y, lam)
    ref_l, ref_g = O.l1_dssim_loss_and_grad(x, y, lam=lam)
    assert np.all(np.isfinite(got_g))
    assert abs(got_l - ref_l) <= 5e-5, (got_l, ref_l)
    rel = np.linalg.norm(got_g - ref_g) / max(np.linalg.norm(ref_g), 1e-30)
    assert rel <= 1e-3, rel
    assert np.abs(got_g - ref_g).max() <= 1e-2 * np.abs(ref_g).max()


def test_l1_dssim_full_training_image():
    from paper_2508_05343_b300 import binding as B
    x, y = images((3, 1064, 1600), 7, flat=True)
    got_l, got_g = gpu_l1_dssim(B, x, y, 0.2)
    ref_l, ref_g = O.l1_dssim_loss_and_grad(x, y, lam=0.2)
    assert abs(got_l - ref_l) <= 5e-5, (got_l, ref_l)
    rel = np.linalg.norm(got_g - ref_g) / np.linalg.norm(ref_g)
    assert rel <= 1e-3, rel
    assert np.abs(got_g - ref_g).max() <= 1e-2 * np.abs(ref_g).max()


def test_l1_dssim_rejects_bad_arguments():
    from paper_2508_05343_b300 import binding as B
    x = torch.zeros(3, 8, 8, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    scratch = torch.empty(64, dtype=torch.uint8, device="cuda")
    for lam in (-0.1, 1.5, float("nan")):
        with pytest.raises(B.GabsplatError):
            B.gabsplat_loss_l1_dssim(x, x, lam, loss, x, scratch)
    assert B.gabsplat_loss_l1_dssim_scratch_bytes(0, 8, 8) == 0
    assert B.gabsplat_loss_l1_dssim_scratch_bytes(3, 8, 40000) == 0


@pytest.mark.parametrize("kind", ["l1", "l2"])
def test_photometric_loss_matches_oracle(kind):
    from paper_2508_05343_b300 import binding as B
    for shape, seed in (((3, 1064, 1600), 11), ((3, 17, 29), 12)):
        x, y = images(shape, seed)
        X, Y = torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        dL = torch.empty_like(X)
        scratch = torch.empty(B.gabsplat_loss_scratch_bytes(X.numel()), dtype=torch.uint8, device="cuda")
        B.gabsplat_loss(X, Y, B.GS_LOSS_L1 if kind == "l1" else B.GS_LOSS_L2, loss, dL, scratch)
        torch.cuda.synchronize()
        ref_l, ref_g = O.loss_and_grad(x, y, kind)
        # x - y is rounded to float32 once (2^-24 relative), |d| exactly and d^2 once more; the
        # compensated sum adds ~1e-13
        np.testing.assert_allclose(loss.item(), ref_l, rtol=1e-7 if kind == "l1" else 2e-7)
        if kind == "l1":
            np.testing.assert_array_equal(dL.cpu().numpy(), ref_g.astype(np.float32))
        else:
            # 2 d / N: the float32 difference, then the float32 result: two roundings
            np.testing.assert_allclose(dL.cpu().numpy(), ref_g, rtol=1.5e-7, atol=0)
