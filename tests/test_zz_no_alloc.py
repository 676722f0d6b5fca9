"""gabsplat_loss_noalloc: the loss entry point for callers that cannot allocate device memory.

Such callers (a plug-in inside another engine's frame loop that owns the device heap, a service
under a fixed memory budget) cannot provide the scratch buffer gabsplat_loss asks for; this entry
point keeps its per-block partial sums in a fixed array inside the library instead.  The test
calls it through the C ABI twice in a row, on different inputs (the second smaller than the first,
so stale partial sums from the first call would show), and compares each result with
gabsplat_loss.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from tests.conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def _reference_loss(B, img, tgt, kind):
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dL = torch.empty_like(img)
    scratch = torch.empty(B.gabsplat_loss_scratch_bytes(img.numel()), dtype=torch.uint8, device="cuda")
    B.gabsplat_loss(img, tgt, kind, loss, dL, scratch)
    return loss, dL


def test_noalloc_loss_matches_gabsplat_loss_on_two_calls():
    from paper_2508_05343_b300 import binding as B
    gen = torch.Generator(device="cuda").manual_seed(7)
    shapes = [(3, 1064, 1600), (3, 333, 517)]            # second call smaller than the first
    for call, (shape, kind) in enumerate(zip(shapes, (B.GS_LOSS_L1, B.GS_LOSS_L2))):
        img = torch.rand(shape, device="cuda", generator=gen)
        tgt = torch.rand(shape, device="cuda", generator=gen)
        ref_loss, ref_dL = _reference_loss(B, img, tgt, kind)
        loss = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        dL = torch.full_like(img, float("nan"))
        st = B.lib.gabsplat_loss_noalloc(C.c_void_p(img.data_ptr()), C.c_void_p(tgt.data_ptr()), img.numel(), kind,
                                         C.c_void_p(loss.data_ptr()), C.c_void_p(dL.data_ptr()),
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == B.GS_OK, (call, B.status_string(st))
        torch.cuda.synchronize()
        np.testing.assert_allclose(loss.item(), ref_loss.item(), rtol=1e-12)
        np.testing.assert_allclose(dL.cpu().numpy(), ref_dL.cpu().numpy(), rtol=1e-6, atol=0)


def test_noalloc_loss_rejects_counts_beyond_its_fixed_scratch():
    from paper_2508_05343_b300 import binding as B
    p = C.c_void_p(0x1000)      # never dereferenced: the size check comes first
    too_many = 33554432 + 1
    assert B.lib.gabsplat_loss_noalloc(p, p, too_many, B.GS_LOSS_L1, p, p, None) == B.GS_ERR_INVALID_ARG
