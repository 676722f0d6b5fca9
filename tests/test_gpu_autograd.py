"""The differentiable rasterizer as a torch.autograd.Function (raster.render / GabSplatRender).

Gradients of a loss through the Function are checked against the FP64 oracle's analytic gradients
(1e-3 relative L2 per attribute group), for FP32 storage and for BF16 storage of the SH, frequency
and weight tensors; the dtype rules for BF16 inputs are checked; and a second forward on the same
rasterizer before the first one's backward does not change the first one's gradients.  The loss is
linear in the image, L = sum(image * G) with a fixed seeded G (zero at the pixels the oracle flags),
so dL/dimage is the same on both sides.
"""
import numpy as np
import pytest
import torch

from oracle import gabsplat_oracle as O
from paper_2508_05343_b300 import scenes
from tests.conftest import cuda_available
from tests.gpu_util import ATTRS, GRAD_TOL, bf16_prims, cfg_pair, rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def _scene():
    spec = scenes.SceneSpec(n=800, K=4, sh_degree=2, layout="uniform", box=1.0, log_scale=(-2.8, 0.5))
    return scenes.make_scene(spec, 515), scenes.orbit_camera(96, 80, 35.0, 12.0, 3.5)


def _leaves(prims, dtypes=None):
    dtypes = dtypes or {}
    return {k: torch.tensor(np.asarray(prims[k]), dtype=dtypes.get(k, torch.float32), device="cuda",
                            requires_grad=True) for k in ATTRS}


def _render_grads(rast, cam, gc, leaves, G, storage):
    from paper_2508_05343_b300 import raster
    img = raster.render(rast, cam, gc, *[leaves[k] for k in ATTRS], storage=storage)
    loss = (img * G).sum()
    grads = torch.autograd.grad(loss, [leaves[k] for k in ATTRS])
    return img, dict(zip(ATTRS, grads))


def _weight_image(out, cam, seed):
    G = np.random.default_rng(seed).standard_normal((3, cam["height"], cam["width"])) * 1e-2
    G[:, out["ambiguous_bwd"].numpy()] = 0.0
    return G


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_autograd_function_matches_oracle_gradients(storage):
    """FP32 leaves; with storage "bf16" the Function rounds SH / frequencies / weights for the
    kernels and the oracle consumes the same rounded values.  The gradients reach the FP32 leaves
    unrounded (the rounding passes straight through)."""
    from paper_2508_05343_b300 import raster
    prims, cam = _scene()
    oc, gc = cfg_pair(bg=(0.1, 0.2, 0.3))
    ref_prims = bf16_prims(prims) if storage == "bf16" else prims
    out = O.render(ref_prims, cam, oc)
    G = _weight_image(out, cam, 7)
    ref = O.render_backward(ref_prims, cam, oc, G)
    rast = raster.Rasterizer(prims["n"], prims["K"], prims["sh_degree"], cam["width"], cam["height"])
    leaves = _leaves(prims)
    _, g = _render_grads(rast, cam, gc, leaves, torch.as_tensor(G, dtype=torch.float32, device="cuda"), storage)
    assert all(v.dtype == torch.float32 for v in g.values())
    errs = {k: rel_l2(g[k].cpu().numpy(), ref[k]) for k in ATTRS}
    assert all(e <= GRAD_TOL for e in errs.values()), errs


def test_autograd_function_bf16_leaves_get_bf16_gradients():
    """BF16 leaves for SH / frequencies / weights: the same kernels run (the values are already
    BF16), and those leaves receive the FP32 gradient rounded to BF16, while the FP32 leaves keep
    FP32 gradients.  The FP32 reference comes from FP32 master leaves holding the same values."""
    from paper_2508_05343_b300 import raster
    prims, cam = _scene()
    prims = bf16_prims(prims)
    _, gc = cfg_pair(bg=(0.1, 0.2, 0.3))
    G = torch.as_tensor(np.random.default_rng(8).standard_normal((3, cam["height"], cam["width"])) * 1e-2,
                        dtype=torch.float32, device="cuda")
    rast = raster.Rasterizer(prims["n"], prims["K"], prims["sh_degree"], cam["width"], cam["height"])
    bf = {k: torch.bfloat16 for k in ("sh", "freqs", "weights")}
    img_b, g_b = _render_grads(rast, cam, gc, _leaves(prims, bf), G, "bf16")
    img_f, g_f = _render_grads(rast, cam, gc, _leaves(prims), G, "bf16")
    assert torch.equal(img_b, img_f)
    for k in ATTRS:
        assert g_b[k].dtype == (torch.bfloat16 if k in bf else torch.float32), k
        a, b = g_b[k].float().cpu().numpy(), g_f[k].cpu().numpy()
        # rounding to BF16 (8 significant bits) on top of float-atomic ordering differences
        assert rel_l2(a, b) <= 2.0 ** -8, k


def test_second_forward_before_backward_keeps_gradients():
    """Two forwards of different views on one Rasterizer, then the first view's backward: its
    gradients equal those of the first view rendered alone (the Function re-renders its own
    inputs when the workspace has moved on), and the second view's backward is unaffected."""
    from paper_2508_05343_b300 import raster
    prims, cam = _scene()
    cam2 = scenes.orbit_camera(cam["width"], cam["height"], 80.0, -5.0, 3.2)
    _, gc = cfg_pair()
    G = torch.as_tensor(np.random.default_rng(9).standard_normal((3, cam["height"], cam["width"])) * 1e-2,
                        dtype=torch.float32, device="cuda")

    def alone(c):
        r = raster.Rasterizer(prims["n"], prims["K"], prims["sh_degree"], cam["width"], cam["height"])
        return _render_grads(r, c, gc, _leaves(prims), G, "f32")

    img1_ref, g1_ref = alone(cam)
    img2_ref, g2_ref = alone(cam2)
    rast = raster.Rasterizer(prims["n"], prims["K"], prims["sh_degree"], cam["width"], cam["height"])
    l1, l2 = _leaves(prims), _leaves(prims)
    img1 = raster.render(rast, cam, gc, *[l1[k] for k in ATTRS])
    img2 = raster.render(rast, cam2, gc, *[l2[k] for k in ATTRS])
    assert torch.equal(img1, img1_ref) and torch.equal(img2, img2_ref)
    g1 = dict(zip(ATTRS, torch.autograd.grad((img1 * G).sum(), [l1[k] for k in ATTRS])))
    g2 = dict(zip(ATTRS, torch.autograd.grad((img2 * G).sum(), [l2[k] for k in ATTRS])))
    for g, ref in ((g1, g1_ref), (g2, g2_ref)):
        for k in ATTRS:
            assert rel_l2(g[k].cpu().numpy(), ref[k].cpu().numpy()) <= 1e-5, k
    assert rel_l2(g1["means"].cpu().numpy(), g2["means"].cpu().numpy()) > 1e-2   # the views differ
