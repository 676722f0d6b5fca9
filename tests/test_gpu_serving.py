"""Batched frames and the continuous-batching server on the GPU.

Each view rendered in a batch (direct launches or graph replay) or through the server must be
bit-identical to the same view rendered alone with the single-view path; the BF16-storage path is
checked against the float64 oracle evaluated on the same rounded values (>= 60 dB PSNR)."""
import numpy as np
import pytest
import torch

from oracle import gabsplat_oracle as O
from paper_2508_05343_b300 import scenes
from tests.conftest import cuda_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

SIZES = (20_000, 60_000, 35_000)


def small_scenes():
    spec = scenes.CONFIGS[2][0]
    return [scenes.make_scene(spec, 900 + i, n=n) for i, n in enumerate(SIZES)]


VIEWS_A = [(0, 160, 120, 10.0, 0.0), (2, 200, 200, 120.0, 20.0), (1, 96, 64, 300.0, -15.0), (0, 320, 180, 250.0, 5.0)]
VIEWS_B = [(1, 128, 128, 45.0, 10.0), (2, 64, 200, 190.0, -25.0)]


def batch_frame(B, K, deg, storage, max_views=8, max_prims=200_000, max_tiles=2000, max_pixels=400_000,
                pairs=4_000_000):
    f = B.gs_batch_frame()
    f.max_views, f.K, f.sh_degree, f.storage = max_views, K, deg, storage
    f.max_prims, f.max_tiles, f.max_pixels, f.pair_capacity = max_prims, max_tiles, max_pixels, pairs
    nbytes = B.gabsplat_batch_workspace_size(max_views, K, deg, max_prims, max_tiles, max_pixels, pairs)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    f.ws, f.ws_bytes = ws.data_ptr(), nbytes
    B.gabsplat_batch_workspace_init(f)
    return f, ws


def alone(prims, view, storage):
    from paper_2508_05343_b300 import binding as B
    from paper_2508_05343_b300 import raster
    si, w, h, az, el = view
    p = prims[si]
    r = raster.Rasterizer(p["means"].shape[0], p["weights"].shape[1], 3, w, h)
    img = r.forward(raster.to_device(p, storage=storage), scenes.orbit_camera(w, h, az, el), B.make_config(),
                    storage=storage)
    torch.cuda.synchronize()
    return img


def render_views(B, f, dev_scenes, prim_structs, views, launch):
    outs = [torch.full((3, h, w), float("nan"), device="cuda") for (_, w, h, _, _) in views]
    vs = [B.make_view(prim_structs[si], B.make_camera(scenes.orbit_camera(w, h, az, el)), o)
          for (si, w, h, az, el), o in zip(views, outs)]
    launch(vs)
    status = torch.zeros(2, dtype=torch.int64).pin_memory()
    B.gabsplat_batch_status_copy(f, status.data_ptr())
    torch.cuda.synchronize()
    assert int(status[0].item() & 0xFFFFFFFF) == B.GS_OK
    return outs


@pytest.mark.parametrize("storage", [0, 1])
def test_batched_views_bit_identical_to_single_view_renders(storage):
    from paper_2508_05343_b300 import binding as B
    from paper_2508_05343_b300 import raster
    prims = small_scenes()
    dev = [raster.to_device(p, storage=storage) for p in prims]
    ps = [B.make_prims(t, storage) for t in dev]
    f, ws = batch_frame(B, 4, 3, storage)
    cfg = B.make_config()
    outs = render_views(B, f, dev, ps, VIEWS_A, lambda vs: B.gabsplat_render_batch(f, vs, cfg))
    for view, out in zip(VIEWS_A, outs):
        assert torch.equal(out, alone(prims, view, storage)), view


def test_graph_replay_matches_direct_launches_across_batches():
    from paper_2508_05343_b300 import binding as B
    from paper_2508_05343_b300 import raster
    prims = small_scenes()
    dev = [raster.to_device(p) for p in prims]
    ps = [B.make_prims(t) for t in dev]
    cfg = B.make_config(bg=(0.2, 0.1, 0.0))
    f, ws = batch_frame(B, 4, 3, 0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = B.gabsplat_batch_graph_create(f, cfg)
        got = [render_views(B, f, dev, ps, views, lambda vs: B.gabsplat_batch_graph_launch(g, vs))
               for views in (VIEWS_A, VIEWS_B, VIEWS_A)]
        B.gabsplat_batch_graph_destroy(g)
    f2, ws2 = batch_frame(B, 4, 3, 0)
    for views, outs in zip((VIEWS_A, VIEWS_B, VIEWS_A), got):
        ref = render_views(B, f2, dev, ps, views, lambda vs: B.gabsplat_render_batch(f2, vs, cfg))
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)


def test_batch_rejects_views_beyond_capacity():
    from paper_2508_05343_b300 import binding as B
    from paper_2508_05343_b300 import raster
    prims = small_scenes()
    dev = [raster.to_device(p) for p in prims]
    ps = [B.make_prims(t) for t in dev]
    f, ws = batch_frame(B, 4, 3, 0, max_views=2, max_prims=100_000)
    cfg = B.make_config()
    with pytest.raises(B.GabsplatError):          # three views > max_views
        render_views(B, f, dev, ps, VIEWS_A[:3], lambda vs: B.gabsplat_render_batch(f, vs, cfg))
    with pytest.raises(B.GabsplatError) as e:     # 60k + 35k + 20k... two views of 60k + 60k > 100k
        render_views(B, f, dev, ps, [(1, 64, 64, 0.0, 0.0), (1, 64, 64, 90.0, 0.0)],
                     lambda vs: B.gabsplat_render_batch(f, vs, cfg))
    assert e.value.status == B.GS_ERR_CAPACITY


@pytest.mark.parametrize("realtime", [False, True])
def test_server_results_same_alone_and_in_the_mix(realtime):
    from paper_2508_05343_b300 import binding as B
    from paper_2508_05343_b300 import serve
    prims = small_scenes()
    res = [(96, 96), (160, 120), (200, 112)]
    reqs = serve.make_requests(n_req=36, rate=3000.0, n_scenes=len(prims), seed=77, resolutions=res)
    lim = serve.SlotLimits(max_views=6, max_prims=400_000, max_tiles=6 * 130, max_pixels=6 * 200 * 120,
                           pair_capacity=3_000_000)
    srv = serve.Server(prims, B.GS_BF16, 4, 3, limits=lim, n_slots=2)
    srv.calibrate(res)
    out = srv.run(reqs, realtime=realtime, keep_images=True)
    assert len(out["images"]) == len(reqs) and out["refused"] == 0
    if not realtime:
        assert out["mean_batch"] > 1.0             # offered at once, requests are batched together
    for r in reqs:
        ref = alone(prims, (r.scene, r.width, r.height, r.azimuth, r.elevation), B.GS_BF16)
        assert torch.equal(out["images"][r.rid], ref), r


def test_bf16_storage_error_against_the_oracle():
    """BF16 storage with float32 evaluation: against the oracle on the same rounded values the
    evaluation error must stay above 60 dB PSNR; the quantisation error against the float32-valued
    oracle is reported (no bar)."""
    from paper_2508_05343_b300 import binding as B
    prims = scenes.make_scene(scenes.CONFIGS[2][0], 1234, n=120_000)
    cam = scenes.orbit_camera(320, 240, 33.0, 12.0)
    oc = O.default_config()
    img = alone([prims], (0, 320, 240, 33.0, 12.0), B.GS_BF16).cpu().numpy()
    rounded = dict(prims, **{k: scenes.bf16_round(prims[k]) for k in ("sh", "freqs", "weights")})
    ref_r = O.render(rounded, cam, oc)["image"].numpy()
    ref_f = O.render(prims, cam, oc)["image"].numpy()
    psnr = lambda a, b: 10 * np.log10(1.0 / max(np.mean((a - b) ** 2), 1e-30))
    assert psnr(img, ref_r) >= 60.0, psnr(img, ref_r)
    print(f"bf16 evaluation PSNR {psnr(img, ref_r):.1f} dB, quantisation PSNR {psnr(img, ref_f):.1f} dB")
