"""Frequency-adaptive density control on the GPU against the oracle (Sec. 3.4.2, supplement B).

Selection and order are decided by single correctly rounded float32 operations on both sides, so
the counts, the source of every output row, the copied attributes, the reset values and the split
children's scales must match bit for bit.  Split children's positions mu + R(q) (s z) are float32
on the GPU and float64 in the oracle: within 2e-6 of max(1, |mu|)."""
import numpy as np
import pytest
import torch

from oracle import gabsplat_oracle as O
from paper_2508_05343_b300 import scenes
from tests.conftest import cuda_available
from tests.gpu_util import cfg_pair, gpu_render

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

KEYS = ("means", "scales", "quats", "opacity", "sh", "freqs", "weights")


def inputs(seed, n, K=3, bf16=False):
    rng = np.random.default_rng(seed)
    spec = scenes.SceneSpec(n=n, K=K, sh_degree=3, layout="uniform", box=1.0, log_scale=(-3.0, 0.5))
    prims = scenes.make_scene(spec, seed)
    prims["opacity"][: n // 8] = (rng.random(n // 8) * 0.02).astype(np.float32)
    if bf16:
        prims = dict(prims, **{k: scenes.bf16_round(prims[k]) for k in ("sh", "freqs", "weights")})
    acc = (rng.random(n) * 2e-3).astype(np.float32)
    den = rng.integers(0, 4, n).astype(np.float32)
    noise = rng.standard_normal((n, 2, 3)).astype(np.float32)
    return prims, acc, den, noise


def gpu_densify(prims, acc, den, noise, cfg, storage):
    from paper_2508_05343_b300 import binding as B
    from paper_2508_05343_b300 import raster
    n = prims["means"].shape[0]
    t = raster.to_device(prims, storage=storage)
    out = {k: torch.full((2 * n,) + tuple(v.shape[1:]), float("nan"), dtype=v.dtype, device="cuda")
           for k, v in t.items() if k in KEYS}
    counts = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    scratch = torch.empty(B.gabsplat_densify_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    dev = lambda a: torch.tensor(a, device="cuda")
    B.gabsplat_densify(B.make_prims(t, storage), dev(acc), dev(den), dev(noise), B.make_densify_config(**cfg),
                       B.make_prim_arrays(out), 2 * n, counts, scratch)
    torch.cuda.synchronize()
    c = counts.cpu().numpy()
    return {k: v[: c[0]].float().cpu().numpy() for k, v in out.items()}, c


@pytest.mark.parametrize("storage,max_scale", [(0, 0.0), (0, 0.12), (1, 0.0)])
def test_densify_matches_oracle(storage, max_scale):
    prims, acc, den, noise = inputs(31 + storage, 5000, bf16=storage == 1)
    cfg = dict(O.densify_defaults(dense_scale=0.06), max_scale=max_scale)
    got, c = gpu_densify(prims, acc, den, noise, cfg, storage)
    ref, rc = O.densify(prims, acc, den, noise.astype(np.float64), cfg)
    assert list(c) == [rc["originals"] + rc["clones"] + rc["children"], rc["originals"], rc["clones"], rc["children"]]
    assert rc["clones"] > 0 and rc["children"] > 0 and rc["originals"] < 5000
    nref = {k: np.asarray(v, np.float64) for k, v in ref.items()}
    if storage == 1:                                     # new primitives' reset values in BF16
        for k in ("freqs", "weights"):
            nref[k] = scenes.bf16_round(ref[k]).astype(np.float64)
    for k in ("scales", "quats", "opacity", "sh", "freqs", "weights"):
        np.testing.assert_array_equal(got[k].reshape(nref[k].shape), nref[k], err_msg=k)
    nc = rc["originals"] + rc["clones"]
    np.testing.assert_array_equal(got["means"][:nc], nref["means"][:nc])
    ch, rch = got["means"][nc:], nref["means"][nc:]
    assert np.abs(ch - rch).max() <= 2e-6 * max(1.0, np.abs(rch).max())


def test_densify_accumulate_on_a_rendered_view():
    from paper_2508_05343_b300 import binding as B
    prims = scenes.config_scene(0)
    cam = scenes.orbit_camera(128, 128, 30.0, 10.0, 1.2)   # inside the cloud: some primitives are not seen
    oc, gc = cfg_pair()
    spec = O.bin_spec(prims, cam, oc)
    r, _, _, _ = gpu_render(prims, cam, gc)
    n = prims["means"].shape[0]
    rng = np.random.default_rng(4)
    acc = torch.zeros(n, device="cuda")
    den = torch.zeros(n, device="cuda")
    ra, rd = np.zeros(n, np.float32), np.zeros(n, np.float32)
    for _ in range(3):
        g = rng.standard_normal((n, 2)).astype(np.float32) * 1e-3
        B.gabsplat_densify_accumulate(r.frame, torch.tensor(g, device="cuda"), acc, den)
        ra, rd = O.densify_accumulate(ra, rd, g, spec["touched"] > 0)
    torch.cuda.synchronize()
    assert 0 < (spec["touched"] > 0).sum() < n
    np.testing.assert_array_equal(acc.cpu().numpy(), ra)
    np.testing.assert_array_equal(den.cpu().numpy(), rd)


@pytest.mark.parametrize("storage", [0, 1])
def test_reset_opacity_weights(storage):
    from paper_2508_05343_b300 import binding as B
    from paper_2508_05343_b300 import raster
    prims, _, _, _ = inputs(35, 3000, bf16=storage == 1)
    t = raster.to_device(prims, storage=storage)
    B.gabsplat_reset_opacity_weights(B.make_prim_arrays(t), 3000, 3, storage, 0.02, 0.01)
    torch.cuda.synchronize()
    ref = O.reset_opacity_weights(prims)
    np.testing.assert_array_equal(t["opacity"].cpu().numpy(), ref["opacity"])
    w = ref["weights"] if storage == 0 else scenes.bf16_round(ref["weights"])
    np.testing.assert_array_equal(t["weights"].float().cpu().numpy(), w)


def test_densify_empty_input_and_capacity_check():
    from paper_2508_05343_b300 import binding as B
    from paper_2508_05343_b300 import raster
    prims, acc, den, noise = inputs(36, 64)
    t = raster.to_device(prims)
    out = {k: torch.empty((100,) + tuple(v.shape[1:]), dtype=v.dtype, device="cuda") for k, v in t.items() if k in KEYS}
    counts = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    scratch = torch.empty(B.gabsplat_densify_scratch_bytes(64), dtype=torch.uint8, device="cuda")
    dev = lambda a: torch.tensor(a, device="cuda")
    cfg = B.make_densify_config()
    with pytest.raises(B.GabsplatError):                 # 100 rows < 2 x 64
        B.gabsplat_densify(B.make_prims(t), dev(acc), dev(den), dev(noise), cfg, B.make_prim_arrays(out), 100,
                           counts, scratch)
    empty = B.make_prims(t)
    empty.n = 0
    B.gabsplat_densify(empty, None, None, None, cfg, B.make_prim_arrays(out), 0, counts, scratch)
    torch.cuda.synchronize()
    assert counts.cpu().tolist() == [0, 0, 0, 0]
