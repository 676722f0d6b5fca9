"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and compare it with
the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

from oracle import gabsplat_oracle as O

IMG_TOL = 2e-4      # max-abs per channel, float32 image vs float64 oracle
GRAD_TOL = 1e-3     # relative L2 per attribute group
MAX_FLAGGED = 1e-3  # flagged pixels (a threshold decision float32 may take the other way) per image pixel
FLAGS_PER_PAIR = 2e-5   # ... or per listed pixel-pair, whichever allows more (see assert_image_parity)
ATTRS = ("means", "scales", "quats", "opacity", "sh", "freqs", "weights")


def cfg_pair(eps2d=0.3, bg=(0.0, 0.0, 0.0), z_atten=False):
    from paper_2508_05343_b300 import binding as B
    oc = O.default_config(eps2d=eps2d, bg=bg, z_atten=z_atten)
    return oc, B.make_config(eps2d=oc["eps2d"], alpha_max=oc["alpha_max"], alpha_min=oc["alpha_min"],
                             T_min=oc["T_min"], bg=oc["bg"], flags=B.GS_FLAG_Z_ATTENUATION if z_atten else 0)


def gpu_render(prims, cam, gcfg, storage=0, capacity=None):
    from paper_2508_05343_b300 import raster
    n, K = prims["means"].shape[0], prims["weights"].shape[1]
    deg = int(round(prims["sh"].shape[1] ** 0.5)) - 1
    r = raster.Rasterizer(n, K, deg, cam["width"], cam["height"], pair_capacity=capacity)
    pt = raster.to_device(prims, storage=storage)
    T = torch.empty(cam["height"], cam["width"], device="cuda")
    img = r.forward(pt, cam, gcfg, storage=storage, out_T=T, stats=True)
    torch.cuda.synchronize()
    return r, pt, img, T


def bf16_prims(prims):
    from paper_2508_05343_b300 import scenes
    out = dict(prims)
    for k in ("sh", "freqs", "weights"):
        out[k] = scenes.bf16_round(prims[k])
    return out


def image_errors(gpu_img, out, tol=IMG_TOL, mask=None):
    """Per-pixel check of a [C][H][W] image against the oracle: every channel within tol of the
    oracle, or, at a pixel the oracle flags (a threshold decision float32 may take the other way),
    within tol + the oracle's allowance for that pixel (the result with each flagged decision
    flipped).  Returns (max error at unflagged pixels, largest excess over the allowance at flagged
    ones (<= 0 passes), flagged count); mask restricts the check to some pixels."""
    err = np.abs(np.asarray(gpu_img, np.float64) - out["image"].numpy())
    amb = np.asarray(out["ambiguous"].numpy(), bool)
    allow = out["allowance"].numpy()
    if mask is None:
        mask = np.ones(amb.shape, bool)
    clean = mask & ~amb
    flagged = mask & amb
    e_clean = float(err.max(0)[clean].max()) if clean.any() else 0.0
    excess = float((err - tol - allow).max(0)[flagged].max()) if flagged.any() else -tol
    return e_clean, excess, int(flagged.sum())


def listed_pixel_pairs(spec, shape, mask=None):
    """Sum over the (masked) pixels of their tile's list length: the threshold decisions a pixel
    can face, an upper bound on its evaluated pairs."""
    L = (spec["ranges"][:, 1].astype(np.int64) - spec["ranges"][:, 0]).reshape(spec["tiles_y"], spec["tiles_x"])
    per_px = np.repeat(np.repeat(L, 16, 0), 16, 1)[:shape[0], :shape[1]]
    return int(per_px[mask].sum()) if mask is not None else int(per_px.sum())


def assert_image_parity(gpu_img, out, tol=IMG_TOL, max_flagged=None, mask=None):
    """Image bars of the parity tests.  Every pixel within tol, or, if flagged, within tol + its
    flip allowance.  The flagged count is capped: each of a pixel's threshold decisions can fall
    inside its float32 window, so the expected count grows with the pairs a pixel evaluates; the
    cap is 0.1% of the pixels or 2e-5 per listed pixel-pair (tile list length summed over the
    pixels), whichever is larger (measured: at most 1.2e-5 per listed pixel-pair at config 2,
    4e-5 per pixel-pair and 0.06% of the pixels at config 1).  max_flagged overrides it as a
    fraction of the pixels."""
    e_clean, excess, namb = image_errors(gpu_img, out, tol, mask)
    npx = int(np.asarray(mask).sum()) if mask is not None else gpu_img.shape[1] * gpu_img.shape[2]
    assert e_clean <= tol, f"max |gpu - oracle| = {e_clean:.3e} at unflagged pixels"
    assert excess <= 0.0, f"a flagged pixel exceeds tol + its flip allowance by {excess:.3e}"
    if max_flagged is not None:
        cap = max(1.0, max_flagged * npx)
    else:
        pairs = listed_pixel_pairs(out["spec"], gpu_img.shape[1:], mask) if "spec" in out else 0
        cap = max(1.0, MAX_FLAGGED * npx, FLAGS_PER_PAIR * pairs)
    assert namb <= cap, f"{namb} flagged pixels of {npx} (cap {cap:.0f})"
    return e_clean, namb


def assert_decisions_flagged(v, out, mask=None):
    """The flags are a valid account of float32 / float64 branch differences: at every pixel where
    the GPU's composited-pair count or last contributor differs from the oracle's, the oracle has
    flagged a decision."""
    amb = out["ambiguous"].numpy()
    diff = (v["n_comp"].cpu().numpy() != out["n_comp"].numpy()) | (v["n_contrib"].cpu().numpy() != out["n_contrib"].numpy())
    if mask is not None:
        diff &= mask
    assert not (diff & ~amb).any(), f"{int((diff & ~amb).sum())} unflagged pixels take another branch on the GPU"
    return int(diff.sum())


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def gpu_grads(r, dL):
    g = r.backward(torch.as_tensor(dL, dtype=torch.float32, device="cuda").contiguous())
    torch.cuda.synchronize()
    return {k: v.float().cpu().numpy() for k, v in g.items()}


def by_prim(v, key, n):
    """Rows of a rank-indexed workspace view (records, grad2d) at their primitives' indices
    (zeros for primitives that reach no tile)."""
    rows = v[key].cpu().numpy().astype(np.float64)
    out = np.zeros((n, rows.shape[1]))
    out[v["order"].cpu().numpy().astype(np.int64)] = rows
    return out
