"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and compare it with
the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

from oracle import gabsplat_oracle as O

IMG_TOL = 2e-4      # max-abs per channel, float32 image vs float64 oracle
GRAD_TOL = 1e-3     # relative L2 per attribute group
AMBIG_EXTRA = 1e-2  # extra allowance at pixels where float32/float64 may take a different threshold branch
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
    img = r.forward(pt, cam, gcfg, storage=storage, out_T=T)
    torch.cuda.synchronize()
    return r, pt, img, T


def bf16_prims(prims):
    from paper_2508_05343_b300 import scenes
    out = dict(prims)
    for k in ("sh", "freqs", "weights"):
        out[k] = scenes.bf16_round(prims[k])
    return out


def compare_images(gpu_img, ref, amb, tol=IMG_TOL):
    """Returns (max error at unambiguous pixels, max error at ambiguous ones, ambiguous count)."""
    err = np.abs(gpu_img - ref).max(0)
    amb = np.asarray(amb, bool)
    e_clean = float(err[~amb].max()) if (~amb).any() else 0.0
    e_amb = float(err[amb].max()) if amb.any() else 0.0
    return e_clean, e_amb, int(amb.sum())


def assert_image_parity(gpu_img, out, tol=IMG_TOL, max_amb_frac=0.02):
    e_clean, e_amb, namb = compare_images(gpu_img, out["image"].numpy(), out["ambiguous"].numpy())
    npx = gpu_img.shape[1] * gpu_img.shape[2]
    assert e_clean <= tol, f"max |gpu - oracle| = {e_clean:.3e} at unambiguous pixels"
    assert e_amb <= tol + AMBIG_EXTRA, f"ambiguous pixel error {e_amb:.3e}"
    assert namb <= max_amb_frac * npx, f"{namb} ambiguous pixels of {npx}"
    return e_clean, namb


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
