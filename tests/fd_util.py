"""Central finite differences of the FP64 oracle's image, rendered only where a perturbation can
change it: the tiles of the perturbed primitives' rectangles, composited from the primitives
listed in those tiles (every other primitive's bins are its own, so the result on those tiles is
the full scene's)."""
import numpy as np

from oracle import gabsplat_oracle as O

PRIM_KEYS = ("means", "scales", "quats", "opacity", "sh", "freqs", "weights")


def _sub(prims, ids):
    return {k: (np.asarray(prims[k])[ids] if k in PRIM_KEYS else prims[k]) for k in prims}


def local_loss(prims, cam, oc, dL, spec, ids, u, h):
    """sum(dL * image) over the tiles the primitives ids can touch, at prims + h u and prims - h u,
    with a flag telling whether any pixel of those tiles changed a compositing decision between the
    two (the image is not differentiable there).  u holds per-attribute arrays for the ids only."""
    tx = spec["tiles_x"]
    tiles = set()
    for s in (h, -h):
        q = _sub(prims, ids)
        for k, v in u.items():
            q[k] = np.asarray(q[k], np.float64) + s * v
        sp = O.bin_spec(q, cam, oc)
        for j in range(len(ids)):
            if sp["valid"][j]:
                x0, x1, y0, y1 = sp["rect"][j]
                tiles |= {ty * tx + t for ty in range(y0, y1 + 1) for t in range(x0, x1 + 1)}
    tiles = sorted(tiles)
    if not tiles:
        return 0.0, 0.0, False
    r = spec["ranges"]
    listed = np.concatenate([spec["sorted_vals"][r[t, 0]:r[t, 1]] for t in tiles] + [np.asarray(ids)])
    sub_ids = np.unique(listed.astype(np.int64))
    pos = np.searchsorted(sub_ids, ids)
    res = []
    for s in (h, -h):
        q = _sub(prims, sub_ids)
        for k, v in u.items():
            a = np.asarray(q[k], np.float64).copy()
            a[pos] += s * v
            q[k] = a
        out = O.render(q, cam, oc, tiles=tiles)
        res.append(out)
    mask = np.zeros((cam["height"], cam["width"]), bool)
    for t in tiles:
        mask[(t // tx) * 16:(t // tx) * 16 + 16, (t % tx) * 16:(t % tx) * 16 + 16] = True
    live = mask & (np.abs(dL).sum(0) > 0)
    flip = ((res[0]["n_comp"].numpy() != res[1]["n_comp"].numpy()) |
            (res[0]["n_contrib"].numpy() != res[1]["n_contrib"].numpy())) & live
    lp = float((res[0]["image"].numpy() * dL)[:, mask].sum())
    lm = float((res[1]["image"].numpy() * dL)[:, mask].sum())
    return lp, lm, bool(flip.any())


# ---- a spawn-started process pool over local_loss (the GPU test process already holds CUDA) ----
_G = {}


def _init(prims, cam, oc, dL, spec):
    import torch
    torch.set_num_threads(1)
    _G.update(prims=prims, cam=cam, oc=oc, dL=dL, spec=spec)


def _job(args):
    ids, u, h = args
    lp, lm, flip = local_loss(_G["prims"], _G["cam"], _G["oc"], _G["dL"], _G["spec"], ids, u, h)
    return (lp - lm) / (2 * h), flip


def directional_fds(prims, cam, oc, dL, spec, jobs, workers=None):
    """[(fd, flipped)] for jobs [(ids, u, h)], computed in a spawn-started process pool."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    workers = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"), initializer=_init,
                                initargs=(prims, cam, oc, dL, spec)) as ex:
        return list(ex.map(_job, jobs, chunksize=8))
