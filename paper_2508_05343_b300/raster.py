"""Frame-level helpers over the C ABI: a workspace-owning Rasterizer and the autograd Function.

Device memory comes from PyTorch's caching allocator; the library itself never allocates.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

ATTRS = ("means", "scales", "quats", "opacity", "sh", "freqs", "weights")


def to_device(prims: dict, device="cuda", storage=B.GS_F32) -> dict:
    """numpy scene (scenes.make_scene) -> contiguous CUDA tensors; sh/freqs/weights in bf16 if asked."""
    out = {}
    for k in ATTRS:
        a = torch.as_tensor(np.ascontiguousarray(prims[k]), dtype=torch.float32)
        if storage == B.GS_BF16 and k in ("sh", "freqs", "weights"):
            a = a.to(torch.bfloat16)     # round-to-nearest-even
        out[k] = a.to(device).contiguous()
    return out


class Rasterizer:
    """One frame's workspace: n primitives with K Gabor components, one camera resolution."""

    def __init__(self, n, K, sh_degree, width, height, pair_capacity=None, device="cuda"):
        self.n, self.K, self.sh_degree, self.width, self.height = n, K, sh_degree, width, height
        self.device = torch.device(device)
        self.frame = B.gs_frame()
        self._alloc(pair_capacity if pair_capacity is not None else max(1 << 16, 8 * n))
        self._loss_scratch = None
        self.generation = 0     # counts forwards: the workspace holds the state of the last one

    def _alloc(self, cap):
        cap = int(cap)
        nbytes = B.gabsplat_workspace_size(self.n, self.K, self.sh_degree, self.width, self.height, cap)
        if nbytes == 0:
            raise ValueError("invalid frame sizes")
        self.ws = None
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        f = self.frame
        f.n, f.K, f.sh_degree, f.width, f.height = self.n, self.K, self.sh_degree, self.width, self.height
        f.storage, f.pair_capacity, f.ws, f.ws_bytes = getattr(self, 'storage', B.GS_F32), cap, self.ws.data_ptr(), nbytes
        B.gabsplat_workspace_init(f)
        self.capacity = cap

    # ---- stages -------------------------------------------------------------------------
    def forward(self, prims_t: dict, camera: dict, cfg: B.gs_config, storage=B.GS_F32, out_rgb=None, out_T=None,
                auto_capacity=True, forward_only=False, stats=False):
        """preprocess -> bin_sort -> render_fwd.  With auto_capacity the pair count is read back once
        (a host synchronisation) and the workspace regrown if it overflowed.  forward_only renders
        without the state a backward pass needs (gabsplat_render_fwd_only); stats also writes the
        per-pixel work counters n_eval / n_reach / n_comp (gabsplat_render_fwd_stats)."""
        self.generation += 1
        self._prims = B.make_prims(prims_t, storage)
        self.storage = storage
        self.frame.storage = storage        # the frame carries the storage type to every stage
        self._cam = B.make_camera(camera)
        self._cfg = cfg
        self._keep = prims_t
        if out_rgb is None:
            out_rgb = torch.empty(3, self.height, self.width, device=self.device)
        for _ in range(2):
            B.gabsplat_preprocess(self.frame, self._prims, self._cam, cfg)
            B.gabsplat_bin_sort(self.frame)
            fwd = B.gabsplat_render_fwd_only if forward_only else (
                B.gabsplat_render_fwd_stats if stats else B.gabsplat_render_fwd)
            fwd(self.frame, out_rgb, out_T)
            if not auto_capacity:
                break
            st, pairs = B.gabsplat_device_status(self.frame)
            if st == B.GS_ERR_CAPACITY:
                self._alloc(int(pairs * 1.25) + 1024)
                continue
            if st != B.GS_OK:
                raise B.GabsplatError("render (device status)", st)
            break
        return out_rgb

    def frequency_map(self, out_map=None):
        """The [3][H][W] frequency maps of the frame that forward() last rendered: weighted
        |f2D|, |f2D_x| and |f2D_y| blended like colours, without background."""
        if out_map is None:
            out_map = torch.empty(3, self.height, self.width, device=self.device)
        B.gabsplat_render_freq_map(self.frame, out_map)
        return out_map

    def backward(self, dL_drgb: torch.Tensor, grads: dict | None = None):
        if grads is None:
            grads = {k: torch.empty(self._keep[k].shape, dtype=torch.float32, device=self.device) for k in ATTRS}
            grads["means2d"] = torch.empty(self.n, 2, device=self.device)
        g = B.gs_prim_grads()
        for k in ATTRS + ("means2d",):
            t = grads.get(k)
            setattr(g, k, t.data_ptr() if (t is not None and t.numel() > 0) else None)
        B.gabsplat_render_bwd(self.frame, dL_drgb.contiguous(), g)
        return grads

    def loss(self, image, target, kind=B.GS_LOSS_L1):
        if self._loss_scratch is None:
            self._loss_scratch = torch.empty(B.gabsplat_loss_scratch_bytes(image.numel()), dtype=torch.uint8,
                                             device=self.device)
            self._loss_val = torch.empty(1, dtype=torch.float64, device=self.device)
        dL = torch.empty_like(image)
        B.gabsplat_loss(image, target, kind, self._loss_val, dL, self._loss_scratch)
        return self._loss_val, dL

    def status(self):
        return B.gabsplat_device_status(self.frame)

    # ---- workspace inspection (tests) ----------------------------------------------------
    def views(self) -> dict:
        v = B.gabsplat_workspace_views(self.frame)
        base = self.ws.data_ptr()
        _, pairs = self.status()
        P = min(pairs, self.capacity)
        ntiles = v.tiles_x * v.tiles_y
        npix = self.width * self.height

        def sl(ptr, count, dtype):
            off = ptr - base
            nb = count * torch.empty(0, dtype=dtype).element_size()
            return self.ws[off:off + nb].view(dtype)

        na = v.n_active   # rows of records / grad2d / offsets / order are depth ranks 0 .. na - 1
        return dict(
            records=sl(v.records, na * v.record_floats, torch.float32).view(na, v.record_floats),
            touched=sl(v.touched, self.n, torch.int32), offsets=sl(v.offsets, na, torch.int32),
            order=sl(v.order, na, torch.int32), n_active=na, keys_sorted=sl(v.keys_sorted, P, torch.int64),
            ranges=sl(v.ranges, 2 * ntiles, torch.int32).view(ntiles, 2),
            T_final=sl(v.T_final, npix, torch.float32).view(self.height, self.width),
            n_contrib=sl(v.n_contrib, npix, torch.int32).view(self.height, self.width),
            n_eval=sl(v.n_eval, npix, torch.int32).view(self.height, self.width),
            n_reach=sl(v.n_reach, npix, torch.int32).view(self.height, self.width),
            n_comp=sl(v.n_comp, npix, torch.int32).view(self.height, self.width),
            grad2d=sl(v.grad2d, na * v.grad2d_floats, torch.float32).view(na, v.grad2d_floats),
            pairs=pairs, tiles_x=v.tiles_x, tiles_y=v.tiles_y,
            record_floats=v.record_floats, grad2d_floats=v.grad2d_floats)


class GabSplatRender(torch.autograd.Function):
    """image = render(primitives, camera), differentiable in every primitive attribute; the backward
    runs the hand-written adjoint kernels (gabsplat_render_bwd), which recompute transmittance
    instead of storing per-pair state.

    Inputs are activated attributes (exp / sigmoid are applied by the caller in torch).

    Storage: with storage="bf16" the SH, frequency and weight tensors are rounded to BF16 (nearest
    even) for the kernels, which evaluate and composite in FP32.  Gradients are always computed in
    FP32 and returned in each input's own dtype: FP32 master tensors (the usual mixed-precision
    setup) receive the FP32 gradient, the rounding being passed straight through; BF16 inputs
    receive the FP32 gradient rounded to BF16 (autograd requires a gradient of the input's dtype).

    The rasterizer's workspace holds the state of its last forward only.  If another forward ran
    on the same Rasterizer before this one's backward, the backward first re-renders this forward's
    inputs (same inputs, same frame), so the gradients always belong to this forward."""

    @staticmethod
    def forward(ctx, rast: Rasterizer, camera: dict, cfg, storage, means, scales, quats, opacity, sh, freqs,
                weights):
        if storage not in ("f32", "bf16"):
            raise ValueError("storage is 'f32' or 'bf16'")
        st = B.GS_BF16 if storage == "bf16" else B.GS_F32
        prims = dict(means=means.float().contiguous(), scales=scales.float().contiguous(),
                     quats=quats.float().contiguous(), opacity=opacity.float().contiguous())
        for k, t in (("sh", sh), ("freqs", freqs), ("weights", weights)):
            prims[k] = (t.to(torch.bfloat16) if st == B.GS_BF16 else t.float()).contiguous()
        img = rast.forward(prims, camera, cfg, storage=st)
        ctx.rast, ctx.camera, ctx.cfg, ctx.storage = rast, camera, cfg, st
        ctx.generation = rast.generation
        ctx.prims = prims            # the tensors the kernels read (kept for a re-render)
        ctx.dtypes = [t.dtype for t in (means, scales, quats, opacity, sh, freqs, weights)]
        return img

    @staticmethod
    def backward(ctx, grad_img):
        rast = ctx.rast
        if rast.generation != ctx.generation:
            rast.forward(ctx.prims, ctx.camera, ctx.cfg, storage=ctx.storage)
        g = rast.backward(grad_img.float().contiguous())
        outs = [g[k] if g[k].dtype == dt else g[k].to(dt) for k, dt in zip(ATTRS, ctx.dtypes)]
        return (None, None, None, None, *outs)


def render(rast: Rasterizer, camera: dict, cfg, means, scales, quats, opacity, sh, freqs, weights, storage="f32"):
    """Differentiable render of one view (see GabSplatRender): a [3][H][W] FP32 image."""
    return GabSplatRender.apply(rast, camera, cfg, storage, means, scales, quats, opacity, sh, freqs, weights)
