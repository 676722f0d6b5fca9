"""Continuous-batching novel-view server over the batched C ABI.

Scenes stay resident in HBM (BF16 storage of SH and Gabor coefficients by default).  Requests
(scene, camera, resolution) arrive over time; whenever one of the server's slots is free, the
admission controller forms a batch from the waiting requests in arrival order -- different scenes
and resolutions together -- within the slot's capacity (views, primitives, tiles, pixels, an
estimate of the (tile, primitive) pairs) and the HBM admission cap, and the slot replays its
captured CUDA graph with the new view table on its own stream.  Batches on different slots run
concurrently on the device, so requests that arrive while others render are admitted as soon as a
slot frees up.  The plain baseline renders one request at a time with the single-view float32 path.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

TILE = 16


def tiles_of(w, h):
    return ((w + TILE - 1) // TILE) * ((h + TILE - 1) // TILE)


@dataclasses.dataclass
class SlotLimits:
    max_views: int = 16
    max_prims: int = 24_000_000
    max_tiles: int = 16 * 8160
    max_pixels: int = 16 * 1920 * 1080
    pair_capacity: int = 160_000_000


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    scene: int
    width: int
    height: int
    azimuth: float
    elevation: float


class AdmissionController:
    """Host-side batch formation and memory ledger (no device access; testable with fakes).

    scene_prims[s] = primitive count of scene s; pair_estimate(scene, w, h) = an upper estimate
    of the pairs one view produces; bytes_per_view(w, h) = output bytes of one view.
    """

    def __init__(self, limits: SlotLimits, scene_prims, pair_estimate, bytes_per_view, hbm_cap_bytes,
                 resident_bytes):
        self.limits = limits
        self.scene_prims = scene_prims
        self.pair_estimate = pair_estimate
        self.bytes_per_view = bytes_per_view
        self.cap = hbm_cap_bytes
        self.in_flight_bytes = 0
        self.resident_bytes = resident_bytes
        self.pending = collections.deque()
        self.refused = 0

    def submit(self, req: Request):
        self.pending.append(req)

    def fits_alone(self, r: Request) -> bool:
        L = self.limits
        return (self.scene_prims[r.scene] <= L.max_prims and tiles_of(r.width, r.height) <= L.max_tiles and
                r.width * r.height <= L.max_pixels and self.pair_estimate(r.scene, r.width, r.height) <= L.pair_capacity)

    def next_batch(self, max_views=None):
        """Pop the longest arrival-order prefix of waiting requests that fits one slot."""
        L = self.limits
        mv = L.max_views if max_views is None else min(max_views, L.max_views)
        batch, prims, tiles, pixels, pairs, out_bytes = [], 0, 0, 0, 0, 0
        while self.pending and len(batch) < mv:
            r = self.pending[0]
            if not self.fits_alone(r):
                self.pending.popleft()
                self.refused += 1
                continue
            n, t, px = self.scene_prims[r.scene], tiles_of(r.width, r.height), r.width * r.height
            pe, ob = self.pair_estimate(r.scene, r.width, r.height), self.bytes_per_view(r.width, r.height)
            if (prims + n > L.max_prims or tiles + t > L.max_tiles or pixels + px > L.max_pixels or
                    pairs + pe > L.pair_capacity):
                break
            if self.resident_bytes + self.in_flight_bytes + out_bytes + ob > self.cap:
                break
            batch.append(self.pending.popleft())
            prims, tiles, pixels, pairs, out_bytes = prims + n, tiles + t, pixels + px, pairs + pe, out_bytes + ob
        self.in_flight_bytes += out_bytes
        return batch, out_bytes

    def release(self, out_bytes):
        self.in_flight_bytes -= out_bytes

    def requeue_front(self, reqs):
        for r in reversed(reqs):
            self.pending.appendleft(r)


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, np.float64), q)) if len(xs) else float("nan")


class Server:
    """Continuous-batching renderer: n_slots workspaces, each with a captured graph and a stream."""

    def __init__(self, scenes: list, storage, K, sh_degree, limits: SlotLimits = None, n_slots=3, cfg=None,
                 hbm_cap_bytes=120 << 30, use_graphs=True, device="cuda"):
        import torch

        from . import binding as B
        from . import raster
        self.B, self.torch = B, torch
        self.limits = limits or SlotLimits()
        self.storage, self.K, self.deg = storage, K, sh_degree
        self.cfg = cfg or B.make_config()
        self.dev = torch.device(device)
        self.scene_t = [raster.to_device(s, self.dev, storage) for s in scenes]
        self.scene_s = [B.make_prims(t, storage) for t in self.scene_t]
        self.scene_n = [s["means"].shape[0] for s in scenes]
        self.resident_bytes = sum(sum(v.numel() * v.element_size() for v in t.values()) for t in self.scene_t)
        self.use_graphs = use_graphs
        self.slots = []
        L = self.limits
        for _ in range(n_slots):
            f = B.gs_batch_frame()
            f.max_views, f.K, f.sh_degree, f.storage = L.max_views, K, sh_degree, storage
            f.max_prims, f.max_tiles, f.max_pixels, f.pair_capacity = L.max_prims, L.max_tiles, L.max_pixels, L.pair_capacity
            nbytes = B.gabsplat_batch_workspace_size(L.max_views, K, sh_degree, L.max_prims, L.max_tiles,
                                                     L.max_pixels, L.pair_capacity)
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.dev)
            f.ws, f.ws_bytes = ws.data_ptr(), nbytes
            stream = torch.cuda.Stream(self.dev)
            with torch.cuda.stream(stream):
                B.gabsplat_batch_workspace_init(f)
                graph = B.gabsplat_batch_graph_create(f, self.cfg) if use_graphs else None
            status = torch.zeros(2, dtype=torch.int64).pin_memory()
            self.slots.append(dict(frame=f, ws=ws, stream=stream, graph=graph, status=status, busy=False,
                                   batch=None, event=None, outs=None, out_bytes=0, launched_s=0.0))
        self.ws_bytes = sum(s["ws"].numel() for s in self.slots)
        self.pair_est = {}

    # ---- calibration of the pair estimate (host reads, before serving) -------------------------
    def calibrate(self, resolutions, poses=((0.0, 0.0), (90.0, 25.0), (200.0, -25.0), (300.0, 10.0)), margin=1.3):
        from . import scenes as S
        torch, B = self.torch, self.B
        slot = self.slots[0]
        with torch.cuda.stream(slot["stream"]):
            for si in range(len(self.scene_t)):
                for (w, h) in resolutions:
                    worst = 0
                    for az, el in poses:
                        cam = B.make_camera(S.orbit_camera(w, h, az, el))
                        out = torch.empty(3, h, w, device=self.dev)
                        B.gabsplat_render_batch(slot["frame"], [B.make_view(self.scene_s[si], cam, out)], self.cfg)
                        B.gabsplat_batch_status_copy(slot["frame"], slot["status"].data_ptr())
                        slot["stream"].synchronize()
                        st = int(slot["status"][0].item() & 0xFFFFFFFF)
                        if st not in (B.GS_OK, B.GS_ERR_CAPACITY):
                            raise B.GabsplatError("calibration", st)
                        worst = max(worst, int(slot["status"][1].item()))
                    self.pair_est[(si, w, h)] = int(worst * margin) + 4096
        return self.pair_est

    def _estimate(self, scene, w, h):
        return self.pair_est.get((scene, w, h), self.limits.pair_capacity)

    # ---- serving loop ------------------------------------------------------------------------
    def run(self, requests: list, realtime=True, max_views=None, keep_images=False):
        """Serve `requests` (arrival times in seconds from the start when realtime, else all at t=0).

        Returns per-request latency (arrival -> completion observed on the host), makespan and
        frames/s, batch-size statistics and the images when keep_images."""
        from . import scenes as S
        torch, B = self.torch, self.B
        ac = AdmissionController(self.limits, self.scene_n, self._estimate, lambda w, h: 3 * 4 * w * h,
                                 120 << 30, self.resident_bytes + self.ws_bytes)
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        cams = {r.rid: B.make_camera(S.orbit_camera(r.width, r.height, r.azimuth, r.elevation)) for r in reqs}
        done_t, images, batch_sizes, retries = {}, {}, [], 0
        nxt = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while len(done_t) < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and (not realtime or reqs[nxt].arrival_s <= now):
                ac.submit(reqs[nxt])
                nxt += 1
            progressed = False
            for slot in self.slots:
                if slot["busy"] and slot["event"].query():
                    st = int(slot["status"][0].item() & 0xFFFFFFFF)
                    tdone = time.perf_counter() - t0
                    ac.release(slot["out_bytes"])
                    if st == B.GS_ERR_CAPACITY and len(slot["batch"]) > 1:
                        half = len(slot["batch"]) // 2     # estimate too low: split and retry
                        ac.requeue_front(slot["batch"])
                        retries += 1
                        slot["retry_views"] = half
                    elif st != B.GS_OK:
                        raise B.GabsplatError("serve (device status)", st)
                    else:
                        for r, out in zip(slot["batch"], slot["outs"]):
                            done_t[r.rid] = tdone
                            if keep_images:
                                images[r.rid] = out
                    slot["busy"] = False
                    progressed = True
            for slot in self.slots:
                if slot["busy"] or not ac.pending:
                    continue
                mv = slot.pop("retry_views", None) or max_views
                batch, out_bytes = ac.next_batch(mv)
                if not batch:
                    continue
                with torch.cuda.stream(slot["stream"]):
                    outs = [torch.empty(3, r.height, r.width, device=self.dev) for r in batch]
                    views = [B.make_view(self.scene_s[r.scene], cams[r.rid], o) for r, o in zip(batch, outs)]
                    if self.use_graphs:
                        B.gabsplat_batch_graph_launch(slot["graph"], views)
                    else:
                        B.gabsplat_render_batch(slot["frame"], views, self.cfg)
                    B.gabsplat_batch_status_copy(slot["frame"], slot["status"].data_ptr())
                    ev = torch.cuda.Event()
                    ev.record(slot["stream"])
                slot.update(busy=True, batch=batch, outs=outs, event=ev, out_bytes=out_bytes)
                batch_sizes.append(len(batch))
                progressed = True
            if not progressed and realtime and not ac.pending and nxt < len(reqs):
                wait = reqs[nxt].arrival_s - (time.perf_counter() - t0)
                if wait > 2e-4 and not any(s["busy"] for s in self.slots):
                    time.sleep(wait - 1e-4)
        lat = [done_t[r.rid] - (r.arrival_s if realtime else 0.0) for r in reqs]
        first = reqs[0].arrival_s if realtime else 0.0
        span = max(done_t.values()) - first
        return dict(latency_ms_p50=1e3 * percentile(lat, 50), latency_ms_p99=1e3 * percentile(lat, 99),
                    frames_per_s=len(reqs) / span, makespan_s=span, batches=len(batch_sizes),
                    mean_batch=float(np.mean(batch_sizes)), retries=retries, refused=ac.refused,
                    images=images if keep_images else None)


class PlainRenderer:
    """The baseline: one request at a time, float32 storage, the single-view ABI path."""

    def __init__(self, scenes: list, pair_est: dict, cfg=None, device="cuda"):
        import torch

        from . import binding as B
        from . import raster
        self.B, self.torch, self.raster = B, torch, raster
        self.cfg = cfg or B.make_config()
        self.dev = torch.device(device)
        self.scene_t = [raster.to_device(s, self.dev, B.GS_F32) for s in scenes]
        self.meta = [(s["means"].shape[0], s["weights"].shape[1], int(round(s["sh"].shape[1] ** 0.5)) - 1)
                     for s in scenes]
        self.pair_est = pair_est
        self.rast = {}

    def _rast(self, si, w, h):
        key = (si, w, h)
        if key not in self.rast:
            n, K, deg = self.meta[si]
            self.rast[key] = self.raster.Rasterizer(n, K, deg, w, h, pair_capacity=self.pair_est.get(key),
                                                    device=self.dev)
        return self.rast[key]

    def prepare(self, requests):
        for r in requests:
            self._rast(r.scene, r.width, r.height)

    def run(self, requests: list, realtime=True, keep_images=False):
        from . import scenes as S
        torch, B = self.torch, self.B
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        done_t, images = {}, {}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in reqs:
            if realtime:
                wait = r.arrival_s - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
            rast = self._rast(r.scene, r.width, r.height)
            out = torch.empty(3, r.height, r.width, device=self.dev)
            rast.forward(self.scene_t[r.scene], S.orbit_camera(r.width, r.height, r.azimuth, r.elevation), self.cfg,
                         out_rgb=out, auto_capacity=True, forward_only=True)   # reads the status each request
            done_t[r.rid] = time.perf_counter() - t0
            if keep_images:
                images[r.rid] = out
        lat = [done_t[r.rid] - (r.arrival_s if realtime else 0.0) for r in reqs]
        first = reqs[0].arrival_s if realtime else 0.0
        span = max(done_t.values()) - first
        return dict(latency_ms_p50=1e3 * percentile(lat, 50), latency_ms_p99=1e3 * percentile(lat, 99),
                    frames_per_s=len(reqs) / span, makespan_s=span, images=images if keep_images else None)


def make_requests(n_req=2000, rate=200.0, n_scenes=8, seed=2000, resolutions=None):
    from . import scenes as S
    return [Request(i, **d) for i, d in enumerate(S.serve_requests(n_req, rate, n_scenes, seed, resolutions))]
