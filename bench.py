#!/usr/bin/env python
"""Benchmark of the 3D Gabor splatting rasterizer (fwd+bwd ms/iter at 1.5M primitives, 1600x1064).

One step = one training iteration of the rasterizer on one view: gabsplat_preprocess ->
gabsplat_bin_sort -> gabsplat_render_fwd -> L1 loss -> the two halves of gabsplat_render_bwd (2D
adjoint with the gradient zero-fill folded in, then the attribute chain rule), on the 1.5M-primitive, K=4, SH-degree-3 synthetic scene cycling through
its 16 orbit poses.  Primitives (450 MB in float32) are larger than L2, so no flush is needed.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--storage bf16]

Multi-GPU runs (torchrun, one rank per GPU) are independent replicas: each rank renders its own
poses with no collective on the data path (weak scaling); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/iter @1.5M prims 1600x1064; serve p50/p99 ms & frames/s vs plain"
UNIT = "ms/iter"
SM_COUNT_B300 = 148
# fused L1 + D-SSIM per image value: five windowed moments and three windowed adjoint maps, each
# separable (2 x 11 taps, an FMA = 2 flops), the SSIM index and its partials (~25), the gradient (5)
SSIM_FLOPS_PER_VALUE = 2 * 11 * 2 * (5 + 3) + 25 + 5
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["f32", "bf16"], default="f32")
    ap.add_argument("--config", type=int, default=2, choices=[2, 4])
    ap.add_argument("--K", type=int, default=None, help="override the number of Gabor components")
    ap.add_argument("--n", type=int, default=None, help="override the primitive count")
    ap.add_argument("--loss", choices=["l1", "l1-dssim"], default="l1",
                    help="loss in the step: mean L1 (the training-iteration configuration) or Eq. 11's "
                         "0.8 L1 + 0.2 D-SSIM")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement (config 3)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-only", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="config 4: K in {0,1,2,4,8} x {f32, bf16}, one line each, with the oracle crop error")
    ap.add_argument("--no-oracle-crop", action="store_true",
                    help="skip the comparison of pose 0 with the FP64 oracle on the 256x256 centre crop")
    ap.add_argument("--no-bf16", action="store_true",
                    help="skip the BF16-storage run of the same step beside the float32 one")
    return ap.parse_args()


def workload_name(args, n, K, W, H, poses=16):
    st = "bf16-storage" if args.storage == "bf16" else "f32"
    loss = "L1 loss" if getattr(args, "loss", "l1") == "l1" else "0.8 L1 + 0.2 D-SSIM loss"
    return f"3DGabSplat train iteration: {n} prims K={K} SH3, {W}x{H}, {poses} orbit poses, {loss}, {st}"


# ----------------------------------------------------------------------------------------------
# clocks sampled with nvidia-smi while the timed region runs
# ----------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, pci_bus_id):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={pci_bus_id}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # nvidia-smi takes a moment to start: wait (at most 5 s) for its first sample, so the
        # samples cover the whole timed region that follows
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 5.0 and self.proc.poll() is None:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)
        self.t_ready = time.time()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = [s for s in sm if s > 0.5 * (max(mx) if mx else 2032)]
        return {"sm_mhz": float(np.median(busy if busy else sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline / reference arm)
# ----------------------------------------------------------------------------------------------
_SPEC_CACHE = {}


def oracle_sample_ms(scene, cam, seed, n_tiles=4, prim_slice=8, pose_key=None):
    """Time the FP64 oracle on a bounded sample of one training iteration; return the estimated
    ms for the whole iteration, a description and the wall seconds spent.

    The iteration is projection + binning of every primitive, forward + backward compositing of
    every non-empty tile, and the backward through the projection.  The sample times:
    - projection + binning of a contiguous 1/prim_slice of the primitives, scaled by prim_slice;
    - forward + backward compositing of n_tiles tiles drawn with probability proportional to their
      pair count, each timed alone; the estimate is sum(L) x mean(t_i / L_i) (Hansen-Hurwitz), so
      a few tiles suffice whatever the spread of list lengths;
    - the backward through the projection of the same 1/prim_slice of the primitives (seeded
      upstream gradients), scaled by prim_slice.
    The full binning that lists the tiles is computed once per pose and not timed."""
    import torch

    from oracle import gabsplat_oracle as O
    oc = O.default_config()
    keys = ("means", "scales", "quats", "opacity", "sh", "freqs", "weights")
    n = scene["means"].shape[0]
    w0 = time.perf_counter()
    key = pose_key if pose_key is not None else id(cam)
    if key not in _SPEC_CACHE:
        _SPEC_CACHE[key] = O.bin_spec(scene, cam, oc)
    spec = _SPEC_CACHE[key]
    rng = np.random.default_rng(seed)
    m = max(1, n // prim_slice)
    off = int(rng.integers(0, n - m + 1))
    part = {k: scene[k][off:off + m] for k in keys}
    t0 = time.perf_counter()
    O.bin_spec(part, cam, oc)
    with torch.no_grad():
        O.project(O._to_f64(part), cam, oc)
    t_proj = (time.perf_counter() - t0) * (n / m)
    leaves_p = O._to_f64(part, requires_grad=True)
    proj_p = O.project(leaves_p, cam, oc)
    outs_p = [proj_p[k] for k in O.REC_KEYS if proj_p[k].requires_grad]
    gouts_p = [torch.from_numpy(rng.standard_normal(tuple(o.shape))) for o in outs_p]
    t2 = time.perf_counter()
    torch.autograd.backward(outs_p, gouts_p)
    t_pbwd = (time.perf_counter() - t2) * (n / m)
    L = (spec["ranges"][:, 1].astype(np.int64) - spec["ranges"][:, 0]).astype(np.float64)
    tiles = rng.choice(len(L), n_tiles, replace=True, p=L / L.sum())
    ids = np.unique(np.concatenate([spec["sorted_vals"][spec["ranges"][t, 0]:spec["ranges"][t, 1]] for t in tiles]))
    sub = {k: scene[k][ids] for k in keys}
    spec_sub = O.bin_spec(sub, cam, oc)
    with torch.no_grad():
        proj = O.project(O._to_f64(sub), cam, oc)
    rec = {k: proj[k].clone().requires_grad_(True) for k in O.REC_KEYS}
    tx = spec["tiles_x"]
    per_pair = []
    for t in tiles:
        g = torch.zeros(3, cam["height"], cam["width"], dtype=torch.float64)
        ty_, tx_ = divmod(int(t), tx)
        g[:, ty_ * 16:ty_ * 16 + 16, tx_ * 16:tx_ * 16 + 16] = 1e-3
        t1 = time.perf_counter()
        O._render_tiles(rec, spec_sub, cam, oc, dL_dC=g, tiles=[int(t)], prims=sub)
        per_pair.append((time.perf_counter() - t1) / L[t])
    t_tiles = L.sum() * float(np.mean(per_pair))
    ms = 1e3 * (t_proj + t_tiles + t_pbwd)
    if os.environ.get("GS_ORACLE_SAMPLE_DEBUG"):
        print("oracle sample: proj %.0f tiles %.0f pbwd %.0f ms; L %s" % (1e3 * t_proj, 1e3 * t_tiles, 1e3 * t_pbwd,
                                                                        L[tiles].astype(int).tolist()), flush=True)
    desc = (f"projection+binning of 1/{prim_slice} of the {n} primitives, fwd+bwd compositing of {n_tiles} "
            f"tiles drawn by pair count from {int((L > 0).sum())} non-empty ones (Hansen-Hurwitz estimate), "
            f"projection backward of the same 1/{prim_slice}; each part scaled to the full iteration")
    return ms, desc, time.perf_counter() - w0


ORACLE_DRAWS = 16   # the fixed draws (seed s at pose s) that both the baseline and the reference arm use


def oracle_baseline(scene, cams, samples, threads, seed0=0):
    """Mean of oracle_sample_ms over draws seed0 .. seed0 + samples - 1 (draw s at pose s mod the
    poses), on `threads` host threads: the reference arm's step s is draw s mod ORACLE_DRAWS."""
    import torch
    prev = torch.get_num_threads()
    torch.set_num_threads(threads)
    try:
        oracle_sample_ms(scene, cams[0], 10_000 + seed0, pose_key=0)        # untimed first call
        runs = [oracle_sample_ms(scene, cams[(seed0 + s) % len(cams)], seed0 + s, pose_key=(seed0 + s) % len(cams))
                for s in range(samples)]
    finally:
        torch.set_num_threads(prev)
    return float(np.mean([r[0] for r in runs])), runs[0][1], float(sum(r[2] for r in runs))


SERVE_RATES = (200.0, 1000.0, 2000.0)


def run_serve(args):
    """Config 3: 8 resident scenes (100k..3M primitives, K=4, SH3, BF16 storage), a Poisson stream of
    novel-view requests at 200 req/s with resolutions from {400x400, 800x800, 1280x720, 1920x1080}.
    The continuous-batching server (graph replays on 3 slots) against the plain float32 path that
    renders one request at a time.  Both replay the stream in real time (latency) at the specified
    200 req/s and, with the same scenes, poses and resolutions, at 1000 and 2000 req/s (the plain
    path saturates near 1100 frames/s, so batching and overlap only matter above that), and then
    serve the whole stream offered at once (frames/s at saturation)."""
    import torch

    from paper_2508_05343_b300 import binding as B
    from paper_2508_05343_b300 import scenes, serve
    t0 = time.time()
    sc = scenes.serve_scenes()
    reqs = serve.make_requests(n_req=args.serve_requests)
    res = scenes.SERVE_RESOLUTIONS
    scaled = {rate: [dataclasses.replace(r, arrival_s=r.arrival_s * SERVE_RATES[0] / rate) for r in reqs]
              for rate in SERVE_RATES}
    srv = serve.Server(sc, B.GS_BF16, 4, 3, n_slots=3)
    est = srv.calibrate(res)
    warm = serve.make_requests(n_req=64, rate=1e6, seed=2001)
    srv.run(warm, realtime=False)
    live = {rate: srv.run(scaled[rate], realtime=True) for rate in SERVE_RATES}
    sat = srv.run(reqs, realtime=False)
    del srv
    torch.cuda.empty_cache()
    plain = serve.PlainRenderer(sc, est)
    plain.prepare(reqs)
    plain.run(warm, realtime=False)
    p_live = {rate: plain.run(scaled[rate], realtime=True) for rate in SERVE_RATES}
    p_sat = plain.run(reqs, realtime=False)
    del plain
    torch.cuda.empty_cache()
    r3 = lambda x: round(float(x), 3)
    first = live[SERVE_RATES[0]]
    sweep = [{"rate_req_per_s": rate,
              "served": {"p50_ms": r3(live[rate]["latency_ms_p50"]), "p99_ms": r3(live[rate]["latency_ms_p99"]),
                         "frames_per_s": r3(live[rate]["frames_per_s"]), "mean_batch": r3(live[rate]["mean_batch"])},
              "plain": {"p50_ms": r3(p_live[rate]["latency_ms_p50"]), "p99_ms": r3(p_live[rate]["latency_ms_p99"]),
                        "frames_per_s": r3(p_live[rate]["frames_per_s"])}} for rate in SERVE_RATES]
    return {"workload": "8 resident scenes {100k..3M} prims K=4 SH3 BF16; %d Poisson requests at 200 req/s; "
                        "resolutions 400x400/800x800/1280x720/1920x1080; random orbit poses" % len(reqs),
            "p50_ms": r3(first["latency_ms_p50"]), "p99_ms": r3(first["latency_ms_p99"]),
            "frames_per_s": r3(sat["frames_per_s"]), "frames_per_s_at_200rps": r3(first["frames_per_s"]),
            "mean_batch_saturated": r3(sat["mean_batch"]), "mean_batch_200rps": r3(first["mean_batch"]),
            "retries": sum(v["retries"] for v in live.values()) + sat["retries"],
            "plain": {"p50_ms": r3(p_live[SERVE_RATES[0]]["latency_ms_p50"]),
                      "p99_ms": r3(p_live[SERVE_RATES[0]]["latency_ms_p99"]),
                      "frames_per_s": r3(p_sat["frames_per_s"]), "storage": "f32", "mode": "one request at a time"},
            "speedup_frames_per_s": r3(sat["frames_per_s"] / p_sat["frames_per_s"]),
            "rate_sweep": sweep,
            "wall_s": round(time.time() - t0, 1)}


def oracle_crop_error(scene, cam, gpu_img, storage_bf16):
    """Error of the GPU image against the FP64 oracle on the 256x256 centre crop of the view:
    evaluation error against the oracle on the same (BF16-rounded when stored so) values, and for
    BF16 storage also the quantisation error against the float32 values.  Per variant: the largest
    error at pixels the oracle does not flag, the largest excess over tolerance + flip allowance at
    flagged ones (<= 0: within the bar), the flagged count and the PSNR (peak 1)."""
    import torch

    from oracle import gabsplat_oracle as O
    from paper_2508_05343_b300 import scenes
    torch.set_num_threads(os.cpu_count() or 1)
    W, H = cam["width"], cam["height"]
    x0, y0 = (W - 256) // 2, (H - 256) // 2
    x1, y1 = x0 + 256, y0 + 256
    tx = (W + 15) // 16
    tiles = [ty * tx + t for ty in range(y0 // 16, (y1 - 1) // 16 + 1) for t in range(x0 // 16, (x1 - 1) // 16 + 1)]
    oc = O.default_config()
    psnr = lambda e: float(10 * np.log10(1.0 / max(float(np.mean(e ** 2)), 1e-30)))
    out = {}
    variants = [("eval", {k: scenes.bf16_round(scene[k]) if storage_bf16 and k in ("sh", "freqs", "weights")
                          else scene[k] for k in scene})]
    if storage_bf16:
        variants.append(("quant", scene))
    t0 = time.time()
    key = ("crop", id(cam))
    if key not in _SPEC_CACHE:                       # the binning does not depend on the storage
        _SPEC_CACHE[key] = O.bin_spec(scene, cam, oc)
    for name, prims in variants:
        ref = O.render(prims, cam, oc, tiles=tiles, spec=_SPEC_CACHE[key])
        e = gpu_img[:, y0:y1, x0:x1] - ref["image"].numpy()[:, y0:y1, x0:x1]
        amb = ref["ambiguous"].numpy()[y0:y1, x0:x1]
        allow = ref["allowance"].numpy()[:, y0:y1, x0:x1]
        err = np.abs(e)
        out[name] = {"max_abs_unflagged": float(err.max(0)[~amb].max()), "max_abs": float(err.max()),
                     "psnr_db": round(psnr(e), 2), "flagged_px": int(amb.sum())}
        if name == "eval":      # the image bar applies to the evaluation error only
            out[name]["max_excess_over_allowance"] = float((err - 2e-4 - allow).max(0)[amb].max()) if amb.any() else None
    out["crop"] = f"[{x0},{x1})x[{y0},{y1})"
    out["oracle_wall_s"] = round(time.time() - t0, 1)
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle timed per step on the host cores, each step one bounded
    sample (oracle_sample_ms) of the training iteration at the step's pose."""
    import torch
    from paper_2508_05343_b300 import scenes
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    torch.set_num_threads(os.cpu_count() or 1)
    scene = scenes.config_scene(args.config, n=args.n, K=args.K)
    cams = scenes.config_cameras(args.config)
    for i in range(args.warmup):
        oracle_sample_ms(scene, cams[i % len(cams)], 10_000 + i, pose_key=i % len(cams))
    times = []
    w0 = time.time()
    for s in range(args.steps):
        d = s % ORACLE_DRAWS   # the same fixed draws as bench's cpu_baseline
        ms, desc, _ = oracle_sample_ms(scene, cams[d % len(cams)], d, pose_key=d % len(cams))
        times.append(ms)
    v = float(np.mean(times))
    W, H = cams[0]["width"], cams[0]["height"]
    cores = torch.get_num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args, scene["n"], scene["K"], W, H, len(cams)) + " (FP64 CPU oracle)"},
            "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                             "sample_wall_s": round(time.time() - w0, 1)},
            "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------------
# replicas (one process per GPU, no collective on the data path)
# ----------------------------------------------------------------------------------------------
def replica_pose(s, rank, n_poses):
    """Pose that replica `rank` renders at step s: replicas start 7 poses apart (7 is coprime to
    the 16 orbit poses), so at every step the first 16 replicas render different views."""
    return (s + 7 * rank) % n_poses


def max_over_ranks(value, world, device):
    """The slowest replica's time (the job ends when it does); a no-op on one process."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_iter(ms_step_max, world):
    """Whole-job time per training iteration: `world` replicas each finish one iteration every
    ms_step_max milliseconds."""
    return ms_step_max / world


# ----------------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------------
class TrainStep:
    """One frame's workspace and buffers for the training step at one storage type, and the step's
    launch sequence through the C ABI: preprocess -> bin_sort -> render_fwd -> loss -> the two
    halves of render_bwd (2D adjoint with the gradient zero-fill, then the chain rule)."""

    STAGES = ["preprocess", "bin_sort", "render_fwd", "loss", "render_bwd", "preprocess_bwd"]

    def __init__(self, scene, cams, storage, dev, loss, targets, pose_of):
        import torch

        from paper_2508_05343_b300 import binding as B
        from paper_2508_05343_b300 import raster
        self.B, self.storage, self.loss_kind, self.targets, self.pose_of = B, storage, loss, targets, pose_of
        W, H = cams[0]["width"], cams[0]["height"]
        n, K, deg = scene["n"], scene["K"], scene["sh_degree"]
        self.pt = raster.to_device(scene, dev, storage)
        self.cfg = B.make_config()
        self.rast = raster.Rasterizer(n, K, deg, W, H, device=dev)
        # size the pair capacity for every pose once (host reads; outside the timed region)
        self.pose_stats = []
        for c in cams:   # the work counters come from the forward that writes them
            self.rast.forward(self.pt, c, self.cfg, storage=storage, stats=True)
            v = self.rast.views()
            self.pose_stats.append(dict(pairs=v["pairs"], n_eval=int(v["n_eval"].sum().item()),
                                        active=int((v["touched"] > 0).sum().item()),
                                        n_reach=int(v["n_reach"].sum().item()), n_comp=int(v["n_comp"].sum().item()),
                                        n_contrib=int(v["n_contrib"].sum().item())))
        maxP = max(st["pairs"] for st in self.pose_stats)
        if self.rast.capacity < maxP * 1.02:
            self.rast._alloc(int(maxP * 1.05) + 4096)
        self.frame = self.rast.frame
        self.prims_s = B.make_prims(self.pt, storage)
        self.cams_s = [B.make_camera(c) for c in cams]
        self.img = torch.empty(3, H, W, device=dev)
        self.dL = torch.empty_like(self.img)
        self.loss_val = torch.zeros(1, dtype=torch.float64, device=dev)
        self.scratch = torch.empty(max(B.gabsplat_loss_scratch_bytes(self.img.numel()),
                                       B.gabsplat_loss_l1_dssim_scratch_bytes(3, H, W)), dtype=torch.uint8, device=dev)
        self.grads = {k: torch.empty(self.pt[k].shape, dtype=torch.float32, device=dev) for k in raster.ATTRS}
        self.grads["means2d"] = torch.empty(n, 2, device=dev)
        self.g_s = B.gs_prim_grads()
        for k, t in self.grads.items():
            setattr(self.g_s, k, t.data_ptr() if t.numel() else None)
        vv = self.rast.views()
        self.tiles = vv["tiles_x"] * vv["tiles_y"]

    def step(self, s, evs=None, target=None):
        B = self.B
        j = self.pose_of(s)
        if evs: evs[0].record()
        B.gabsplat_preprocess(self.frame, self.prims_s, self.cams_s[j], self.cfg)
        if evs: evs[1].record()
        B.gabsplat_bin_sort(self.frame)
        if evs: evs[2].record()
        B.gabsplat_render_fwd(self.frame, self.img, None)
        if evs: evs[3].record()
        tj = self.targets[j] if target is None else target
        if self.loss_kind == "l1":
            B.gabsplat_loss(self.img, tj, B.GS_LOSS_L1, self.loss_val, self.dL, self.scratch)
        else:
            B.gabsplat_loss_l1_dssim(self.img, tj, 0.2, self.loss_val, self.dL, self.scratch)
        if evs: evs[4].record()
        B.gabsplat_render_bwd_2d_zero(self.frame, self.dL, self.g_s)
        if evs: evs[5].record()
        B.gabsplat_preprocess_bwd_prezeroed(self.frame, self.g_s)
        if evs: evs[6].record()

    def timed(self, steps, warmup, barrier, dev):
        """W untimed steps, then K steps between a barrier + synchronize on each side, with CUDA
        events on the launching stream around the whole region; clocks sampled throughout.  Then
        the same K steps again with an event between every two stages for the per-stage split
        (an event between two kernels keeps the second from starting in the first one's tail, so
        the split comes from its own pass).  Returns (ms per step, {stage: ms}, clocks)."""
        import torch
        sampler = ClockSampler(_pci_id(torch.cuda.get_device_properties(dev)))
        for s in range(warmup):
            self.step(s)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        start.record()
        for s in range(steps):
            self.step(s)
        end.record()
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop()
        st, _ = self.rast.status()
        if st != self.B.GS_OK:
            raise RuntimeError(f"device status after timed region: {self.B.status_string(st)}")
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(steps)]
        for s in range(steps):
            self.step(s, evs[s])
        torch.cuda.synchronize()
        stage_ms = {nm: float(np.mean([evs[s][i].elapsed_time(evs[s][i + 1]) for s in range(steps)]))
                    for i, nm in enumerate(self.STAGES)}
        return start.elapsed_time(end) / steps, stage_ms, clocks


def stage_work(n, K, deg, bf16, P, n_eval, n_contrib, n_act, npix, loss, tpasses, dpasses):
    """Algorithmic work per stage of one step: ("hbm", bytes) or ("alu", FP32 operations) or
    ("flop", FLOPs).  Per-unit figures as stated in the design notes (kernels, bounds and work)."""
    sh_b = (deg + 1) ** 2 * 3 * (2 if bf16 else 4)
    g_b = K * 4 * (2 if bf16 else 4)
    param_b = 12 + 12 + 16 + 4 + sh_b + g_b
    rec_b = (12 + 4 * ((3 * K + 3) // 4)) * 4
    g2d_b = 4 * ((9 + 3 * K + 3) // 4) * 4
    grad_b = 4 * (3 + 3 + 4 + 1 + (deg + 1) ** 2 * 3 + 3 * K + K + 2)
    # Algorithmic FP32 work of the blending kernels: every evaluated pixel-pair costs 14 + 4K FP32
    # operations in the forward (offset and quadratic form, exp argument, the K-term filter bank
    # after cycle-domain reduction, alpha, blend; an FMA is one operation) and three times that in
    # the backward, whose evaluated pixel-pairs are those up to each pixel's last contributor.
    ops_eval = 14 + 4 * K
    return {
        # all primitives: mean/scale/quat read, counts written and scanned; active ones: depth key
        # written, compacted (16) and depth-sorted (16 per pass), rank scan (key, count, order,
        # offset: 20), order and offset read by emission and records (12), attributes read and
        # record written; one 8-byte pair written per kept tile
        "preprocess": ("hbm", n * (40 + 8) + n_act * (8 + 16 + 16 * dpasses + 20 + 12 + param_b + rec_b) + P * 8),
        # tile histogram read, each tile pass reads and writes 8-byte pairs, ranges read
        "bin_sort": ("hbm", P * (8 + tpasses * 16 + 8)),
        "render_fwd": ("alu", n_eval * ops_eval),
        "loss": ("hbm", npix * 12) if loss == "l1" else ("flop", npix * SSIM_FLOPS_PER_VALUE),
        "render_bwd": ("alu", n_contrib * 3 * ops_eval),
        # active primitives read their inputs and grad2d row and write their gradients (the other
        # rows were zero-filled inside render_bwd)
        "preprocess_bwd": ("hbm", n_act * (4 + param_b + g2d_b + grad_b)),
    }, param_b


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2508_05343_b300 import binding as B
    from paper_2508_05343_b300 import raster, scenes

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    storage = B.GS_BF16 if args.storage == "bf16" else B.GS_F32

    scene = scenes.config_scene(args.config, n=args.n, K=args.K)
    cams = scenes.config_cameras(args.config)
    W, H = cams[0]["width"], cams[0]["height"]
    n, K, deg = scene["n"], scene["K"], scene["sh_degree"]
    targets = [torch.as_tensor(scenes.make_target(W, H, 5000 + j)).to(dev) for j in range(len(cams))]

    def pose_of(s):
        return replica_pose(s, rank, len(cams))

    def barrier():
        if world > 1:
            dist.barrier()

    ts = TrainStep(scene, cams, storage, dev, args.loss, targets, pose_of)
    tbits = max(0, math.ceil(math.log2(max(1, ts.tiles))))
    tpasses = math.ceil(tbits / 8)                           # tile-sort passes (launched = needed)
    zb = lambda z: int(np.float32(z).view(np.uint32))
    dbits = max(1, (zb(cams[0]["zfar"]) - zb(cams[0]["znear"])).bit_length())
    dpasses = min(4, math.ceil(dbits / 8))                   # depth-sort passes that do work (4 launched)
    # my kernels per step: setup; bin, active count + scan, 4 depth passes, rank count + scan, emit,
    # records; tile histogram + tile passes + ranges + tile schedule; render_fwd; loss (2);
    # grad2d clear + render_bwd (with the attribute-gradient zero-fill); preprocess_bwd
    launches_per_step = 1 + 11 + (1 + tpasses + 2) + 1 + 2 + 2 + 1

    ms_step, stage_ms, clocks = ts.timed(args.steps, args.warmup, barrier, dev)
    ms_step_max = max_over_ranks(ms_step, world, dev)

    # ---- end to end through the public API with host buffers --------------------------------
    # Every step's target image goes host -> device from pinned memory inside the timed region, on a
    # copy stream into one of two device buffers: step s + 1's upload overlaps step s's compute (the
    # input pipeline a training loop would run); each step waits for its own upload, and an upload
    # waits until the step that last used its buffer is done.  The loss comes back after every step.
    e2e = None
    if not args.no_e2e:
        host_t = [targets[j].cpu().pin_memory() for j in range(len(cams))]
        loss_host = torch.zeros(1, dtype=torch.float64).pin_memory()
        dev_t = [torch.empty_like(ts.img), torch.empty_like(ts.img)]
        main, copy_s = torch.cuda.current_stream(), torch.cuda.Stream()
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        freed = [torch.cuda.Event(), torch.cuda.Event()]

        def upload(s, after=None):
            b = s % 2
            with torch.cuda.stream(copy_s):
                copy_s.wait_event(after if after is not None else freed[b])
                dev_t[b].copy_(host_t[pose_of(s)], non_blocking=True)
                ready[b].record(copy_s)

        def run(nsteps, start_event):
            for b in range(2):
                freed[b].record(main)
            upload(0, after=start_event)
            for s in range(nsteps):
                if s + 1 < nsteps:
                    upload(s + 1)
                main.wait_event(ready[s % 2])
                ts.step(s, target=dev_t[s % 2])
                freed[s % 2].record(main)
                loss_host.copy_(ts.loss_val, non_blocking=True)

        w0 = torch.cuda.Event()
        w0.record(main)
        run(min(3, args.steps), w0)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        run(args.steps, e0)
        e1.record(main)
        torch.cuda.synchronize()
        te = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
        e2e = {"value": round(job_ms_per_iter(te, world), 4), "unit": UNIT,
               "h2d_bytes_per_step": int(ts.img.numel() * 4), "d2h_bytes_per_step": 8}

    # ---- roofline of the dominant kernel ------------------------------------------------------
    poses = [pose_of(s) for s in range(args.steps)]

    def mean_stats(t):
        m = lambda key: float(np.mean([t.pose_stats[j][key] for j in poses]))
        return m("pairs"), m("n_eval"), m("n_contrib"), m("active"), m("n_reach"), m("n_comp")

    P, n_eval, n_contrib, n_act, n_reach, n_comp = mean_stats(ts)
    work, param_b = stage_work(n, K, deg, storage == B.GS_BF16, P, n_eval, n_contrib, n_act, ts.img.numel(),
                               args.loss, tpasses, dpasses)
    # A finer count, which charges the filter bank only to pixel-pairs passing o G >= alpha_min and
    # the adjoints only to composited ones (7 per walked pixel-pair, 6 + 6K per reached, 7 per
    # composited; in the backward 7 per walked and 43 + 16K per composited), is reported as "fine".
    ops_eval = 14 + 4 * K
    ops_walk, ops_reach, ops_comp, ops_bwd = 7, 6 + 6 * K, 7, 43 + 16 * K
    sm_mhz = (clocks or {}).get("sm_mhz") or 2032.0
    alu_peak = SM_COUNT_B300 * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12          # T FP32 operations/s (issue)
    flop_peak = 2 * alu_peak                                                      # TFLOP/s with FMA = 2 FLOPs
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    stage_peak = {"hbm": hbm_peak, "alu": alu_peak, "flop": flop_peak}

    def fractions(work, stage_ms):
        out = {}
        for nm, (bd, amt) in work.items():
            s_ = stage_ms[nm] * 1e-3
            out[nm] = round((amt / s_ / 1e9 / hbm_peak) if bd == "hbm" else (amt / s_ / 1e12 / stage_peak[bd]), 4)
        return out

    top = max(stage_ms, key=stage_ms.get)
    bound, amount = work[top]
    sec = stage_ms[top] * 1e-3
    fine = {"render_fwd": n_eval * ops_walk + n_reach * ops_reach + n_comp * ops_comp,
            "render_bwd": n_contrib * ops_walk + n_comp * ops_bwd}
    if bound == "hbm":
        achieved, peak, unit = amount / sec / 1e9, hbm_peak, "GB/s"
    else:
        achieved, peak, unit = amount / sec / 1e12, stage_peak[bound], "TFLOP/s"
    traffic = _measured_traffic(top, W, H, n)
    roofline = {"kernel": top, "bound": "alu" if bound == "flop" else bound, "achieved": round(achieved, 3),
                "peak": round(peak, 3), "unit": unit, "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json)" if bound == "hbm" else
                f"derived FP32 issue peak: 148 SMs x 128 lanes x {sm_mhz:.0f} MHz (median SM clock under load), "
                "one FP32 operation (an FMA is one) per lane per cycle"}
    if top in fine:
        roofline["work_per_unit"] = (f"{ops_eval} FP32 operations per evaluated pixel-pair" +
                                     (" x 3 (backward)" if top == "render_bwd" else ""))
        fa = fine[top] / sec / 1e12
        roofline["fine"] = {"achieved": round(fa, 3), "frac": round(fa / peak, 4)}
        ex = _executed_fp32_ops(top, W, H, n)
        if ex is not None:
            # FP32 operations the kernel executed per launch (ncu instruction counts, see profiles/)
            # at the live launch time, against the same peak
            ea = ex / sec / 1e12
            roofline["executed"] = {"ops_per_launch": ex, "achieved": round(ea, 3), "frac": round(ea / peak, 4)}
    stage_fracs = fractions(work, stage_ms)

    # ---- the same step with BF16 storage of SH / frequencies / weights --------------------------
    bf16 = None
    if storage == B.GS_F32 and not args.no_bf16:
        ts_b = TrainStep(scene, cams, B.GS_BF16, dev, args.loss, targets, pose_of)
        ms_b, stage_b, clocks_b = ts_b.timed(args.steps, args.warmup, barrier, dev)
        ms_b = max_over_ranks(ms_b, world, dev)
        Pb, ne_b, nc_b, na_b, _, _ = mean_stats(ts_b)
        work_b, _ = stage_work(n, K, deg, True, Pb, ne_b, nc_b, na_b, ts.img.numel(), args.loss, tpasses, dpasses)
        bf16 = {"value": round(job_ms_per_iter(ms_b, world), 4), "unit": UNIT, "ms_per_step": round(ms_b, 4),
                "storage": "bf16 SH, frequencies and weights; FP32 evaluation and compositing",
                "stages_ms": {k: round(v, 4) for k, v in stage_b.items()},
                "stage_roofline_frac": fractions(work_b, stage_b), "clocks": clocks_b,
                "speedup_vs_f32": round(ms_step_max / ms_b, 4)}
        if rank == 0 and not args.no_oracle_crop:
            img0 = ts_b.rast.forward(ts_b.pt, cams[0], ts_b.cfg, storage=B.GS_BF16)
            torch.cuda.synchronize()
            bf16["oracle_crop"] = oracle_crop_error({k: scene[k] for k in raster.ATTRS}, cams[0],
                                                    img0.cpu().numpy().astype(np.float64), True)
        del ts_b
        torch.cuda.empty_cache()

    # the fused L1 + D-SSIM loss (Eq. 11) timed on its own on the same images, whatever --loss is
    img, dL, loss_val, scratch = ts.img, ts.dL, ts.loss_val, ts.scratch
    ssim_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for r in range(3):
        B.gabsplat_loss_l1_dssim(img, targets[0], 0.2, loss_val, dL, scratch)
    ssim_ev[0].record()
    for r in range(20):
        B.gabsplat_loss_l1_dssim(img, targets[r % len(targets)], 0.2, loss_val, dL, scratch)
    ssim_ev[1].record()
    torch.cuda.synchronize()
    ssim_ms = ssim_ev[0].elapsed_time(ssim_ev[1]) / 20
    ssim_tf = img.numel() * SSIM_FLOPS_PER_VALUE / (ssim_ms * 1e-3) / 1e12
    l1_dssim = {"ms": round(ssim_ms, 4), "bound": "alu", "achieved": round(ssim_tf, 3), "peak": round(flop_peak, 3),
                "unit": "TFLOP/s", "frac": round(ssim_tf / flop_peak, 4),
                "hbm_frac": round(img.numel() * 12 / (ssim_ms * 1e-3) / 1e9 / hbm_peak, 4)}

    # frequency-adaptive density control on the same scene: about 10% of the primitives reach the
    # gradient threshold, half of them small (cloned) and half large (split); 20 timed compactions
    rng_d = np.random.default_rng(77)
    d_acc = torch.tensor((rng_d.random(n) * 2.22e-4).astype(np.float32), device=dev)
    d_den = torch.ones(n, device=dev)
    d_noise = torch.tensor(rng_d.standard_normal((n, 2, 3)).astype(np.float32), device=dev)
    d_cfg = B.make_densify_config(dense_scale=float(np.median(scene["scales"].max(1))))
    d_out = {k: torch.empty((2 * n,) + tuple(v.shape[1:]), dtype=v.dtype, device=dev) for k, v in ts.pt.items()}
    d_counts = torch.zeros(4, dtype=torch.int32, device=dev)
    d_scr = torch.empty(B.gabsplat_densify_scratch_bytes(n), dtype=torch.uint8, device=dev)
    d_args = (ts.prims_s, d_acc, d_den, d_noise, d_cfg, B.make_prim_arrays(d_out), 2 * n, d_counts, d_scr)
    B.gabsplat_densify(*d_args)
    d_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    d_ev[0].record()
    for r in range(20):
        B.gabsplat_densify(*d_args)
    d_ev[1].record()
    torch.cuda.synchronize()
    d_ms = d_ev[0].elapsed_time(d_ev[1]) / 20
    dc = d_counts.cpu().tolist()
    d_bytes = n * (param_b + 8) + (dc[3] // 2) * 24 + dc[0] * param_b
    densify = {"ms": round(d_ms, 4), "rows_in": n, "rows_out": dc[0], "clones": dc[2], "split_children": dc[3],
               "bound": "hbm", "achieved": round(d_bytes / (d_ms * 1e-3) / 1e9, 1), "peak": hbm_peak, "unit": "GB/s",
               "frac": round(d_bytes / (d_ms * 1e-3) / 1e9 / hbm_peak, 4)}
    del d_out, d_noise, d_scr

    crop = None
    if rank == 0 and not args.no_oracle_crop:
        img0 = ts.rast.forward(ts.pt, cams[0], ts.cfg, storage=storage)
        torch.cuda.synchronize()
        crop = oracle_crop_error({k: scene[k] for k in raster.ATTRS}, cams[0], img0.cpu().numpy().astype(np.float64),
                                 storage == B.GS_BF16)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        ms, desc, wall = oracle_baseline(scene, cams, ORACLE_DRAWS, cores)
        ms1, _, wall1 = oracle_baseline(scene, cams, 1, 1)
        cpu = {"value": round(ms, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": desc + f"; mean of the {ORACLE_DRAWS} fixed draws (seed s at pose s) that the "
                                "reference arm's steps cycle through",
               "wall_s": round(wall, 1), "single_thread": {"value": round(ms1, 1), "cores": 1, "wall_s": round(wall1, 1)}}

    serve_out = None
    if rank == 0 and world == 1 and not args.no_serve:
        del ts, targets, img, dL
        torch.cuda.empty_cache()
        try:
            serve_out = run_serve(args)
        except Exception as e:          # the training line is still reported
            serve_out = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(job_ms_per_iter(ms_step_max, world), 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step_max, 4),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if storage == B.GS_F32 else "f32 (bf16 storage)", "data": "synthetic",
            "config": {"workload": workload_name(args, n, K, W, H, len(cams)), "n": n, "K": K, "sh_degree": deg,
                       "width": W, "height": H, "storage": args.storage, "poses": len(cams),
                       "pairs_per_view": round(P), "evaluated_pixel_pairs": round(n_eval),
                       "walked_pixel_pairs_bwd": round(n_contrib), "reached_pixel_pairs": round(n_reach),
                       "composited_pixel_pairs": round(n_comp),
                       "l2": "inputs larger than L2 (primitive arrays %.0f MB)" % (n * param_b / 1e6),
                       "parallelism": f"replicas x{world}"},
            "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "stage_roofline_frac": stage_fracs,
            "bf16": bf16,
            "l1_dssim": l1_dssim,
            "densify": densify,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "serve": serve_out,
            "oracle_crop": crop,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _pci_id(props):
    try:
        return "%08X:%02X:%02X.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]


KERNEL_SOURCES = {"preprocess": "preprocess.cu", "bin_sort": "sort.cu", "render_fwd": "render.cu",
                  "loss": "loss.cu", "render_bwd": "render.cu", "preprocess_bwd": "preprocess.cu"}


def kernel_source_sha(stage):
    """Hash of the sources that define a stage's kernels: its .cu file, common.cuh and the header."""
    import hashlib
    h = hashlib.sha1()
    for f in (os.path.join(ROOT, "paper_2508_05343_b300", "csrc", KERNEL_SOURCES[stage]),
              os.path.join(ROOT, "paper_2508_05343_b300", "csrc", "common.cuh"),
              os.path.join(ROOT, "include", "gabsplat.h")):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:12]


def _measured_traffic(stage, W, H, n):
    """DRAM bytes per launch of a stage's kernel from the ncu summary in profiles/ (lines
    `stage source_sha width height n bytes`), if it was taken on these kernel sources and this
    workload; else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_train_iter.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(stage)
    for line in open(path):
        if line.startswith("#"):
            continue
        f = line.split()
        if len(f) == 6 and f[0] == stage and f[1] == sha and (int(f[2]), int(f[3]), int(f[4])) == (W, H, n):
            return int(f[5])
    return None


def _executed_fp32_ops(stage, W, H, n):
    """FP32 operations one launch of a stage's kernel executed, from the ncu instruction counts in
    profiles/ (lines `stage source_sha width height n ops`: FADD + FMUL + FFMA + 2 x the packed
    FADD2 / FMUL2 / FFMA2 thread instructions), if taken on these kernel sources and this workload."""
    path = os.path.join(ROOT, "profiles", "fp32_ops_train_iter.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(stage)
    for line in open(path):
        if line.startswith("#"):
            continue
        f = line.split()
        if len(f) == 6 and f[0] == stage and f[1] == sha and (int(f[2]), int(f[3]), int(f[4])) == (W, H, n):
            return int(f[5])
    return None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        base = list(sys.argv[1:])
        for K in (0, 1, 2, 4, 8):
            for st in ("f32", "bf16"):
                sys.argv = [sys.argv[0], "--config", "4", "--K", str(K), "--storage", st, "--steps", str(args.steps),
                            "--warmup", str(args.warmup), "--no-cpu-baseline", "--no-e2e", "--no-serve",
                            "--no-bf16"]
                run_ours(parse())
        sys.argv = [sys.argv[0]] + base
    elif args.serve_only:
        print(json.dumps({"serve": run_serve(args)}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
