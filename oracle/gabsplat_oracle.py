"""FP64 CPU oracle of the 3D Gabor splatting rasterizer -- TEST INFRASTRUCTURE ONLY.

This module exists to check the CUDA path.  Only the tests, the package smoke check and the
CPU-baseline leg of the benchmark may import it; the product path never does, and it shares
no code with the CUDA kernels (the only common module is the seeded input generator).

What it computes (paper: "3DGabSplat", arXiv 2508.05343), per camera:

1. project():   the 3D Gabor primitive of Sec. 3.2 (Eq. 5: a Gaussian envelope times the
   weighted filter bank (1 - sum w_i) + sum w_i cos(2 pi f_i . (x - mu))) is mapped to ray space
   with the EWA local affine map JW (Sec. 3.1, Eq. 2; supplement A.1).  The envelope becomes the
   top-left 2x2 of J W Sigma W^T J^T (Sec. 3.1), each frequency becomes f_proj = ((JW)^-1)^T f
   (Eq. 7), and z-integration turns it into f2D = f_proj_xy - (S_02, S_12)/S_22 * f_proj_z with S the
   inverse of the ray-space covariance (Eq. 8-9; supplement A.2).  Colour is the SH expansion at
   the viewing direction.  Everything here is float64 and differentiable with torch.autograd.
2. bin_spec():  the tile binning.  Which 16x16 tiles a primitive touches and the depth used for
   ordering are integer/bit decisions, so they are defined by a written float32 procedure (the
   binning specification, op order fixed, no fused multiply-add) which the GPU follows
   independently.  Pairs are ordered by (tile, float32 depth bits, primitive index) - the
   "sorted by depth" step of Sec. 3.1 and the tile-based rasterizer of Sec. 3.3.3.
3. render():    per pixel, front-to-back alpha compositing (Eq. 10) of the 2D Gabor primitives
   (Eq. 9 text: G2D(x) [(1 - sum w) + sum w cos(2 pi f2D . (x - mu2D))]) with the conventions
   of the tile rasterizer the paper adopts: alpha = min(alpha_max, o * Gabor2D), pairs with
   alpha < alpha_min are skipped, compositing stops before the pair whose transmittance
   T (1 - alpha) would fall below T_min, and the background is added with the final T.
4. render_backward(): the exact adjoint of 1-3 by reverse-mode autodiff in float64, with the
   skip/stop decisions held fixed and zero gradient through the clamps.

Readings of points the paper leaves open (frame of f, S in ray space, dropped z-integration
constants, 3DGS conventions) are listed in the design notes; they are fixed here as:
S is the inverse of the undilated ray-space covariance; J's third row is (0, 0, 1); the
z-integration constants C1, C2 are dropped as in Eq. 9; the envelope is unnormalised (Eq. 1);
frequencies are world-frame cycles per unit; pixel centres sit at (i + 0.5, j + 0.5).
"""
from __future__ import annotations

import math

import numpy as np
import torch

F64 = torch.float64
TILE = 16


def default_config(eps2d=0.3, bg=(0.0, 0.0, 0.0), z_atten=False):
    """Rasterizer constants (float32 values, so both sides compare against identical thresholds).
    z_atten selects the z-attenuation variant (see z_attenuation)."""
    f = lambda v: float(np.float32(v))
    return dict(eps2d=f(eps2d), alpha_max=f(0.99), alpha_min=f(1.0 / 255.0), T_min=f(1e-4),
                bg=tuple(f(b) for b in bg), z_atten=bool(z_atten))


# ----------------------------------------------------------------------------------------------
# Primitive geometry (Sec. 3.1: Sigma = R S S^T R^T)
# ----------------------------------------------------------------------------------------------
def rotation_from_quaternion(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of the normalised quaternion (w, x, y, z); q: [n,4] -> [n,3,3]."""
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    rows = [
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ]
    return torch.stack(rows, -2)


def covariance_3d(scales: torch.Tensor, quats: torch.Tensor) -> torch.Tensor:
    """Sigma = R S S^T R^T with S = diag(scales) (Sec. 3.1)."""
    R = rotation_from_quaternion(quats)
    M = R * scales[:, None, :]
    return M @ M.transpose(-1, -2)


# ----------------------------------------------------------------------------------------------
# Real spherical harmonics up to degree 3 (view-dependent colour c_k of Sec. 3.1)
# Index l*l + l + m, m = -l..l; the standard orthonormal real basis on the unit sphere.
# ----------------------------------------------------------------------------------------------
def sh_basis(d: torch.Tensor, degree: int) -> torch.Tensor:
    """d: [n,3] unit directions -> [n,(degree+1)^2] real SH values."""
    x, y, z = d.unbind(-1)
    pi = math.pi
    out = [torch.full_like(x, 0.5 * math.sqrt(1.0 / pi))]
    if degree >= 1:
        c1 = math.sqrt(3.0 / (4.0 * pi))
        out += [c1 * y, c1 * z, c1 * x]
    if degree >= 2:
        out += [0.5 * math.sqrt(15.0 / pi) * x * y,
                0.5 * math.sqrt(15.0 / pi) * y * z,
                0.25 * math.sqrt(5.0 / pi) * (3.0 * z * z - 1.0),
                0.5 * math.sqrt(15.0 / pi) * x * z,
                0.25 * math.sqrt(15.0 / pi) * (x * x - y * y)]
    if degree >= 3:
        out += [0.25 * math.sqrt(35.0 / (2.0 * pi)) * y * (3.0 * x * x - y * y),
                0.5 * math.sqrt(105.0 / pi) * x * y * z,
                0.25 * math.sqrt(21.0 / (2.0 * pi)) * y * (5.0 * z * z - 1.0),
                0.25 * math.sqrt(7.0 / pi) * z * (5.0 * z * z - 3.0),
                0.25 * math.sqrt(21.0 / (2.0 * pi)) * x * (5.0 * z * z - 1.0),
                0.25 * math.sqrt(105.0 / pi) * z * (x * x - y * y),
                0.25 * math.sqrt(35.0 / (2.0 * pi)) * x * (x * x - 3.0 * y * y)]
    return torch.stack(out, -1)


# ----------------------------------------------------------------------------------------------
# Projection and splatting (Sec. 3.1, Sec. 3.3.1-3.3.2, supplement A)
# ----------------------------------------------------------------------------------------------
def camera_tensors(cam):
    W = torch.tensor(np.asarray(cam["R"], np.float64).reshape(3, 3), dtype=F64)
    tc = torch.tensor(np.asarray(cam["t"], np.float64).reshape(3), dtype=F64)
    return W, tc


def jacobian(t: torch.Tensor, cam, third_row: str = "z") -> torch.Tensor:
    """Local affine Jacobian J of the perspective map at camera-space mean t ([n,3] -> [n,3,3]).

    Rows 0 and 1 are the derivative of (fx x/z, fy y/z) with the 3DGS field-of-view guard (x/z and
    y/z clamped to 1.3 tan(fov/2)).  The paper needs a square J for (JW)^-1 (Eq. 7) but never gives
    the third row; "z" uses (0, 0, 1), "ewa" the EWA row t/|t|.  The splatted frequency does not
    depend on this choice (it only reparametrises the integrated coordinate).
    """
    fx, fy = cam["fx"], cam["fy"]
    limx = 1.3 * (0.5 * cam["width"] / fx)
    limy = 1.3 * (0.5 * cam["height"] / fy)
    tx, ty, tz = t.unbind(-1)
    ux = torch.clamp(tx / tz, -limx, limx)
    uy = torch.clamp(ty / tz, -limy, limy)
    zero = torch.zeros_like(tz)
    r0 = torch.stack([fx / tz, zero, -fx * ux / tz], -1)
    r1 = torch.stack([zero, fy / tz, -fy * uy / tz], -1)
    if third_row == "z":
        r2 = torch.stack([zero, zero, torch.ones_like(tz)], -1)
    else:
        r2 = t / torch.linalg.norm(t, dim=-1, keepdim=True)
    return torch.stack([r0, r1, r2], -2)


def splat_frequency(f_proj: torch.Tensor, sigma_ray: torch.Tensor) -> torch.Tensor:
    """Eq. 8: f2D = f_proj_xy - (S_02, S_12) / S_22 * f_proj_z with S = inverse(ray-space covariance).

    f_proj: [n,K,3]; sigma_ray: [n,3,3] -> [n,K,2].
    """
    S = torch.linalg.inv(sigma_ray)
    ratio = S[:, 0:2, 2] / S[:, 2:3, 2]                       # [n,2]
    return f_proj[..., 0:2] - ratio[:, None, :] * f_proj[..., 2:3]


def z_attenuation(f_proj: torch.Tensor, sigma_ray: torch.Tensor) -> torch.Tensor:
    """The variant that keeps the z-integration constant C2 (supplement A.2): integrating a cosine
    component over z multiplies it, relative to the envelope, by C2 = exp(-2 pi^2 f_proj_z^2 / S_22)
    with S = inverse(ray-space covariance).  [n,K,3], [n,3,3] -> [n,K]."""
    S = torch.linalg.inv(sigma_ray)
    return torch.exp(-2.0 * math.pi ** 2 * f_proj[..., 2] ** 2 / S[:, 2:3, 2])


def project(prims: dict, cam, cfg, third_row: str = "z") -> dict:
    """Per-primitive 2D Gabor parameters in float64 (differentiable in every attribute)."""
    W, tc = camera_tensors(cam)
    means, scales, quats = prims["means"], prims["scales"], prims["quats"]
    t = means @ W.T + tc                                        # camera-space mean
    J = jacobian(t, cam, third_row)
    M = J @ W                                                   # the local affine map JW
    sigma = covariance_3d(scales, quats)
    sigma_ray = M @ sigma @ M.transpose(-1, -2)                 # Sigma' = J W Sigma W^T J^T (Eq. 2)
    eye2 = torch.eye(2, dtype=F64)
    cov2d = sigma_ray[:, 0:2, 0:2] + cfg["eps2d"] * eye2        # top-left 2x2 (+ dilation)
    conic_m = torch.linalg.inv(cov2d)
    conic = torch.stack([conic_m[:, 0, 0], conic_m[:, 0, 1], conic_m[:, 1, 1]], -1)
    mu2d = torch.stack([cam["fx"] * t[:, 0] / t[:, 2] + cam["cx"], cam["fy"] * t[:, 1] / t[:, 2] + cam["cy"]], -1)
    K = prims["weights"].shape[1]
    cos_weights = prims["weights"]
    if K > 0:
        f_proj = torch.einsum("nji,nkj->nki", torch.linalg.inv(M), prims["freqs"])   # ((JW)^-1)^T f  (Eq. 7)
        f2d = splat_frequency(f_proj, sigma_ray)
        if cfg.get("z_atten"):
            cos_weights = prims["weights"] * z_attenuation(f_proj, sigma_ray)
    else:
        f2d = torch.zeros(means.shape[0], 0, 2, dtype=F64)
    campos = -(W.T @ tc)
    v = means - campos
    dirs = v / torch.linalg.norm(v, dim=-1, keepdim=True)
    deg = int(round(math.sqrt(prims["sh"].shape[1]))) - 1
    basis = sh_basis(dirs, deg)                                 # [n, (d+1)^2]
    rgb = torch.clamp_min(torch.einsum("nc,ncj->nj", basis, prims["sh"]) + 0.5, 0.0)
    return dict(mu2d=mu2d, conic=conic, opacity=prims["opacity"], rgb=rgb, f2d=f2d,
                weights=prims["weights"], cos_weights=cos_weights, depth=t[:, 2], cov2d=cov2d)


# ----------------------------------------------------------------------------------------------
# Binning specification (float32, fixed op order; integer results must match the GPU bit for bit)
# ----------------------------------------------------------------------------------------------
LN2_UP = np.float32(0.693147182464599609375)   # the float32 just above ln 2


def _tile_reachable(prims_np, prim_of, tile_x, tile_y, mux, muy, ca, cb, cc, det, cfg):
    """Which (primitive, tile) pairs of the 3-sigma squares can give some pixel alpha >= alpha_min.

    alpha = o G(x) bank(x) <= o G(x) because the filter bank is at most 1, so a pixel needs
    q(x) = (x - mu)^T Sigma2D^-1 (x - mu) <= 2 ln(o / alpha_min).  The set {q <= thr} is an ellipse,
    and the pixel centres of a row of tiles lie in a horizontal strip, so the centres of that row
    which the ellipse can reach lie in one x-interval: between the ellipse's leftmost and rightmost
    points within the strip.  A tile is kept if its pixel-centre x-range meets that interval (in exact
    arithmetic this is the same as its box of pixel centres meeting the ellipse); dropping the other
    tiles removes only pairs that every pixel skips, so the image is unchanged.  thr bounds the
    threshold from above and the interval is widened slightly, so float32 rounding keeps the rule
    conservative.  All in float32, single correctly rounded operations in the written order:
      conic A = c / det32, B = -b / det32, C = a / det32;  x = o / alpha_min = m 2^e (frexp);
      m2 = 2 m, t = (e - 1) LN2_UP + (m2 - 1) / sqrt(m2)  (>= ln x since ln m2 <= (m2 - 1)/sqrt m2);
      thr = (2 t) (1 + 2^-10) + 2^-6;  o < alpha_min reaches nothing;
      per primitive: D = A C - B B;  ye = sqrt((thr A) / D), xe = sqrt((thr C) / D) (the half extents),
      ys = ((-B) xe) / C (the y of the rightmost point; the leftmost is at -ys),
      ye' = ye (1 + 2^-10) + 2^-8;  unless D, A, C > 0 and D, ys, ye' are finite, every tile of the
      square is kept;
      per row: yl = (16 ty + 0.5) - mu_y, yh = (16 ty + 15.5) - mu_y, lo = max(yl, -ye'),
      hi = min(yh, ye'), an empty row if lo > hi;
      x+-(y) = ((-B) y +- sqrt(max((A thr) - (D y) y, 0))) / A:  xr = x+(clip(ys, lo, hi)),
      xl = x-(clip(-ys, lo, hi)), widened to xr' = (xr + |xr| 2^-10) + 2^-8, xl' = (xl - |xl| 2^-10) - 2^-8;
      kept tiles tx in [ceil(((xl' + mu_x) - 15.5) / 16), floor(((xr' + mu_x) - 0.5) / 16)].
    """
    f32 = np.float32
    with np.errstate(all="ignore"):
        op = np.asarray(prims_np["opacity"], f32)
        amin = f32(cfg["alpha_min"])
        det32 = det.astype(f32)
        A, B, C = cc / det32, -cb / det32, ca / det32
        xq = op / amin
        mq, eq = np.frexp(xq)
        m2 = mq * f32(2)
        t = (eq - 1).astype(f32) * LN2_UP + (m2 - f32(1)) / np.sqrt(m2)
        thr = (f32(2) * t) * f32(1 + 2 ** -10) + f32(2 ** -6)
        D = A * C - B * B
        ye = np.sqrt((thr * A) / D)
        xe = np.sqrt((thr * C) / D)
        ys = ((-B) * xe) / C
        yew = ye * f32(1 + 2 ** -10) + f32(2 ** -8)
        ok = (D > f32(0)) & (A > f32(0)) & (C > f32(0)) & np.isfinite(D) & np.isfinite(ys) & np.isfinite(yew)
        A, B, C, D, thr, ys, yew, ok, mx, my = (v[prim_of] for v in (A, B, C, D, thr, ys, yew, ok, mux, muy))
        reach = (op >= amin)[prim_of]
        by = (tile_y * 16).astype(f32)
        lo = np.maximum((by + f32(0.5)) - my, -yew)
        hi = np.minimum((by + f32(15.5)) - my, yew)

        def x_at(y, sign):
            root = np.sqrt(np.maximum(A * thr - (D * y) * y, f32(0)))
            return ((-B) * y + root) / A if sign > 0 else ((-B) * y - root) / A

        xr = x_at(np.minimum(np.maximum(ys, lo), hi), +1)
        xl = x_at(np.minimum(np.maximum(-ys, lo), hi), -1)
        xr = (xr + np.abs(xr) * f32(2 ** -10)) + f32(2 ** -8)
        xl = (xl - np.abs(xl) * f32(2 ** -10)) - f32(2 ** -8)
        t_lo = np.ceil((((xl + mx) - f32(15.5)) * f32(0.0625)))
        t_hi = np.floor((((xr + mx) - f32(0.5)) * f32(0.0625)))
        row_ok = lo <= hi
        tx = tile_x.astype(f32)
        in_row = row_ok & (tx >= t_lo) & (tx <= t_hi)
    return reach & np.where(ok, in_row, True)


def bin_spec(prims_np: dict, cam, cfg, cull: bool = True) -> dict:
    """Tile binning per the written float32 specification.

    Every float32 operation below is a single IEEE round-to-nearest operation in the stated order
    (numpy never fuses multiply-add).  The determinant of the dilated 2D covariance is a float64
    function of its float32 entries; eigenvalue and radius are float32 from the rounded determinant;
    the tile rectangle is integer arithmetic.  A primitive's tiles are those of its 3-sigma square that some
    pixel can reach (see _tile_reachable; cull=False keeps the whole square, which renders the same
    image).  Returns per-primitive depth/mean/covariance/radius/rect, the emitted (key, value) pairs
    in emission order, the stably sorted pairs and tile ranges.
    """
    f32 = np.float32
    mu = np.asarray(prims_np["means"], f32)
    sc = np.asarray(prims_np["scales"], f32)
    q = np.asarray(prims_np["quats"], f32)
    n = mu.shape[0]
    Wm = np.asarray(cam["R"], f32).reshape(3, 3)
    tc = np.asarray(cam["t"], f32).reshape(3)
    fx, fy, cx, cy = f32(cam["fx"]), f32(cam["fy"]), f32(cam["cx"]), f32(cam["cy"])
    width, height = int(cam["width"]), int(cam["height"])
    znear, zfar, eps = f32(cam["znear"]), f32(cam["zfar"]), f32(cfg["eps2d"])
    tiles_x, tiles_y = (width + TILE - 1) // TILE, (height + TILE - 1) // TILE

    # camera-space mean: t_i = ((W_i0 m0 + W_i1 m1) + W_i2 m2) + tc_i
    t = [((Wm[i, 0] * mu[:, 0] + Wm[i, 1] * mu[:, 1]) + Wm[i, 2] * mu[:, 2]) + tc[i] for i in range(3)]
    tx, ty, tz = t
    mux = (fx * tx) / tz + cx
    muy = (fy * ty) / tz + cy
    # normalised quaternion and rotation
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    nrm = np.sqrt(((w * w + x * x) + y * y) + z * z)
    w, x, y, z = w / nrm, x / nrm, y / nrm, z / nrm
    one, two = f32(1.0), f32(2.0)
    R = [[one - two * (y * y + z * z), two * (x * y - w * z), two * (x * z + w * y)],
         [two * (x * y + w * z), one - two * (x * x + z * z), two * (y * z - w * x)],
         [two * (x * z - w * y), two * (y * z + w * x), one - two * (x * x + y * y)]]
    M = [[R[i][j] * sc[:, j] for j in range(3)] for i in range(3)]
    Sig = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(i, 3):
            Sig[i][j] = (M[i][0] * M[j][0] + M[i][1] * M[j][1]) + M[i][2] * M[j][2]
            Sig[j][i] = Sig[i][j]
    # J rows 0-1 (field-of-view guarded) and T = J[0:2] W
    limx = f32(1.3) * ((f32(0.5) * f32(width)) / fx)
    limy = f32(1.3) * ((f32(0.5) * f32(height)) / fy)
    ux = np.minimum(np.maximum(tx / tz, -limx), limx)
    uy = np.minimum(np.maximum(ty / tz, -limy), limy)
    J00, J02 = fx / tz, -((fx * ux) / tz)
    J11, J12 = fy / tz, -((fy * uy) / tz)
    T = [[J00 * Wm[0, j] + J02 * Wm[2, j] for j in range(3)],
         [J11 * Wm[1, j] + J12 * Wm[2, j] for j in range(3)]]
    U = [[(T[a][0] * Sig[0][j] + T[a][1] * Sig[1][j]) + T[a][2] * Sig[2][j] for j in range(3)] for a in range(2)]
    A00 = (U[0][0] * T[0][0] + U[0][1] * T[0][1]) + U[0][2] * T[0][2]
    A01 = (U[0][0] * T[1][0] + U[0][1] * T[1][1]) + U[0][2] * T[1][2]
    A11 = (U[1][0] * T[1][0] + U[1][1] * T[1][1]) + U[1][2] * T[1][2]
    ca, cb, cc = A00 + eps, A01, A11 + eps
    # float64 determinant of the dilated 2D covariance (where near-degenerate footprints cancel)
    da, db, dc = ca.astype(np.float64), cb.astype(np.float64), cc.astype(np.float64)
    det = da * dc - db * db
    # largest eigenvalue and 3-sigma radius in float32 from the rounded determinant
    with np.errstate(invalid="ignore", over="ignore"):
        det32 = det.astype(f32)
        mid = f32(0.5) * (ca + cc)
        lam = mid + np.sqrt(np.maximum(mid * mid - det32, f32(0)))
        rad = np.ceil(f32(3) * np.sqrt(np.maximum(lam, f32(0))))
    lim = f32(2.0 ** 30)
    finite = (np.isfinite(mux) & np.isfinite(muy) & np.isfinite(det) & np.isfinite(rad) &
              (np.abs(mux) < lim) & (np.abs(muy) < lim) & (rad < lim))
    valid = (tz > znear) & (tz <= zfar) & (det > 0.0) & finite
    # rectangle: floor((mu -+ r) / 16) = floor_div(floor(mu) -+ r, 16) exactly, r being an integer
    ix = np.where(finite, np.floor(mux), 0).astype(np.int64)
    iy = np.where(finite, np.floor(muy), 0).astype(np.int64)
    ir = np.where(finite, rad, 0).astype(np.int64)
    x0, x1 = (ix - ir) // TILE, (ix + ir) // TILE
    y0, y1 = (iy - ir) // TILE, (iy + ir) // TILE
    valid &= (x1 >= 0) & (x0 <= tiles_x - 1) & (y1 >= 0) & (y0 <= tiles_y - 1)
    x0 = np.where(valid, np.clip(x0, 0, tiles_x - 1), 0).astype(np.int64)
    x1 = np.where(valid, np.clip(x1, 0, tiles_x - 1), -1).astype(np.int64)
    y0 = np.where(valid, np.clip(y0, 0, tiles_y - 1), 0).astype(np.int64)
    y1 = np.where(valid, np.clip(y1, 0, tiles_y - 1), -1).astype(np.int64)
    # tiles of the 3-sigma square, in emission order: primitive ascending, then row-major
    sq_count = np.where(valid, (x1 - x0 + 1) * (y1 - y0 + 1), 0).astype(np.int64)
    sq_off = np.concatenate([[0], np.cumsum(sq_count)[:-1]]) if n else np.zeros(0, np.int64)
    prim_of = np.repeat(np.arange(n), sq_count)
    local = np.arange(int(sq_count.sum())) - np.repeat(sq_off, sq_count)
    wx = (x1 - x0 + 1)[prim_of]
    tile_y = y0[prim_of] + local // wx
    tile_x = x0[prim_of] + local % wx
    if cull:
        keep = _tile_reachable(prims_np, prim_of, tile_x, tile_y, mux, muy, ca, cb, cc, det, cfg)
        prim_of, tile_x, tile_y = prim_of[keep], tile_x[keep], tile_y[keep]
    touched = np.bincount(prim_of, minlength=n).astype(np.int64)
    offsets = np.concatenate([[0], np.cumsum(touched)[:-1]]) if n else np.zeros(0, np.int64)
    P = int(touched.sum())
    depth_bits = tz.astype(f32).view(np.uint32).astype(np.uint64)
    tid = (tile_y * tiles_x + tile_x).astype(np.uint64)
    keys = (tid << np.uint64(32)) | depth_bits[prim_of]
    vals = prim_of.astype(np.uint32)
    order = np.argsort(keys, kind="stable")
    skeys, svals = keys[order], vals[order]
    ntiles = tiles_x * tiles_y
    tile_of = (skeys >> np.uint64(32)).astype(np.int64)
    starts = np.searchsorted(tile_of, np.arange(ntiles), side="left")
    ends = np.searchsorted(tile_of, np.arange(ntiles), side="right")
    ranges = np.stack([starts, ends], -1).astype(np.uint32)
    return dict(depth=tz, mu2d=np.stack([mux, muy], -1), cov2d=np.stack([ca, cb, cc], -1), radius=rad,
                valid=valid, rect=np.stack([x0, x1, y0, y1], -1), touched=touched, offsets=offsets, P=P,
                square_count=sq_count,
                keys=keys, vals=vals, sorted_keys=skeys, sorted_vals=svals, ranges=ranges,
                tiles_x=tiles_x, tiles_y=tiles_y)


def _box_min_q(a, b, c, x0, x1, y0, y1):
    """Smallest q(x, y) = a x^2 + 2 b x y + c y^2 over the box [x0, x1] x [y0, y1] (positive definite
    q, coordinates relative to the mean): 0 if the box holds the mean, else the least of the four
    edge minima, each the 1D quadratic's vertex clipped to its edge."""
    inside = (x0 <= 0) & (0 <= x1) & (y0 <= 0) & (0 <= y1)
    best = np.full(np.shape(a), np.inf)
    for x in (x0, x1):
        y = np.clip(-b * x / c, y0, y1)
        best = np.minimum(best, a * x * x + 2 * b * x * y + c * y * y)
    for y in (y0, y1):
        x = np.clip(-b * y / a, x0, x1)
        best = np.minimum(best, a * x * x + 2 * b * x * y + c * y * y)
    return np.where(inside, 0.0, best)


def bin_fp64(prims_np: dict, cam, cfg) -> dict:
    """The binning in float64 throughout, with no float32 step: depth, projected mean and dilated 2D
    covariance from project() (Sec. 3.1), the largest eigenvalue and the 3-sigma radius
    ceil(3 sqrt(lambda_max)), the tile rectangle floor((mu -+ r) / 16), and the reach rule of
    _tile_reachable in exact form: a tile is kept when the ellipse q <= 2 ln(o / alpha_min) meets
    the box of its pixel centres.  It is the reference that the float32 binning specification of
    bin_spec() is measured against (binning_differences); its pair set defines no image."""
    with torch.no_grad():
        proj = project(_to_f64(prims_np), cam, cfg)
    mu = proj["mu2d"].numpy()
    cov = proj["cov2d"].numpy()
    ca, cb, cc = cov[:, 0, 0], cov[:, 0, 1], cov[:, 1, 1]
    depth = proj["depth"].numpy()
    op = np.asarray(prims_np["opacity"], np.float64)
    n = mu.shape[0]
    tiles_x = (int(cam["width"]) + TILE - 1) // TILE
    tiles_y = (int(cam["height"]) + TILE - 1) // TILE
    with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
        det = ca * cc - cb * cb
        mid = 0.5 * (ca + cc)
        lam = mid + np.sqrt(np.maximum(mid * mid - det, 0.0))
        rad = np.ceil(3.0 * np.sqrt(np.maximum(lam, 0.0)))
        finite = np.isfinite(mu).all(1) & np.isfinite(det) & np.isfinite(rad)
        valid = (depth > cam["znear"]) & (depth <= cam["zfar"]) & (det > 0) & finite
        x0 = np.floor((mu[:, 0] - rad) / TILE)
        x1 = np.floor((mu[:, 0] + rad) / TILE)
        y0 = np.floor((mu[:, 1] - rad) / TILE)
        y1 = np.floor((mu[:, 1] + rad) / TILE)
    valid &= (x1 >= 0) & (x0 <= tiles_x - 1) & (y1 >= 0) & (y0 <= tiles_y - 1)
    x0 = np.where(valid, np.clip(x0, 0, tiles_x - 1), 0).astype(np.int64)
    x1 = np.where(valid, np.clip(x1, 0, tiles_x - 1), -1).astype(np.int64)
    y0 = np.where(valid, np.clip(y0, 0, tiles_y - 1), 0).astype(np.int64)
    y1 = np.where(valid, np.clip(y1, 0, tiles_y - 1), -1).astype(np.int64)
    cnt = np.where(valid, (x1 - x0 + 1) * (y1 - y0 + 1), 0)
    prim_of = np.repeat(np.arange(n), cnt)
    local = np.arange(int(cnt.sum())) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    wx = (x1 - x0 + 1)[prim_of]
    ty = y0[prim_of] + local // wx
    tx = x0[prim_of] + local % wx
    with np.errstate(invalid="ignore", divide="ignore"):
        ia, ib, ic = cc / det, -cb / det, ca / det                  # the conic Sigma2D^-1
        thr = 2.0 * np.log(np.maximum(op, 1e-300) / cfg["alpha_min"])
        m = prim_of
        qmin = _box_min_q(ia[m], ib[m], ic[m], 16.0 * tx + 0.5 - mu[m, 0], 16.0 * tx + 15.5 - mu[m, 0],
                          16.0 * ty + 0.5 - mu[m, 1], 16.0 * ty + 15.5 - mu[m, 1])
    keep = (op[m] >= cfg["alpha_min"]) & (qmin <= thr[m])
    return dict(valid=valid, radius=rad, rect=np.stack([x0, x1, y0, y1], -1), prim_of=prim_of[keep],
                tile=(ty * tiles_x + tx)[keep], qmin=qmin[keep], thr=thr, tiles_x=tiles_x)


def binning_differences(prims_np: dict, cam, cfg, spec=None) -> dict:
    """How the float32 binning specification (bin_spec) differs from the pure float64 binning
    (bin_fp64): primitives whose validity or rectangle differs, and (primitive, tile) pairs listed
    by only one of them.  spec_only pairs are reported with the float64 margin of their tile
    (min q over the tile minus the threshold; > 0 means no pixel of the tile reaches alpha_min, so
    the pair leaves the image unchanged); fp64_only pairs are ones the float32 rule drops."""
    spec = bin_spec(prims_np, cam, cfg) if spec is None else spec
    ref = bin_fp64(prims_np, cam, cfg)
    tiles_x = spec["tiles_x"]
    rect_s = np.where(spec["valid"][:, None], spec["rect"], -1)
    rect_d = np.where(ref["valid"][:, None], ref["rect"], -1)
    rect_diff = int(np.any(rect_s != rect_d, axis=1).sum())
    key_s = spec["vals"].astype(np.int64) * (tiles_x * spec["tiles_y"]) + (spec["keys"] >> np.uint64(32)).astype(np.int64)
    key_d = ref["prim_of"].astype(np.int64) * (tiles_x * spec["tiles_y"]) + ref["tile"]
    only_s = np.setdiff1d(key_s, key_d)
    only_d = np.setdiff1d(key_d, key_s)
    # float64 margin of the spec-only pairs: min q over their tile minus the reach threshold
    ntile = tiles_x * spec["tiles_y"]
    ps, ts = only_s // ntile, only_s % ntile
    with torch.no_grad():
        proj = project(_to_f64({k: np.asarray(prims_np[k])[ps] for k in
                                ("means", "scales", "quats", "opacity", "sh", "freqs", "weights")}), cam, cfg)
    mu, cov = proj["mu2d"].numpy(), proj["cov2d"].numpy()
    det = cov[:, 0, 0] * cov[:, 1, 1] - cov[:, 0, 1] ** 2
    tx, ty = ts % tiles_x, ts // tiles_x
    with np.errstate(invalid="ignore", divide="ignore"):
        qmin = _box_min_q(cov[:, 1, 1] / det, -cov[:, 0, 1] / det, cov[:, 0, 0] / det,
                          16.0 * tx + 0.5 - mu[:, 0], 16.0 * tx + 15.5 - mu[:, 0],
                          16.0 * ty + 0.5 - mu[:, 1], 16.0 * ty + 15.5 - mu[:, 1])
    margin = qmin - ref["thr"][ps]
    r = rect_d[ps]
    in_rect = (tx >= r[:, 0]) & (tx <= r[:, 1]) & (ty >= r[:, 2]) & (ty <= r[:, 3])
    return dict(P_spec=int(key_s.size), P_fp64=int(key_d.size), rect_diff=rect_diff,
                spec_only=int(only_s.size), fp64_only=int(only_d.size),
                spec_only_unreachable=int((in_rect & (margin > 0)).sum()),
                spec_only_outside_fp64_rect=int((~in_rect).sum()),
                spec_only_margin=margin, spec_only_in_fp64_rect=in_rect, fp64_only_pairs=only_d)


# ----------------------------------------------------------------------------------------------
# Compositing (Eq. 10 with the 2D Gabor primitive of Eq. 9)
# ----------------------------------------------------------------------------------------------
# Threshold decisions that float32 may take differently (survey reading c16).  The GPU evaluates
# alpha in float32 from the float32 projection that the binning specification rounds (projected
# mean and 2D covariance), so its alpha differs from this float64 alpha by (1) the effect of that
# rounding, which is computed here exactly by evaluating alpha a second time from the rounded
# projection, and (2) the rounding of the evaluation itself, bounded below from the size of the
# terms.  A decision is ambiguous when alpha_min (or alpha_max, or T_min) lies between the float64
# value and the float32 window; such a pixel is flagged, and its result "the other way" is
# computed by flipping that decision (flip_allowance).
U32 = 2.0 ** -24          # float32 unit roundoff
COS_ERR = 2e-6            # absolute error of the single-precision cosine at |angle| <= 4 pi
PHASE_BLOCK = 8           # pixels per side of the blocks that share a range-reduction decision
FAST_PHASE_CYCLES = 2.0   # a block whose |f2D . (x - mu)| stays within this takes no range reduction
F2D_ROUNDINGS = 8         # roundings charged to each float32 entry behind f2D (see f2d_rounding_bound)
EVAL_SAFETY = 2.0         # factor over the first-order bounds below


def f2d_rounding_bound(prims_np: dict, cam, cfg, ids=None):
    """First-order bound on how far a float32 evaluation of Eq. 7-8 can move f2D (and, in the
    z-attenuation variant, the cosine weights w C2): [m,K,2] and [m,K] for primitives ids.

    Forming the ray-space covariance Sigma'' = M R S^2 R^T M^T (M = JW) and f_proj = M^-T f in
    float32 perturbs each entry by a few roundings of its terms' magnitudes, |M||R| S^2 |R|^T |M|^T
    and |M^-T||f|.  The bound is F2D_ROUNDINGS u times the sum, over those entries, of |d f2D /
    d entry| times that magnitude (torch.autograd through splat_frequency).  For elongated
    primitives, whose Sigma'' is ill-conditioned, it is far larger than u |f2D|.  Eight roundings
    per entry: an entry of a product of three 3x3 factors is a sum of nine products, each formed
    from three roundings, added in a chain."""
    p = _to_f64({k: np.asarray(prims_np[k])[ids] if ids is not None else prims_np[k]
                 for k in ("means", "scales", "quats", "opacity", "sh", "freqs", "weights")})
    K = p["weights"].shape[1]
    m = p["means"].shape[0]
    if K == 0 or m == 0:
        return torch.zeros(m, K, 2, dtype=F64), torch.zeros(m, K, dtype=F64)
    W, tc = camera_tensors(cam)
    t = p["means"] @ W.T + tc
    M = jacobian(t, cam) @ W
    R = rotation_from_quaternion(p["quats"])
    S2 = p["scales"] ** 2
    MR, MRa = M @ R, M.abs() @ R.abs()
    sig = ((MR * S2[:, None, :]) @ MR.transpose(-1, -2)).requires_grad_(True)
    sig_mag = (MRa * S2[:, None, :]) @ MRa.transpose(-1, -2)
    MinvT = torch.linalg.inv(M).transpose(-1, -2)
    fp = torch.einsum("nij,nkj->nki", MinvT, p["freqs"]).requires_grad_(True)
    fp_mag = torch.einsum("nij,nkj->nki", MinvT.abs(), p["freqs"].abs())
    f2d = splat_frequency(fp, sig)
    cw = p["weights"] * z_attenuation(fp, sig) if cfg.get("z_atten") else None
    bf = torch.zeros(m, K, 2, dtype=F64)
    bw = torch.zeros(m, K, dtype=F64)
    for k in range(K):
        outs = [(f2d[:, k, 0], bf[:, k, 0]), (f2d[:, k, 1], bf[:, k, 1])] + ([(cw[:, k], bw[:, k])] if cw is not None else [])
        for y, dst in outs:
            gs, gf = torch.autograd.grad(y.sum(), [sig, fp], retain_graph=True)
            dst.copy_((gs.abs() * sig_mag).sum((1, 2)) + (gf.abs() * fp_mag).sum((1, 2)))
    return F2D_ROUNDINGS * U32 * bf, F2D_ROUNDINGS * U32 * bw


def gabor_alpha(px, py, rec, cfg):
    """alpha_raw = o * G2D(x) * [(1 - sum w) + sum w' cos(2 pi f2D . (x - mu2D))] for pixels x pairs,
    w' = w (the method) or w C2 (the z-attenuation variant)."""
    dx = px[:, None] - rec["mu2d"][None, :, 0]
    dy = py[:, None] - rec["mu2d"][None, :, 1]
    a, b, c = rec["conic"][:, 0], rec["conic"][:, 1], rec["conic"][:, 2]
    G = torch.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
    w = rec["weights"]
    if w.shape[1] > 0:
        phase = 2.0 * math.pi * (dx[..., None] * rec["f2d"][None, :, :, 0] + dy[..., None] * rec["f2d"][None, :, :, 1])
        bank = (1.0 - w.sum(-1))[None, :] + (rec["cos_weights"][None] * torch.cos(phase)).sum(-1)
    else:
        bank = torch.ones_like(G)
    return rec["opacity"][None, :] * G * bank


def phase_rounding_bound(px, py, mu2d, f2d):
    """[P, L, K] bound on the float32 rounding error (radians) of the Gabor phase 2 pi f2D . (x - mu)
    at pixels (px, py) for pairs with projected means mu2d [L, 2] and frequencies f2d [L, K, 2].

    The float32 evaluation takes d = x - mu (one rounding per axis), F = 2 pi f2D (one rounding of a
    product with a float32 2 pi) and F_x d_x + F_y d_y by a product and a fused sum.  With
    |phase| = 2 pi (|f2D_x d_x| + |f2D_y d_y|) that is at most u |phase| for d, 1.5 u |phase| for F,
    u |phase| for the product and u |phase| for the sum: 5 u |phase| charged.  A pixel of a block
    (PHASE_BLOCK x PHASE_BLOCK pixels, aligned to the tiles) where some component's |f2D . (x - mu)|
    can exceed FAST_PHASE_CYCLES reduces the phase by whole cycles before the cosine: the product
    with a float32 1 / (2 pi) and the final scaling by 2 pi charge another 2 u |phase| + 2 pi u.  It
    is charged wherever the float64 test is within 1e-4 cycles of the threshold or above."""
    fx, fy = f2d[None, :, :, 0].abs(), f2d[None, :, :, 1].abs()
    dx, dy = (px[:, None] - mu2d[None, :, 0]).abs(), (py[:, None] - mu2d[None, :, 1]).abs()   # [P, L]
    ph = 2.0 * math.pi * (dx[..., None] * fx + dy[..., None] * fy)
    x0 = PHASE_BLOCK * torch.floor(px / PHASE_BLOCK) + 0.5      # the block's first and last pixel centres
    y0 = PHASE_BLOCK * torch.floor(py / PHASE_BLOCK) + 0.5
    x1, y1 = x0 + (PHASE_BLOCK - 1), y0 + (PHASE_BLOCK - 1)
    ax = torch.maximum((x0[:, None] - mu2d[None, :, 0]).abs(), (x1[:, None] - mu2d[None, :, 0]).abs())
    ay = torch.maximum((y0[:, None] - mu2d[None, :, 1]).abs(), (y1[:, None] - mu2d[None, :, 1]).abs())
    reach = (ax[..., None] * fx + ay[..., None] * fy).amax(-1, keepdim=True)   # cycles, [P, L, 1]
    slow = reach > FAST_PHASE_CYCLES - 1e-4
    return 5 * U32 * ph + torch.where(slow, 2 * U32 * ph + 2 * math.pi * U32, torch.zeros_like(ph))


def alpha_window(px, py, rec, cfg, alpha_raw, rounded=None):
    """[lo, hi] holding both this float64 alpha_raw and every float32 evaluation of it.

    rounded: the float32 projected means and conics that the binning specification produces for the
    same pairs (float64 tensors).  The float32 evaluation then lies within e of the alpha of that
    rounded projection, with e the first-order rounding bound of: the envelope exponent
    (8 u per term of 1/2 d^T Q d, and 2^-19 for the exponential); each bank component
    (COS_ERR + the phase error of a float32 f2D, 2 pi (|df2D_x| |dx| + |df2D_y| |dy|) with df2D from
    f2d_rounding_bound, + the roundings of the phase itself; the cosine weight's own error in the
    z-attenuation variant); and the products (4 u).  The phase's own roundings are
    phase_rounding_bound's."""
    with torch.no_grad():
        src = rec if rounded is None else dict(rec, mu2d=rounded["mu2d"], conic=rounded["conic"])
        alt = alpha_raw if rounded is None else gabor_alpha(px, py, src, cfg)
        dx = px[:, None] - src["mu2d"][None, :, 0]
        dy = py[:, None] - src["mu2d"][None, :, 1]
        a, b, c = src["conic"][:, 0], src["conic"][:, 1], src["conic"][:, 2]
        terms = 0.5 * (a.abs() * dx * dx + c.abs() * dy * dy) + (b * dx * dy).abs()
        G = torch.exp(-(0.5 * (a * dx * dx + c * dy * dy) + b * dx * dy))
        e = alt.abs() * (8 * U32 * terms + 2.0 ** -19 + 4 * U32)
        w = rec["cos_weights"]
        if w.shape[1] > 0:
            f = rec["f2d"]
            err = COS_ERR + phase_rounding_bound(px, py, src["mu2d"], f)
            if rounded is not None and "f2d_err" in rounded:
                fe = rounded["f2d_err"]
                err = err + 2.0 * math.pi * (dx.abs()[..., None] * fe[None, :, :, 0] + dy.abs()[..., None] * fe[None, :, :, 1])
            e_bank = (w.abs()[None] * err).sum(-1) + 4 * U32 * (1 + w.abs().sum(-1))[None]
            if rounded is not None and "cw_err" in rounded:
                e_bank = e_bank + rounded["cw_err"].sum(-1)[None]
            e = e + rec["opacity"][None, :] * G * e_bank
        e = EVAL_SAFETY * e
        lo = torch.minimum(alpha_raw, alt - e)
        hi = torch.maximum(alpha_raw, alt + e)
    return lo, hi


def composite(px, py, rec, cfg, rounded=None):
    """Front-to-back compositing of L depth-ordered pairs at P pixels (Eq. 10).

    Returns colour [P,3], final transmittance [P], the 1-based list position of the last
    composited pair [P] (0 if none), ambiguity flags for forward / backward comparisons, the
    number of composited pairs [P], and the allowance [P,3] of each flagged pixel: the sum over
    its ambiguous decisions of |result with that decision flipped - result|, background included.
    """
    L = rec["mu2d"].shape[0]
    alpha_raw = gabor_alpha(px, py, rec, cfg)
    alpha = torch.clamp_max(alpha_raw, cfg["alpha_max"])
    amin, amax, Tmin = cfg["alpha_min"], cfg["alpha_max"], cfg["T_min"]
    with torch.no_grad():
        keep = alpha >= amin
    a_eff = torch.where(keep, alpha, torch.zeros_like(alpha))
    T_after = torch.cumprod(1.0 - a_eff, dim=1)
    idx = torch.arange(L)
    with torch.no_grad():
        stop = keep & (T_after < Tmin)
        s = torch.where(stop.any(1), stop.int().argmax(1), torch.full((px.shape[0],), L, dtype=torch.long))
        include = keep & (idx[None, :] < s[:, None])
        evaluated = idx[None, :] <= s[:, None]
        last = torch.where(include, idx[None, :] + 1, torch.zeros_like(idx)[None, :]).amax(1)
        ar = alpha_raw.detach()
        lo, hi = alpha_window(px, py, {k: v.detach() for k, v in rec.items()}, cfg, ar, rounded)
        near_min = (torch.clamp_max(lo, amax) < amin) & (amin <= torch.clamp_max(hi, amax))
        near_max = (lo < amax) & (amax <= hi)
        # relative error of the float32 transmittance after each pair: the alpha windows of the
        # composited pairs so far (relative to 1 - alpha) plus two roundings per pair
        rel = torch.where(keep, (hi - lo) / (1.0 - a_eff.detach()) + 2 * U32, torch.zeros_like(ar))
        near_T = keep & ((T_after.detach() - Tmin).abs() <= 1.5 * T_after.detach() * torch.cumsum(rel, 1))
        flip_min = near_min & evaluated
        flip_T = near_T & evaluated
        amb_f = (flip_min | flip_T).any(1)
        amb_b = amb_f | (near_max & evaluated).any(1)
        allow = torch.zeros(px.shape[0], 3, dtype=F64)
        for p in torch.nonzero(amb_f)[:, 0].tolist():
            allow[p] = flip_allowance(ar[p], rec["rgb"].detach(), cfg,
                                      torch.nonzero(flip_min[p])[:, 0].tolist(), torch.nonzero(flip_T[p])[:, 0].tolist())
    ones = torch.ones(px.shape[0], 1, dtype=F64)
    T_before = torch.cat([ones, T_after[:, :-1]], 1)
    weight = torch.where(include, a_eff * T_before, torch.zeros_like(a_eff))
    C = weight @ rec["rgb"]
    T_ext = torch.cat([T_before, T_after[:, -1:]], 1) if L > 0 else ones
    T_final = torch.gather(T_ext, 1, s[:, None])[:, 0]
    return C, T_final, last, amb_f, amb_b, include.sum(1), allow


def composite_pixel(alpha_raw, rgb, cfg, flip_keep=(), flip_stop=()):
    """One pixel composited pair by pair (Eq. 10), with the alpha_min decision of the pairs in
    flip_keep and the T_min decision of those in flip_stop inverted.  Returns C + T bg [3]."""
    T, C = 1.0, torch.zeros(3, dtype=F64)
    for j in range(alpha_raw.shape[0]):
        a = min(float(alpha_raw[j]), cfg["alpha_max"])
        if (a >= cfg["alpha_min"]) == (j in flip_keep):
            continue
        test = T * (1.0 - a)
        if (test < cfg["T_min"]) != (j in flip_stop):
            break
        C = C + rgb[j] * (a * T)
        T = test
    return C + T * torch.tensor(cfg["bg"], dtype=F64)


def flip_allowance(alpha_raw, rgb, cfg, flips_min, flips_T):
    """Sum over the ambiguous decisions of a pixel of |result with that decision flipped - result|."""
    base = composite_pixel(alpha_raw, rgb, cfg)
    out = torch.zeros(3, dtype=F64)
    for j in flips_min:
        out += (composite_pixel(alpha_raw, rgb, cfg, flip_keep=(j,)) - base).abs()
    for j in flips_T:
        out += (composite_pixel(alpha_raw, rgb, cfg, flip_stop=(j,)) - base).abs()
    return out


def _tile_pixels(tx, ty, width, height):
    xs = torch.arange(tx * TILE, min((tx + 1) * TILE, width), dtype=F64)
    ys = torch.arange(ty * TILE, min((ty + 1) * TILE, height), dtype=F64)
    gy, gx = torch.meshgrid(ys, xs, indexing="ij")
    return gx.reshape(-1) + 0.5, gy.reshape(-1) + 0.5, gx.reshape(-1).long(), gy.reshape(-1).long()


REC_KEYS = ("mu2d", "conic", "opacity", "rgb", "f2d", "weights", "cos_weights")


def _to_f64(prims, requires_grad=False):
    out = {}
    for k in ("means", "scales", "quats", "opacity", "sh", "freqs", "weights"):
        out[k] = torch.tensor(np.asarray(prims[k], np.float64), dtype=F64, requires_grad=requires_grad)
    return out


def _render_tiles(proj, spec, cam, cfg, dL_dC=None, tiles=None, max_elems=1 << 22, prims=None):
    """Composite every tile (or the listed tile ids); optionally back-propagate dL/dC per tile.
    prims (the numpy inputs) lets the ambiguity windows include the float32 f2D bound."""
    width, height = cam["width"], cam["height"]
    tiles_x = spec["tiles_x"]
    bg = torch.tensor(cfg["bg"], dtype=F64)
    img = torch.zeros(3, height, width, dtype=F64)
    Tf = torch.ones(height, width, dtype=F64)
    last = torch.zeros(height, width, dtype=torch.long)
    comp = torch.zeros(height, width, dtype=torch.long)
    amb_f = torch.zeros(height, width, dtype=torch.bool)
    amb_b = torch.zeros(height, width, dtype=torch.bool)
    allow = torch.zeros(3, height, width, dtype=F64)
    K = proj["weights"].shape[1]
    # the float32 projection of the binning specification (what a float32 evaluation consumes)
    cov32 = spec["cov2d"].astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        det32 = cov32[:, 0] * cov32[:, 2] - cov32[:, 1] * cov32[:, 1]
        conic32 = np.stack([cov32[:, 2] / det32, -cov32[:, 1] / det32, cov32[:, 0] / det32], -1)
    rounded_all = dict(mu2d=torch.from_numpy(spec["mu2d"].astype(np.float64)), conic=torch.from_numpy(conic32))
    if prims is not None and K > 0:
        # f2D bound for the primitives of the rendered tiles only
        tl = range(spec["tiles_x"] * spec["tiles_y"]) if tiles is None else tiles
        sel = [spec["sorted_vals"][int(spec["ranges"][t, 0]):int(spec["ranges"][t, 1])] for t in tl]
        used = np.unique(np.concatenate(sel)).astype(np.int64) if sel else np.zeros(0, np.int64)
        fe, we = f2d_rounding_bound(prims, cam, cfg, used)
        n_all = proj["mu2d"].shape[0]
        rounded_all["f2d_err"] = torch.zeros(n_all, K, 2, dtype=F64).index_copy_(0, torch.from_numpy(used), fe)
        rounded_all["cw_err"] = torch.zeros(n_all, K, dtype=F64).index_copy_(0, torch.from_numpy(used), we)
    tile_list = range(spec["tiles_x"] * spec["tiles_y"]) if tiles is None else tiles
    for tid in tile_list:
        s0, s1 = int(spec["ranges"][tid, 0]), int(spec["ranges"][tid, 1])
        gxp, gyp, gxi, gyi = _tile_pixels(tid % tiles_x, tid // tiles_x, width, height)
        if s1 == s0:
            img[:, gyi, gxi] = bg[:, None]
            continue
        ids = torch.from_numpy(spec["sorted_vals"][s0:s1].astype(np.int64))
        L = s1 - s0
        chunk = max(1, max_elems // (L * max(K, 1)))
        for c0 in range(0, gxp.shape[0], chunk):
            sl = slice(c0, c0 + chunk)
            rec = {k: proj[k].index_select(0, ids) for k in REC_KEYS}   # fresh graph per pixel chunk
            rounded = {k: v.index_select(0, ids) for k, v in rounded_all.items()}
            C, T, lst, af, ab, nc, al = composite(gxp[sl], gyp[sl], rec, cfg, rounded)
            out = C + T[:, None] * bg[None, :]
            if dL_dC is not None:
                g = dL_dC[:, gyi[sl], gxi[sl]].T
                (out * g).sum().backward()
            img[:, gyi[sl], gxi[sl]] = out.detach().T
            Tf[gyi[sl], gxi[sl]] = T.detach()
            last[gyi[sl], gxi[sl]] = lst
            comp[gyi[sl], gxi[sl]] = nc
            amb_f[gyi[sl], gxi[sl]] = af
            amb_b[gyi[sl], gxi[sl]] = ab
            allow[:, gyi[sl], gxi[sl]] = al.T
    return dict(image=img, T=Tf, n_contrib=last, n_comp=comp, ambiguous=amb_f, ambiguous_bwd=amb_b,
                allowance=allow)


def render(prims: dict, cam, cfg, tiles=None, third_row="z", cull=True, spec=None) -> dict:
    """Forward render in float64.  prims: numpy arrays (means, scales, quats, opacity, sh, freqs, weights).
    spec: bin_spec(prims, cam, cfg, cull) when the caller already has it."""
    spec = bin_spec(prims, cam, cfg, cull=cull) if spec is None else spec
    with torch.no_grad():
        proj = project(_to_f64(prims), cam, cfg, third_row)
    out = _render_tiles(proj, spec, cam, cfg, tiles=tiles, prims=prims)
    out["spec"] = spec
    out["proj"] = {k: v.detach() for k, v in proj.items()}
    return out


def frequency_features(proj: dict) -> torch.Tensor:
    """Per primitive [n, 3]: sum_i w_i |f2D_i|, sum_i w_i |f2D_i,x|, sum_i w_i |f2D_i,y| -- the
    weighted Gabor frequencies (cycles per pixel) that the frequency maps blend (Sec. 4)."""
    f, w = proj["f2d"], proj["cos_weights"]
    if w.shape[1] == 0:
        return torch.zeros(w.shape[0], 3, dtype=F64)
    mag = torch.sqrt((f * f).sum(-1))
    return torch.stack([(w * mag).sum(-1), (w * f[..., 0].abs()).sum(-1), (w * f[..., 1].abs()).sum(-1)], -1)


def render_frequency_map(prims: dict, cam, cfg) -> dict:
    """Frequency maps: the compositing of render() (same pairs, same weights alpha T) with each
    primitive's colour replaced by its frequency features and no background."""
    spec = bin_spec(prims, cam, cfg)
    with torch.no_grad():
        proj = project(_to_f64(prims), cam, cfg)
    proj = dict(proj, rgb=frequency_features(proj))
    out = _render_tiles(proj, spec, cam, dict(cfg, bg=(0.0, 0.0, 0.0)), prims=prims)
    out["map"] = out.pop("image")
    out["spec"] = spec
    return out


def render_backward(prims: dict, cam, cfg, dL_dC) -> dict:
    """Gradients of sum(dL_dC * image) w.r.t. every primitive attribute (float64, exact adjoint).

    Also returns the per-primitive 2D gradients (w.r.t. mu2d, conic (a, b, c), opacity, rgb, f2d,
    weights as used by the compositing step) under the key "grad2d".
    """
    spec = bin_spec(prims, cam, cfg)
    leaves = _to_f64(prims, requires_grad=True)
    proj = project(leaves, cam, cfg)
    rec = {k: proj[k].detach().clone().requires_grad_(True) for k in REC_KEYS}
    g = torch.as_tensor(np.asarray(dL_dC, np.float64), dtype=F64)
    out = _render_tiles(rec, spec, cam, cfg, dL_dC=g, prims=prims)
    g2d = {k: (rec[k].grad if rec[k].grad is not None else torch.zeros_like(rec[k])) for k in REC_KEYS}
    outs = [proj[k] for k in REC_KEYS if proj[k].requires_grad]
    gouts = [g2d[k] for k in REC_KEYS if proj[k].requires_grad]
    torch.autograd.backward(outs, gouts)
    grads = {k: (v.grad if v.grad is not None else torch.zeros_like(v)).numpy() for k, v in leaves.items()}
    grads["grad2d"] = {k: v.numpy() for k, v in g2d.items()}
    grads["image"] = out["image"].numpy()
    grads["ambiguous_bwd"] = out["ambiguous_bwd"].numpy()
    return grads


# ----------------------------------------------------------------------------------------------
# Photometric loss (Sec. 3.4.1, the L1 part; L2 for the gradient-check configuration)
# ----------------------------------------------------------------------------------------------
def loss_and_grad(image, target, kind="l1"):
    """Mean L1 or mean squared error over all pixels and channels, and dL/dimage."""
    image = np.asarray(image, np.float64)
    target = np.asarray(target, np.float64)
    diff = image - target
    N = diff.size
    if kind == "l1":
        return float(np.abs(diff).sum() / N), np.sign(diff) / N
    return float((diff * diff).sum() / N), 2.0 * diff / N


# ----------------------------------------------------------------------------------------------
# Training loss with the structural term (Sec. 3.4.1, Eq. 11): L = (1 - lambda) L1 + lambda D-SSIM
# ----------------------------------------------------------------------------------------------
SSIM_WINDOW = 11       # Gaussian window of the SSIM index (Wang et al. 2004, the paper's metric)
SSIM_SIGMA = 1.5
SSIM_C1 = 0.01 ** 2    # (K1 L)^2 with K1 = 0.01, dynamic range L = 1
SSIM_C2 = 0.03 ** 2    # (K2 L)^2 with K2 = 0.03


def ssim_window() -> torch.Tensor:
    """The 11 x 11 circular Gaussian window (sigma 1.5) normalised to unit sum."""
    i = torch.arange(SSIM_WINDOW, dtype=F64) - SSIM_WINDOW // 2
    g = torch.exp(-(i * i) / (2.0 * SSIM_SIGMA ** 2))
    g = g / g.sum()
    return torch.outer(g, g)


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Per-pixel SSIM of two [C][H][W] images, channels separately: local means, variances and
    covariance are window-weighted moments with zeros outside the image, and
    SSIM = (2 mu_x mu_y + C1)(2 cov_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(var_x + var_y + C2))."""
    C = x.shape[0]
    w = ssim_window()[None, None].expand(C, 1, SSIM_WINDOW, SSIM_WINDOW).contiguous()
    filt = lambda t: torch.nn.functional.conv2d(t[None], w, padding=SSIM_WINDOW // 2, groups=C)[0]
    mx, my = filt(x), filt(y)
    vx = filt(x * x) - mx * mx
    vy = filt(y * y) - my * my
    cxy = filt(x * y) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * cxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (vx + vy + SSIM_C2))


def l1_dssim_loss_and_grad(image, target, lam=0.2):
    """L = (1 - lam) mean|x - y| + lam (1 - mean SSIM(x, y)) over all pixels and channels (D-SSIM
    read as 1 - SSIM), and dL/dimage by autodiff in float64 (|.| has derivative sign, 0 at 0)."""
    x = torch.tensor(np.asarray(image, np.float64), requires_grad=True)
    y = torch.tensor(np.asarray(target, np.float64))
    L = (1.0 - lam) * (x - y).abs().mean() + lam * (1.0 - ssim_map(x, y).mean())
    L.backward()
    return float(L.detach()), x.grad.numpy()


# ----------------------------------------------------------------------------------------------
# Frequency-adaptive density control (Sec. 3.4.2; supplement B), on top of the 3DGS rules
# ----------------------------------------------------------------------------------------------
def densify_defaults(dense_scale=0.05):
    """Constants: 3DGS's gradient threshold, split into two children whose scales are divided by
    0.8 x 2; the paper's opacity threshold 0.01 and the reset values of new primitives' frequencies
    (0.001 per coordinate) and weights (0.01)."""
    return dict(grad_threshold=2e-4, dense_scale=dense_scale, min_opacity=0.01, max_scale=0.0,
                split_divisor=1.6, child_freq=1e-3, child_weight=1e-2)


def densify_accumulate(grad_accum, denom, means2d_grad, visible):
    """One training view's statistics: every primitive visible in the view (at least one tile)
    adds the norm of dL/dmu2D (pixels) to grad_accum and 1 to denom.  float32, single correctly
    rounded operations: sqrt((gx gx) + (gy gy)), then the sum."""
    f32 = np.float32
    g = np.asarray(means2d_grad, f32)
    norm = np.sqrt(g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1])
    vis = np.asarray(visible, bool)
    acc = np.asarray(grad_accum, f32).copy()
    den = np.asarray(denom, f32).copy()
    acc[vis] = acc[vis] + norm[vis]
    den[vis] = den[vis] + f32(1.0)
    return acc, den


def densify_decisions(prims, grad_accum, denom, cfg):
    """Per primitive, in float32 with correctly rounded operations:
      mean gradient  g = grad_accum / denom (0 where denom = 0);
      candidate      g >= grad_threshold;  s_max = the largest scale;
      clone          candidate and s_max <= dense_scale;  split: candidate and s_max > dense_scale;
      pruned         opacity < min_opacity, or max_scale > 0 and s_max > max_scale (children of a
                     split are tested with their own scale s / split_divisor).
    Returns (keep_original, keep_clone, keep_children) boolean arrays."""
    f32 = np.float32
    acc, den = np.asarray(grad_accum, f32), np.asarray(denom, f32)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(den > 0, acc / np.where(den > 0, den, f32(1)), f32(0))
    sc = np.asarray(prims["scales"], f32)
    smax = sc.max(1)
    cand = g >= f32(cfg["grad_threshold"])
    clone = cand & (smax <= f32(cfg["dense_scale"]))
    split = cand & (smax > f32(cfg["dense_scale"]))
    low = np.asarray(prims["opacity"], f32) < f32(cfg["min_opacity"])
    ms = f32(cfg["max_scale"])
    big = (ms > 0) & (smax > ms)
    child_big = (ms > 0) & ((sc / f32(cfg["split_divisor"])).max(1) > ms)
    return ~split & ~low & ~big, clone & ~low & ~big, split & ~low & ~child_big


def densify(prims, grad_accum, denom, split_noise, cfg):
    """Clone / split / prune with the frequency-adaptive reset of new primitives.

    Output rows, in this order: the kept originals (index order), then one clone per kept clone
    (index order), then two children per kept split (index order; child c at
    mu + R(q) (s * z_c) with z = split_noise[i, c], scale s / split_divisor).  Clones and children
    copy rotation, opacity and SH; every frequency coordinate of a new primitive is child_freq and
    every weight child_weight.  Returns the output attribute arrays (float64 means, float32 scales)
    and the three segment counts."""
    keep_o, keep_c, keep_s = densify_decisions(prims, grad_accum, denom, cfg)
    f32 = np.float32
    K = prims["weights"].shape[1]
    io, ic, isp = np.nonzero(keep_o)[0], np.nonzero(keep_c)[0], np.nonzero(keep_s)[0]
    isp2 = np.repeat(isp, 2)
    which = np.tile([0, 1], isp.shape[0])
    src = np.concatenate([io, ic, isp2])
    out = {k: np.asarray(prims[k])[src].copy() for k in ("means", "scales", "quats", "opacity", "sh", "freqs", "weights")}
    out["means"] = out["means"].astype(np.float64)
    new = slice(io.shape[0], src.shape[0])
    out["freqs"][new] = f32(cfg["child_freq"])
    out["weights"][new] = f32(cfg["child_weight"])
    if isp.shape[0]:
        s = np.asarray(prims["scales"], f32)[isp2]
        R = rotation_from_quaternion(torch.tensor(np.asarray(prims["quats"], np.float64)[isp2])).numpy()
        z = np.asarray(split_noise, np.float64)[isp2, which]
        off = np.einsum("nij,nj->ni", R, s.astype(np.float64) * z)
        ch = slice(io.shape[0] + ic.shape[0], src.shape[0])
        out["means"][ch] = np.asarray(prims["means"], np.float64)[isp2] + off
        out["scales"][ch] = s / f32(cfg["split_divisor"])
    counts = dict(originals=int(io.shape[0]), clones=int(ic.shape[0]), children=int(2 * isp.shape[0]))
    return out, counts


def reset_opacity_weights(prims, opacity_cap=0.02, weight=0.01):
    """The periodic reset (every 3000 iterations in the paper): opacity capped, every weight set."""
    out = dict(prims)
    out["opacity"] = np.minimum(np.asarray(prims["opacity"], np.float32), np.float32(opacity_cap))
    out["weights"] = np.full_like(np.asarray(prims["weights"], np.float32), np.float32(weight))
    return out
