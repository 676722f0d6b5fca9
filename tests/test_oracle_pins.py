"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks the oracle against mathematics the paper fixes or against a library routine:
closed forms, numerical quadrature of the z-integral (supplement A.2), the stated special cases
(Sec. 3.2.2), brute-force sequential compositing, finite differences, scipy's spherical
harmonics and rotations.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import gabsplat_oracle as O
from paper_2508_05343_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny_scene(seed, n=24, K=2, sh_degree=1, box=0.6, log_scale=(-2.0, 0.3)):
    spec = scenes.SceneSpec(n=n, K=K, sh_degree=sh_degree, layout="uniform", box=box, log_scale=log_scale)
    return scenes.make_scene(spec, seed)


def tiny_camera(w=40, h=36, dist=3.0, az=20.0, el=10.0):
    return scenes.orbit_camera(w, h, az, el, dist)


def t64(a, rg=False):
    return torch.tensor(np.asarray(a, np.float64), requires_grad=rg)


# ------------------------------------------------------------------------------------------
# Library pins: spherical harmonics, rotations
# ------------------------------------------------------------------------------------------
def test_sh_basis_matches_scipy():
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(0)
    d = rng.standard_normal((64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    ours = O.sh_basis(t64(d), 3).numpy()
    for l in range(4):
        for m in range(-l, l + 1):
            if m > 0:
                ref = math.sqrt(2) * (-1) ** m * sph_harm_y(l, m, theta, phi).real
            elif m < 0:
                ref = math.sqrt(2) * (-1) ** m * sph_harm_y(l, -m, theta, phi).imag
            else:
                ref = sph_harm_y(l, 0, theta, phi).real
            np.testing.assert_allclose(ours[:, l * l + l + m], ref, atol=1e-13, err_msg=f"l={l} m={m}")


def test_rotation_matches_scipy():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(1)
    q = rng.standard_normal((32, 4)) * rng.uniform(0.2, 3.0, (32, 1))      # any norm > 0
    ours = O.rotation_from_quaternion(t64(q)).numpy()
    ref = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()               # scipy is scalar-last
    np.testing.assert_allclose(ours, ref, atol=1e-13)


def test_covariance_is_rotated_scale():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(2)
    q = rng.standard_normal((16, 4))
    s = np.exp(rng.normal(-1, 0.5, (16, 3)))
    ours = O.covariance_3d(t64(s), t64(q)).numpy()
    R = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    ref = np.einsum("nij,nj,nkj->nik", R, s * s, R)
    np.testing.assert_allclose(ours, ref, atol=1e-14)


# ------------------------------------------------------------------------------------------
# Projection pins (Sec. 3.1, Eq. 2; Sec. 3.3.1, Eq. 7)
# ------------------------------------------------------------------------------------------
def test_jacobian_is_derivative_of_pinhole_projection():
    cam = tiny_camera(64, 48)
    W, tc = O.camera_tensors(cam)
    rng = np.random.default_rng(3)
    mu = rng.uniform(-0.5, 0.5, (10, 3))
    t = t64(mu) @ W.T + tc
    JW = (O.jacobian(t, cam) @ W).numpy()

    def pi(x):
        c = W.numpy() @ x + tc.numpy()
        return np.array([cam["fx"] * c[0] / c[2] + cam["cx"], cam["fy"] * c[1] / c[2] + cam["cy"]])

    for k in range(mu.shape[0]):
        num = np.zeros((2, 3))
        for j in range(3):
            e = np.zeros(3); e[j] = 1e-6
            num[:, j] = (pi(mu[k] + e) - pi(mu[k] - e)) / 2e-6
        np.testing.assert_allclose(JW[k, :2], num, rtol=1e-7, atol=1e-6)


def test_jacobian_field_of_view_guard_closed_form():
    """Means outside the guarded field of view on each axis (x/z and y/z beyond 1.3 tan(fov/2),
    the 3DGS convention the paper keeps): J's first two rows are the pinhole derivative taken at
    the clamped ray, with the x guard from width / fx and the y guard from height / fy.  A camera
    with width != height and fx != fy tells the two guards apart.  Expected rows worked by hand:
    at depth 2 with W = 200, fx = 150, H = 100, fy = 90 the guards are 1.3 * 100 / 150 and
    1.3 * 50 / 90, so -fx ux / z = -1.3 * 100 / 2 = -65 and -fy uy / z = +1.3 * 50 / 2 = 32.5."""
    cam = dict(R=np.eye(3).reshape(-1).tolist(), t=[0.0, 0.0, 0.0], fx=150.0, fy=90.0, cx=100.0, cy=50.0,
               width=200, height=100, znear=0.2, zfar=100.0)
    t = t64([[3.0, -2.4, 2.0],      # x/z = 1.5 > 0.8667 (clamped), y/z = -1.2 < -0.7222 (clamped)
             [1.0, 0.5, 2.0],       # x/z = 0.5, y/z = 0.25: inside, plain pinhole derivative
             [-4.0, 0.2, 2.0]])     # x/z = -2 (clamped to -0.8667), y/z = 0.1
    J = O.jacobian(t, cam).numpy()
    expected = np.array([[[75.0, 0.0, -65.0], [0.0, 45.0, 32.5], [0.0, 0.0, 1.0]],
                         [[75.0, 0.0, -37.5], [0.0, 45.0, -11.25], [0.0, 0.0, 1.0]],
                         [[75.0, 0.0, 65.0], [0.0, 45.0, -4.5], [0.0, 0.0, 1.0]]])
    np.testing.assert_allclose(J, expected, rtol=1e-14, atol=1e-12)
    # the guard shapes only the Jacobian: the projected mean of the first point stays at 1.5 fx + cx
    prims = dict(means=np.array([[3.0, -2.4, 2.0]], np.float32), scales=np.full((1, 3), 0.1, np.float32),
                 quats=np.array([[1.0, 0, 0, 0]], np.float32), opacity=np.array([0.5], np.float32),
                 sh=np.zeros((1, 1, 3), np.float32), freqs=np.zeros((1, 0, 3), np.float32),
                 weights=np.zeros((1, 0), np.float32))
    mu = O.project(O._to_f64(prims), cam, O.default_config())["mu2d"].numpy()[0]
    np.testing.assert_allclose(mu, [1.5 * 150.0 + 100.0, -1.2 * 90.0 + 50.0], rtol=1e-6)


def test_mean_projection_is_pinhole():
    cam = tiny_camera()
    prims = tiny_scene(4)
    proj = O.project(O._to_f64(prims), cam, O.default_config())
    c = prims["means"].astype(np.float64) @ np.asarray(cam["R"], np.float64).T + np.asarray(cam["t"], np.float64)
    ref = np.stack([cam["fx"] * c[:, 0] / c[:, 2] + cam["cx"], cam["fy"] * c[:, 1] / c[:, 2] + cam["cy"]], -1)
    np.testing.assert_allclose(proj["mu2d"].detach().numpy(), ref, rtol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_z_integration_by_quadrature(seed):
    """Supplement A.2: integrating exp(-x^T S x / 2) cos(2 pi f.x) over z gives
    C1 C2 G2D(x, y) cos(2 pi f2D.(x, y)) with G2D built from the top-left 2x2 of S^-1, f2D from Eq. 8,
    C1 = sqrt(2 pi / S22) and C2 = exp(-2 pi^2 f_z^2 / S22).  Pins the reading of S (ray space)."""
    from scipy.integrate import quad
    rng = np.random.default_rng(100 + seed)
    A = rng.standard_normal((3, 3))
    sigma = A @ A.T + 0.3 * np.eye(3)
    f = rng.normal(0, 0.4, 3)
    f2d = O.splat_frequency(t64(f[None, None, :]), t64(sigma[None])).numpy()[0, 0]
    S = np.linalg.inv(sigma)
    cov2 = sigma[:2, :2]
    C1 = math.sqrt(2 * math.pi / S[2, 2])
    C2 = math.exp(-2 * math.pi ** 2 * f[2] ** 2 / S[2, 2])
    for _ in range(6):
        x, y = rng.normal(0, 1.0, 2)
        integrand = lambda z: math.exp(-0.5 * np.array([x, y, z]) @ S @ np.array([x, y, z])) * \
            math.cos(2 * math.pi * (f[0] * x + f[1] * y + f[2] * z))
        val, _ = quad(integrand, -np.inf, np.inf, epsabs=1e-14, epsrel=1e-12, limit=400)
        xy = np.array([x, y])
        ref = C1 * C2 * math.exp(-0.5 * xy @ np.linalg.inv(cov2) @ xy) * math.cos(2 * math.pi * f2d @ xy)
        assert abs(val - ref) < 1e-10 * max(1.0, abs(ref)), (val, ref)


def test_f2d_independent_of_jacobian_third_row():
    cam = tiny_camera(64, 64, az=35.0, el=-15.0)
    prims = tiny_scene(5, K=3)
    cfg = O.default_config()
    pz = O.project(O._to_f64(prims), cam, cfg, third_row="z")
    pe = O.project(O._to_f64(prims), cam, cfg, third_row="ewa")
    np.testing.assert_allclose(pz["f2d"].detach().numpy(), pe["f2d"].detach().numpy(), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(pz["conic"].detach().numpy(), pe["conic"].detach().numpy(), rtol=1e-12)


def test_f2d_conditional_mean_form():
    """-S_xz/S_zz equals A^-1 b (A, b = blocks of the ray-space covariance): a second formula for Eq. 8."""
    rng = np.random.default_rng(6)
    for _ in range(20):
        X = rng.standard_normal((3, 3))
        sig = X @ X.T + 0.1 * np.eye(3)
        fp = rng.standard_normal(3)
        ours = O.splat_frequency(t64(fp[None, None]), t64(sig[None])).numpy()[0, 0]
        r = np.linalg.solve(sig[:2, :2], sig[:2, 2])
        np.testing.assert_allclose(ours, fp[:2] + r * fp[2], rtol=1e-10, atol=1e-12)


def test_fixed_direction_frequencies_project_along_one_direction():
    """The 2DGabSplat case (Sec. 3.2.2): with every frequency of a primitive a multiple m_i of one
    world axis a, Eq. 7 ((JW)^-T f) and Eq. 8 (the S-ratio correction) are linear in f, so
    f2D_i = m_i f2D(a): all of the primitive's projected frequencies lie along one image direction.
    Checked against a separate projection of the axis alone."""
    cam = tiny_camera()
    prims = tiny_scene(31, n=16, K=3)
    a = np.array([0.75, 0.0, 0.5])
    m = np.random.default_rng(32).uniform(-6, 6, (16, 3))
    prims["freqs"] = m[:, :, None] * a[None, None, :]
    f2d = O.project(O._to_f64(prims), cam, O.default_config())["f2d"].detach().numpy()
    axis_only = dict(prims, freqs=np.broadcast_to(a, (16, 1, 3)).copy(), weights=prims["weights"][:, :1])
    fa = O.project(O._to_f64(axis_only), cam, O.default_config())["f2d"].detach().numpy()[:, 0]
    np.testing.assert_allclose(f2d, m[:, :, None] * fa[:, None, :], rtol=1e-12, atol=1e-14)
    cross = f2d[:, :, 0] * fa[:, None, 1] - f2d[:, :, 1] * fa[:, None, 0]
    assert np.abs(cross).max() < 1e-12 * np.abs(f2d).max() * np.abs(fa).max()


def test_frequency_projection_camera_aligned():
    """Axis-aligned primitive on the optical axis, f along camera x: f2D = (f tz / fx, 0) cycles/pixel."""
    cam = scenes.make_camera(64, 64, 60.0, eye=(0, 0, -4.0))
    prims = dict(means=np.array([[0, 0, 1.0]], np.float32), scales=np.array([[0.1, 0.2, 0.3]], np.float32),
                 quats=np.array([[1, 0, 0, 0]], np.float32), opacity=np.array([0.8], np.float32),
                 sh=np.zeros((1, 1, 3), np.float32), freqs=np.array([[[2.5, 0, 0]]], np.float32),
                 weights=np.array([[0.5]], np.float32))
    p = O.project(O._to_f64(prims), cam, O.default_config())
    tz = 5.0
    np.testing.assert_allclose(p["f2d"].detach().numpy()[0, 0], [2.5 * tz / cam["fx"], 0.0], atol=1e-14)


# ------------------------------------------------------------------------------------------
# Rendering pins (Eq. 9-10)
# ------------------------------------------------------------------------------------------
def test_single_primitive_closed_form():
    """One axis-aligned primitive on the optical axis: the image is rgb*alpha + bg*(1-alpha) with alpha
    from the analytic 2D footprint sigma_x = fx s_x / tz, f2D = f tz / fx (no matrices involved)."""
    Wd, Hd = 96, 80
    cam = scenes.make_camera(Wd, Hd, 60.0, eye=(0, 0, -4.0))
    cfg = O.default_config(eps2d=0.3, bg=(0.1, 0.2, 0.3))
    sx, sy, tz, fw, w, o = 0.07, 0.11, 4.0, 3.0, 0.45, 0.9
    sh = np.array([[[0.3, -0.2, 0.1]]], np.float32)
    prims = dict(means=np.array([[0, 0, 0.0]], np.float32), scales=np.array([[sx, sy, 0.05]], np.float32),
                 quats=np.array([[1, 0, 0, 0]], np.float32), opacity=np.array([o], np.float32), sh=sh,
                 freqs=np.array([[[fw, 0, 0]]], np.float32), weights=np.array([[w]], np.float32))
    out = O.render(prims, cam, cfg)
    fx = cam["fx"]
    vx = (fx * np.float64(np.float32(sx)) / tz) ** 2 + cfg["eps2d"]
    vy = (fx * np.float64(np.float32(sy)) / tz) ** 2 + cfg["eps2d"]
    f2 = np.float64(np.float32(fw)) * tz / fx
    rgb = np.maximum(0, 0.5 / math.sqrt(math.pi) * sh[0, 0].astype(np.float64) + 0.5)
    r = math.ceil(3 * math.sqrt(max(vx, vy)))
    xs = np.arange(Wd) + 0.5
    ys = np.arange(Hd) + 0.5
    dx = xs[None, :] - Wd / 2
    dy = ys[:, None] - Hd / 2
    alpha = np.float64(np.float32(o)) * np.exp(-0.5 * (dx ** 2 / vx + dy ** 2 / vy)) * \
        ((1 - np.float64(np.float32(w))) + np.float64(np.float32(w)) * np.cos(2 * math.pi * f2 * dx))
    alpha = np.minimum(alpha, cfg["alpha_max"])
    alpha = np.where(alpha >= cfg["alpha_min"], alpha, 0.0)
    tx0, tx1 = math.floor((Wd / 2 - r) / 16), math.floor((Wd / 2 + r) / 16)
    ty0, ty1 = math.floor((Hd / 2 - r) / 16), math.floor((Hd / 2 + r) / 16)
    tile_x = (np.arange(Wd) // 16)[None, :]
    tile_y = (np.arange(Hd) // 16)[:, None]
    inside = (tile_x >= tx0) & (tile_x <= tx1) & (tile_y >= ty0) & (tile_y <= ty1)
    alpha = np.where(inside, alpha, 0.0)
    bg = np.array(cfg["bg"])
    ref = rgb[:, None, None] * alpha[None] + bg[:, None, None] * (1 - alpha[None])
    np.testing.assert_allclose(out["image"].numpy(), ref, atol=1e-12)
    np.testing.assert_allclose(out["T"].numpy(), 1 - alpha, atol=1e-12)


def _special_cases():
    with open(os.path.join(GOLDEN, "special_cases.json")) as fh:
        return json.load(fh)


def test_gaussian_special_case_reduction():
    """Sec. 3.2.2: f = 0 or w = 0 is 3DGS; K = 0 is the plain Gaussian splatter.  All three agree."""
    sc = _special_cases()["gaussian_special_case"]
    cam = tiny_camera(48, 40)
    cfg = O.default_config()
    base = tiny_scene(7, n=30, K=3)
    a = dict(base, weights=np.full_like(base["weights"], sc["w"]))
    b = dict(base, freqs=np.full_like(base["freqs"], sc["f"]))
    c = dict(base, freqs=np.zeros((30, 0, 3), np.float32), weights=np.zeros((30, 0), np.float32))
    ia, ib, ic = (O.render(p, cam, cfg)["image"].numpy() for p in (a, b, c))
    np.testing.assert_allclose(ia, ic, atol=1e-13)
    np.testing.assert_allclose(ib, ic, atol=1e-13)
    assert np.abs(O.render(base, cam, cfg)["image"].numpy() - ic).max() > 1e-3   # Gabor terms matter


def test_initialisation_values_avoid_degenerate_gradients():
    """Sec. 3.4.1: at f = 0 the Gabor terms have zero gradient; at the stated initial values they do not."""
    sc = _special_cases()
    cam = tiny_camera(32, 32)
    cfg = O.default_config()
    base = tiny_scene(8, n=10, K=2, log_scale=(-1.5, 0.2))
    rng = np.random.default_rng(8)
    g = rng.standard_normal((3, 32, 32))
    deg = dict(base, freqs=np.zeros_like(base["freqs"]), weights=np.full_like(base["weights"], 0.3))
    gd = O.render_backward(deg, cam, cfg, g)
    assert np.abs(gd["freqs"]).max() == 0.0 and np.abs(gd["weights"]).max() < 1e-15
    ini = sc["initialisation"]
    init = dict(base, freqs=np.full_like(base["freqs"], ini["f"]), weights=np.full_like(base["weights"], ini["w"]))
    gi = O.render_backward(init, cam, cfg, g)
    assert np.abs(gi["freqs"]).max() > 0 and np.abs(gi["weights"]).max() > 0


def test_constant_colour_weights_telescope():
    """With every primitive white and a black background, C = 1 - T_final exactly (sum of weights)."""
    cam = scenes.orbit_camera(64, 48, 0.0, 0.0, 4.0)
    cfg = O.default_config()
    prims = scenes.config_scene(0)
    c0 = 0.5 / math.sqrt(math.pi)
    prims = dict(prims, sh=np.full_like(prims["sh"], 0.5 / c0))
    out = O.render(prims, cam, cfg)
    img, T = out["image"].numpy(), out["T"].numpy()
    for ch in range(3):
        np.testing.assert_allclose(img[ch], 1 - T, atol=1e-12)
    assert (T >= cfg["T_min"]).all() and (T <= 1).all() and (img >= 0).all()


def test_transmittance_monotone_and_bounded():
    cam = scenes.config_cameras(0)[0]
    cfg = O.default_config()
    prims = scenes.config_scene(0)
    out = O.render(prims, cam, cfg)
    spec, proj = out["spec"], out["proj"]
    for tid in range(spec["tiles_x"] * spec["tiles_y"]):
        s0, s1 = spec["ranges"][tid]
        if s1 == s0:
            continue
        ids = torch.from_numpy(spec["sorted_vals"][s0:s1].astype(np.int64))
        rec = {k: proj[k].index_select(0, ids) for k in O.REC_KEYS}
        gx, gy, _, _ = O._tile_pixels(tid % spec["tiles_x"], tid // spec["tiles_x"], 128, 128)
        alpha = torch.clamp_max(O.gabor_alpha(gx, gy, rec, cfg), cfg["alpha_max"])
        assert (alpha <= cfg["alpha_max"]).all()
    T = out["T"].numpy()
    assert (T >= cfg["T_min"]).all() and (T <= 1.0).all()
    assert (out["image"].numpy() >= 0).all()


def test_flip_allowance_hand_worked():
    """Sequential compositing with one decision inverted, on cases worked by hand (bg 0.2):
    pairs alpha 0.5 (red) then 0.25 (green).  Plain: C = (0.5, 0.125, 0), T = 0.375, so the result
    is (0.575, 0.2, 0.075).  Skipping pair 0: C = (0, 0.25, 0), T = 0.75 -> (0.15, 0.4, 0.15).
    Stopping before pair 1: C = (0.5, 0, 0), T = 0.5 -> (0.6, 0.1, 0.1)."""
    cfg = dict(O.default_config(bg=(0.2, 0.2, 0.2)), bg=(0.2, 0.2, 0.2))
    a = torch.tensor([0.5, 0.25], dtype=torch.float64)
    rgb = torch.tensor([[1.0, 0, 0], [0, 1.0, 0]], dtype=torch.float64)
    np.testing.assert_allclose(O.composite_pixel(a, rgb, cfg).numpy(), [0.575, 0.2, 0.075], atol=1e-15)
    np.testing.assert_allclose(O.composite_pixel(a, rgb, cfg, flip_keep=(0,)).numpy(), [0.15, 0.4, 0.15], atol=1e-15)
    np.testing.assert_allclose(O.composite_pixel(a, rgb, cfg, flip_stop=(1,)).numpy(), [0.6, 0.1, 0.1], atol=1e-15)
    np.testing.assert_allclose(O.flip_allowance(a, rgb, cfg, [0], [1]).numpy(),
                               [0.425 + 0.025, 0.2 + 0.1, 0.075 + 0.025], atol=1e-15)


def test_threshold_flags_follow_the_float32_error():
    """One primitive, one pixel at its mean: alpha = o (G = 1, no bank).  An opacity within a few
    float32 roundings of alpha_min is flagged (either branch is a correct float32 result), one
    0.1% away is not; the same for alpha_max.  The flagged pixel's allowance is the whole pair."""
    cfg = O.default_config()
    amin, amax = cfg["alpha_min"], cfg["alpha_max"]
    rec = dict(mu2d=torch.tensor([[8.5, 8.5]], dtype=torch.float64), conic=torch.tensor([[0.5, 0.0, 0.5]], dtype=torch.float64),
               rgb=torch.tensor([[1.0, 1.0, 1.0]], dtype=torch.float64), f2d=torch.zeros(1, 0, 2, dtype=torch.float64),
               weights=torch.zeros(1, 0, dtype=torch.float64), cos_weights=torch.zeros(1, 0, dtype=torch.float64))
    px = py = torch.tensor([8.5], dtype=torch.float64)
    for o, flag_f, flag_b in [(amin * (1 + 1e-7), True, True), (amin * (1 - 1e-7), True, True),
                              (amin * 1.001, False, False), (amax * (1 + 1e-7), False, True), (amax * 0.999, False, False)]:
        r = dict(rec, opacity=torch.tensor([o], dtype=torch.float64))
        _, _, _, af, ab, _, allow = O.composite(px, py, r, cfg)
        assert bool(af[0]) == flag_f and bool(ab[0]) == flag_b, o
        if flag_f:
            assert abs(float(allow[0, 0]) - o) < 1e-9      # the pair composited or not: alpha T c


def _brute_force(prims, cam, cfg, feature=None):
    """Sequential per-pixel compositing with scalar math, independent of the tile vectorisation:
    gather every primitive whose 3-sigma square overlaps the pixel's tile, order by (float32 depth
    bits, index) with Python's sort, and walk front to back.  feature(P, k) replaces the colour
    (and the background is then zero)."""
    spec = O.bin_spec(prims, cam, cfg)
    proj = O.project(O._to_f64(prims), cam, cfg)
    P = {k: v.detach().numpy() for k, v in proj.items()}
    Wd, Hd = cam["width"], cam["height"]
    img = np.zeros((3, Hd, Wd)); Tf = np.zeros((Hd, Wd)); last = np.zeros((Hd, Wd), np.int64)
    dbits = spec["depth"].astype(np.float32).view(np.uint32)
    n = prims["means"].shape[0]
    for py in range(Hd):
        for px in range(Wd):
            tx, ty = px // 16, py // 16
            plist = []
            for k in range(n):
                if not spec["valid"][k]:
                    continue
                mx, my = float(spec["mu2d"][k, 0]), float(spec["mu2d"][k, 1])
                r = float(spec["radius"][k])
                if 16 * tx <= mx + r and 16 * tx + 16 > mx - r and 16 * ty <= my + r and 16 * ty + 16 > my - r:
                    plist.append(k)
            plist.sort(key=lambda k: (int(dbits[k]), k))
            T, C, lst = 1.0, np.zeros(3), 0
            for pos, k in enumerate(plist):
                dx, dy = px + 0.5 - P["mu2d"][k, 0], py + 0.5 - P["mu2d"][k, 1]
                a, b, c = P["conic"][k]
                G = math.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
                bank = 1.0
                for i in range(P["weights"].shape[1]):
                    wi = P["weights"][k, i]
                    wc = P["cos_weights"][k, i]
                    bank += wc * math.cos(2 * math.pi * (P["f2d"][k, i, 0] * dx + P["f2d"][k, i, 1] * dy)) - wi
                alpha = min(cfg["alpha_max"], P["opacity"][k] * G * bank)
                if alpha < cfg["alpha_min"]:
                    continue
                if T * (1 - alpha) < cfg["T_min"]:
                    break
                C += (P["rgb"][k] if feature is None else feature(P, k)) * alpha * T
                T *= (1 - alpha)
                lst = pos + 1
            img[:, py, px] = C + (T * np.array(cfg["bg"]) if feature is None else 0.0)
            Tf[py, px] = T
            last[py, px] = lst
    return img, Tf, last


@pytest.mark.parametrize("seed,n,K", [(11, 40, 2), (12, 24, 0), (13, 32, 4)])
def test_brute_force_matches_tiled_oracle(seed, n, K):
    cam = tiny_camera(40, 36, dist=2.5)                       # ragged tiles: 40x36 is not a multiple of 16
    cfg = O.default_config(bg=(0.2, 0.0, 0.5))
    prims = tiny_scene(seed, n=n, K=K, log_scale=(-2.2, 0.4))
    prims["opacity"] = np.clip(prims["opacity"] * 1.4, 0, 0.999).astype(np.float32)   # exercise the stop rule
    out = O.render(prims, cam, cfg)                     # tiles culled to those a pixel can reach
    img, T, last = _brute_force(prims, cam, cfg)        # every tile of the 3-sigma squares
    np.testing.assert_allclose(out["image"].numpy(), img, atol=1e-12)
    np.testing.assert_allclose(out["T"].numpy(), T, atol=1e-12)
    full = O.render(prims, cam, cfg, cull=False)       # list positions refer to the full squares
    np.testing.assert_array_equal(full["n_contrib"].numpy(), last)


def test_binning_rects_and_sorted_keys_brute_force():
    """Pairs = tiles of each primitive's 3-sigma square (interval overlap, brute force) that some pixel
    centre can reach with o G >= alpha_min (float64 over the 256 centres): every such pair must be
    emitted, and every emitted pair must be within the specification's margin of reaching; the
    sorted keys must be Python's sort of the emission list."""
    cam = tiny_camera(72, 56, dist=2.0)
    cfg = O.default_config()
    prims = tiny_scene(14, n=60, K=1, log_scale=(-2.0, 0.6))
    spec = O.bin_spec(prims, cam, cfg)
    tx_n, ty_n = spec["tiles_x"], spec["tiles_y"]
    emitted = {(int(k) >> 32, int(v)) for k, v in zip(spec["keys"], spec["vals"])}
    must, may = set(), set()
    for k in range(60):
        if not spec["valid"][k]:
            continue
        mx, my, r = float(spec["mu2d"][k, 0]), float(spec["mu2d"][k, 1]), float(spec["radius"][k])
        a, b, c = (float(x) for x in spec["cov2d"][k])
        det = a * c - b * b
        Qa, Qb, Qc = c / det, -b / det, a / det
        o = float(np.float32(prims["opacity"][k]))
        thr = 2 * math.log(o / cfg["alpha_min"]) if o >= cfg["alpha_min"] else -1.0
        for ty in range(ty_n):
            for tx in range(tx_n):
                if not (16 * tx <= mx + r and 16 * tx + 16 > mx - r and 16 * ty <= my + r and 16 * ty + 16 > my - r):
                    continue
                px = 16 * tx + 0.5 + np.arange(16) - mx
                py = 16 * ty + 0.5 + np.arange(16) - my
                q = (Qa * px[None] ** 2 + 2 * Qb * px[None] * py[:, None] + Qc * py[:, None] ** 2).min()
                if q <= thr:
                    must.add((ty * tx_n + tx, k))
                if q <= thr * 1.01 + 0.1 and thr > 0:
                    may.add((ty * tx_n + tx, k))
    assert must and must <= emitted <= may, (len(must), len(emitted), len(may))
    pairs = [(int(key), int(v)) for key, v in zip(spec["keys"], spec["vals"])]
    ref = sorted(enumerate(pairs), key=lambda e: (e[1][0], e[0]))
    np.testing.assert_array_equal(spec["sorted_keys"], np.array([p[1][0] for p in ref], np.uint64))
    np.testing.assert_array_equal(spec["sorted_vals"], np.array([p[1][1] for p in ref], np.uint32))
    for tid in range(tx_n * ty_n):
        cnt = sum(1 for p in pairs if p[0] >> 32 == tid)
        assert spec["ranges"][tid, 1] - spec["ranges"][tid, 0] == cnt


@pytest.mark.parametrize("cfgi", [0, 1])
def test_tile_culling_leaves_the_image_unchanged(cfgi):
    """Dropping the tiles no pixel can reach changes no pixel: culled and full 3-sigma lists render the
    same float64 image and transmittance up to summation order (config 1 on a block of tiles)."""
    prims, cam = scenes.config_scene(cfgi), scenes.config_cameras(cfgi)[0]
    cfg = O.default_config()
    tiles = None if cfgi == 0 else [ty * 50 + tx for ty in range(20, 26) for tx in range(20, 28)]
    a = O.render(prims, cam, cfg, tiles=tiles)
    b = O.render(prims, cam, cfg, tiles=tiles, cull=False)
    assert a["spec"]["P"] < 0.8 * b["spec"]["P"]
    np.testing.assert_allclose(a["image"].numpy(), b["image"].numpy(), rtol=0, atol=1e-13)
    np.testing.assert_allclose(a["T"].numpy(), b["T"].numpy(), rtol=0, atol=1e-13)


@pytest.mark.parametrize("cfgi", [0, 1])
def test_float32_binning_against_pure_float64_binning(cfgi):
    """The float32 binning specification against the same binning done in float64 throughout
    (bin_fp64: float64 projection, radius ceil(3 sqrt(lambda_max)), exact ellipse-meets-tile-box
    reach test).  No pair that float64 reaches is dropped; every extra float32 pair inside the
    float64 rectangle is one no pixel reaches in float64 (the rule's float32 safety margins), so it
    leaves the image unchanged; radius flips (ceil at an integer boundary) touch a handful of
    primitives."""
    prims, cam = scenes.config_scene(cfgi), scenes.config_cameras(cfgi)[0]
    d = O.binning_differences(prims, cam, O.default_config())
    assert d["fp64_only"] == 0
    inside = d["spec_only_in_fp64_rect"]
    assert (d["spec_only_margin"][inside] > 0).all()
    assert d["spec_only"] <= 0.005 * d["P_fp64"]
    assert d["rect_diff"] <= max(2, 1e-4 * prims["means"].shape[0])
    assert d["spec_only_outside_fp64_rect"] <= d["rect_diff"]


def test_binning_float32_close_to_float64():
    cam = scenes.config_cameras(0)[0]
    cfg = O.default_config()
    prims = scenes.config_scene(0)
    spec = O.bin_spec(prims, cam, cfg)
    proj = O.project(O._to_f64(prims), cam, cfg)
    v = spec["valid"]
    np.testing.assert_allclose(spec["mu2d"][v], proj["mu2d"].detach().numpy()[v], rtol=1e-5)
    c64 = proj["cov2d"].detach().numpy()[v]
    np.testing.assert_allclose(spec["cov2d"][v][:, 0], c64[:, 0, 0], rtol=1e-4)
    np.testing.assert_allclose(spec["cov2d"][v][:, 2], c64[:, 1, 1], rtol=1e-4)


# ------------------------------------------------------------------------------------------
# Gradients: analytic (reverse mode) vs central finite differences
# ------------------------------------------------------------------------------------------
def _scalar_loss(prims, cam, cfg, g):
    return float((O.render(prims, cam, cfg)["image"].numpy() * g).sum())


@pytest.mark.parametrize("seed,K,deg", [(21, 2, 1), (22, 1, 3)])
def test_gradients_match_finite_differences(seed, K, deg):
    cam = tiny_camera(32, 32, dist=2.2, az=30.0, el=-20.0)
    cfg = O.default_config(bg=(0.3, 0.1, 0.2))
    prims = tiny_scene(seed, n=6, K=K, sh_degree=deg, box=0.35, log_scale=(-1.8, 0.3))
    prims = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in prims.items()}
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((3, 32, 32))
    an = O.render_backward(prims, cam, cfg, g)
    bad, total = 0, 0
    for key in ("means", "scales", "quats", "opacity", "sh", "freqs", "weights"):
        arr = prims[key]
        flat = arr.reshape(-1)
        num = np.zeros_like(flat)
        for i in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[i]))
            p = dict(prims); q = flat.copy(); q[i] += h; p[key] = q.reshape(arr.shape)
            lp = _scalar_loss(p, cam, cfg, g)
            q[i] -= 2 * h; p[key] = q.reshape(arr.shape)
            lm = _scalar_loss(p, cam, cfg, g)
            num[i] = (lp - lm) / (2 * h)
        a = an[key].reshape(-1)
        err = np.abs(a - num) / np.maximum(1e-4, np.abs(num))
        total += flat.size
        bad += int((err > 1e-5).sum())
        rel = np.linalg.norm(a - num) / max(np.linalg.norm(num), 1e-12)
        assert rel < 1e-6, (key, rel)
    assert bad <= max(1, total // 200), (bad, total)


def test_loss_gradients():
    rng = np.random.default_rng(5)
    img, tgt = rng.uniform(0, 1, (3, 8, 8)), rng.uniform(0, 1, (3, 8, 8))
    for kind in ("l1", "l2"):
        L, g = O.loss_and_grad(img, tgt, kind)
        i, j, k = 1, 3, 5
        h = 1e-7
        im2 = img.copy(); im2[i, j, k] += h
        L2, _ = O.loss_and_grad(im2, tgt, kind)
        assert abs((L2 - L) / h - g[i, j, k]) < 1e-6


# ---- training loss with the structural term (Sec. 3.4.1, Eq. 11) ------------------------------
def _window_1d():
    g = [math.exp(-((i - 5) ** 2) / (2 * 1.5 ** 2)) for i in range(11)]
    s = sum(g)
    return [v / s for v in g]


def _moments_brute(x, y, c, i, j):
    """Window-weighted moments at pixel (i, j) of channel c by explicit sums (zeros outside)."""
    g = _window_1d()
    H, W = x.shape[1:]
    m = [0.0] * 5
    for a in range(-5, 6):
        for b in range(-5, 6):
            r, q = i + a, j + b
            if 0 <= r < H and 0 <= q < W:
                w = g[a + 5] * g[b + 5]
                u, v = float(x[c, r, q]), float(y[c, r, q])
                m[0] += w * u; m[1] += w * v; m[2] += w * u * u; m[3] += w * v * v; m[4] += w * u * v
    return m


def test_ssim_brute_force_tiny():
    """Every pixel of a 2 x 9 x 13 image pair (smaller than the window in one direction, so every
    pixel sees the zero border): explicit windowed sums, then the SSIM index."""
    rng = np.random.default_rng(41)
    x, y = rng.random((2, 9, 13)), rng.random((2, 9, 13))
    got = O.ssim_map(torch.tensor(x), torch.tensor(y)).numpy()
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    for c in range(2):
        for i in range(9):
            for j in range(13):
                mx, my, exx, eyy, exy = _moments_brute(x, y, c, i, j)
                vx, vy, cv = exx - mx * mx, eyy - my * my, exy - mx * my
                ref = (2 * mx * my + C1) * (2 * cv + C2) / ((mx * mx + my * my + C1) * (vx + vy + C2))
                assert abs(got[c, i, j] - ref) < 1e-12, (c, i, j)


def test_ssim_closed_forms():
    rng = np.random.default_rng(42)
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    x = rng.random((3, 24, 30))
    # identical images: 1 everywhere, zero loss
    np.testing.assert_allclose(O.ssim_map(torch.tensor(x), torch.tensor(x)).numpy(), 1.0, atol=1e-12)
    assert O.l1_dssim_loss_and_grad(x, x)[0] == 0.0
    # constant images a, b: away from the border only the luminance factor is left
    a, b = 0.7, 0.2
    s = O.ssim_map(torch.full((1, 24, 30), a, dtype=torch.float64), torch.full((1, 24, 30), b, dtype=torch.float64))
    np.testing.assert_allclose(s[0, 5:-5, 5:-5].numpy(), (2 * a * b + C1) / (a * a + b * b + C1), rtol=1e-12)
    # y = x + c: equal variances and covariance, so the contrast-structure factor is 1
    s = O.ssim_map(torch.tensor(x), torch.tensor(x + 0.3)).numpy()
    for (c, i, j) in [(0, 7, 9), (1, 12, 20), (2, 18, 6)]:
        mx = _moments_brute(x, x, c, i, j)[0]
        my = mx + 0.3
        assert abs(s[c, i, j] - (2 * mx * my + C1) / (mx * mx + my * my + C1)) < 1e-12
    # y = 1 - x: covariance = -variance, so the contrast-structure factor is (C2 - 2 var)/(C2 + 2 var)
    s = O.ssim_map(torch.tensor(x), torch.tensor(1.0 - x)).numpy()
    for (c, i, j) in [(0, 6, 11), (2, 15, 24)]:
        mx, _, exx, _, _ = _moments_brute(x, x, c, i, j)
        var, my = exx - mx * mx, 1.0 - mx
        ref = (2 * mx * my + C1) / (mx * mx + my * my + C1) * (C2 - 2 * var) / (C2 + 2 * var)
        assert abs(s[c, i, j] - ref) < 1e-12


def test_l1_dssim_is_the_weighted_sum_and_its_gradient():
    """lambda = 0 is the mean L1 loss with gradient sign(x - y)/N; lambda = 1 is 1 - mean SSIM;
    the value is affine in lambda; the gradient matches central finite differences."""
    rng = np.random.default_rng(43)
    x, y = rng.random((2, 12, 15)), rng.random((2, 12, 15))
    N = x.size
    l0, g0 = O.l1_dssim_loss_and_grad(x, y, lam=0.0)
    assert abs(l0 - np.abs(x - y).mean()) < 1e-14
    np.testing.assert_allclose(g0, np.sign(x - y) / N, atol=1e-18)
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    ssum = 0.0
    for c in range(2):
        for i in range(12):
            for j in range(15):
                mx, my, exx, eyy, exy = _moments_brute(x, y, c, i, j)
                ssum += (2 * mx * my + C1) * (2 * (exy - mx * my) + C2) / (
                    (mx * mx + my * my + C1) * (exx - mx * mx + eyy - my * my + C2))
    l1, _ = O.l1_dssim_loss_and_grad(x, y, lam=1.0)
    assert abs(l1 - (1.0 - ssum / N)) < 1e-12
    l2, g2 = O.l1_dssim_loss_and_grad(x, y, lam=0.2)
    assert abs(l2 - (0.8 * l0 + 0.2 * l1)) < 1e-14
    h = 1e-6
    for (c, i, j) in [(0, 0, 0), (1, 5, 7), (0, 11, 14), (1, 3, 12)]:
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (O.l1_dssim_loss_and_grad(xp, y)[0] - O.l1_dssim_loss_and_grad(xm, y)[0]) / (2 * h)
        assert abs(fd - g2[c, i, j]) < 1e-8 * max(1.0, abs(g2[c, i, j]) * N), (c, i, j, fd, g2[c, i, j])


# ---- frequency maps (the visualisation of Sec. 4) --------------------------------------------
def _weighted_frequencies(P, k):
    m = mx = my = 0.0
    for i in range(P["weights"].shape[1]):
        fx, fy, w = P["f2d"][k, i, 0], P["f2d"][k, i, 1], P["weights"][k, i]
        m += w * math.hypot(fx, fy)
        mx += w * abs(fx)
        my += w * abs(fy)
    return np.array([m, mx, my])


@pytest.mark.parametrize("seed,n,K", [(5, 24, 2), (6, 30, 3)])
def test_frequency_map_brute_force(seed, n, K):
    """The maps are the compositing of the image with each primitive's colour replaced by its
    weighted |f2D|, |f2D_x|, |f2D_y| and no background: brute-force sequential compositing."""
    cam = tiny_camera(40, 32, dist=2.0)
    cfg = O.default_config(bg=(0.3, 0.2, 0.1))
    prims = tiny_scene(seed, n=n, K=K, log_scale=(-2.2, 0.4))
    got = O.render_frequency_map(prims, cam, cfg)["map"].numpy()
    ref, _, _ = _brute_force(prims, cam, cfg, feature=_weighted_frequencies)
    np.testing.assert_allclose(got, ref, atol=1e-12)
    assert np.abs(ref).max() > 1e-3                       # the maps are not trivially zero


def test_frequency_map_special_cases():
    cam = tiny_camera(40, 32, dist=2.0)
    cfg = O.default_config()
    # K = 0 (or all weights zero): a pure Gaussian scene has no frequency content
    p0 = tiny_scene(7, n=20, K=0)
    assert np.all(O.render_frequency_map(p0, cam, cfg)["map"].numpy() == 0.0)
    # one primitive: map = alpha * features, alpha read off the image of a constant colour
    p1 = tiny_scene(8, n=1, K=2, log_scale=(-1.0, 0.0))
    p1["means"][:] = 0.0
    p1["sh"][:] = 0.0
    p1["sh"][0, 0, :] = 0.5 / 0.28209479177387814     # SH band 0 -> colour 1.0 in every channel
    out = O.render(p1, cam, cfg)
    alpha = out["image"].numpy()[0]                     # colour 1, background 0: image = alpha
    proj = {k: v.numpy() for k, v in out["proj"].items()}
    feat = _weighted_frequencies(proj, 0)
    got = O.render_frequency_map(p1, cam, cfg)["map"].numpy()
    np.testing.assert_allclose(got, alpha[None] * feat[:, None, None], atol=1e-14)
    assert alpha.max() > 0.1


# ---- frequency-adaptive density control (Sec. 3.4.2) -----------------------------------------
def _densify_loop(prims, acc, den, noise, cfg):
    """The rules written per primitive with float32 scalars, output segments built by appending."""
    f32 = np.float32
    orig, clones, kids = [], [], []
    for i in range(prims["means"].shape[0]):
        g = f32(acc[i]) / f32(den[i]) if den[i] > 0 else f32(0)
        s = [f32(v) for v in prims["scales"][i]]
        smax = max(s)
        cand = g >= f32(cfg["grad_threshold"])
        low = f32(prims["opacity"][i]) < f32(cfg["min_opacity"])
        ms = f32(cfg["max_scale"])
        too_big = lambda m: ms > 0 and m > ms
        split = cand and smax > f32(cfg["dense_scale"])
        if not split and not low and not too_big(smax):
            orig.append(i)
            if cand:
                clones.append(i)
        if split and not low and not too_big(max(v / f32(cfg["split_divisor"]) for v in s)):
            kids.append(i)
    return orig, clones, kids


def _densify_inputs(seed, n=80):
    rng = np.random.default_rng(seed)
    prims = tiny_scene(seed, n=n, K=2, log_scale=(-3.0, 0.5))
    prims["opacity"][: n // 8] = rng.random(n // 8).astype(np.float32) * 0.02   # some below 0.01
    acc = (rng.random(n) * 2e-3).astype(np.float32)
    den = rng.integers(0, 4, n).astype(np.float32)
    return prims, acc, den, rng.standard_normal((n, 2, 3))


def _golden_f32(v):
    if isinstance(v, dict):
        (k, x), = v.items()
        return np.nextafter(np.float32(x), np.float32(0.0 if k == "below" else np.inf))
    return np.float32(v)


@pytest.mark.parametrize("case", [0, 1])
def test_densify_hand_worked_cases(case):
    """Decisions, output order and new rows against cases worked by hand from the paper's rules and
    values (tests/golden/densify_cases.json): the >= / > edges at the gradient threshold, at
    dense_scale and at the 0.01 opacity threshold; pruning by max_scale of originals, clones and
    split children; children's scale s / 1.6 and position mu + R (s z); new primitives' frequency
    0.001 and weight 0.01 (supplement B)."""
    g = json.load(open(os.path.join(GOLDEN, "densify_cases.json")))
    rows, want = g["primitives"], g["cases"][case]
    n, K = len(rows), 2
    prims = dict(
        means=np.array([r.get("means", [0.0, 0.0, 0.0]) for r in rows], np.float32),
        scales=np.array([[_golden_f32(v) for v in r["scales"]] for r in rows], np.float32),
        quats=np.tile(np.array([1.0, 0.0, 0.0, 0.0], np.float32), (n, 1)),
        opacity=np.array([_golden_f32(r["opacity"]) for r in rows], np.float32),
        sh=np.arange(n * 4 * 3, dtype=np.float32).reshape(n, 4, 3),
        freqs=np.full((n, K, 3), 0.7, np.float32), weights=np.full((n, K), 0.4, np.float32))
    acc = np.array([_golden_f32(r["acc"]) for r in rows], np.float32)
    den = np.array([r["den"] for r in rows], np.float32)
    noise = np.zeros((n, 2, 3))
    for r in rows:
        if "noise" in r:
            noise[r["i"]] = r["noise"]
    cfg = dict(O.densify_defaults(), **g["config"], max_scale=want["max_scale"])
    out, cnt = O.densify(prims, acc, den, noise, cfg)
    assert cnt == dict(originals=len(want["originals"]), clones=len(want["clones"]),
                       children=2 * len(want["children"]))
    src = want["originals"] + want["clones"] + [i for i in want["children"] for _ in (0, 1)]
    np.testing.assert_array_equal(out["sh"], prims["sh"][src])          # rows in the stated order
    np.testing.assert_array_equal(out["opacity"], prims["opacity"][src])
    no = len(want["originals"])
    np.testing.assert_array_equal(out["freqs"][:no], np.float32(0.7))
    np.testing.assert_array_equal(out["weights"][:no], np.float32(0.4))
    assert np.all(out["freqs"][no:] == np.float32(0.001)) and np.all(out["weights"][no:] == np.float32(0.01))
    ch0 = no + len(want["clones"])
    for i, sx in want["child_scale_x"].items():
        k = ch0 + 2 * want["children"].index(int(i))
        assert out["scales"][k, 0] == np.float32(sx) and out["scales"][k + 1, 0] == np.float32(sx)
    for i, pos in want["child_means"].items():
        k = ch0 + 2 * want["children"].index(int(i))
        np.testing.assert_allclose(out["means"][k:k + 2], pos, atol=1e-7)


def test_densify_hand_worked_accumulate_and_reset():
    g = json.load(open(os.path.join(GOLDEN, "densify_cases.json")))
    a = g["accumulate"]
    acc, den = O.densify_accumulate(np.array(a["acc"], np.float32), np.array(a["den"], np.float32),
                                    np.array(a["grad"], np.float32), np.array(a["visible"]))
    np.testing.assert_allclose(acc, a["acc_after"], rtol=1e-6)
    np.testing.assert_array_equal(den, a["den_after"])
    r = g["periodic_reset"]
    p = dict(opacity=np.array(r["opacity"], np.float32), weights=np.full((4, 2), 0.6, np.float32))
    out = O.reset_opacity_weights(p)
    np.testing.assert_array_equal(out["opacity"], np.array(r["opacity_after"], np.float32))
    assert np.all(out["weights"] == np.float32(r["weight_after"]))


@pytest.mark.parametrize("seed,max_scale", [(21, 0.0), (22, 0.12)])
def test_densify_vectorised_rules_match_per_primitive_loop(seed, max_scale):
    """A vectorisation check only (the rules themselves are pinned by the hand-worked cases): the
    array form of the rules gives the per-primitive loop's segments on random inputs."""
    prims, acc, den, noise = _densify_inputs(seed)
    cfg = dict(O.densify_defaults(dense_scale=0.06), max_scale=max_scale)
    out, cnt = O.densify(prims, acc, den, noise, cfg)
    orig, clones, kids = _densify_loop(prims, acc, den, noise, cfg)
    assert (cnt["originals"], cnt["clones"], cnt["children"]) == (len(orig), len(clones), 2 * len(kids))
    assert len(orig) and len(clones) and len(kids) and len(orig) < prims["means"].shape[0]
    src = orig + clones + [i for i in kids for _ in (0, 1)]
    for k in ("quats", "opacity", "sh"):
        np.testing.assert_array_equal(out[k], np.asarray(prims[k])[src])
    no = len(orig)
    np.testing.assert_array_equal(out["freqs"][:no], prims["freqs"][orig])
    np.testing.assert_array_equal(out["weights"][:no], prims["weights"][orig])
    assert np.all(out["freqs"][no:] == np.float32(1e-3)) and np.all(out["weights"][no:] == np.float32(1e-2))
    nc = no + len(clones)
    np.testing.assert_array_equal(out["means"][:nc], np.asarray(prims["means"], np.float64)[orig + clones])
    np.testing.assert_array_equal(out["scales"][:nc], prims["scales"][orig + clones])
    np.testing.assert_array_equal(out["scales"][nc:], np.repeat(prims["scales"][kids], 2, 0) / np.float32(1.6))


def test_densify_split_children_geometry():
    """Children sit at mu + R(q) (s * z): with antithetic noise (z, -z) they average to the parent,
    and R^T (child - mu) / s recovers z (R from scipy's quaternion convention, scalar last)."""
    from scipy.spatial.transform import Rotation
    prims, acc, den, noise = _densify_inputs(23)
    noise[:, 1] = -noise[:, 0]
    cfg = O.densify_defaults(dense_scale=0.06)
    out, cnt = O.densify(prims, acc, den, noise, cfg)
    _, _, kids = _densify_loop(prims, acc, den, noise, cfg)
    ch = out["means"][cnt["originals"] + cnt["clones"]:].reshape(-1, 2, 3)
    mu = np.asarray(prims["means"], np.float64)[kids]
    np.testing.assert_allclose(ch.mean(1), mu, atol=1e-12)
    q = np.asarray(prims["quats"], np.float64)[kids]
    R = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    z = np.einsum("nji,nj->ni", R, ch[:, 0] - mu) / prims["scales"][kids].astype(np.float64)
    np.testing.assert_allclose(z, noise[kids, 0], atol=1e-9)


def test_densify_special_cases_accumulate_and_reset():
    prims, acc, den, noise = _densify_inputs(24)
    cfg = O.densify_defaults(dense_scale=0.06)
    n = prims["means"].shape[0]
    # no statistics: nothing is densified, only low-opacity primitives go
    out, cnt = O.densify(prims, np.zeros(n, np.float32), np.zeros(n, np.float32), noise, cfg)
    keep = prims["opacity"] >= np.float32(0.01)
    assert cnt == dict(originals=int(keep.sum()), clones=0, children=0)
    np.testing.assert_array_equal(out["sh"], prims["sh"][keep])
    # everything below the opacity threshold: nothing survives
    out, cnt = O.densify(dict(prims, opacity=np.zeros(n, np.float32)), acc, den, noise, cfg)
    assert cnt == dict(originals=0, clones=0, children=0)
    # accumulation: visible primitives add |g| and one visit, the others are unchanged
    rng = np.random.default_rng(5)
    g = rng.standard_normal((n, 2)).astype(np.float32)
    vis = rng.random(n) < 0.5
    a2, d2 = O.densify_accumulate(acc, den, g, vis)
    np.testing.assert_allclose(a2[vis], acc[vis] + np.hypot(g[vis, 0], g[vis, 1]), rtol=1e-6)
    np.testing.assert_array_equal(a2[~vis], acc[~vis])
    np.testing.assert_array_equal(d2, den + vis)
    # periodic reset
    r = O.reset_opacity_weights(prims)
    np.testing.assert_array_equal(r["opacity"], np.minimum(prims["opacity"], np.float32(0.02)))
    assert np.all(r["weights"] == np.float32(0.01))



# ---- the z-attenuation variant (supplement A.2 with C2 kept) ---------------------------------
@pytest.mark.parametrize("seed", [3, 4])
def test_z_attenuation_variant_is_the_z_integral(seed):
    """With C2 kept, the 2D bank (1 - w) + w C2 cos(2 pi f2D.(x, y)) is the z-integral of the 3D
    primitive's bank weighted by its envelope, divided by the z-integral of the envelope
    (adaptive quadrature), so C1 cancels and only C2 remains."""
    from scipy.integrate import quad
    rng = np.random.default_rng(200 + seed)
    A = rng.standard_normal((3, 3))
    sigma = A @ A.T + 0.3 * np.eye(3)
    f = rng.normal(0, 0.4, 3)
    S22 = np.linalg.inv(sigma)[2, 2]
    f *= math.sqrt(0.7 * S22 / (2 * math.pi ** 2 * f[2] ** 2))   # 2 pi^2 f_z^2 / S22 = 0.7
    w = 0.7
    f2d = O.splat_frequency(t64(f[None, None, :]), t64(sigma[None])).numpy()[0, 0]
    C2 = float(O.z_attenuation(t64(f[None, None, :]), t64(sigma[None])).numpy()[0, 0])
    S = np.linalg.inv(sigma)
    assert abs(C2 - math.exp(-0.7)) < 1e-12
    for _ in range(5):
        x, y = rng.normal(0, 1.0, 2)
        env = lambda z: math.exp(-0.5 * np.array([x, y, z]) @ S @ np.array([x, y, z]))
        num, _ = quad(lambda z: env(z) * ((1 - w) + w * math.cos(2 * math.pi * (f @ np.array([x, y, z])))),
                      -np.inf, np.inf, epsabs=1e-14, epsrel=1e-12, limit=400)
        den, _ = quad(env, -np.inf, np.inf, epsabs=1e-14, epsrel=1e-12, limit=400)
        bank = (1 - w) + w * C2 * math.cos(2 * math.pi * (f2d @ np.array([x, y])))
        assert abs(num / den - bank) < 1e-9, (num / den, bank)


def test_z_attenuation_variant_render_brute_force():
    cam = tiny_camera(40, 32, dist=2.0)
    cfg = O.default_config(z_atten=True)
    prims = tiny_scene(9, n=24, K=2, log_scale=(-2.2, 0.4))
    prims["freqs"] = prims["freqs"] * 6.0                  # frequencies high enough to be attenuated
    out = O.render(prims, cam, cfg)
    img, T, _ = _brute_force(prims, cam, cfg)
    np.testing.assert_allclose(out["image"].numpy(), img, atol=1e-12)
    plain = O.render(prims, cam, O.default_config())["image"].numpy()
    assert np.abs(plain - img).max() > 1e-3                # and it differs from the method
    proj = O.project(O._to_f64(prims), cam, cfg)
    c2 = (proj["cos_weights"] / proj["weights"]).detach().numpy()
    assert np.all(c2 <= 1.0) and c2.min() < 0.9


def _fma32(a, b, c):
    """float32 fused multiply-add: the float32 product is exact in float64, so one float64 sum then
    one rounding to float32 (a double rounding differs from a single one only at float64 ties)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def test_phase_rounding_bound_covers_a_float32_evaluation():
    """phase_rounding_bound against a float32 emulation of the compositing kernels' phase:
    d = x - mu, F = 2 pi f, theta = F_x d_x + F_y d_y (a product and a fused sum), and in a block
    (8 x 8 pixels) where some |f . (x - mu)| can exceed 2 cycles, theta reduced by whole cycles
    (t = theta / (2 pi), 2 pi (t - rint t)).  The float32 angle stays within the bound of the exact
    phase 2 pi f . (x - mu) of the same float32 inputs (modulo 2 pi), over means up to 600 pixels
    away and frequencies up to about 1 cycle per pixel (both paths taken)."""
    f32 = np.float32
    rng = np.random.default_rng(11)
    two_pi, inv_two_pi = f32(2 * np.pi), f32(1 / (2 * np.pi))
    n_slow = n_fast = 0
    ratio = 0.0
    for trial in range(40):
        L = 64
        mu = (rng.uniform(-600, 600, (L, 2)) * rng.choice([0.01, 0.1, 1.0], (L, 1)) + 40).astype(f32)
        f = (rng.standard_normal((L, 1, 2)) * rng.choice([0.01, 0.1, 0.3], (L, 1, 1))).astype(f32)
        tx, ty = rng.integers(0, 6, 2)
        xs, ys = np.meshgrid(np.arange(16 * tx, 16 * tx + 16), np.arange(16 * ty, 16 * ty + 16))
        px, py = xs.reshape(-1) + 0.5, ys.reshape(-1) + 0.5
        bound = O.phase_rounding_bound(torch.tensor(px), torch.tensor(py), torch.tensor(mu, dtype=torch.float64),
                                       torch.tensor(f, dtype=torch.float64)).numpy()[:, :, 0]
        fx, fy = f[None, :, 0, 0], f[None, :, 0, 1]
        dx = (px.astype(f32)[:, None] - mu[None, :, 0]).astype(f32)
        dy = (py.astype(f32)[:, None] - mu[None, :, 1]).astype(f32)
        Fx, Fy = (two_pi * fx).astype(f32), (two_pi * fy).astype(f32)
        theta = _fma32(np.broadcast_to(Fx, dx.shape), dx, (Fy * dy).astype(f32))
        # the block's range-reduction decision, from float32 bounds of |f . (x - mu)| over its pixels
        x0, y0 = (8 * np.floor(px / 8) + 0.5).astype(f32), (8 * np.floor(py / 8) + 0.5).astype(f32)
        ax = np.maximum(np.abs(x0[:, None] - mu[None, :, 0]), np.abs(x0[:, None] + f32(7) - mu[None, :, 0]))
        ay = np.maximum(np.abs(y0[:, None] - mu[None, :, 1]), np.abs(y0[:, None] + f32(7) - mu[None, :, 1]))
        slow = (np.abs(fx) * ax + np.abs(fy) * ay).astype(f32) > f32(2.0)
        t = (theta * inv_two_pi).astype(f32)
        theta = np.where(slow, (two_pi * (t - np.rint(t)).astype(f32)).astype(f32), theta)
        n_slow += int(slow.sum())
        n_fast += int((~slow).sum())
        exact = 2 * np.pi * (fx.astype(np.float64) * (px[:, None] - mu[None, :, 0]) +
                             fy.astype(np.float64) * (py[:, None] - mu[None, :, 1]))
        d = np.abs(np.angle(np.exp(1j * (theta.astype(np.float64) - exact))))
        assert (d <= bound).all(), float((d / bound).max())
        ratio = max(ratio, float((d / bound).max()))
    assert n_slow > 1000 and n_fast > 1000
    assert ratio > 0.2   # the bound is not vacuous
