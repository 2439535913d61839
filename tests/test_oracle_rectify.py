"""Pins of the oracle's rectification and depth registration (arxiv
2201.11924 Sec. VI-D names both; the camera model is a reading: pinhole with
Brown-Conrady distortion, fixed-point bilinear resampling, nearest-pixel
z-buffered splatting).

The pins are exact geometric cases (identity, integer shifts, a quarter turn,
a half-pixel shift against a library bilinear interpolation), the distortion
polynomial at points where it is known in closed form, and the z-buffer and
coverage properties of the registration."""
import numpy as np
import pytest
import scipy.ndimage

import oracle


def _img(H=40, W=48, seed=1):
    return np.random.default_rng(seed).integers(0, 256, (H, W), dtype=np.uint8)


@pytest.mark.parametrize("fx,fy", [(300.0, 300.0), (250.0, 400.0)])
def test_identity_camera_returns_the_image(fx, fy):
    img = _img()
    cam = oracle.camera(fx, fy, 23.5, 19.5)
    assert np.array_equal(oracle.rectify(img, cam), img)


@pytest.mark.parametrize("dx,dy", [(3, 0), (0, -2), (-5, 4)])
def test_principal_point_shift_is_an_integer_translation(dx, dy):
    # rectified cx' = cx + dx maps rectified u to raw u - dx
    img = _img(seed=100 + dx * 10 + dy)
    H, W = img.shape
    cam = oracle.camera(250.0, 250.0, 20.0, 18.0, rcx=20.0 + dx, rcy=18.0 + dy)
    out = oracle.rectify(img, cam)
    want = np.zeros_like(img)
    ys, xs = np.mgrid[0:H, 0:W]
    sx, sy = xs - dx, ys - dy
    ok = (sx >= 0) & (sx < W) & (sy >= 0) & (sy < H)
    want[ok] = img[sy[ok], sx[ok]]
    assert np.array_equal(out, want)


def test_quarter_turn_about_the_axis_rotates_the_image():
    img = _img(32, 32, seed=4)
    c = 15.5                                   # centre of a 32 x 32 image
    R = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]     # rectified ray = R raw ray
    out = oracle.rectify(img, oracle.camera(100.0, 100.0, c, c, R=R))
    # raw ray = R^T rectified ray = (yr, -xr, 1): out[v, u] = img[2c - u, v],
    # the image turned a quarter clockwise
    assert np.array_equal(out, np.rot90(img, k=-1))


def test_half_pixel_shift_matches_library_bilinear():
    img = _img(seed=7)
    H, W = img.shape
    cam = oracle.camera(200.0, 200.0, 22.0, 17.0, rcx=22.5, rcy=17.25)
    out = oracle.rectify(img, cam).astype(int)
    ys, xs = np.mgrid[0:H, 0:W].astype(float)
    ref = scipy.ndimage.map_coordinates(img.astype(float), [ys - 0.25, xs - 0.5], order=1, mode="constant", cval=0)
    inner = (slice(1, H - 1), slice(1, W - 1))
    assert np.abs(out[inner] - ref[inner]).max() <= 0.5 + 1e-9   # the fixed point holds 1/256 steps


def test_radial_distortion_moves_points_by_the_polynomial():
    # on the x axis y = 0: x_d = x (1 + k1 x^2 + k2 x^4 + k3 x^6); a raw image
    # that is a ramp in x (value = raw column) reads back the distorted column
    # (x reaches 1.5, where each of the three terms moves the point by more
    # than a pixel)
    W, H = 64, 9
    ramp = np.tile(np.arange(W, dtype=np.uint8), (H, 1))
    f, cx, cy = 20.0, 4.0, 4.0
    k1, k2, k3 = 0.05, -0.02, 0.01
    out = oracle.rectify(ramp, oracle.camera(f, f, cx, cy, k1=k1, k2=k2, k3=k3))
    for u in (10, 15, 20, 25, 30, 34):
        x = (u - cx) / f
        ur = f * x * (1 + k1 * x * x + k2 * x ** 4 + k3 * x ** 6) + cx
        assert abs(int(out[4, u]) - ur) <= 0.5 + 1.0 / 256, u


def test_tangential_terms_are_symmetric_in_their_axes():
    # Brown-Conrady on an axis: p1 alone shifts v on the y axis by p1 (3 y^2)
    # and leaves u on the x axis alone; p2 alone does the same with the axes
    # exchanged (shifts of 1-3 px here, well above the rounding)
    W, H = 40, 40
    rampx = np.tile(np.arange(W, dtype=np.uint8), (H, 1))
    rampy = rampx.T.copy()
    f, c, p = 30.0, 8.0, 0.1
    for p1, p2 in ((0.0, p), (p, 0.0)):
        cam = oracle.camera(f, f, c, c, p1=p1, p2=p2)
        outx, outy = oracle.rectify(rampx, cam), oracle.rectify(rampy, cam)
        for t in (12, 18, 24):
            x = (t - c) / f
            # along the x axis (v = c) the column read moves by p2 (3 x^2) only
            assert abs(int(outx[int(c), t]) - (f * (x + p2 * 3 * x * x) + c)) <= 0.5 + 1.0 / 256
            # along the y axis (u = c) the row read moves by p1 (3 y^2) only
            assert abs(int(outy[t, int(c)]) - (f * (x + p1 * 3 * x * x) + c)) <= 0.5 + 1.0 / 256


def test_registration_identity_and_zbuffer():
    rng = np.random.default_rng(2)
    depth = rng.uniform(0.4, 2.0, (30, 40)).astype(np.float32)
    depth[rng.random(depth.shape) < 0.2] = 0.0
    f, cx, cy = 100.0, 19.5, 14.5
    same = oracle.register(depth, f, f, cx, cy, f, f, cx, cy, np.eye(3), [0, 0, 0], 40, 30)
    assert np.array_equal(same, depth)
    # a camera half the focal length: 2x2 depth blocks land on one pixel, the nearest wins
    half = oracle.register(depth, f, f, cx, cy, f / 2, f / 2, cx / 2 - 0.25, cy / 2 - 0.25, np.eye(3), [0, 0, 0], 20, 15)
    blocks = np.where(depth > 0, depth, np.inf).reshape(15, 2, 20, 2).min(axis=(1, 3))
    want = np.where(np.isfinite(blocks), blocks, 0).astype(np.float32)
    assert np.array_equal(half, want)


def test_registration_translation_along_the_axis():
    # a fronto-parallel plane at Z moved by tz: every pixel keeps its ray
    # direction scaled by Z / (Z + tz) about the principal point, depth Z + tz
    depth = np.full((21, 31), 1.5, dtype=np.float32)
    f, cx, cy, tz = 80.0, 15.0, 10.0, 1.5
    out = oracle.register(depth, f, f, cx, cy, f, f, cx, cy, np.eye(3), [0, 0, tz], 31, 21)
    filled = out > 0
    assert np.allclose(out[filled], 3.0)
    # the plane shrinks by half about the principal point: columns 8..22 only
    cols = np.flatnonzero(filled.any(axis=0))
    assert cols.min() >= 7 and cols.max() <= 23 and filled.sum() == len(np.unique(np.floor((np.arange(31) - cx) / 2 + cx + 0.5))) * len(np.unique(np.floor((np.arange(21) - cy) / 2 + cy + 0.5)))


@pytest.mark.parametrize("tx,ty", [(0.05, 0.0), (0.0, -0.075), (0.05, 0.025)])
def test_registration_sideways_translation_shifts_the_image(tx, ty):
    # the RGB camera sees the point X + t: on a fronto-parallel plane at Z
    # every pixel moves by (f tx / Z, f ty / Z) = whole pixels here, with its
    # depth unchanged
    depth = np.full((21, 31), 2.0, dtype=np.float32)
    f, cx, cy, Z = 80.0, 15.0, 10.0, 2.0
    out = oracle.register(depth, f, f, cx, cy, f, f, cx, cy, np.eye(3), [tx, ty, 0.0], 31, 21)
    sx, sy = int(round(f * tx / Z)), int(round(f * ty / Z))
    want = np.zeros_like(depth)
    want[max(sy, 0):21 + min(sy, 0), max(sx, 0):31 + min(sx, 0)] = Z
    assert np.array_equal(out, want)


def test_registration_camera_facing_away_sees_nothing():
    # turned half a turn about the y axis, the RGB camera looks away from every
    # point in front of the depth camera (Z' = -Z < 0): nothing is splatted
    depth = np.full((12, 16), 1.2, dtype=np.float32)
    R = [[-1, 0, 0], [0, 1, 0], [0, 0, -1]]
    out = oracle.register(depth, 50.0, 50.0, 7.5, 5.5, 50.0, 50.0, 7.5, 5.5, np.array(R, float), [0, 0, 0], 16, 12)
    assert not out.any()


def test_registration_through_an_anisotropic_rgb_camera():
    # one depth pixel (u, v) = (12, 3) at Z through the pinhole model:
    # X = (u - cx) / f Z, Y = (v - cy) / f Z; the RGB camera (fx2 = 100,
    # fy2 = 50, cx2 = 20, cy2 = 5.5) sees it at (100 * 4.5 / 50 + 20,
    # 50 * (-2.5) / 50 + 5.5) = (29, 3)
    depth = np.zeros((12, 16), dtype=np.float32)
    depth[3, 12] = 1.75
    out = oracle.register(depth, 50.0, 50.0, 7.5, 5.5, 100.0, 50.0, 20.0, 5.5, np.eye(3), [0, 0, 0], 40, 12)
    assert list(zip(*np.nonzero(out))) == [(3, 29)] and out[3, 29] == np.float32(1.75)
