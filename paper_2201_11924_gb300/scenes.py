"""Seeded synthetic rectified IR pairs (random-dot active stereo scenes).

This module stands in for the paper's ray-traced IR rendering with a textured
spot-light projector (Sec. VI-A/VI-B) and its sensor-noise step (Sec. VI-C,
here reduced to additive Gaussian noise): it ray-casts analytic scenes on the
CPU with numpy.  It holds none of the depth stage's arithmetic (no census, no
matching cost, no aggregation, no selection); both the CUDA path and the CPU
oracle take its images as their inputs.

Camera model: pinhole, fx = fy = f, cx = (W-1)/2, cy = (H-1)/2.  The left
camera sits at the origin looking down +Z, the right one at (+b, 0, 0), so a
point at depth Z appears at x_r = x_l - f b / Z on the same row.  The
projector sits with the left camera and throws an H x W random-dot pattern
(dot probability, dot and background intensity ranges from the scene recipe).

Left pixel value   = albedo * pattern(x, y) of the surface its ray hits.
Right pixel value  = albedo * pattern(x_l, y), linearly interpolated in x,
                     when the right ray's hit point is also seen by the left
                     camera; otherwise albedo * a background-only value.
"Translucent-like" objects use albedo * (40 + c * (pattern - 40)) with a
small contrast c, so their dots nearly vanish.  Each view then gets
independent N(0, sigma^2) noise, is rounded half to even and clamped to
[0, 255].  Random numbers come from numpy's PCG64 (``default_rng(seed)``).
"""
from __future__ import annotations

import numpy as np

from .configs import Scene, Workload


def _rays(W, H, f):
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    xs = (np.arange(W, dtype=np.float64) - cx) / f
    ys = (np.arange(H, dtype=np.float64) - cy) / f
    dx = np.broadcast_to(xs[None, :], (H, W))
    dy = np.broadcast_to(ys[:, None], (H, W))
    return dx, dy


def _make_objects(rng, W, H, f, sc: Scene):
    """Random objects: dicts with kind, geometry, albedo and translucency."""
    objs = []
    zr = sc.z_max - sc.z_min
    albedo = lambda: float(rng.uniform(sc.albedo_lo, sc.albedo_hi)) if sc.albedo_hi > sc.albedo_lo else float(sc.albedo_lo)
    # back wall: full frame, fronto-parallel, Z from the top 20% of the range
    zw = float(rng.uniform(sc.z_max - 0.2 * zr, sc.z_max))
    objs.append(dict(kind="wall", z=zw, albedo=albedo(), translucent=False))
    n_obj = (sc.n_planes - 1) + sc.n_spheres
    kinds = ["plane"] * (sc.n_planes - 1) + ["sphere"] * sc.n_spheres
    for k in kinds[:n_obj]:
        z = float(rng.uniform(sc.z_min, sc.z_min + 0.8 * zr))
        px = float(rng.uniform(0.1 * W, 0.9 * W))
        py = float(rng.uniform(0.1 * H, 0.9 * H))
        cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
        centre = np.array([(px - cx) / f * z, (py - cy) / f * z, z])
        translucent = bool(rng.random() < sc.translucent_frac)
        if k == "plane":
            tilt = np.deg2rad(float(rng.uniform(0.0, 30.0)))
            az = float(rng.uniform(0.0, 2 * np.pi))
            n = np.array([np.sin(tilt) * np.cos(az), np.sin(tilt) * np.sin(az), -np.cos(tilt)])
            # in-plane axes
            a = np.cross(n, [0.0, 1.0, 0.0])
            a /= np.linalg.norm(a)
            bvec = np.cross(n, a)
            frac = float(rng.uniform(0.10, 0.40))
            area = frac * W * H * (z / f) ** 2
            aspect = float(rng.uniform(0.5, 2.0))
            hu = 0.5 * np.sqrt(area * aspect)
            hv = 0.5 * np.sqrt(area / aspect)
            objs.append(dict(kind="plane", c=centre, n=n, u=a, v=bvec, hu=hu, hv=hv,
                             albedo=albedo(), translucent=translucent))
        else:
            r = float(rng.uniform(0.03, 0.15))
            objs.append(dict(kind="sphere", c=centre, r=r, albedo=albedo(), translucent=translucent))
    return objs


def _hit_t(obj, ox, dx, dy):
    """Ray parameter t (= depth Z, rays have unit z) of the hit, +inf if none.

    Rays start at (ox, 0, 0) with direction (dx, dy, 1)."""
    inf = np.inf
    if obj["kind"] == "wall":
        return np.full(dx.shape, obj["z"])
    if obj["kind"] == "plane":
        n, c = obj["n"], obj["c"]
        denom = n[0] * dx + n[1] * dy + n[2]
        num = n[0] * (c[0] - ox) + n[1] * c[1] + n[2] * c[2]
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(np.abs(denom) > 1e-12, num / denom, inf)
        hx = ox + t * dx - c[0]
        hy = t * dy - c[1]
        hz = t - c[2]
        pu = hx * obj["u"][0] + hy * obj["u"][1] + hz * obj["u"][2]
        pv = hx * obj["v"][0] + hy * obj["v"][1] + hz * obj["v"][2]
        ok = (t > 1e-6) & (np.abs(pu) <= obj["hu"]) & (np.abs(pv) <= obj["hv"])
        return np.where(ok, t, inf)
    # sphere
    c, r = obj["c"], obj["r"]
    ocx, ocy, ocz = ox - c[0], -c[1], -c[2]
    a = dx * dx + dy * dy + 1.0
    b = dx * ocx + dy * ocy + ocz
    cc = ocx * ocx + ocy * ocy + ocz * ocz - r * r
    disc = b * b - a * cc
    with np.errstate(invalid="ignore"):
        t = (-b - np.sqrt(np.maximum(disc, 0.0))) / a
    ok = (disc >= 0) & (t > 1e-6)
    return np.where(ok, t, inf)


def _nearest(objs, ox, dx, dy):
    best = np.full(dx.shape, np.inf)
    idx = np.full(dx.shape, -1, dtype=np.int64)
    for i, o in enumerate(objs):
        t = _hit_t(o, ox, dx, dy)
        closer = t < best
        best = np.where(closer, t, best)
        idx = np.where(closer, i, idx)
    return best, idx


def _shade(pattern_val, albedo, translucent, contrast):
    return np.where(translucent, albedo * (40.0 + contrast * (pattern_val - 40.0)), albedo * pattern_val)


def make_pattern(rng, W, H, sc: Scene):
    dots = rng.random((H, W)) < sc.dot_density
    dot_v = rng.integers(sc.dot_lo, sc.dot_hi + 1, size=(H, W))
    bg_v = rng.integers(sc.bg_lo, sc.bg_hi + 1, size=(H, W))
    return np.where(dots, dot_v, bg_v).astype(np.float64)


def _noisy_u8(rng, img, sigma):
    if sigma > 0:
        img = img + rng.normal(0.0, sigma, size=img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def make_pair(wl: Workload, seed: int | None = None):
    """Render one seeded pair for workload ``wl``.

    Returns dict(left, right: uint8 H x W; depth_gt, disp_gt: float64 H x W
    for the left view)."""
    sc = wl.scene
    rng = np.random.default_rng(wl.seed if seed is None else seed)
    W, H, f, b = wl.W, wl.H, float(wl.f), float(wl.baseline)
    objs = _make_objects(rng, W, H, f, sc)
    pattern = make_pattern(rng, W, H, sc)
    bg_only = rng.integers(sc.bg_lo, sc.bg_hi + 1, size=(H, W)).astype(np.float64)
    alb = np.array([o["albedo"] for o in objs])
    trans = np.array([o["translucent"] for o in objs])
    dx, dy = _rays(W, H, f)

    # left view: the projector shares the left camera's rays
    tl, il = _nearest(objs, 0.0, dx, dy)
    left = _shade(pattern, alb[il], trans[il], sc.translucent_contrast)

    # right view: cast, re-project the hit into the left camera, test visibility
    tr, ir = _nearest(objs, b, dx, dy)
    px = b + tr * dx                      # hit point (px, py, pz = tr)
    xl = f * px / tr + (W - 1) / 2.0      # its column in the left image (same row)
    dxl = px / tr
    tl2, _ = _nearest(objs, 0.0, dxl, dy)
    visible = (tl2 >= tr * (1.0 - 1e-9) - 1e-9) & (xl >= 0.0) & (xl <= W - 1)
    x0 = np.clip(np.floor(xl), 0, W - 1).astype(np.int64)
    x1 = np.clip(x0 + 1, 0, W - 1)
    wgt = np.clip(xl - x0, 0.0, 1.0)
    rows = np.broadcast_to(np.arange(H)[:, None], (H, W))
    pat_r = (1.0 - wgt) * pattern[rows, x0] + wgt * pattern[rows, x1]
    lit = _shade(pat_r, alb[ir], trans[ir], sc.translucent_contrast)
    right = np.where(visible, lit, alb[ir] * bg_only)

    left_u8 = _noisy_u8(rng, left, sc.noise_sigma)
    right_u8 = _noisy_u8(rng, right, sc.noise_sigma)
    depth_gt = tl
    disp_gt = f * b / tl
    return dict(left=left_u8, right=right_u8, depth_gt=depth_gt, disp_gt=disp_gt)


def make_plane_pair(W: int, H: int, d0: int, seed: int, sc: Scene | None = None, sigma: float = 0.0):
    """A fronto-parallel plane at integer disparity d0 filling the frame.

    right(x, y) = left(x + d0, y) where x + d0 < W; the strip the left camera
    does not see gets background-only values.  Used for exact-recovery tests."""
    sc = sc or Scene()
    rng = np.random.default_rng(seed)
    pattern = make_pattern(rng, W, H, sc)
    bg_only = rng.integers(sc.bg_lo, sc.bg_hi + 1, size=(H, W)).astype(np.float64)
    right = bg_only.copy()
    if d0 < W:
        right[:, : W - d0] = pattern[:, d0:]
    return dict(left=_noisy_u8(rng, pattern, sigma), right=_noisy_u8(rng, right, sigma))


def make_multiplane_pair(W: int, H: int, disps, seed: int, sc: Scene | None = None):
    """Noise-free vertical bands, band k a fronto-parallel plane at integer
    disparity disps[k] (bands of equal width, left to right).

    right(x_r, y) = left(x_r + d(x_r + d), y) when that left pixel's band has
    disparity d; right pixels no left pixel maps to get background-only
    values.  Returns dict(left, right, disp_gt: int H x W for the left view)."""
    sc = sc or Scene()
    rng = np.random.default_rng(seed)
    pattern = make_pattern(rng, W, H, sc)
    bg_only = rng.integers(sc.bg_lo, sc.bg_hi + 1, size=(H, W)).astype(np.float64)
    nb = len(disps)
    band = np.minimum((np.arange(W) * nb) // W, nb - 1)
    dmap = np.asarray(disps, dtype=np.int64)[band]
    right = bg_only.copy()
    zbuf = np.full(W, -1, dtype=np.int64)   # larger disparity = nearer surface wins
    owner = np.full(W, -1, dtype=np.int64)
    for xl in range(W):
        xr = xl - dmap[xl]
        if 0 <= xr < W and dmap[xl] > zbuf[xr]:
            zbuf[xr] = dmap[xl]
            owner[xr] = xl
    has = owner >= 0
    right[:, has] = pattern[:, owner[has]]
    disp_gt = np.broadcast_to(dmap[None, :], (H, W)).copy()
    return dict(left=pattern.astype(np.uint8), right=right.astype(np.uint8), disp_gt=disp_gt)
