"""Pins of the oracle's IR renderer (arxiv 2201.11924 Sec. VI-A/VI-B: a
textured spot-light projector and the BSDF mix f = w_d f_d + (1 - w_d) f_s,
w_d = (1 - metallic)(1 - transmission); the direct-light ray caster and its
parameters are readings).

Pins: the cosine-cubed falloff of a fronto-parallel Lambertian wall lit from
the camera centre (closed form), the stereo shift d = f b / Z between the two
views, projector shadows and nearest hits against an independent ray-sphere
test, no shadow from behind the projector, Helmholtz reciprocity of the BSDF,
linearity of the mix in the transmission weight, and the specular highlight of
a glossy metal sphere at the point facing the light, and the Fresnel factor
of the specular lobe against the exact Fresnel equations of a dielectric
(n = 1.5): F0 = 0.04 at normal incidence, Schlick's exponent 5 within its
deviation from the exact reflectance from grazing to normal incidence."""
import numpy as np
import pytest

import oracle

W, H, F = 80, 60, 60.0
CX, CY = 40.0, 30.0


def _wall(Z, **mat):
    return oracle.rectangle((0, 0, Z), (5, 0, 0), (0, 5, 0), **mat)


def _render(prims, pattern, baseline=0.05, proj=(0, 0, 0), power=1.0, ambient=0.05, gain=400.0):
    return oracle.render(prims, pattern, W, H, F, CX, CY, baseline, proj, F, CX, CY, power, ambient, gain)


def test_lambert_wall_follows_the_cosine_cubed_law():
    rng = np.random.default_rng(1)
    pat = rng.integers(1, 256, (H, W), dtype=np.uint8)
    Z, albedo, power, amb, gain = 1.3, 0.7, 2.0, 0.05, 400.0
    _, _, lf, _ = _render([_wall(Z, albedo=albedo)], pat, power=power, ambient=amb, gain=gain)
    us, vs = np.meshgrid(np.arange(W), np.arange(H))
    dn = np.sqrt(((us - CX) / F) ** 2 + ((vs - CY) / F) ** 2 + 1.0)      # |d| of the pixel ray
    want = gain * (albedo / np.pi * power * (pat / 255.0) / (Z * Z * dn ** 3) + amb * albedo)
    np.testing.assert_allclose(lf, want, rtol=1e-12)


@pytest.mark.parametrize("Z", [0.5, 1.0])
def test_right_view_is_the_left_view_shifted_by_the_disparity(Z):
    # Lambertian radiance does not depend on the viewer: right(u) = left(u + f b / Z)
    rng = np.random.default_rng(2)
    pat = rng.integers(1, 256, (H, W), dtype=np.uint8)
    b = 5.0 * Z / F                                  # an integer disparity of 5 px
    _, _, lf, rf = _render([_wall(Z)], pat, baseline=b)
    np.testing.assert_allclose(rf[:, :W - 5], lf[:, 5:], rtol=1e-9)


def test_projector_shadow_of_a_sphere():
    pat = np.full((H, W), 255, dtype=np.uint8)
    Z, c, r = 1.0, np.array([0.05, 0.02, 0.5]), 0.08
    proj = np.array([0.02, 0.0, 0.0])
    amb, albedo, gain = 0.05, 0.6, 400.0
    wall = _wall(Z, albedo=albedo)
    ball = oracle.sphere(tuple(c), r, albedo=0.3)
    _, _, lf, _ = _render([wall, ball], pat, proj=tuple(proj), ambient=amb, gain=gain)
    # the sphere alone: the wall lies behind it, so it neither hides nor shadows it
    _, _, lf_ball, _ = _render([ball], pat, proj=tuple(proj), ambient=amb, gain=gain)
    us, vs = np.meshgrid(np.arange(W), np.arange(H))
    seen = 0
    for u, v in [(int(x), int(y)) for x, y in zip(us.ravel()[::7], vs.ravel()[::7])]:
        d = np.array([(u - CX) / F, (v - CY) / F, 1.0])
        # the camera ray first: pixels that see the sphere (nearer than the
        # wall) show the sphere, not the wall
        oc = -c
        bq, cq = 2 * d @ oc, oc @ oc - r * r
        if bq * bq - 4 * (d @ d) * cq >= 0:
            assert lf[v, u] == lf_ball[v, u] and lf_ball[v, u] > 0, (u, v)
            seen += 1
            continue
        p = Z * d                                    # the wall point
        X = p - proj                                 # outside the projector's texture: unlit anyway
        up, vp = np.floor(F * X[0] / X[2] + CX + 0.5), np.floor(F * X[1] / X[2] + CY + 0.5)
        if not (0 <= up < W and 0 <= vp < H):
            continue
        L = proj - p                                 # towards the projector: does it pass the sphere?
        pc = p - c
        a2, b2, c2 = L @ L, 2 * L @ pc, pc @ pc - r * r
        disc = b2 * b2 - 4 * a2 * c2
        shadowed = disc >= 0 and 0 < (-b2 - np.sqrt(disc)) / (2 * a2) < 1
        if shadowed:
            assert abs(lf[v, u] - gain * amb * albedo) < 1e-9, (u, v)
        else:
            assert lf[v, u] > gain * amb * albedo + 1.0, (u, v)
    assert seen > 10


def test_no_shadow_from_behind_the_projector():
    # only what lies between a point and the projector blocks its light: a
    # large panel behind the projector and the cameras changes nothing
    pat = np.full((H, W), 255, dtype=np.uint8)
    proj = (0.02, 0.0, 0.0)
    scene = [_wall(1.0, albedo=0.6), oracle.sphere((0.05, 0.02, 0.5), 0.08, albedo=0.3)]
    panel = oracle.rectangle((0.0, 0.0, -0.5), (3, 0, 0), (0, 3, 0), albedo=0.9)
    _, _, a, _ = _render(scene, pat, proj=proj)
    _, _, b, _ = _render(scene + [panel], pat, proj=proj)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("metallic,roughness", [(0.0, 0.3), (0.5, 0.25), (1.0, 0.4)])
def test_bsdf_is_reciprocal(metallic, roughness):
    # Helmholtz reciprocity: f(i, o) = f(o, i).  Light a fronto-parallel wall
    # at Z from the left camera's centre and look from the right camera, then
    # swap the two roles.  A wall point p seen at right pixel u is seen at
    # left pixel u + f b / Z; with ambient 0 and a uniform pattern its value
    # is gain f E, E = power (n.i) / |p - light|^2 and n.i = Z / |p - light|,
    # so value * |p - light|^3 must agree between the two renders.
    pat = np.full((H, W), 255, dtype=np.uint8)
    Z, disp = 0.8, 6
    b = disp * Z / F
    wall = _wall(Z, albedo=0.7, metallic=metallic, roughness=roughness)
    _, _, _, rf = _render([wall], pat, baseline=b, proj=(0.0, 0.0, 0.0), ambient=0.0)
    _, _, lf, _ = _render([wall], pat, baseline=b, proj=(b, 0.0, 0.0), ambient=0.0)
    for v in range(8, H - 8, 5):
        for u in range(8, W - disp - 8, 5):
            p = np.array([(u - CX) * Z / F + b, (v - CY) * Z / F, Z])
            da, db = np.linalg.norm(p), np.linalg.norm(p - np.array([b, 0.0, 0.0]))
            np.testing.assert_allclose(rf[v, u] * da ** 3, lf[v, u + disp] * db ** 3, rtol=1e-9)


def test_mix_is_linear_in_the_transmission_weight():
    rng = np.random.default_rng(3)
    pat = rng.integers(1, 256, (H, W), dtype=np.uint8)
    ball = dict(c=(0.0, 0.0, 0.8), radius=0.3, albedo=0.6, metallic=0.0, roughness=0.4)
    out = {}
    for t in (0.0, 0.35, 1.0):
        _, _, lf, _ = _render([_wall(1.5), oracle.sphere(transmission=t, **ball)], pat, ambient=0.0)
        out[t] = lf
    np.testing.assert_allclose(out[0.35], 0.65 * out[0.0] + 0.35 * out[1.0], rtol=1e-9, atol=1e-9)


def test_glossy_metal_highlight_faces_the_light():
    pat = np.full((H, W), 255, dtype=np.uint8)
    c = (0.03, -0.02, 0.7)
    _, _, lf, _ = _render([oracle.sphere(c, 0.2, albedo=0.9, metallic=1.0, roughness=0.15)], pat, ambient=0.0)
    v, u = np.unravel_index(np.argmax(lf), lf.shape)
    # projector at the camera centre: the mirror point lies on the line to the centre
    assert abs(u - (F * c[0] / c[2] + CX)) <= 1 and abs(v - (F * c[1] / c[2] + CY)) <= 1


def test_rays_that_miss_give_zero_and_rounding():
    pat = np.full((H, W), 255, dtype=np.uint8)
    l, r, lf, rf = _render([oracle.sphere((0, 0, 1.0), 0.1)], pat)
    assert l[0, 0] == 0 and lf[0, 0] == 0.0
    assert np.array_equal(l, np.clip(np.rint(lf), 0, 255).astype(np.uint8))


def test_rectangle_silhouette_is_its_projected_extent():
    # a fronto-parallel rectangle at Z = 1 with half-sizes 0.2 x 0.1 m, seen
    # by the f = 60 px left camera, covers |u - cx| <= 12, |v - cy| <= 6;
    # rays that miss give 0, hits at least the ambient term (pixels on the
    # edge itself are left out: the edge is one rounding away either way)
    pat = np.full((H, W), 255, dtype=np.uint8)
    rect = oracle.rectangle((0.0, 0.0, 1.0), (0.2, 0, 0), (0, 0.1, 0), albedo=0.5)
    _, _, lf, _ = _render([rect], pat, ambient=0.05)
    us, vs = np.meshgrid(np.arange(W), np.arange(H))
    du, dv = np.abs(us - CX), np.abs(vs - CY)
    inside, outside = (du < 12) & (dv < 6), (du > 12) | (dv > 6)
    assert (lf[inside] >= 400.0 * 0.05 * 0.5 - 1e-9).all()
    assert (lf[outside] == 0.0).all()


# --- the Fresnel factor of the specular term ---------------------------------
#
# Two renders of the same geometry that differ only in the material isolate the
# Fresnel factor F of the specular lobe: with transmission 1 (dielectric,
# metallic 0) the diffuse weight w_d is 0 and F0 is the dielectric one; with
# metallic 1 and albedo 1, w_d is 0 again and F0 = 1, so F = 1 at every angle.
# D, G, the light and the geometry are identical, so the ratio of the two
# unrounded radiances is the dielectric F at cos(theta_d) = v.h of the pixel.
# The reference is independent of the oracle: the exact Fresnel reflectance
# of unpolarised light at a dielectric of refractive index 1.5 (the usual
# value for the dielectrics the F0 = 0.04 convention stands for), from the
# Fresnel equations.

N_DIELECTRIC = 1.5


def _fresnel_exact(c, n=N_DIELECTRIC):
    """Unpolarised reflectance at incidence cos(theta) = c from the Fresnel
    equations (s and p averaged)."""
    s2 = 1.0 - c * c
    ct = np.sqrt(1.0 - s2 / (n * n))
    rs = ((c - n * ct) / (c + n * ct)) ** 2
    rp = ((n * c - ct) / (n * c + ct)) ** 2
    return 0.5 * (rs + rp)


def _fresnel_row(z0, b, Wr=401, f=8.0):
    """F of every pixel of a one-row render: camera at the origin, projector
    at (b, 0, 0), a wall z = z0 facing them; returns (cos theta_d, F)."""
    cx = (Wr - 1) / 2.0
    pat = np.full((1, 4001), 255, dtype=np.uint8)
    wall = dict(c=(b / 2.0, 0.0, z0), u=(50.0, 0.0, 0.0), v=(0.0, 50.0, 0.0), roughness=1.0)
    out = []
    for mat in (dict(albedo=0.6, metallic=0.0, transmission=1.0), dict(albedo=1.0, metallic=1.0, transmission=0.0)):
        _, _, lf, _ = oracle.render([oracle.rectangle(**wall, **mat)], pat, Wr, 1, f, cx, 0.0, 0.05,
                                    (b, 0.0, 0.0), 1.0, 2000.0, 0.0, 1.0, 0.0, 1.0)
        out.append(lf[0])
    ok = out[1] > 0
    ratio = out[0][ok] / out[1][ok]
    # v.h from the geometry of each pixel's hit point
    u = np.arange(Wr)[ok]
    p = np.stack([z0 * (u - cx) / f, np.zeros_like(u, dtype=float), np.full(u.shape, z0)], axis=1)
    v = -p / np.linalg.norm(p, axis=1, keepdims=True)
    li = np.array([b, 0.0, 0.0]) - p
    i = li / np.linalg.norm(li, axis=1, keepdims=True)
    h = (v + i) / np.linalg.norm(v + i, axis=1, keepdims=True)
    return np.sum(v * h, axis=1), ratio


def test_dielectric_f0_is_the_normal_incidence_reflectance():
    # projector at the camera: v = i = h for every pixel, so F = F0, which
    # must equal the reflectance at normal incidence ((n - 1) / (n + 1))^2
    c, F = _fresnel_row(1.0, 0.0)
    assert len(F) > 300
    np.testing.assert_allclose(c, 1.0, atol=1e-12)
    want = ((N_DIELECTRIC - 1.0) / (N_DIELECTRIC + 1.0)) ** 2
    np.testing.assert_allclose(F, want, rtol=1e-12)
    np.testing.assert_allclose(F, _fresnel_exact(np.ones(1))[0], rtol=1e-12)


def test_fresnel_factor_follows_the_exact_reflectance_within_schlicks_bound():
    # Over cos(theta_d) in [0.05, 1], Schlick's form F0 + (1 - F0)(1 - c)^5
    # stays within 0.036 of the exact reflectance at n = 1.5 (its largest
    # deviations near grazing incidence); with the exponent 4 or 6 the
    # deviation reaches 0.10 or 0.055.  The oracle's F must stay within 0.04
    # at every sampled angle, sampled densely from grazing to normal
    # incidence, and be monotone in the angle as the exact reflectance is.
    cs, Fs = [], []
    for z0, b in ((0.02, 2.0), (0.1, 2.0), (0.3, 1.5), (1.0, 1.0), (3.0, 0.5)):
        c, F = _fresnel_row(z0, b)
        cs.append(c)
        Fs.append(F)
    c = np.concatenate(cs)
    F = np.concatenate(Fs)
    assert c.min() < 0.06 and c.max() > 0.99
    for lo, hi in ((0.05, 0.2), (0.2, 0.5), (0.5, 0.9), (0.9, 1.0)):
        assert ((c >= lo) & (c <= hi)).sum() >= 20, (lo, hi)     # every part of the range is sampled
    sel = c >= 0.05
    err = np.abs(F[sel] - _fresnel_exact(c[sel]))
    assert err.max() <= 0.04, err.max()
    order = np.argsort(c)
    assert np.all(np.diff(F[order]) <= 1e-12)                    # more grazing -> more reflective
