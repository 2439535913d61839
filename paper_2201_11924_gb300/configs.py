"""Named workloads of the depth stage (sizes, sensor parameters, scene recipes).

Each workload is a rectified IR pair of a given size and disparity range,
the matcher's parameters (census window, P1/P2, path count, uniqueness
ratio, left-right tolerance, sub-pixel on/off) and the pinhole parameters
that turn disparity into depth (focal length f in pixels, baseline b in
metres).  The scene recipe (object counts, depth range, dot pattern, noise)
feeds the synthetic generator in ``scenes.py``; it stands in for the paper's
ray-traced IR rendering (Sec. VI-A/VI-B), which this package does not do.

Nothing here computes any step of the method.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace


@dataclass(frozen=True)
class Scene:
    """Recipe for one synthetic random-dot stereo scene."""
    n_planes: int = 3            # including the back wall
    n_spheres: int = 0
    z_min: float = 0.3           # metres
    z_max: float = 1.5
    dot_density: float = 0.15
    dot_lo: int = 180            # dot intensity, inclusive range
    dot_hi: int = 255
    bg_lo: int = 20              # background intensity, inclusive range
    bg_hi: int = 60
    albedo_lo: float = 1.0       # per-object albedo, uniform
    albedo_hi: float = 1.0
    noise_sigma: float = 2.0     # Gaussian sensor noise per view, in grey levels
    translucent_frac: float = 0.0  # share of objects whose dot contrast is scaled down
    translucent_contrast: float = 0.1


@dataclass(frozen=True)
class Workload:
    name: str
    W: int
    H: int
    D: int
    win_w: int
    win_h: int
    P1: int = 7
    P2: int = 86
    paths: int = 8
    uniq: int = 0                # integer percentage; 0 disables the test
    lr_max_diff: int = 1         # < 0 disables the left-right check
    subpixel: bool = True
    f: float = 920.0             # focal length in pixels
    baseline: float = 0.055      # metres
    seed: int = 0
    scene: Scene = field(default_factory=Scene)
    # variants Sec. VI-D names: centre-symmetric census, SGBM block (bw, bh),
    # k x k median filter (0 = off)
    census_cs: bool = False
    block: tuple = (1, 1)
    median: int = 0
    # IR sensor noise of Sec. VI-C with the D415 values, seeded by `seed`
    noise: bool = False

    @property
    def nbits(self) -> int:
        full = self.win_w * self.win_h - 1
        return full // 2 if self.census_cs else full

    @property
    def census_win(self) -> int:
        """Window code passed to ``simsense_create``: w | (h << 8)."""
        return self.win_w | (self.win_h << 8)

    @property
    def cells(self) -> int:
        return self.W * self.H * self.D

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# 320x240, D=64, 5x5 census, 4-path SGM, no uniqueness, L/R 1, no sub-pixel;
# 3 planes at 0.3-1.5 m, f = 300 px, b = 0.055 m, noise sigma 2.
SMALL_320 = Workload(
    name="320x240_D64_census5x5_4path",
    W=320, H=240, D=64, win_w=5, win_h=5, P1=7, P2=86, paths=4, uniq=0, lr_max_diff=1,
    subpixel=False, f=300.0, baseline=0.055, seed=1001,
    scene=Scene(n_planes=3, n_spheres=0, z_min=0.3, z_max=1.5, noise_sigma=2.0),
)

# 1280x720 (D415-like IR size), D=128, 7x7 census (48-bit codes), 8-path SGM,
# uniqueness 15, L/R 1, sub-pixel, f = 920 px, b = 0.055 m; 6 planes plus
# 8 spheres at 0.25-2.0 m, albedo 0.2-1.0, noise sigma 3.
HD_720 = Workload(
    name="1280x720_D128_census7x7_8path",
    W=1280, H=720, D=128, win_w=7, win_h=7, P1=7, P2=86, paths=8, uniq=15, lr_max_diff=1,
    subpixel=True, f=920.0, baseline=0.055, seed=1002,
    scene=Scene(n_planes=6, n_spheres=8, z_min=0.25, z_max=2.0, albedo_lo=0.2, albedo_hi=1.0,
                noise_sigma=3.0),
)

# 1920x1080, D=256, 9x7 census (62 bits), 8-path SGM, uniqueness 10, L/R 1,
# sub-pixel; 20 mixed planes and spheres at 0.2-3.0 m, 30% of the objects with
# the dot contrast scaled by 0.1, noise sigma 4.
FHD_1080 = Workload(
    name="1920x1080_D256_census9x7_8path",
    W=1920, H=1080, D=256, win_w=9, win_h=7, P1=7, P2=86, paths=8, uniq=10, lr_max_diff=1,
    subpixel=True, f=920.0, baseline=0.055, seed=1004,
    scene=Scene(n_planes=10, n_spheres=10, z_min=0.2, z_max=3.0, albedo_lo=0.2, albedo_hi=1.0,
                noise_sigma=4.0, translucent_frac=0.3),
)

# Size classes of the batched workload (64 pairs): census 7x7, 8 paths, the
# small workload's post-processing (no uniqueness, L/R 1, no sub-pixel).
BATCH_SIZES = [(640, 360, 64), (848, 480, 96), (1280, 720, 128), (1280, 720, 256)]


def batch_workloads(n: int = 64, seed0: int = 3000):
    """The batched mix: pair i has seed seed0 + i and a size drawn by that seed."""
    import numpy as np
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        W, H, D = BATCH_SIZES[int(rng.integers(0, len(BATCH_SIZES)))]
        out.append(Workload(
            name=f"batch_{i}_{W}x{H}_D{D}", W=W, H=H, D=D, win_w=7, win_h=7, P1=7, P2=86,
            paths=8, uniq=0, lr_max_diff=1, subpixel=False, f=300.0, baseline=0.055,
            seed=seed0 + i, scene=SMALL_320.scene))
    return out


# Size classes of the serving mix: 50% 848x480 D=96, 40% 1280x720 D=128,
# 10% 1920x1080 D=256; census 7x7, 8 paths, uniqueness 15, L/R 1, sub-pixel.
SERVE_SIZES = [((848, 480, 96), 0.5), ((1280, 720, 128), 0.4), ((1920, 1080, 256), 0.1)]


def serve_camera(cam: int, seed0: int = 5000) -> Workload:
    """Camera ``cam`` of the serving workload (its size class is drawn by its seed)."""
    import numpy as np
    rng = np.random.default_rng(seed0 + cam)
    u = float(rng.random())
    acc = 0.0
    size = SERVE_SIZES[-1][0]
    for s, p in SERVE_SIZES:
        acc += p
        if u < acc:
            size = s
            break
    W, H, D = size
    return Workload(
        name=f"cam_{cam}_{W}x{H}_D{D}", W=W, H=H, D=D, win_w=7, win_h=7, P1=7, P2=86, paths=8,
        uniq=15, lr_max_diff=1, subpixel=True, f=300.0, baseline=0.055, seed=seed0 + cam,
        scene=SMALL_320.scene)


ALL = {w.name: w for w in (SMALL_320, HD_720, FHD_1080)}
