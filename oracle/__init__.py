"""CPU oracle for the depth stage of arxiv 2201.11924 (Sec. VI-D).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module, and this module never imports the product.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, int32 for the
integer steps, fp64 for sub-pixel and depth); this file only compiles it with
gcc and marshals numpy arrays through ctypes.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against facts that do not come from the oracle itself (hand-computed codes,
invariants, brute-force minimum-energy label sequences, closed forms, exact
disparity recovery on fronto-parallel planes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

# Path index -> direction (rx, ry); the value at p comes from p - r.
PATH_DIRS = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, 1), (1, -1), (-1, -1)]


def build(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile oracle.c (or ``src``, a copy of it) into a shared library next
    to it (or at ``out``) with gcc -O2."""
    src = src or _SRC
    out = out or _LIB_PATH
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + f".tmp{os.getpid()}.{threading.get_ident()}"
    # -ffp-contract=off: no fused multiply-adds, so the fp64 camera arithmetic
    # rounds after every operation as written
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            I = ctypes.c_int
            Dd = ctypes.c_double
            lib.oracle_census.argtypes = [P, I, I, I, I, P]
            lib.oracle_cost.argtypes = [P, P, I, I, I, I, P]
            lib.oracle_path.argtypes = [P, I, I, I, I, I, I, I, P]
            lib.oracle_aggregate.argtypes = [P, I, I, I, I, I, I, P]
            lib.oracle_select.argtypes = [P, I, I, I, I, I, I, Dd, P, P, P, P]
            lib.oracle_compute.argtypes = [P, P, I, I, I, I, I, I, I, I, I, I, I, Dd, Dd,
                                           P, P, P, P, P, P, P]
            lib.oracle_census_cs.argtypes = [P, I, I, I, I, P]
            lib.oracle_cost_block.argtypes = [P, I, I, I, I, I, P]
            lib.oracle_median.argtypes = [P, I, I, I, P]
            lib.oracle_compute_ex.argtypes = [P, P, I, I, I, I, I, I, I, I, I, I, I, Dd, Dd, I, I, I, I,
                                              P, P, P, P, P, P, P]
            U64 = ctypes.c_uint64
            U32 = ctypes.c_uint32
            lib.oracle_philox4x64.argtypes = [P, P, P]
            lib.oracle_philox4x64.restype = None
            lib.oracle_noise.argtypes = [P, I, I, Dd, Dd, Dd, Dd, U64, U32, U32, P, P, P]
            lib.oracle_render.argtypes = [P, I, P, P, P, P, P, P]
            lib.oracle_render.restype = ctypes.c_int
            lib.oracle_rectify.argtypes = [P, I, I, P, P]
            lib.oracle_register.argtypes = [P, I, I, Dd, Dd, Dd, Dd, P, P, I, I]
            lib.oracle_rectify.restype = ctypes.c_int
            lib.oracle_register.restype = ctypes.c_int
            for fn in ("oracle_census", "oracle_cost", "oracle_path", "oracle_aggregate",
                       "oracle_select", "oracle_compute", "oracle_census_cs", "oracle_cost_block",
                       "oracle_median", "oracle_compute_ex", "oracle_noise"):
                getattr(lib, fn).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def census(img: np.ndarray, ww: int, wh: int) -> np.ndarray:
    """Census codes (uint64, H x W) of one uint8 view."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.empty((H, W), dtype=np.uint64)
    _check(_load().oracle_census(_ptr(img), W, H, ww, wh, _ptr(out)), "census")
    return out


def cost(cl: np.ndarray, cr: np.ndarray, D: int, nbits: int) -> np.ndarray:
    """Hamming cost volume C (uint8, H x W x D)."""
    cl = np.ascontiguousarray(cl, dtype=np.uint64)
    cr = np.ascontiguousarray(cr, dtype=np.uint64)
    H, W = cl.shape
    out = np.empty((H, W, D), dtype=np.uint8)
    _check(_load().oracle_cost(_ptr(cl), _ptr(cr), W, H, D, nbits, _ptr(out)), "cost")
    return out


def path(C: np.ndarray, rx: int, ry: int, P1: int, P2: int) -> np.ndarray:
    """One SGM path L_r (int32, H x W x D) along r = (rx, ry)."""
    C = np.ascontiguousarray(C, dtype=np.uint8)
    H, W, D = C.shape
    out = np.empty((H, W, D), dtype=np.int32)
    _check(_load().oracle_path(_ptr(C), W, H, D, rx, ry, P1, P2, _ptr(out)), "path")
    return out


def aggregate(C: np.ndarray, paths: int, P1: int, P2: int) -> np.ndarray:
    """Aggregated cost S = sum of the paths' L_r (int32, H x W x D)."""
    C = np.ascontiguousarray(C, dtype=np.uint8)
    H, W, D = C.shape
    out = np.empty((H, W, D), dtype=np.int32)
    _check(_load().oracle_aggregate(_ptr(C), W, H, D, paths, P1, P2, _ptr(out)), "aggregate")
    return out


def select(S: np.ndarray, uniq: int, lr_max_diff: int, subpixel: bool, fb: float):
    """Selection and post-processing of an aggregated volume.

    Returns (dstar int32, mask uint8, disp float64, depth float64), each H x W.
    """
    S = np.ascontiguousarray(S, dtype=np.int32)
    H, W, D = S.shape
    dstar = np.empty((H, W), dtype=np.int32)
    mask = np.empty((H, W), dtype=np.uint8)
    disp = np.empty((H, W), dtype=np.float64)
    depth = np.empty((H, W), dtype=np.float64)
    _check(_load().oracle_select(_ptr(S), W, H, D, uniq, lr_max_diff, int(bool(subpixel)), float(fb),
                                 _ptr(dstar), _ptr(mask), _ptr(disp), _ptr(depth)), "select")
    return dstar, mask, disp, depth


def census_cs(img: np.ndarray, ww: int, wh: int) -> np.ndarray:
    """Centre-symmetric census codes ((ww*wh-1)/2 bits) of one view (uint64, H x W)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.empty((H, W), dtype=np.uint64)
    _check(_load().oracle_census_cs(_ptr(img), W, H, ww, wh, _ptr(out)), "census_cs")
    return out


def cost_block(C: np.ndarray, bw: int, bh: int) -> np.ndarray:
    """SGBM block cost: the mean of C over a bw x bh block, rounded half up (uint8, H x W x D)."""
    C = np.ascontiguousarray(C, dtype=np.uint8)
    H, W, D = C.shape
    out = np.empty((H, W, D), dtype=np.uint8)
    _check(_load().oracle_cost_block(_ptr(C), W, H, D, bw, bh, _ptr(out)), "cost_block")
    return out


def median(img: np.ndarray, k: int) -> np.ndarray:
    """k x k median of a float map with replicated borders (float64, H x W)."""
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    out = np.empty((H, W), dtype=np.float64)
    _check(_load().oracle_median(_ptr(img), W, H, k, _ptr(out)), "median")
    return out


def philox4x64(ctr, key) -> np.ndarray:
    """Philox4x64-10 of a 4-word counter under a 2-word key (4 uint64)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, dtype=np.uint64)
    _load().oracle_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return out


# D415 noise parameters the paper estimates (Sec. VII, sensor parameters)
D415_NOISE = dict(mu=-0.231, sigma=0.83, k=3.98, theta=0.254)


def noise(clean, mu, sigma, k, theta, seed, frame=0, view=0):
    """Sensor noise of one view (Sec. VI-C).  Returns (noisy uint8, value
    float64 before rounding, margin float64 = distance of the nearest
    decision to its threshold)."""
    clean = np.ascontiguousarray(clean, dtype=np.uint8)
    H, W = clean.shape
    noisy = np.empty((H, W), dtype=np.uint8)
    value = np.empty((H, W), dtype=np.float64)
    margin = np.empty((H, W), dtype=np.float64)
    _check(_load().oracle_noise(_ptr(clean), W, H, float(mu), float(sigma), float(k), float(theta),
                                int(seed), int(frame), int(view), _ptr(value), _ptr(noisy), _ptr(margin)),
           "noise")
    return noisy, value, margin


def camera(fx, fy, cx, cy, k1=0.0, k2=0.0, p1=0.0, p2=0.0, k3=0.0, R=None, rfx=None, rfy=None, rcx=None,
           rcy=None) -> np.ndarray:
    """Raw and rectified camera of one view as the 22 doubles the oracle takes
    (rectified intrinsics default to the raw ones, R to the identity)."""
    R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
    return np.array([fx, fy, cx, cy, k1, k2, p1, p2, k3, *R.ravel(),
                     fx if rfx is None else rfx, fy if rfy is None else rfy,
                     cx if rcx is None else rcx, cy if rcy is None else rcy], dtype=np.float64)


def rectify(raw, cam) -> np.ndarray:
    """Rectified view (uint8, same size) of a raw view under `camera(...)`."""
    raw = np.ascontiguousarray(raw, dtype=np.uint8)
    H, W = raw.shape
    c = np.ascontiguousarray(cam, dtype=np.float64)
    out = np.empty((H, W), dtype=np.uint8)
    _check(_load().oracle_rectify(_ptr(raw), W, H, _ptr(c), _ptr(out)), "rectify")
    return out


def register(depth, fx, fy, cx, cy, fx2, fy2, cx2, cy2, R, t, W2, H2) -> np.ndarray:
    """Depth (float32, W x H, 0 invalid) of camera (fx, fy, cx, cy) splatted
    into an RGB camera (fx2, fy2, cx2, cy2) at pose (R, t), W2 x H2."""
    depth = np.ascontiguousarray(depth, dtype=np.float32)
    H, W = depth.shape
    reg = np.array([fx2, fy2, cx2, cy2, *np.asarray(R, dtype=np.float64).ravel(), *t], dtype=np.float64)
    out = np.empty((H2, W2), dtype=np.float32)
    _check(_load().oracle_register(_ptr(depth), W, H, float(fx), float(fy), float(cx), float(cy), _ptr(reg),
                                   _ptr(out), W2, H2), "register")
    return out


PRIM_DTYPE = np.dtype([("kind", np.int32), ("pad", np.int32), ("c", np.float64, 3), ("u", np.float64, 3),
                       ("v", np.float64, 3), ("radius", np.float64), ("albedo", np.float64),
                       ("metallic", np.float64), ("roughness", np.float64), ("transmission", np.float64)])
RENDER_DTYPE = np.dtype([("W", np.int32), ("H", np.int32), ("f", np.float64), ("cx", np.float64),
                         ("cy", np.float64), ("baseline", np.float64), ("proj", np.float64, 3), ("pf", np.float64),
                         ("pcx", np.float64), ("pcy", np.float64), ("PW", np.int32), ("PH", np.int32),
                         ("power", np.float64), ("ambient", np.float64), ("gain", np.float64)])


def sphere(c, radius, albedo=0.8, metallic=0.0, roughness=0.5, transmission=0.0):
    return (0, 0, c, (0, 0, 0), (0, 0, 0), radius, albedo, metallic, roughness, transmission)


def rectangle(c, u, v, albedo=0.8, metallic=0.0, roughness=0.5, transmission=0.0):
    return (1, 0, c, u, v, 0.0, albedo, metallic, roughness, transmission)


def render(prims, pattern, W, H, f, cx, cy, baseline, proj, pf, pcx, pcy, power, ambient, gain):
    """IR images (left, right uint8) and their values before rounding (float64)
    of a scene of spheres and rectangles lit by a textured projector."""
    pr = np.array(list(prims), dtype=PRIM_DTYPE)
    pattern = np.ascontiguousarray(pattern, dtype=np.uint8)
    PH, PW = pattern.shape
    rp = np.array([(W, H, f, cx, cy, baseline, proj, pf, pcx, pcy, PW, PH, power, ambient, gain)], dtype=RENDER_DTYPE)
    left = np.empty((H, W), dtype=np.uint8)
    right = np.empty((H, W), dtype=np.uint8)
    lf = np.empty((H, W), dtype=np.float64)
    rf = np.empty((H, W), dtype=np.float64)
    _check(_load().oracle_render(_ptr(pr), len(pr), _ptr(rp), _ptr(pattern), _ptr(left), _ptr(right), _ptr(lf),
                                 _ptr(rf)), "render")
    return left, right, lf, rf


def compute(left, right, D, ww, wh, P1, P2, paths, uniq, lr_max_diff, subpixel, f, baseline,
            want_codes=False, want_S=False, census_cs=False, block=(1, 1), median=0):
    """The whole stage for one pair.  Returns a dict of numpy arrays.

    ``f`` and ``baseline`` are converted to float32 first, as the library
    receives them, and their product is then formed in fp64.  census_cs,
    block = (bw, bh) and median = k select the variants (centre-symmetric
    census, SGBM block cost, k x k median filter).
    """
    left = np.ascontiguousarray(left, dtype=np.uint8)
    right = np.ascontiguousarray(right, dtype=np.uint8)
    H, W = left.shape
    f32 = float(np.float32(f))
    b32 = float(np.float32(baseline))
    out = {
        "depth": np.empty((H, W), dtype=np.float64),
        "disp": np.empty((H, W), dtype=np.float64),
        "dstar": np.empty((H, W), dtype=np.int32),
        "mask": np.empty((H, W), dtype=np.uint8),
    }
    cl = np.empty((H, W), dtype=np.uint64) if want_codes else None
    cr = np.empty((H, W), dtype=np.uint64) if want_codes else None
    S = np.empty((H, W, D), dtype=np.int32) if want_S else None
    rc = _load().oracle_compute_ex(_ptr(left), _ptr(right), W, H, D, ww, wh, P1, P2, paths, uniq,
                                   lr_max_diff, int(bool(subpixel)), f32, b32, int(bool(census_cs)),
                                   int(block[0]), int(block[1]), int(median),
                                   _ptr(out["depth"]), _ptr(out["disp"]), _ptr(out["dstar"]),
                                   _ptr(out["mask"]), _ptr(cl), _ptr(cr), _ptr(S))
    _check(rc, "compute")
    if want_codes:
        out["codes_left"], out["codes_right"] = cl, cr
    if want_S:
        out["S"] = S
    return out
