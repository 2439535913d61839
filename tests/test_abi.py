"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/simsense.h declares, and argument validation rejects
out-of-range parameters before any CUDA call is made."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(simsense_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_11924_gb300 import _build, simsense
    _build.build()
    return simsense.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("simsense_create", "simsense_compute", "simsense_destroy", "simsense_compute_host",
                 "simsense_compute_debug", "simsense_set_option", "simsense_strerror"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_strerror(lib):
    from paper_2201_11924_gb300 import simsense
    assert simsense.strerror(0) == "ok"
    assert simsense.strerror(-1) == "invalid argument"
    assert simsense.strerror(-4).startswith("device-side wait")


@pytest.mark.parametrize("args", [
    # W, H, D, win, P1, P2, paths, uniq, lr, f, b
    (64, 32, 0, 5 | (5 << 8), 7, 86, 4, 0, 1, 300.0, 0.055),       # D < 1
    (64, 32, 257, 5 | (5 << 8), 7, 86, 4, 0, 1, 300.0, 0.055),     # D > 256
    (64, 32, 65, 5 | (5 << 8), 7, 86, 4, 0, 1, 300.0, 0.055),      # D > W
    (64, 32, 16, 4 | (5 << 8), 7, 86, 4, 0, 1, 300.0, 0.055),      # even window
    (64, 32, 16, 9 | (9 << 8), 7, 86, 4, 0, 1, 300.0, 0.055),      # 80 bits > 64
    (64, 32, 16, 5 | (5 << 8), 9, 8, 4, 0, 1, 300.0, 0.055),       # P1 > P2
    (64, 32, 16, 9 | (7 << 8), 7, 200, 4, 0, 1, 300.0, 0.055),     # nbits + P2 > 255
    (64, 32, 16, 5 | (5 << 8), 7, 86, 6, 0, 1, 300.0, 0.055),      # paths
    (64, 32, 16, 5 | (5 << 8), 7, 86, 8, 100, 1, 300.0, 0.055),    # uniqueness ratio
    (64, 32, 16, 5 | (5 << 8), 7, 86, 8, 0, 1, 0.0, 0.055),        # f
    (64, 32, 16, 5 | (5 << 8), 7, 86, 8, 0, 1, 300.0, -1.0),       # baseline
    (4, 32, 4, 5 | (5 << 8), 7, 86, 8, 0, 1, 300.0, 0.055),        # W < window
    (8193, 32, 64, 5 | (5 << 8), 7, 86, 8, 0, 1, 300.0, 0.055),    # W above the row limit
])
def test_create_rejects_bad_arguments(lib, args):
    h = ctypes.c_void_p()
    assert lib.simsense_create(ctypes.byref(h), *args) == -1
    assert not h.value


def test_null_handles_are_rejected(lib):
    assert lib.simsense_compute(None, None, None, None, None) == -1
    assert lib.simsense_set_option(None, 1, 0) == -1
    assert lib.simsense_set_noise(None, 1, -0.231, 0.83, 3.98, 0.254, 1) == -1
    assert lib.simsense_destroy(None) == 0


def test_geometry_calls_reject_bad_arguments(lib):
    from paper_2201_11924_gb300 import simsense
    import oracle
    fake = ctypes.c_void_p(0x1000)
    cam = simsense.camera_t(oracle.camera(300.0, 300.0, 10.0, 10.0))
    bad = simsense.camera_t(oracle.camera(0.0, 300.0, 10.0, 10.0))
    assert lib.simsense_set_rectify(None, ctypes.byref(cam), ctypes.byref(cam)) == -1
    assert lib.simsense_rectify(None, fake, 8, 8, ctypes.byref(cam), None) == -1
    assert lib.simsense_rectify(fake, fake, 0, 8, ctypes.byref(cam), None) == -1
    assert lib.simsense_rectify(fake, fake, 8, 8, ctypes.byref(bad), None) == -1
    reg = simsense.registration_t(100.0, 100.0, 4.0, 4.0, 100.0, 100.0, 4.0, 4.0, np.eye(3), [0, 0, 0], 0, 8)
    assert lib.simsense_register_depth(fake, 8, 8, ctypes.byref(reg), fake, None) == -1


def test_render_rejects_bad_arguments(lib):
    from paper_2201_11924_gb300 import simsense
    fake = ctypes.c_void_p(0x1000)
    good = simsense.RenderT(8, 8, 10.0, 4.0, 4.0, 0.05, (ctypes.c_double * 3)(0, 0, 0), 10.0, 4.0, 4.0, 8, 8,
                            1.0, 0.1, 100.0)
    bad = simsense.RenderT(8, 8, 0.0, 4.0, 4.0, 0.05, (ctypes.c_double * 3)(0, 0, 0), 10.0, 4.0, 4.0, 8, 8,
                           1.0, 0.1, 100.0)
    assert lib.simsense_render_ir(fake, 1, ctypes.byref(bad), fake, fake, fake, None) == -1
    assert lib.simsense_render_ir(None, 1, ctypes.byref(good), fake, fake, fake, None) == -1
    assert lib.simsense_render_ir(fake, -1, ctypes.byref(good), fake, fake, fake, None) == -1
    assert lib.simsense_render_ir(fake, 1, None, fake, fake, fake, None) == -1


@pytest.mark.parametrize("W,H,k,theta,sigma", [
    (0, 8, 3.98, 0.254, 0.83),           # empty image
    (8, 8, 0.5, 0.254, 0.83),            # k < 1 (the rejection sampler needs k >= 1)
    (8, 8, 3.98, 0.0, 0.83),             # theta
    (8, 8, 3.98, 0.254, -1.0),           # sigma
    (8, 8, float("nan"), 0.254, 0.83),
])
def test_add_noise_rejects_bad_arguments(lib, W, H, k, theta, sigma):
    # argument checks come before any CUDA call: the buffers are never touched
    fake = ctypes.c_void_p(0x1000)
    assert lib.simsense_add_noise(fake, fake, W, H, -0.231, sigma, k, theta, 1, 0, 0, None) == -1
    assert lib.simsense_add_noise(None, fake, 8, 8, -0.231, 0.83, 3.98, 0.254, 1, 0, 0, None) == -1


def test_batch_create_rejects_bad_arguments(lib):
    from paper_2201_11924_gb300 import configs, simsense
    blib = simsense._load_batch()
    h = ctypes.c_void_p()
    good = simsense.pair_params(configs.SMALL_320)
    bad = simsense.pair_params(configs.SMALL_320.with_(D=0))
    arr = (simsense.PairParamsT * 2)(good, bad)
    assert blib.simsense_batch_create(ctypes.byref(h), arr, 2) == -1 and not h.value
    assert blib.simsense_batch_create(ctypes.byref(h), arr, 0) == -1
    assert blib.simsense_batch_create(None, arr, 1) == -1
    assert blib.simsense_batch_destroy(None) == 0
    assert blib.simsense_batch_num_classes(None) == -1


_C_CALLER = r"""
#include "simsense.h"
#include <stdio.h>
#include <string.h>

typedef void (*fn_t)(void);
static const fn_t every_entry_point[] = {
%(table)s
};

int main(void)
{
    simsense_t h = (simsense_t)0;
    /* a window larger than the image: rejected before any CUDA call */
    int rc = simsense_create(&h, 4, 4, 2, 7, 7, 86, 8, 15, 1, 920.0f, 0.055f);
    if (rc != SIMSENSE_ERR_INVALID_ARG || h != (simsense_t)0) return 1;
    if (simsense_destroy((simsense_t)0) != SIMSENSE_OK) return 2;
    if (simsense_scratch_bytes((simsense_t)0) != 0) return 3;
    if (strcmp(simsense_strerror(SIMSENSE_ERR_INVALID_ARG), "invalid argument") != 0) return 4;
    printf("%%d entry points\n", (int)(sizeof every_entry_point / sizeof every_entry_point[0]));
    return 0;
}
"""


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c99"), ("g++", "-std=c++17")])
def test_plain_c_and_cpp_callers_compile_link_and_run(lib, tmp_path, compiler, std):
    # the boundary needs nothing but the header and the shared library: a C99
    # (and a C++) caller that takes the address of every declared entry point
    # compiles without warnings, links, and gets the documented status codes
    # from the calls that fail before touching the GPU
    from paper_2201_11924_gb300 import simsense
    names = _declared_functions()
    src = tmp_path / ("caller.c" if compiler == "gcc" else "caller.cpp")
    src.write_text(_C_CALLER % {"table": ",\n".join(f"    (fn_t){n}" for n in names)})
    exe = tmp_path / "caller"
    libdir = os.path.dirname(simsense.LIB_PATH)
    subprocess.run([compiler, std, "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), f"-L{libdir}", "-lsimsense", f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == f"{len(names)} entry points"


def _documented_valid(W, H, D, w, h, P1, P2, paths, uniq, f, b):
    """The limits simsense.h states for simsense_create."""
    hh = h or w
    nbits = w * hh - 1
    return (w % 2 == 1 and hh % 2 == 1 and 1 <= w <= 15 and 1 <= hh <= 15 and 1 <= nbits <= 64
            and w <= W <= 8192 and hh <= H <= 16384 and 1 <= D <= 256 and D <= W
            and 0 <= P1 <= P2 and nbits + P2 <= 255 and paths in (4, 8) and 0 <= uniq <= 99
            and f > 0 and b > 0 and np.isfinite(f) and np.isfinite(b))


def test_create_validation_matches_the_documented_limits(lib):
    # one field of a valid argument set at a time, set to values on both
    # sides of its documented limits: the invalid ones are refused with
    # SIMSENSE_ERR_INVALID_ARG before any CUDA call, the valid ones get past
    # validation (on this GPU-less host the device query then fails with
    # SIMSENSE_ERR_CUDA)
    import torch
    if torch.cuda.is_available():
        pytest.skip("on a GPU the valid sets would allocate their scratch")
    base = dict(W=64, H=32, D=16, w=5, h=5, P1=7, P2=86, paths=4, uniq=15, f=920.0, b=0.055)
    cand = {
        "W": [0, 4, 5, 16, 8192, 8193], "H": [0, 4, 5, 16384, 16385],
        "D": [-1, 0, 1, 63, 64, 65, 256, 257],
        "w": [0, 1, 2, 3, 13, 15, 17], "h": [0, 1, 2, 3, 13, 15, 17],
        "P1": [-1, 0, 86, 87], "P2": [-1, 6, 7, 230, 231, 255],
        "paths": [0, 2, 4, 6, 8, 16], "uniq": [-1, 0, 1, 99, 100],
        "f": [920.0, 1e-6, 0.0, -1.0, float("inf"), float("nan")],
        "b": [0.055, 0.0, -0.1, float("inf"), float("nan")],
    }
    outcomes = {True: 0, False: 0}
    for field, values in cand.items():
        for v in values:
            a = dict(base, **{field: v})
            if field in ("w", "h"):                    # a big window needs a big enough image
                a.update(W=8192, H=64, D=16)
            valid = _documented_valid(a["W"], a["H"], a["D"], a["w"], a["h"], a["P1"], a["P2"], a["paths"],
                                      a["uniq"], a["f"], a["b"])
            hdl = ctypes.c_void_p()
            rc = lib.simsense_create(ctypes.byref(hdl), a["W"], a["H"], a["D"], a["w"] | (a["h"] << 8), a["P1"],
                                     a["P2"], a["paths"], a["uniq"], 1, a["f"], a["b"])
            assert rc == (-3 if valid else -1), (field, v, rc)
            assert not hdl.value
            outcomes[valid] += 1
    assert outcomes[True] >= 15 and outcomes[False] >= 30      # both sides of the limits


def test_binding_constants_match_the_header(lib):
    # the Python binding repeats the header's status and option codes
    from paper_2201_11924_gb300 import simsense
    text = open(os.path.join(ROOT, "include", "simsense.h")).read()
    defs = dict(re.findall(r"^#define SIMSENSE_((?:OK|ERR_\w+|OPT_\w+))\s+(-?\d+)", text, flags=re.M))
    assert set(defs) >= {"OK", "ERR_INVALID_ARG", "ERR_OOM", "ERR_CUDA", "ERR_TIMEOUT", "OPT_SUBPIXEL"}
    for name, value in defs.items():
        assert getattr(simsense, name) == int(value), name
    # every status has its own description, and an unknown one is named as such
    texts = {code: simsense.strerror(int(v)) for code, v in defs.items() if code == "OK" or code.startswith("ERR_")}
    assert len(set(texts.values())) == len(texts)
    assert simsense.strerror(-99) == "unknown status"
