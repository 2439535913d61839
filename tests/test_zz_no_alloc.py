"""simsense_compute_noalloc against simsense_compute, through the C ABI.

The no-allocation entry point serves callers that may not allocate device
memory (a plugin whose host application owns all device memory, a real-time
loop that bans cudaMalloc after start-up because it can block the host and
synchronise the device, a process whose memory another framework's caching
allocator already holds).  It runs the same kernels on a fixed scratch array
inside the library, so its depth maps must match those of the handle-based
call on the same pairs, call after call (the array keeps the previous call's
contents, which must not leak into the next result).

This file is named to be collected last, so a run that stops at the first
failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest

from paper_2201_11924_gb300 import configs, scenes

pytestmark = pytest.mark.gpu

DEPTH_RTOL = 1e-5   # the tolerance the parity tests use for fp32 depth


@pytest.fixture(scope="module")
def lib():
    from paper_2201_11924_gb300 import _build, simsense
    _build.build()
    lib = simsense.load()
    P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    lib.simsense_compute_noalloc.argtypes = [P, P, P, I, I, I, I, I, I, I, I, I, F, F, I, P]
    lib.simsense_compute_noalloc.restype = ctypes.c_int
    return lib


def _handle_depth(lib, wl, left, right, stream):
    import torch
    h = ctypes.c_void_p()
    rc = lib.simsense_create(ctypes.byref(h), wl.W, wl.H, wl.D, wl.census_win, wl.P1, wl.P2, wl.paths,
                             wl.uniq, wl.lr_max_diff, wl.f, wl.baseline)
    assert rc == 0
    try:
        if not wl.subpixel:
            assert lib.simsense_set_option(h, 1, 0) == 0
        depth = torch.empty((wl.H, wl.W), dtype=torch.float32, device="cuda")
        rc = lib.simsense_compute(h, ctypes.c_void_p(left.data_ptr()), ctypes.c_void_p(right.data_ptr()),
                                  ctypes.c_void_p(depth.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        return depth.cpu().numpy()
    finally:
        lib.simsense_destroy(h)


def _noalloc_depth(lib, wl, left, right, stream):
    import torch
    depth = torch.full((wl.H, wl.W), -7.0, dtype=torch.float32, device="cuda")
    rc = lib.simsense_compute_noalloc(ctypes.c_void_p(left.data_ptr()), ctypes.c_void_p(right.data_ptr()),
                                      ctypes.c_void_p(depth.data_ptr()), wl.W, wl.H, wl.D, wl.census_win,
                                      wl.P1, wl.P2, wl.paths, wl.uniq, wl.lr_max_diff, wl.f, wl.baseline,
                                      int(wl.subpixel), stream)
    assert rc == 0
    torch.cuda.synchronize()
    return depth.cpu().numpy()


def _same(a, b):
    valid = b != 0
    assert np.array_equal(a != 0, valid)
    np.testing.assert_allclose(a[valid], b[valid], rtol=DEPTH_RTOL, atol=0)


@pytest.mark.parametrize("wl", [
    configs.SMALL_320,
    configs.SMALL_320.with_(name="160x96_D48_7x7_8path_subpixel", W=160, H=96, D=48, win_w=7, win_h=7,
                            paths=8, uniq=15, subpixel=True),
], ids=lambda w: w.name)
def test_noalloc_matches_handle_call_twice_in_a_row(lib, wl):
    import torch
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    pairs = [scenes.make_pair(wl, seed=wl.seed + k) for k in range(2)]
    for p in pairs:   # two calls in a row on different pairs share the array
        left = torch.from_numpy(p["left"]).cuda()
        right = torch.from_numpy(p["right"]).cuda()
        want = _handle_depth(lib, wl, left, right, stream)
        got = _noalloc_depth(lib, wl, left, right, stream)
        _same(got, want)


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    import torch
    wl = configs.HD_720
    buf = torch.zeros((wl.H, wl.W), dtype=torch.uint8, device="cuda")
    out = torch.zeros((wl.H, wl.W), dtype=torch.float32, device="cuda")
    rc = lib.simsense_compute_noalloc(ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), wl.W, wl.H, wl.D, wl.census_win,
                                      wl.P1, wl.P2, wl.paths, wl.uniq, wl.lr_max_diff, wl.f, wl.baseline, 1,
                                      None)
    assert rc == -1
