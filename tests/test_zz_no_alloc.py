"""simsense_compute_noalloc against simsense_compute and the oracle, through
the C ABI.

The no-allocation entry point serves callers that may not allocate device
memory: a plugin whose host application owns all device memory, a real-time
loop that bans cudaMalloc after start-up (it can block the host and
synchronise the device), or a process whose memory another framework's caching
allocator already holds.  It runs the same kernels as the handle-based call,
on a fixed scratch array inside the library, so on the same pair it must give
the same depth map bit for bit, call after call: the array keeps the previous
call's contents, which must not leak into the next result, even when the
previous call was a larger problem with another layout.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest

from paper_2201_11924_gb300 import configs, scenes

pytestmark = pytest.mark.gpu

DEPTH_RTOL = 1e-5   # the tolerance the parity tests use for fp32 depth against the oracle

SMALL_8PATH = configs.SMALL_320.with_(name="160x96_D48_7x7_8path_subpixel", W=160, H=96, D=48, win_w=7, win_h=7,
                                      paths=8, uniq=15, subpixel=True)


@pytest.fixture(scope="module")
def lib():
    from paper_2201_11924_gb300 import _build, simsense
    _build.build()
    lib = simsense.load()
    P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    lib.simsense_compute_noalloc.argtypes = [P, P, P, I, I, I, I, I, I, I, I, I, F, F, I, P]
    lib.simsense_compute_noalloc.restype = ctypes.c_int
    lib.simsense_noalloc_status.argtypes = [P]
    lib.simsense_noalloc_status.restype = ctypes.c_int
    return lib


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _handle_depth(lib, wl, left, right):
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
                                  ctypes.c_void_p(depth.data_ptr()), _stream())
        assert rc == 0
        assert lib.simsense_device_status(h, _stream()) == 0
        return depth.cpu().numpy()
    finally:
        lib.simsense_destroy(h)


def _noalloc_depth(lib, wl, left, right):
    import torch
    depth = torch.full((wl.H, wl.W), -7.0, dtype=torch.float32, device="cuda")
    rc = lib.simsense_compute_noalloc(ctypes.c_void_p(left.data_ptr()), ctypes.c_void_p(right.data_ptr()),
                                      ctypes.c_void_p(depth.data_ptr()), wl.W, wl.H, wl.D, wl.census_win,
                                      wl.P1, wl.P2, wl.paths, wl.uniq, wl.lr_max_diff, wl.f, wl.baseline,
                                      int(wl.subpixel), _stream())
    assert rc == 0
    assert lib.simsense_noalloc_status(_stream()) == 0      # no bounded wait gave up
    return depth.cpu().numpy()


def _oracle_depth(wl, pair):
    import oracle
    o = oracle.compute(pair["left"], pair["right"], wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq,
                       wl.lr_max_diff, wl.subpixel, wl.f, wl.baseline)
    return o["depth"], o["mask"] == 0


def _check(lib, wl, pair):
    """One no-allocation call: the same bits as the handle call on the same
    pair, and the oracle's valid pixels and depth within the parity tolerance."""
    import torch
    left = torch.from_numpy(pair["left"]).cuda()
    right = torch.from_numpy(pair["right"]).cuda()
    want = _handle_depth(lib, wl, left, right)
    got = _noalloc_depth(lib, wl, left, right)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    ref, valid = _oracle_depth(wl, pair)
    assert np.array_equal(got != 0, valid)
    np.testing.assert_allclose(got[valid], ref[valid], rtol=DEPTH_RTOL, atol=0)


@pytest.mark.parametrize("wl", [configs.SMALL_320, SMALL_8PATH], ids=lambda w: w.name)
def test_noalloc_matches_handle_call_twice_in_a_row(lib, wl):
    for k in range(2):   # two calls in a row on different pairs share the array
        _check(lib, wl, scenes.make_pair(wl, seed=wl.seed + k))


def test_noalloc_alternating_layouts(lib):
    # a larger problem with another layout (320x240, D = 64, 4 paths, 32-bit
    # codes) directly before a smaller one (160x96, D = 48, 8 paths, 64-bit
    # codes) and back: the leftovers of each call in the shared array must not
    # reach the next call's result
    a, b = configs.SMALL_320, SMALL_8PATH
    for wl, k in ((a, 0), (b, 0), (a, 1)):
        _check(lib, wl, scenes.make_pair(wl, seed=wl.seed + 10 + k))


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
    assert lib.simsense_noalloc_status(None) == 0
