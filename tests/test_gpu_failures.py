"""Out-of-memory paths of the C ABI, driven by the allocation test hook
(simsense_test_fail_allocation): the nth device allocation fails as if the
device were full.  No real memory pressure, no GPU fault.  Each failing call
must return SIMSENSE_ERR_OOM, give back everything it had allocated, and
leave the library usable: the next calls compute the same depth as before.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2201_11924_gb300 import configs, scenes

pytestmark = pytest.mark.gpu

CREATE_ALLOCS = 8          # codes x2, cost, paths, status, staging x3
RECTIFY_ALLOCS = 4         # map and image per view
BATCH_ALLOCS = 2           # scratch, status
SLACK = 2 << 20            # bytes of free-memory reading noise tolerated


@pytest.fixture(scope="module")
def lib():
    from paper_2201_11924_gb300 import _build, simsense
    _build.build()
    L = simsense.load()
    L.simsense_test_fail_allocation.argtypes = [ctypes.c_int]
    L.simsense_test_fail_allocation.restype = None
    yield simsense
    L.simsense_test_fail_allocation(0)


class _Armed:
    """The nth allocation from here fails; disarmed on leaving the block."""

    def __init__(self, L, n):
        self.L, self.n = L, n

    def __enter__(self):
        self.L.simsense_test_fail_allocation(self.n)

    def __exit__(self, *exc):
        self.L.simsense_test_fail_allocation(0)


def _create(L, wl):
    h = ctypes.c_void_p()
    rc = L.simsense_create(ctypes.byref(h), wl.W, wl.H, wl.D, wl.win_w | (wl.win_h << 8), wl.P1, wl.P2,
                           wl.paths, wl.uniq, wl.lr_max_diff, wl.f, wl.baseline)
    return rc, h


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _depth(lib, wl, pair):
    import torch
    with lib.SimSense.from_workload(wl) as m:
        d = m.compute(torch.from_numpy(pair["left"]).cuda(), torch.from_numpy(pair["right"]).cuda())
        torch.cuda.synchronize()
        assert m.device_status() == 0
        return d.cpu().numpy()


def test_each_failed_allocation_of_create_is_reported_and_released(lib):
    L = lib.load()
    wl = configs.HD_720            # every scratch buffer of this size is >= 0.9 MB
    rc, h = _create(L, wl)
    assert rc == lib.OK
    L.simsense_destroy(h)
    free0 = _free_bytes()
    for rep in range(4):
        for n in range(1, CREATE_ALLOCS + 1):
            with _Armed(L, n):
                rc, h = _create(L, wl)
            assert (rc, h.value) == (lib.ERR_OOM, None), (rep, n)
    # one past the last allocation: nothing fails
    with _Armed(L, CREATE_ALLOCS + 1):
        rc, h = _create(L, wl)
    assert rc == lib.OK
    L.simsense_destroy(h)
    # 32 failed creates that each held up to 1.1 GB gave every byte back
    assert abs(_free_bytes() - free0) <= SLACK


def test_library_computes_the_same_depth_after_failed_allocations(lib):
    wl = configs.SMALL_320
    pair = scenes.make_pair(wl)
    before = _depth(lib, wl, pair)
    L = lib.load()
    for n in range(1, CREATE_ALLOCS + 1):
        with _Armed(L, n), pytest.raises(lib.SimsenseError) as ei:
            lib.SimSense.from_workload(wl)
        assert ei.value.code == lib.ERR_OOM
    after = _depth(lib, wl, pair)
    np.testing.assert_array_equal(after, before)
    o = oracle.compute(pair["left"], pair["right"], wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq,
                       wl.lr_max_diff, wl.subpixel, wl.f, wl.baseline)
    valid = o["mask"] == 0
    assert np.array_equal(after != 0, valid)
    np.testing.assert_allclose(after[valid], o["depth"][valid], rtol=1e-5, atol=0)


def test_failed_rectify_allocation_leaves_rectification_off(lib):
    import torch
    wl = configs.SMALL_320
    pair = scenes.make_pair(wl)
    plain = _depth(lib, wl, pair)
    cam = oracle.camera(wl.f, wl.f, (wl.W - 1) / 2, (wl.H - 1) / 2)     # identity rectification
    L = lib.load()
    lt, rt = torch.from_numpy(pair["left"]).cuda(), torch.from_numpy(pair["right"]).cuda()
    out = torch.empty((wl.H, wl.W), dtype=torch.float32, device="cuda")    # no allocation inside the loop
    with lib.SimSense.from_workload(wl) as m:
        free0 = _free_bytes()
        for n in range(1, RECTIFY_ALLOCS + 1):
            with _Armed(L, n), pytest.raises(lib.SimsenseError) as ei:
                m.set_rectify(cam, cam)
            assert ei.value.code == lib.ERR_OOM
            assert abs(_free_bytes() - free0) <= SLACK
            m.compute(lt, rt, out)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), plain)
        # and it still switches on: the identity maps reproduce the plain depth
        m.set_rectify(cam, cam)
        m.compute(lt, rt, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), plain)


def test_failed_batch_allocation_is_reported(lib):
    wls = [configs.SMALL_320, configs.SMALL_320.with_(D=96)]
    L = lib.load()
    blib = lib._load_batch()
    arr = (lib.PairParamsT * 2)(*[lib.pair_params(w) for w in wls])
    for n in range(1, BATCH_ALLOCS + 1):
        h = ctypes.c_void_p()
        with _Armed(L, n):
            rc = blib.simsense_batch_create(ctypes.byref(h), arr, 2)
        assert (rc, h.value) == (lib.ERR_OOM, None), n
    h = ctypes.c_void_p()
    assert blib.simsense_batch_create(ctypes.byref(h), arr, 2) == lib.OK
    blib.simsense_batch_destroy(h)
