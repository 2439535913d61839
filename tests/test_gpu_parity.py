"""Parity of the CUDA depth stage (through the C ABI) with the CPU oracle.

Bar: census codes, the cost volume C, every path's L_r, aggregated costs S,
integer disparities and validity masks bit-exact; fp32 sub-pixel disparity within 1e-4 px and fp32 depth within
1e-5 relative of the oracle's fp64 values (the fp32 rounding of one division
and one sum stays far below both).
"""
import numpy as np
import pytest

import oracle
from paper_2201_11924_gb300 import configs, scenes

pytestmark = pytest.mark.gpu

DISP_TOL = 1e-4
DEPTH_RTOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    from paper_2201_11924_gb300 import _build, simsense
    _build.build()
    return simsense


def _run(lib, wl, left, right, aggregated=True, volumes=False):
    import torch
    dev = torch.device("cuda:0")
    with lib.SimSense.from_workload(wl) as m:
        lt = torch.from_numpy(left).to(dev)
        rt = torch.from_numpy(right).to(dev)
        out = m.compute_debug(lt, rt, aggregated=aggregated, volumes=volumes)
        depth2 = m.compute(lt, rt)
        torch.cuda.synchronize()
        assert m.device_status() == 0     # no bounded device-side wait gave up
        res = {k: v.cpu().numpy() for k, v in out.items()}
        res["depth_plain"] = depth2.cpu().numpy()
    return res


def _oracle(wl, left, right, want_S=True):
    return oracle.compute(left, right, wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq,
                          wl.lr_max_diff, wl.subpixel, wl.f, wl.baseline, want_codes=True, want_S=want_S)


def _compare(g, o, wl, check_S=True):
    np.testing.assert_array_equal(g["census_left"].view(np.uint64), o["codes_left"])
    np.testing.assert_array_equal(g["census_right"].view(np.uint64), o["codes_right"])
    if check_S:
        np.testing.assert_array_equal(g["aggregated"].view(np.uint16).astype(np.int32), o["S"])
    np.testing.assert_array_equal(g["disparity_int"].astype(np.int32), o["dstar"])
    np.testing.assert_array_equal(g["mask"], o["mask"])
    valid = o["mask"] == 0
    assert (g["disparity"][~valid] == -1.0).all()
    np.testing.assert_allclose(g["disparity"][valid], o["disp"][valid], rtol=0, atol=DISP_TOL)
    assert (g["depth"][~valid] == 0.0).all()
    np.testing.assert_allclose(g["depth"][valid], o["depth"][valid], rtol=DEPTH_RTOL, atol=0)
    # the plain call and the debug call run the same kernels
    np.testing.assert_array_equal(g["depth_plain"], g["depth"])


# path directions in the order of the debug dump (the value at p comes from p - r)
PATH_DIRS = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, 1), (1, -1), (-1, -1)]


def _compare_volumes(g, o, wl):
    """The cost volume C and every path's L_r bit for bit against the oracle
    (the cost from the oracle's codes, each L_r from the oracle's path
    recurrence on that cost), every cell including x - d < 0 and the last
    disparities of a padded range."""
    C = oracle.cost(o["codes_left"], o["codes_right"], wl.D, wl.nbits)
    np.testing.assert_array_equal(g["cost"], C)
    assert g["paths"].shape[0] == wl.paths
    for r in range(wl.paths):
        rx, ry = PATH_DIRS[r]
        L = oracle.path(C, rx, ry, wl.P1, wl.P2)
        assert L.max() <= 255
        np.testing.assert_array_equal(g["paths"][r].astype(np.int32), L, err_msg=f"path r={r} ({rx},{ry})")


def _small(name, W, H, D, ww, wh, paths, uniq, lr, sub, P1=7, P2=86, seed=1):
    sc = configs.SMALL_320.scene
    return configs.Workload(name=name, W=W, H=H, D=D, win_w=ww, win_h=wh, P1=P1, P2=P2, paths=paths,
                            uniq=uniq, lr_max_diff=lr, subpixel=sub, f=300.0, baseline=0.055, seed=seed,
                            scene=sc)


SMALL_CASES = [
    # ragged sizes spanning several tiles, every disparity padding class (D
    # per 32-lane group: 2, 4, 6, 8) and every code width
    _small("ragged_5x5_4p", 97, 45, 48, 5, 5, 4, 0, 1, False),
    _small("ragged_7x7_8p_uniq", 150, 70, 96, 7, 7, 8, 15, 1, True, seed=2),
    _small("ragged_9x7_8p_D160", 300, 33, 160, 9, 7, 8, 10, 1, True, seed=3),
    _small("ragged_9x7_8p_D256", 260, 40, 256, 9, 7, 8, 10, 0, True, seed=4),
    _small("D64_exact_4p", 130, 50, 64, 7, 7, 4, 5, 2, True, seed=5),
    _small("D1", 20, 9, 1, 3, 3, 8, 0, 1, True, seed=6),
    _small("D_equals_W", 40, 12, 40, 5, 5, 8, 15, 1, True, seed=7),
    _small("tiny_window_size", 9, 7, 3, 9, 7, 8, 0, 0, True, seed=8),
    _small("zero_penalties", 80, 30, 32, 5, 5, 8, 0, -1, True, P1=0, P2=0, seed=9),
    _small("equal_penalties", 80, 30, 32, 7, 7, 4, 99, 3, True, P1=20, P2=20, seed=10),
    _small("max_P2", 90, 20, 70, 9, 7, 8, 50, 1, True, P1=0, P2=193, seed=11),
    _small("win_15x3", 70, 25, 40, 15, 3, 8, 0, 1, True, seed=12),
    _small("win_1x1", 30, 10, 8, 3, 1, 4, 0, 1, True, seed=13),
    # long rows with slowly forgetting paths: with P1 = 0 and the largest P2,
    # a row's path restarted in its middle reaches the true state only 23-68
    # pixels later (by the oracle's recurrence); and a D = 96 (padded to 128)
    # row of 700 pixels
    _small("split_rows_slow_agreement", 520, 24, 64, 7, 7, 8, 10, 1, True, P1=0, P2=193, seed=21),
    _small("split_rows_D128", 700, 16, 96, 9, 7, 8, 10, 1, True, P1=1, P2=150, seed=23),
]


@pytest.mark.parametrize("wl", SMALL_CASES, ids=lambda w: w.name)
def test_parity_small(lib, wl):
    p = scenes.make_pair(wl)
    g = _run(lib, wl, p["left"], p["right"], volumes=True)
    o = _oracle(wl, p["left"], p["right"])
    _compare(g, o, wl)
    _compare_volumes(g, o, wl)


def test_parity_small_workload_320(lib):
    wl = configs.SMALL_320
    p = scenes.make_pair(wl)
    g = _run(lib, wl, p["left"], p["right"], volumes=True)
    o = _oracle(wl, p["left"], p["right"])
    _compare(g, o, wl)
    _compare_volumes(g, o, wl)


def test_parity_hd_720_full(lib):
    wl = configs.HD_720
    p = scenes.make_pair(wl)
    g = _run(lib, wl, p["left"], p["right"], volumes=True)
    o = _oracle(wl, p["left"], p["right"])
    _compare(g, o, wl)
    _compare_volumes(g, o, wl)


def test_parity_fhd_1080_full(lib):
    wl = configs.FHD_1080
    p = scenes.make_pair(wl)
    _compare(_run(lib, wl, p["left"], p["right"]), _oracle(wl, p["left"], p["right"]), wl)


def test_plane_exact_recovery_gpu(lib):
    # noise-free fronto-parallel plane: d* = d0 on every pixel whose census
    # windows match exactly (the oracle pins the same property)
    W, H, D, d0 = 200, 60, 64, 17
    wl = _small("plane", W, H, D, 7, 7, 8, 0, -1, False)
    p = scenes.make_plane_pair(W, H, d0, seed=3)
    g = _run(lib, wl, p["left"], p["right"], aggregated=False)
    xs = np.arange(W)
    inner = (xs >= d0 + 3) & (xs <= W - 4)
    assert (g["disparity_int"][:, inner] == d0).all()


def test_constant_images(lib):
    # flat images: all codes 0, every cost 0 -> S constant per pixel -> d* = 0
    wl = _small("flat", 64, 16, 16, 5, 5, 8, 0, 1, True)
    left = np.full((16, 64), 90, dtype=np.uint8)
    g = _run(lib, wl, left, left.copy())
    o = _oracle(wl, left, left.copy())
    _compare(g, o, wl)
    assert (g["disparity_int"] == 0).all() and (g["depth"] == 0).all()


def test_host_buffers_match_device_path(lib):
    import torch
    wl = configs.SMALL_320
    p = scenes.make_pair(wl)
    with lib.SimSense.from_workload(wl) as m:
        lt = torch.from_numpy(p["left"]).pin_memory()
        rt = torch.from_numpy(p["right"]).pin_memory()
        dh = torch.empty((wl.H, wl.W), dtype=torch.float32).pin_memory()
        m.compute_host(lt, rt, dh)
        dd = m.compute(lt.cuda(), rt.cuda())
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dh.numpy(), dd.cpu().numpy())


def test_repeat_runs_are_identical(lib):
    import torch
    wl = configs.HD_720
    p = scenes.make_pair(wl)
    with lib.SimSense.from_workload(wl) as m:
        lt, rt = torch.from_numpy(p["left"]).cuda(), torch.from_numpy(p["right"]).cuda()
        a = m.compute(lt, rt).clone()
        for _ in range(3):
            b = m.compute(lt, rt)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_bad_tensor_arguments_raise(lib):
    import torch
    with lib.SimSense(64, 32, 16, 5, 5, 7, 86, 4, 0, 1, 300.0, 0.055) as m:
        good = torch.zeros((32, 64), dtype=torch.uint8, device="cuda")
        with pytest.raises(ValueError):
            m.compute(good.float(), good)
        with pytest.raises(ValueError):
            m.compute(good[:, :32], good)
        with pytest.raises(ValueError):
            m.compute(good.cpu(), good)


@pytest.mark.parametrize("W", [128, 130])
def test_unaligned_image_pointers_give_the_same_depth(lib, W):
    """Images that start at an odd byte address (the census stages its tile
    byte by byte then, a word at a time otherwise) give bit-identical depth."""
    import torch
    wl = _small("odd_base", W, 40, 48, 7, 7, 8, 15, 1, True, seed=21)
    p = scenes.make_pair(wl)
    dev = torch.device("cuda:0")
    n = wl.W * wl.H
    with lib.SimSense.from_workload(wl) as m:
        a = m.compute(torch.from_numpy(p["left"]).to(dev), torch.from_numpy(p["right"]).to(dev)).cpu().numpy()
        lb = torch.zeros(n + 3, dtype=torch.uint8, device=dev)
        rb = torch.zeros(n + 3, dtype=torch.uint8, device=dev)
        lb[1:n + 1] = torch.from_numpy(p["left"]).to(dev).reshape(-1)
        rb[3:n + 3] = torch.from_numpy(p["right"]).to(dev).reshape(-1)
        lo, ro = lb[1:n + 1].view(wl.H, wl.W), rb[3:n + 3].view(wl.H, wl.W)
        assert lo.data_ptr() % 4 == 1 and ro.data_ptr() % 4 == 3
        b = m.compute(lo, ro).cpu().numpy()
        torch.cuda.synchronize()
        assert m.device_status() == 0
    np.testing.assert_array_equal(a, b)
