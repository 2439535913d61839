"""The bounded device-side waits give up with a status instead of hanging.

SIMSENSE_OPT_TEST_STALL makes the cost stage's MMA-issuing thread issue no
tensor-core work, so no wait on its completions can be satisfied (a flag that
nothing sets); each wait runs out after its short test limit, the stage frees
its tensor memory and returns.  The call reports SIMSENSE_ERR_TIMEOUT through
the device status word, and the same handle then computes correctly.
"""
import numpy as np
import pytest

import oracle
from paper_2201_11924_gb300 import configs, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2201_11924_gb300 import _build, simsense
    _build.build()
    return simsense


@pytest.mark.parametrize("D,win", [(64, (7, 7)), (200, (9, 7))])
def test_stalled_cost_stage_reports_timeout_and_recovers(lib, D, win):
    import torch
    wl = configs.SMALL_320.with_(W=300, H=64, D=D, win_w=win[0], win_h=win[1], paths=8, uniq=10, subpixel=True)
    p = scenes.make_pair(wl)
    dev = torch.device("cuda:0")
    L = torch.from_numpy(p["left"]).to(dev)
    R = torch.from_numpy(p["right"]).to(dev)
    with lib.SimSense.from_workload(wl) as m:
        m.compute(L, R)
        torch.cuda.synchronize()
        assert m.device_status() == 0
        m.set_option(lib.OPT_TEST_STALL, 1)
        m.compute(L, R)
        torch.cuda.synchronize()
        assert m.device_status() == lib.ERR_TIMEOUT
        assert m.device_status() == 0            # reading the status clears it
        m.set_option(lib.OPT_TEST_STALL, 0)
        depth = m.compute(L, R)
        torch.cuda.synchronize()
        assert m.device_status() == 0
        got = depth.cpu().numpy()
    o = oracle.compute(p["left"], p["right"], wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq,
                       wl.lr_max_diff, wl.subpixel, wl.f, wl.baseline)
    valid = o["mask"] == 0
    assert np.array_equal(got != 0, valid)
    np.testing.assert_allclose(got[valid], o["depth"][valid], rtol=1e-5, atol=0)


def test_stall_option_range(lib):
    wl = configs.SMALL_320.with_(W=64, H=32, D=16, win_w=5, win_h=5)
    with lib.SimSense.from_workload(wl) as m:
        for bad in (-1, 2):
            with pytest.raises(lib.SimsenseError):
                m.set_option(lib.OPT_TEST_STALL, bad)


def test_fused_batch_wait_gives_up_and_recovers(lib):
    # the fused batch launch's selection rows wait (bounded) for their pair's
    # path work; with that work left out of the task list for pair 0
    # (SIMSENSE_BATCH_OPT_TEST_STALL), every such wait gives up: the launch
    # reports the timeout, the other pair is computed as usual, and the batch
    # then computes every pair again
    import numpy as np
    import torch
    from paper_2201_11924_gb300 import configs, scenes
    mk = lambda name, W, H, D, seed: configs.Workload(
        name=name, W=W, H=H, D=D, win_w=7, win_h=7, P1=7, P2=86, paths=8, uniq=15, lr_max_diff=1, subpixel=True,
        f=300.0, baseline=0.055, seed=seed, scene=configs.SMALL_320.scene)
    wls = [mk("p0", 96, 24, 48, 31), mk("p1", 160, 60, 64, 32)]
    pairs = [scenes.make_pair(w) for w in wls]
    L = [torch.from_numpy(p["left"]).cuda() for p in pairs]
    R = [torch.from_numpy(p["right"]).cuda() for p in pairs]
    Z = [torch.zeros((w.H, w.W), device="cuda") for w in wls]
    with lib.SimSenseBatch(wls) as b:
        b.set_schedule(fused=1)
        b.compute(L, R, Z)
        torch.cuda.synchronize()
        assert b.device_status() == 0
        ref = [z.clone() for z in Z]
        b.set_option(lib.BATCH_OPT_TEST_STALL, 1)
        for z in Z:
            z.fill_(-2.0)
        b.compute(L, R, Z)
        torch.cuda.synchronize()
        assert b.device_status() == lib.ERR_TIMEOUT
        assert torch.equal(Z[1], ref[1])
        assert b.device_status() == 0                    # the status was cleared by the read
        b.set_option(lib.BATCH_OPT_TEST_STALL, 0)
        b.compute(L, R, Z)
        torch.cuda.synchronize()
        assert b.device_status() == 0
        assert all(torch.equal(a, z) for a, z in zip(ref, Z))
        np.testing.assert_array_equal(Z[0].cpu().numpy(), ref[0].cpu().numpy())
