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
