"""Batched depth stage (simsense_batch_*): every pair of a batch must give
exactly what a plain call gives for that pair alone (the same kernels run on
it, only grouped), and so match the oracle; replaying the captured graph,
re-recording it for new buffers and retuning must not change any result."""
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


def _wl(name, W, H, D, ww=7, wh=7, paths=8, uniq=0, lr=1, sub=False, seed=1, P2=86):
    return configs.Workload(name=name, W=W, H=H, D=D, win_w=ww, win_h=wh, P1=7, P2=P2, paths=paths, uniq=uniq,
                            lr_max_diff=lr, subpixel=sub, f=300.0, baseline=0.055, seed=seed,
                            scene=configs.SMALL_320.scene)


MIX = [
    _wl("a_160x90_D64", 160, 90, 64, seed=11),
    _wl("b_212x120_D96", 212, 120, 96, seed=12),
    _wl("a2_160x90_D64", 160, 90, 64, seed=13),            # same class as the first
    _wl("c_180x70_D160_9x7", 180, 70, 160, ww=9, wh=7, uniq=10, sub=True, seed=14),
    _wl("d_300x60_D256", 300, 60, 256, uniq=15, sub=True, seed=15),
    _wl("e_97x45_D48_5x5_4p", 97, 45, 48, ww=5, wh=5, paths=4, seed=16),
]


def _inputs(wls):
    import torch
    pairs = [scenes.make_pair(w) for w in wls]
    L = [torch.from_numpy(p["left"]).cuda() for p in pairs]
    R = [torch.from_numpy(p["right"]).cuda() for p in pairs]
    Z = [torch.full((w.H, w.W), -3.0, device="cuda") for w in wls]
    return pairs, L, R, Z


def _plain(lib, w, l, r):
    import torch
    with lib.SimSense.from_workload(w) as m:
        d = m.compute(l, r)
        torch.cuda.synchronize()
        return d.cpu().numpy()


@pytest.mark.parametrize("fused", [1, 0], ids=["fused", "per_class"])
def test_batch_equals_plain_and_oracle(lib, fused):
    import torch
    pairs, L, R, Z = _inputs(MIX)
    with lib.SimSenseBatch(MIX) as b:
        assert b.num_classes() == len(MIX) - 1
        b.set_schedule(fused=fused)
        b.compute(L, R, Z)
        torch.cuda.synchronize()
        assert b.device_status() == 0
        got = [z.cpu().numpy() for z in Z]
    for i, w in enumerate(MIX):
        np.testing.assert_array_equal(got[i], _plain(lib, w, L[i], R[i]))
        o = oracle.compute(pairs[i]["left"], pairs[i]["right"], w.D, w.win_w, w.win_h, w.P1, w.P2, w.paths,
                           w.uniq, w.lr_max_diff, w.subpixel, w.f, w.baseline)
        valid = o["mask"] == 0
        assert np.array_equal(got[i] != 0, valid)
        np.testing.assert_allclose(got[i][valid], o["depth"][valid], rtol=1e-5, atol=0)


def test_graph_replay_rerecord_and_eager_agree(lib):
    import torch
    _, L, R, Z = _inputs(MIX)
    with lib.SimSenseBatch(MIX) as b:
        b.compute(L, R, Z)
        first = [z.clone() for z in Z]
        for z in Z:
            z.fill_(-1.0)
        b.compute(L, R, Z)                           # replay
        torch.cuda.synchronize()
        assert all(torch.equal(a, z) for a, z in zip(first, Z))
        Z2 = [torch.empty_like(z) for z in Z]       # new buffers: the graph is re-recorded
        b.compute(L, R, Z2)
        b.set_graph(False)
        Z3 = [torch.empty_like(z) for z in Z]
        b.compute(L, R, Z3)                          # eager launches
        torch.cuda.synchronize()
        assert all(torch.equal(a, z) for a, z in zip(first, Z2))
        assert all(torch.equal(a, z) for a, z in zip(first, Z3))


def test_tuning_changes_no_result(lib):
    import torch
    _, L, R, Z = _inputs(MIX)
    with lib.SimSenseBatch(MIX) as b:
        b.compute(L, R, Z)
        ref = [z.clone() for z in Z]
        chosen = b.tune(L, R, Z, reps=1)
        assert len(chosen) == b.num_classes()
        for c, t in enumerate(chosen):
            assert t["prefetch"] in (8, 12, 16) and t["select_blocks"] in (1, 2)
        sc = b.get_schedule()
        assert sc["fused"] == 0 or {k: sc[k] for k in ("keep_paths", "lag", "order")} in \
            [{k: v for k, v in c.items() if k != "fused"} for c in SCHEDULES]
        for z in Z:
            z.fill_(0.0)
        b.compute(L, R, Z)
        torch.cuda.synchronize()
        assert all(torch.equal(a, z) for a, z in zip(ref, Z))
        b.set_schedule(fused=0)                      # the per-class form uses the per-class choices
        for c in range(b.num_classes()):
            for pf, sb in ((8, 1), (16, 2)):
                b.set_tuning(c, pf, sb)
                for z in Z:
                    z.fill_(0.0)
                b.compute(L, R, Z)
                torch.cuda.synchronize()
                assert all(torch.equal(a, z) for a, z in zip(ref, Z))


SCHEDULES = [dict(fused=1, keep_paths=k, lag=g, order=o) for o in (0, 1, 2) for g in (1, 2) for k in (0, 1)]


def test_every_schedule_gives_the_same_depth(lib):
    # the fused launch's task order, lag and store policy change when each
    # pair's work runs, never what it computes; the per-class form agrees
    import torch
    _, L, R, Z = _inputs(MIX)
    with lib.SimSenseBatch(MIX) as b:
        b.set_schedule(fused=0)
        b.compute(L, R, Z)
        torch.cuda.synchronize()
        ref = [z.clone() for z in Z]
        for sc in SCHEDULES:
            b.set_schedule(**sc)
            assert b.get_schedule() == dict(sc, prefetch=16)
            for z in Z:
                z.fill_(-5.0)
            b.compute(L, R, Z)
            torch.cuda.synchronize()
            assert b.device_status() == 0, sc
            assert all(torch.equal(a, z) for a, z in zip(ref, Z)), sc


def test_schedule_rejects_values_outside_its_sets(lib):
    from paper_2201_11924_gb300.simsense import SimsenseError
    with lib.SimSenseBatch(MIX[:2]) as b:
        for bad in (dict(fused=2), dict(prefetch=8), dict(keep_paths=3), dict(lag=0), dict(lag=3), dict(order=3)):
            with pytest.raises(SimsenseError):
                b.set_schedule(**bad)
        assert b.get_schedule() == dict(fused=1, prefetch=16, keep_paths=1, lag=1, order=1)


def test_more_pairs_than_one_launch_takes(lib):
    import torch
    wls = [_wl(f"t{i}", 64, 24, 32, ww=5, wh=5, seed=100 + i) for i in range(35)]   # 32 + 3 in one class
    _, L, R, Z = _inputs(wls)
    with lib.SimSenseBatch(wls) as b:
        assert b.num_classes() == 1
        b.compute(L, R, Z)
        torch.cuda.synchronize()
        for i in (0, 31, 32, 34):
            np.testing.assert_array_equal(Z[i].cpu().numpy(), _plain(lib, wls[i], L[i], R[i]))


def test_batch_rejects_bad_buffers(lib):
    import torch
    with lib.SimSenseBatch(MIX[:2]) as b:
        _, L, R, Z = _inputs(MIX[:2])
        with pytest.raises(ValueError):
            b.compute(L[:1], R, Z)
        with pytest.raises(ValueError):
            b.compute([L[1], L[0]], R, Z)     # wrong shapes for the pairs
