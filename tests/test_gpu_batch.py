"""Batches of scenes (mmpc_batch_*): many scenes with uneven goal counts,
obstacle counts and horizons in one persistent solve launch, one scoring
launch and a per-scene argmin.

Each scene's trajectories are computed by the same per-trajectory code as
the single-scene pair kernel (variant 2), with obstacle terms summed in index
order, so the batch must reproduce the single-scene solves bit for bit, in
any schedule, and inside a CUDA graph.  The single-scene path is itself held
to the oracle by the parity tests; one small batch is also checked against
the oracle directly here."""
import numpy as np
import pytest

from paper_2109_10392_gb300 import mmpc, scenes

from parity_utils import check_parity, f32, oracle_solve

pytestmark = pytest.mark.gpu


def _dev(a, dtype=np.float32):
    import torch
    return torch.tensor(np.asarray(a, dtype=dtype), device="cuda:0").contiguous()


def _params(sc, **kw):
    p = dict(sc.params)
    p.update(tol=1e-2, check_every=10)
    p.update(kw)
    return p


def _scene_dicts(scs, **kw):
    out = []
    for sc in scs:
        m = sc.obst.shape[0]
        out.append(dict(params=_params(sc, **kw), ego=_dev(sc.ego), obst=_dev(sc.obst).reshape(m, 4) if m else None,
                        goals=_dev(sc.goals).reshape(-1, 3)))
    return out


def _single(sd, meta):
    import torch
    p = dict(sd["params"])
    p["variant"] = 2
    s = mmpc.Solver(p, 0 if sd["obst"] is None else sd["obst"].shape[0])
    r = s.solve(sd["ego"], sd["obst"], sd["goals"])
    cost, am = s.score(meta, r.coef)
    torch.cuda.synchronize()
    out = dict(coef=r.coef.cpu().numpy(), lam=r.lam.cpu().numpy(), resid=r.resid.cpu().numpy(),
               iters=r.iters.cpu().numpy(), cost=cost.cpu().numpy(), argmin=int(am.item()))
    s.close()
    return out


def _host(o):
    return {k: (None if v is None else v.cpu().numpy()) for k, v in o.items()}


@pytest.fixture(scope="module")
def mixed():
    """12 scenes of the batching distribution, smaller B so single solves stay quick."""
    return scenes.scene_batch(7, S=12, B_range=(1, 96), m_range=(0, 40))


def test_batch_equals_single_scene_solves(mixed):
    import torch
    meta = mmpc.make_meta(**scenes.META_ABS)
    sds = _scene_dicts(mixed)
    bt = mmpc.Batch(sds, meta, want_lam=True)
    bt.run()
    torch.cuda.synchronize()
    for i, sd in enumerate(sds):
        ref = _single(sd, meta)
        got = _host(bt.out[i])
        for k in ("coef", "lam", "resid", "iters", "cost"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"scene {i} {k}")
        assert int(got["argmin"][0]) == ref["argmin"], i
    bt.close()


@pytest.mark.parametrize("schedule", [1, 2, 3, 4])
def test_schedules_agree(mixed, schedule):
    import torch
    meta = mmpc.make_meta(**scenes.META_ABS)
    sds = _scene_dicts(mixed)
    bt = mmpc.Batch(sds, meta)
    bt.run()
    torch.cuda.synchronize()
    base = [_host(o) for o in bt.out]
    bt.set_schedule(schedule)
    for o in bt.out:
        for v in o.values():
            if v is not None:
                v.zero_()
    bt.run()
    torch.cuda.synchronize()
    for i, o in enumerate(bt.out):
        h = _host(o)
        for k in ("coef", "resid", "iters", "cost", "argmin"):
            np.testing.assert_array_equal(h[k], base[i][k], err_msg=f"scene {i} {k}")
    bt.close()


def test_autotune_and_graph_replay(mixed):
    import torch
    meta = mmpc.make_meta(**scenes.META_ABS)
    sds = _scene_dicts(mixed)
    bt = mmpc.Batch(sds, meta)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        chosen = bt.autotune()
    assert chosen in (1, 2, 3, 4)
    # the launch shapes of the choice: one per horizon group in schedule 4
    # (whole warps, one CTA per trajectory, every trajectory once), else one
    for sch in (1, 4, chosen):
        bt.set_schedule(sch)
        d = bt.describe()
        assert d["schedule"] == sch
        warps = {-(-((sc["params"]["N"] + 1) // 2) // 32) for sc in sds}  # CTA size in warps per scene
        assert len(d["launches"]) == (len(warps) if sch == 4 else 1), (sch, d)
        assert sum(x["trajectories"] for x in d["launches"]) == sum(int(sc["goals"].shape[0]) for sc in sds)
        for x in d["launches"]:
            assert x["kernel"] == "fp32 pair" and x["threads"] % 32 == 0 and x["grid"] >= 1 and x["smem_bytes"] > 0
    with torch.cuda.stream(stream):
        bt.run()
    torch.cuda.synchronize()
    base = [_host(o) for o in bt.out]
    for o in bt.out:
        o["coef"].zero_()
        o["argmin"].fill_(-7)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        bt.run()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for i, o in enumerate(bt.out):
        h = _host(o)
        np.testing.assert_array_equal(h["coef"], base[i]["coef"])
        assert int(h["argmin"][0]) == int(base[i]["argmin"][0])
    ms, mk = bt.times()
    assert ms.shape == (len(sds),)
    assert np.all(ms > 0) and np.isclose(mk, ms.max())
    del g
    bt.close()


def test_batch_against_oracle():
    """Three small scenes of different N and m against the FP64 oracle."""
    import torch
    scs = [scenes.scene_custom(11, 6, 3, N=40, x_range=(-30.0, 120.0)),
           scenes.scene_custom(12, 9, 0, N=60, x_range=(-30.0, 120.0)),
           scenes.scene_custom(13, 5, 6, N=100, x_range=(-30.0, 120.0))]
    meta = mmpc.make_meta(**scenes.META_ABS)
    sds = _scene_dicts(scs, tol=0.0, iters=100)
    bt = mmpc.Batch(sds, meta)
    bt.run()
    torch.cuda.synchronize()
    for sc, sd, o in zip(scs, sds, bt.out):
        p = sd["params"]
        ego, obst, goals = f32(sc.ego), f32(sc.obst).reshape(-1, 4), f32(sc.goals)
        ref = oracle_solve(p, ego, obst, goals)
        check_parity(p, ego, obst, goals, dict(coef=o["coef"].double().cpu().numpy()), ref)
    bt.close()


def test_empty_scene_and_errors(mixed):
    import torch
    meta = mmpc.make_meta(**scenes.META_ABS)
    sds = _scene_dicts(mixed[:2])
    sds.append(dict(params=_params(mixed[0]), ego=sds[0]["ego"], obst=sds[0]["obst"],
                    goals=_dev(np.zeros((0, 3)))))
    bt = mmpc.Batch(sds, meta)
    bt.run()
    torch.cuda.synchronize()
    assert int(bt.out[2]["argmin"].item()) == -1
    with pytest.raises(mmpc.MmpcError):
        bt.set_schedule(5)
    bt.close()
    # n <= 12 and n > 12 contexts cannot share a batch
    sc16 = scenes.scene_custom(3, 4, 2, N=50, n=16)
    with pytest.raises(mmpc.MmpcError) as ei:
        mmpc.Batch(_scene_dicts([mixed[0], sc16]), meta)
    assert ei.value.code == mmpc.MMPC_ERR_SHAPE
