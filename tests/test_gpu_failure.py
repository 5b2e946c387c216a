"""The failure path of the solve kernels, without a GPU fault.

Every device wait is bounded.  A test hook (mmpc_debug_expire_wait) makes the
staging wait of the constants expect 16 bytes that no copy delivers -- a wait
on something nothing completes -- so each CTA's wait runs out after its time
limit (0.2 s, then a second bounded wait), the expiry lands in the context's
error word, the CTA returns, and mmpc_status / mmpc_batch_status report
MMPC_ERR_TIMEOUT.  The context stays usable: with the hook off, the next
solve is bit-identical to one before the failure.
"""
import time

import numpy as np
import pytest

from paper_2109_10392_gb300 import mmpc, scenes

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda:0")


def test_expired_wait_is_reported_and_the_context_stays_usable():
    import torch
    sc = scenes.scene_small(3)
    ego, obst, goals = _dev(sc.ego), _dev(sc.obst), _dev(sc.goals)
    s = mmpc.Solver(sc.params, sc.obst.shape[0])
    ref = s.solve(ego, obst, goals)
    s.status()  # nothing expired
    ref_coef = ref.coef.clone()

    s.expire_waits(True)
    t0 = time.time()
    s.solve(ego, obst, goals)
    with pytest.raises(mmpc.MmpcError) as ei:
        s.status()
    dt = time.time() - t0
    assert ei.value.code == mmpc.MMPC_ERR_TIMEOUT
    assert 0.3 < dt < 20.0, dt  # two bounded passes of 0.2 s, all CTAs at once
    s.status()  # the word was cleared

    s.expire_waits(False)
    again = s.solve(ego, obst, goals)
    s.status()
    torch.cuda.synchronize()
    assert torch.equal(again.coef, ref_coef)
    s.close()


def test_expired_wait_in_a_host_step_is_reported():
    """mmpc_step_host is synchronous: it reports the expiry itself."""
    import torch
    sc = scenes.scene_small(5)
    m, B = sc.obst.shape[0], len(sc.goals)
    s = mmpc.Solver(sc.params, m)
    meta = mmpc.make_meta(**sc.meta)
    pin = lambda a: torch.tensor(np.asarray(a, dtype=np.float32)).pin_memory()  # noqa: E731
    ego, obst, goals = pin(sc.ego), pin(sc.obst), pin(sc.goals)
    coef = torch.zeros((B, 3 * s.n)).pin_memory()
    cost = torch.zeros((B,)).pin_memory()
    am = torch.zeros((1,), dtype=torch.int32).pin_memory()
    mmpc.mmpc_step_host(s.ctx, meta, ego, obst, goals, coef, cost, am)
    ref = coef.clone()
    s.expire_waits(True)
    with pytest.raises(mmpc.MmpcError) as ei:
        mmpc.mmpc_step_host(s.ctx, meta, ego, obst, goals, coef, cost, am)
    assert ei.value.code == mmpc.MMPC_ERR_TIMEOUT
    s.expire_waits(False)
    mmpc.mmpc_step_host(s.ctx, meta, ego, obst, goals, coef, cost, am)
    assert torch.equal(coef, ref)
    s.status()
    s.close()


def test_expired_wait_in_a_batch_is_reported():
    sc = scenes.scene_small(4)
    ego, obst, goals = _dev(sc.ego), _dev(sc.obst), _dev(sc.goals)
    s = mmpc.Solver(sc.params, sc.obst.shape[0])
    s.expire_waits(True)  # taken by batches created from now on
    desc = [dict(params=sc.params, ego=ego, obst=obst, goals=goals, solver=s)]
    bad = mmpc.Batch(desc, sc.meta)
    bad.run()
    with pytest.raises(mmpc.MmpcError) as ei:
        bad.status()
    assert ei.value.code == mmpc.MMPC_ERR_TIMEOUT
    bad.close()
    s.expire_waits(False)
    good = mmpc.Batch(desc, sc.meta)
    good.run()
    good.status()
    assert np.all(np.isfinite(good.out[0]["coef"].cpu().numpy()))
    good.close()
    s.status()
    s.close()


def test_undersized_buffers_are_refused_before_any_launch():
    """The binding knows each context's N, n and m and refuses buffers too
    small for the batch (the kernels would write past them), before anything
    is enqueued; the context keeps working."""
    import torch

    from paper_2109_10392_gb300 import mlp
    sc = scenes.scene_small(6)
    m = sc.obst.shape[0]
    ego, obst, goals = _dev(sc.ego), _dev(sc.obst), _dev(sc.goals)
    B = goals.shape[0]
    s = mmpc.Solver(sc.params, m)
    n = s.n
    meta = mmpc.make_meta(**sc.meta)
    z = lambda *shape: torch.zeros(shape, device="cuda:0")  # noqa: E731
    with pytest.raises(ValueError):
        mmpc.mmpc_solve(s.ctx, ego, obst, goals, z(B, 3 * n - 1))
    with pytest.raises(ValueError):
        mmpc.mmpc_solve(s.ctx, ego, obst, goals, z(B, 3 * n), resid_out=z(B, 3))
    with pytest.raises(ValueError):
        mmpc.mmpc_solve(s.ctx, ego, obst, goals, z(B, 3 * n), warm_coef=z(B - 1, 3 * n))
    with pytest.raises(ValueError):
        mmpc.mmpc_solve(s.ctx, ego, obst, goals.reshape(-1)[: 3 * B - 1].reshape(1, -1), z(B, 3 * n))
    with pytest.raises(ValueError):
        mmpc.mmpc_score(s.ctx, meta, z(B, 3 * n), z(B - 1), torch.zeros(1, dtype=torch.int32, device="cuda:0"))
    pin = lambda *shape: torch.zeros(shape).pin_memory()  # noqa: E731
    with pytest.raises(ValueError):
        mmpc.mmpc_step_host(s.ctx, meta, ego.cpu(), obst.cpu(), goals.cpu(), pin(B, 3 * n - 2), pin(B),
                            torch.zeros(1, dtype=torch.int32))
    with pytest.raises(ValueError):
        mmpc.Batch([dict(params=sc.params, ego=ego, obst=obst, goals=goals, solver=s, warm_coef=z(B, n))], sc.meta)
    with pytest.raises(ValueError):
        mmpc.Batch.from_uniform(sc.params, ego.reshape(1, 4), obst.reshape(1, m, 4), goals.reshape(1, B, 3)[:, :-1]
                                .contiguous().reshape(1, -1), sc.meta)
    res = s.solve(ego, obst, goals)  # still fine
    torch.cuda.synchronize()
    s.status()
    assert torch.isfinite(res.coef).all()
    s.close()
    widths = (64, 32, 16)
    from paper_2109_10392_gb300 import scenes as S_
    Ws, bs = S_.mlp_init(0, widths)
    net = mlp.Mlp(widths, Ws, bs, max_batch=16)
    with pytest.raises(ValueError):
        net.forward(z(8, 64), z(8, 15))
    net.close()
