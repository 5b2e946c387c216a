"""The warm-start kernels (include/mmpc_mlp.h) against the FP64 oracle
(oracle/mlp_oracle.py) on the same seeded inputs: feature rows (the nearest-
obstacle order exactly, values to float32 rounding), encoding and decoding,
the network's outputs, loss and gradients with the same bfloat16-rounded
weights, and the AdamW update.  Tolerances follow from float32 accumulation
over at most 256 terms (relative 1e-5 - 1e-4 of each array's scale)."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2109_10392_gb300 import mlp, scenes

pytestmark = pytest.mark.gpu


def _dev(a, dtype=np.float32):
    import torch
    return torch.tensor(np.asarray(a, dtype=dtype), device="cuda:0").contiguous()


def _host(t):
    return t.double().cpu().numpy()


def _scene_rows(scs):
    import torch
    out, keep = [], []
    for sc in scs:
        ego, goals = _dev(sc.ego), _dev(sc.goals).reshape(-1, 3)
        obst = _dev(sc.obst).reshape(-1, 4) if sc.obst.shape[0] else None
        X = torch.zeros((goals.shape[0], 64), device="cuda:0")
        out.append(mlp.scene_row(ego=ego, obst=obst, goals=goals, X=X))
        keep.append((ego, obst, goals, X))
    return out, keep


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def test_features_match_oracle():
    import torch
    scs = [scenes.scene_custom(1, 37, 50), scenes.scene_custom(2, 5, 3), scenes.scene_custom(3, 1, 0),
           scenes.scene_custom(4, 0, 12), scenes.scene_custom(5, 9, 1024, x_range=(-500.0, 500.0))]
    # a scene with exact ties and a duplicated obstacle
    tie = scenes.scene_custom(6, 4, 6)
    tie.obst[1] = tie.obst[0]
    tie.obst[3, 0] = -tie.obst[2, 0]
    tie.obst[3, 1] = tie.obst[2, 1]
    scs.append(tie)
    rows, keep = _scene_rows(scs)
    table = mlp.SceneTable(rows, "cuda:0")
    mlp.features(table, 5.6, 2.5)
    torch.cuda.synchronize()
    for sc, (_, _, _, X) in zip(scs, keep):
        want = M.features(_f32(sc.ego), _f32(sc.obst), _f32(sc.goals), 5.6, 2.5)
        got = _host(X)
        assert got.shape == want.shape
        if want.size:
            # the slot order is an exact decision: x0 / 100 of every slot matches to rounding
            assert np.allclose(got[:, 4:54:5], want[:, 4:54:5], rtol=1e-6, atol=1e-7)
            assert np.allclose(got, want, rtol=1e-6, atol=1e-6)


def test_encode_decode_match_oracle():
    import torch
    n, T = 12, 8.0
    rng = np.random.default_rng(0)
    egos = [np.array([1.75, 14.0, 0.0, 0.0]), np.array([-5.25, 19.5, 0.02, 0.3])]
    Bs = [7, 3]
    coefs = [rng.normal(size=(B, 3 * n)) * 10 for B in Bs]
    lams = [rng.normal(size=(B, 3 * n)) for B in Bs]
    mu = rng.normal(size=6 * n)
    sigma = rng.uniform(0.5, 3.0, 6 * n)
    rows, keep = [], []
    for ego, c, l in zip(egos, coefs, lams):
        t = dict(ego=_dev(ego), coef=_dev(c), lam=_dev(l), Z=torch.zeros((c.shape[0], 6 * n), device="cuda:0"))
        keep.append(t)
        rows.append(mlp.scene_row(**t))
    table = mlp.SceneTable(rows, "cuda:0")
    mlp.warm_encode(table, n, T, _dev(mu), _dev(sigma))
    torch.cuda.synchronize()
    for ego, c, l, t in zip(egos, coefs, lams, keep):
        want = (M.encode(_f32(c), _f32(l), ego, T, n) - _f32(mu)) / _f32(sigma)
        assert np.allclose(_host(t["Z"]), want, rtol=1e-5, atol=1e-5)
    # decode the encoded rows back
    rows2, keep2 = [], []
    for ego, t in zip(egos, keep):
        B = t["Z"].shape[0]
        d = dict(ego=t["ego"], Y=t["Z"], coef=torch.zeros((B, 3 * n), device="cuda:0"),
                 lam=torch.zeros((B, 3 * n), device="cuda:0"))
        keep2.append(d)
        rows2.append(mlp.scene_row(**d))
    table2 = mlp.SceneTable(rows2, "cuda:0")
    mlp.warm_decode(table2, n, T, _dev(mu), _dev(sigma))  # 6n outputs: multipliers predicted
    torch.cuda.synchronize()
    for ego, c, l, d, t in zip(egos, coefs, lams, keep2, keep):
        wc, wl = M.decode(_host(t["Z"]) * _f32(sigma) + _f32(mu), ego, T, n)
        assert np.allclose(_host(d["coef"]), wc, rtol=1e-5, atol=1e-4)
        assert np.allclose(_host(d["lam"]), wl, rtol=1e-5, atol=1e-5)
        assert np.allclose(_host(d["coef"]), c, rtol=1e-4, atol=1e-3)


def _net(seed=0, max_batch=512):
    Ws, bs = scenes.mlp_init(seed)
    rng = np.random.default_rng(seed + 100)
    bs = [rng.normal(0, 0.1, b.shape).astype(np.float32) for b in bs]
    return Ws, bs, mlp.Mlp(scenes.WARM_WIDTHS, Ws, bs, max_batch=max_batch, weight_decay=1e-2)


def test_forward_matches_oracle():
    import torch
    Ws, bs, net = _net(1)
    rng = np.random.default_rng(2)
    for M_rows in (1, 65, 300):
        X = rng.normal(size=(M_rows, 64)).astype(np.float32)
        Y = torch.zeros((M_rows, 72), device="cuda:0")
        net.forward(_dev(X), Y)
        torch.cuda.synchronize()
        want, _ = M.forward(Ws, bs, X.astype(np.float64), bf16=True)
        got = _host(Y)
        scale = np.abs(want).max()
        assert np.max(np.abs(got - want)) <= 2e-5 * scale, (M_rows, np.max(np.abs(got - want)), scale)
    net.close()


def test_gradients_match_oracle():
    import torch
    Ws, bs, net = _net(3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(203, 64)).astype(np.float32)
    Z = rng.normal(size=(203, 72)).astype(np.float32)
    loss = torch.zeros((1,), device="cuda:0")
    net.loss_grad(_dev(X), _dev(Z), loss)
    torch.cuda.synchronize()
    L, gW, gb = M.loss_and_grads(Ws, bs, X.astype(np.float64), Z.astype(np.float64), bf16=True)
    assert abs(float(loss.item()) - L) <= 1e-5 * L
    for i in range(4):
        dW, db = net.read(mlp.READ_DW, i), net.read(mlp.READ_DB, i)
        sW, sb = np.abs(gW[i]).max(), np.abs(gb[i]).max()
        assert np.max(np.abs(dW - gW[i])) <= 1e-4 * sW, (i, np.max(np.abs(dW - gW[i])), sW)
        assert np.max(np.abs(db - gb[i])) <= 1e-4 * sb, (i, np.max(np.abs(db - gb[i])), sb)
    net.close()


def test_gradients_are_deterministic():
    import torch
    _, _, net = _net(5, max_batch=2048)
    rng = np.random.default_rng(6)
    X, Z = _dev(rng.normal(size=(2048, 64))), _dev(rng.normal(size=(2048, 72)))
    net.loss_grad(X, Z)
    a = [net.read(mlp.READ_DW, i) for i in range(4)]
    net.loss_grad(X, Z)
    torch.cuda.synchronize()
    b = [net.read(mlp.READ_DW, i) for i in range(4)]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    net.close()


def test_adamw_matches_oracle():
    import torch
    Ws, bs, net = _net(7)
    rng = np.random.default_rng(8)
    X, Z = _dev(rng.normal(size=(128, 64))), _dev(rng.normal(size=(128, 72)))
    state = [(np.zeros_like(W, dtype=np.float64), np.zeros_like(W, dtype=np.float64),
              np.zeros_like(b, dtype=np.float64), np.zeros_like(b, dtype=np.float64)) for W, b in zip(Ws, bs)]
    w = [W.astype(np.float64) for W in Ws]
    bb = [b.astype(np.float64) for b in bs]
    lr, b1, b2, eps, wd = 1e-3, 0.9, 0.999, 1e-8, 1e-2
    for step in (1, 2, 3):
        net.loss_grad(X, Z)
        gW = [net.read(mlp.READ_DW, i).astype(np.float64) for i in range(4)]
        gB = [net.read(mlp.READ_DB, i).astype(np.float64) for i in range(4)]
        net.adamw(lr)
        torch.cuda.synchronize()
        for i in range(4):
            mW, vW, mb, vb = state[i]
            w[i], mW, vW = M.adamw(w[i], gW[i], mW, vW, step, lr, b1, b2, eps, wd)
            bb[i], mb, vb = M.adamw(bb[i], gB[i], mb, vb, step, lr, b1, b2, eps, 0.0)
            state[i] = (mW, vW, mb, vb)
            gotW, gotb = net.read(mlp.READ_W, i), net.read(mlp.READ_B, i)
            assert np.max(np.abs(gotW - w[i])) <= 1e-6 + 1e-5 * lr, (step, i, np.max(np.abs(gotW - w[i])))
            assert np.max(np.abs(gotb - bb[i])) <= 1e-6 + 1e-5 * lr
            assert np.allclose(net.read(mlp.READ_MW, i), mW, rtol=1e-4, atol=1e-9)
            assert np.allclose(net.read(mlp.READ_VW, i), vW, rtol=1e-4, atol=1e-12)
    net.close()


def test_training_fits_a_smooth_map():
    """Behaviour: the kernels' training loop fits a smooth synthetic map."""
    import torch
    Ws, bs = scenes.mlp_init(9, (64, 128, 128, 8))
    net = mlp.Mlp((64, 128, 128, 8), Ws, bs, max_batch=1024, weight_decay=0.0)
    rng = np.random.default_rng(10)
    A = rng.normal(size=(64, 8)) / 8
    X = rng.normal(size=(1024, 64))
    Z = np.tanh(X @ A) + 0.1 * (X[:, :8] ** 2)
    Xd, Zd = _dev(X), _dev(Z)
    loss = torch.zeros((1,), device="cuda:0")
    first = None
    for it in range(400):
        net.loss_grad(Xd, Zd, loss)
        if it == 0:
            first = float(loss.item())
        net.adamw(3e-3)
    net.loss_grad(Xd, Zd, loss)
    last = float(loss.item())
    assert last < 0.05 * first, (first, last)
    net.close()


def test_column_stats_and_gather():
    import torch
    rng = np.random.default_rng(11)
    X = rng.normal(3.0, 2.0, size=(1000, 7)).astype(np.float32)
    X[:, 3] = 5.0  # constant column: deviation replaced by 1
    mean, sd = torch.zeros(7, device="cuda:0"), torch.zeros(7, device="cuda:0")
    mlp.column_stats(_dev(X), mean, sd)
    idx = np.array([5, 0, 999, 5, -1, 1000], dtype=np.int32)
    out = torch.zeros((6, 7), device="cuda:0")
    mlp.gather_rows(_dev(X), _dev(idx, np.int32), out)
    torch.cuda.synchronize()
    X64 = X.astype(np.float64)
    assert np.allclose(_host(mean), X64.mean(0), rtol=1e-6, atol=1e-6)
    want_sd = X64.std(0)
    want_sd[3] = 1.0
    assert np.allclose(_host(sd), want_sd, rtol=1e-5)
    got = _host(out)
    assert np.array_equal(got[:4], X64[[5, 0, 999, 5]])
    assert np.all(np.isnan(got[4:]))


def test_decode_coefficients_only_with_consistent_multipliers(orc):
    """3n outputs: the multipliers are Q c per axis (or 0 without Q)."""
    import torch
    n, T = 12, 8.0
    p = dict(scenes.BASE_PARAMS)
    Q = orc.matrices(orc.params(**p), 0)["Q"]
    rng = np.random.default_rng(3)
    ego = np.array([1.75, 12.5, 0.0, 0.0])
    Y = rng.normal(size=(9, 3 * n))
    mu, sigma = rng.normal(size=3 * n), rng.uniform(0.5, 2.0, 3 * n)
    for use_q in (True, False):
        d = dict(ego=_dev(ego), Y=_dev(Y), coef=torch.zeros((9, 3 * n), device="cuda:0"),
                 lam=torch.full((9, 3 * n), 7.0, device="cuda:0"))
        table = mlp.SceneTable([mlp.scene_row(**d)], "cuda:0")
        mlp.warm_decode(table, n, T, _dev(mu), _dev(sigma), Q=_dev(Q) if use_q else None)
        torch.cuda.synchronize()
        t = _f32(Y) * _f32(sigma) + _f32(mu)
        wc, wl = M.decode(t, ego, T, n, Q=_f32(Q) if use_q else None)
        assert np.allclose(_host(d["coef"]), wc, rtol=1e-5, atol=1e-4)
        scale = max(1.0, np.abs(wl).max())
        assert np.max(np.abs(_host(d["lam"]) - wl)) <= 1e-5 * scale


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("widths", [(64, 256, 256, 256, 36), (64, 256, 256, 256, 72), (64, 32, 16),
                                    (64, 320, 40), (60, 256, 36), (8, 16, 8, 24)])
def test_tensor_core_forward_matches_oracle(widths, mode):
    """tcgen05 inference (mode 1: TMA-fed pipeline, mode 2: single-stage
    kernel): bfloat16 layer inputs and weights, float32 accumulation --
    against the oracle with the same roundings (act_bf16), on ragged row
    counts (tails of the 128-row tile), a layer wider than one 256-column
    tile, an input width that is not a multiple of 8 (the pipeline falls back
    to the single-stage kernel), and layers narrower than one K step."""
    import torch
    Ws, bs = scenes.mlp_init(21, widths)
    rng = np.random.default_rng(22)
    bs = [rng.normal(0, 0.1, b.shape).astype(np.float32) for b in bs]
    net = mlp.Mlp(widths, Ws, bs, max_batch=256)
    net.set_tensor_cores(mode)
    for M_rows in (1, 127, 128, 300, 5000):
        X = rng.normal(size=(M_rows, widths[0])).astype(np.float32)
        Y = torch.zeros((M_rows, widths[-1]), device="cuda:0")
        net.forward(_dev(X), Y)
        net.status()
        want, _ = M.forward(Ws, bs, X.astype(np.float64), bf16=True, act_bf16=True)
        got = _host(Y)
        scale = np.abs(want).max()
        assert np.max(np.abs(got - want)) <= 3e-3 * scale, (M_rows, np.max(np.abs(got - want)), scale)
    # against the float32-activation path: the bfloat16 staging is the only difference
    X = rng.normal(size=(700, widths[0])).astype(np.float32)
    Yt = torch.zeros((700, widths[-1]), device="cuda:0")
    Ys = torch.zeros((700, widths[-1]), device="cuda:0")
    net.forward(_dev(X), Yt)
    net.set_tensor_cores(False)
    net.forward(_dev(X), Ys)
    torch.cuda.synchronize()
    d = np.abs(_host(Yt) - _host(Ys)).max() / np.abs(_host(Ys)).max()
    assert 0 < d < 3e-2, d
    net.close()


def test_tensor_core_paths_agree_at_scale():
    """The pipelined and single-stage tcgen05 GEMMs over the warm-start
    network's widths, across the inference chunk boundary (max(65536, SMs x
    512) rows): same roundings, so they differ only by the order of the
    float32 sums and the GELU evaluation; a sample of rows against the
    oracle."""
    import torch
    widths = (64, 256, 256, 256, 36)
    Ws, bs = scenes.mlp_init(5, widths)
    net = mlp.Mlp(widths, Ws, bs, max_batch=256)
    chunk = max(65536, torch.cuda.get_device_properties(0).multi_processor_count * 512)
    rows = chunk + 4465
    X = torch.randn((rows, widths[0]), device="cuda:0", generator=torch.Generator("cuda:0").manual_seed(6))
    Y1 = torch.zeros((rows, widths[-1]), device="cuda:0")
    Y2 = torch.zeros((rows, widths[-1]), device="cuda:0")
    net.set_tensor_cores(1)
    net.forward(X, Y1)
    net.set_tensor_cores(2)
    net.forward(X, Y2)
    net.status()
    scale = Y2.abs().max().item()
    assert (Y1 - Y2).abs().max().item() <= 2e-2 * scale
    idx = np.r_[0:5, chunk - 6:chunk + 5, rows - 5:rows]
    want, _ = M.forward(Ws, bs, _host(X)[idx].astype(np.float64), bf16=True, act_bf16=True)
    assert np.max(np.abs(_host(Y1)[idx] - want)) <= 3e-3 * np.abs(want).max()
    net.close()


def test_tensor_core_mode_checked():
    widths = (64, 32, 16)
    Ws, bs = scenes.mlp_init(1, widths)
    net = mlp.Mlp(widths, Ws, bs, max_batch=16)
    for bad in (-1, 3):
        with pytest.raises(RuntimeError):
            net.set_tensor_cores(bad)
    net.close()


@pytest.mark.parametrize("widths", [(64, 256, 256, 256, 72), (64, 256, 256, 256, 36), (64, 320, 40),
                                    (8, 16, 8, 24), (16, 32, 13)])
def test_tensor_core_gradients_match_oracle(widths):
    """Training on the tensor cores (forward H W, backward D W^T and weight
    gradient H^T D on the tcgen05 pipeline, bfloat16 operands, float32
    accumulation) against the oracle with the same operand roundings
    (op_bf16): ragged row counts (one row, the 128-row tile's tail, several
    tiles, splits of the weight gradient's row sum), an output width that is
    not a multiple of 8 (padded operand rows), a layer wider than one
    256-column tile.  The bfloat16 rounding of an activation or gradient
    can fall the other way where float32 and float64 pre-activations differ
    in the last bits, which moves single terms by 2^-8: hence max 1e-2 and
    RMS 2e-3 of each array's scale."""
    import torch
    Ws, bs = scenes.mlp_init(31, widths)
    rng = np.random.default_rng(32)
    bs = [rng.normal(0, 0.1, b.shape).astype(np.float32) for b in bs]
    net = mlp.Mlp(widths, Ws, bs, max_batch=2100)
    net.set_train_tensor_cores(True)
    loss = torch.zeros((1,), device="cuda:0")
    for M_rows in (1, 127, 300, 2100):
        X = rng.normal(size=(M_rows, widths[0])).astype(np.float32)
        Z = rng.normal(size=(M_rows, widths[-1])).astype(np.float32)
        net.loss_grad(_dev(X), _dev(Z), loss)
        net.status()
        L, gW, gb = M.loss_and_grads(Ws, bs, X.astype(np.float64), Z.astype(np.float64), bf16=True, op_bf16=True)
        assert abs(float(loss.item()) - L) <= 1e-3 * L, (M_rows, float(loss.item()), L)
        for i in range(len(Ws)):
            for got, want, tag in ((net.read(mlp.READ_DW, i), gW[i], "dW"), (net.read(mlp.READ_DB, i), gb[i], "db")):
                scale = np.abs(want).max()
                err = np.abs(got - want)
                assert err.max() <= 1e-2 * scale, (widths, M_rows, i, tag, err.max(), scale)
                assert np.sqrt(np.mean(err ** 2)) <= 2e-3 * scale, (widths, M_rows, i, tag)
    net.close()


def test_tensor_core_training_against_simt():
    """Same network, same batch: the tensor-core gradients differ from the
    float32 SIMT ones only by the bfloat16 operand rounding (nonzero, a few
    per mille of the scale), are bit-identical over repeated calls (fixed
    order of the split partial sums), and switching back restores the SIMT
    results exactly."""
    import torch
    widths = (64, 256, 256, 256, 72)
    Ws, bs = scenes.mlp_init(41, widths)
    net = mlp.Mlp(widths, Ws, bs, max_batch=4096)
    rng = np.random.default_rng(42)
    X, Z = _dev(rng.normal(size=(4096, 64))), _dev(rng.normal(size=(4096, 72)))
    net.loss_grad(X, Z)
    simt = [net.read(mlp.READ_DW, i) for i in range(4)]
    net.set_train_tensor_cores(True)
    net.loss_grad(X, Z)
    a = [net.read(mlp.READ_DW, i) for i in range(4)]
    net.loss_grad(X, Z)
    net.status()
    b = [net.read(mlp.READ_DW, i) for i in range(4)]
    for x, y, s in zip(a, b, simt):
        assert np.array_equal(x, y)
        d = np.abs(x - s).max() / np.abs(s).max()
        assert 0 < d < 3e-2, d
    net.set_train_tensor_cores(False)
    net.loss_grad(X, Z)
    torch.cuda.synchronize()
    for i in range(4):
        assert np.array_equal(net.read(mlp.READ_DW, i), simt[i])
    net.close()


def test_tensor_core_training_fits_a_smooth_map():
    """Behaviour: the tensor-core training loop fits the smooth synthetic map
    of the SIMT test as well."""
    import torch
    Ws, bs = scenes.mlp_init(9, (64, 128, 128, 8))
    net = mlp.Mlp((64, 128, 128, 8), Ws, bs, max_batch=1024, weight_decay=0.0)
    net.set_train_tensor_cores(True)
    rng = np.random.default_rng(10)
    A = rng.normal(size=(64, 8)) / 8
    X = rng.normal(size=(1024, 64))
    Z = np.tanh(X @ A) + 0.1 * (X[:, :8] ** 2)
    Xd, Zd = _dev(X), _dev(Z)
    loss = torch.zeros((1,), device="cuda:0")
    first = None
    for it in range(400):
        net.loss_grad(Xd, Zd, loss)
        if it == 0:
            first = float(loss.item())
        net.adamw(3e-3)
    net.loss_grad(Xd, Zd, loss)
    net.status()
    last = float(loss.item())
    assert last < 0.05 * first, (first, last)
    net.close()


def test_tensor_core_training_mode_checked():
    Ws, bs = scenes.mlp_init(1, (60, 256, 36))
    net = mlp.Mlp((60, 256, 36), Ws, bs, max_batch=16)
    with pytest.raises(RuntimeError):
        net.set_train_tensor_cores(True)  # input width 60: rows of 120 bytes
    for bad in (-1, 2):
        with pytest.raises(RuntimeError):
            net.set_train_tensor_cores(bad)
    net.close()


def test_forward_launch_count():
    """mmpc_mlp_forward_launches: one launch for the single-kernel network of
    mode 1; layer by layer otherwise (per inference chunk one per layer, plus
    the features' rounding in mode 1)."""
    import torch
    widths = (64, 256, 256, 256, 36)
    Ws, bs = scenes.mlp_init(3, widths)
    net = mlp.Mlp(widths, Ws, bs, max_batch=64)
    net.set_tensor_cores(1)
    assert net.forward_launches(0) == 0
    assert net.forward_launches(1_000_000) == 1
    net.set_tensor_cores(0)
    chunk = max(65536, torch.cuda.get_device_properties(0).multi_processor_count * 512)
    assert net.forward_launches(chunk) == 4 and net.forward_launches(chunk + 1) == 8
    net.close()
    Ws, bs = scenes.mlp_init(3, (64, 320, 40))   # a hidden layer wider than 256: layer by layer
    net = mlp.Mlp((64, 320, 40), Ws, bs, max_batch=64)
    net.set_tensor_cores(1)
    assert net.forward_launches(10) == 3
    net.close()
