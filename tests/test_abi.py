"""CPU checks of the C-ABI library: it builds, loads and exports every entry
point include/mmpc.h declares; its host FP64 builder (mmpc_build, an
implementation independent of the oracle's: de Casteljau basis, LU-based KKT
inverse) reproduces the oracle's matrices; and argument errors are reported
before any CUDA call.  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2109_10392_gb300 import mmpc, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mmpc_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol():
    from paper_2109_10392_gb300 import mlp
    L = mmpc.lib()
    names = _declared()
    assert set(names) == set(mmpc.EXPORTED) | set(mlp.EXPORTED)
    for name in names:
        assert hasattr(L, name), name
    assert L.mmpc_version() == 2


def _split(buf, N, n):
    sizes = [("t", N), ("P", N * n), ("Pd", N * n), ("Pdd", N * n), ("lin", n), ("Q", n * n), ("K11x", n * n),
             ("K11y", n * n), ("K11p", n * n), ("K12p", n * 4), ("K12x", n * 5), ("K12y", n * 6), ("C0x", n * 5),
             ("C0y", n * 6), ("C0p", n * 4)]
    out, o = {}, 0
    for k, s in sizes:
        out[k] = buf[o:o + s]
        o += s
    assert o == buf.size
    return out


@pytest.mark.parametrize("N,n,m", [(100, 12, 50), (40, 7, 0), (200, 16, 30), (37, 10, 3)])
def test_builder_matches_oracle(orc, N, n, m):
    kw = dict(scenes.BASE_PARAMS)
    kw.update(N=N, n=n)
    buf = mmpc.mmpc_build(mmpc.make_params(**kw), m)
    assert buf.size == mmpc.mmpc_problem_size(N, n) == N + 3 * N * n + n + 4 * n * n + 30 * n
    S = _split(buf, N, n)
    op = orc.params(**kw)
    M = orc.matrices(op, m)
    for key in ("P", "Pd", "Pdd"):
        assert np.allclose(S[key].reshape(N, n), M[key], rtol=1e-12, atol=1e-12 * np.abs(M[key]).max())
    assert np.allclose(S["Q"].reshape(n, n), M["Q"], rtol=1e-10, atol=1e-10 * np.abs(M["Q"]).max())
    assert np.allclose(S["t"], kw["T"] * np.arange(N) / (N - 1))
    assert np.allclose(M["P"] @ S["lin"], S["t"], atol=1e-12)
    # KKT blocks: the oracle's xy inverse is over (c_x, c_y, mu_x, mu_y)
    Kxy = M["Kxy_inv"]
    tol = dict(rtol=1e-7, atol=1e-9 * np.abs(Kxy).max())
    assert np.allclose(S["K11x"].reshape(n, n), Kxy[:n, :n], **tol)
    assert np.allclose(S["K11y"].reshape(n, n), Kxy[n:2 * n, n:2 * n], **tol)
    assert np.allclose(S["K12x"].reshape(n, 5), Kxy[:n, 2 * n:2 * n + 5], **tol)
    assert np.allclose(S["K12y"].reshape(n, 6), Kxy[n:2 * n, 2 * n + 5:], **tol)
    Kp = M["Kpsi_inv"]
    assert np.allclose(S["K11p"].reshape(n, n), Kp[:n, :n], rtol=1e-7, atol=1e-9 * np.abs(Kp).max())
    assert np.allclose(S["K12p"].reshape(n, 4), Kp[:n, n:], rtol=1e-7, atol=1e-9 * np.abs(Kp).max())
    K0 = M["K0xy_inv"]
    assert np.allclose(S["C0x"].reshape(n, 5), K0[:n, 2 * n:2 * n + 5], rtol=1e-6, atol=1e-8 * np.abs(K0).max())
    assert np.allclose(S["C0y"].reshape(n, 6), K0[n:2 * n, 2 * n + 5:], rtol=1e-6, atol=1e-8 * np.abs(K0).max())
    K0p = M["K0psi_inv"]
    assert np.allclose(S["C0p"].reshape(n, 4), K0p[:n, n:], rtol=1e-6, atol=1e-8 * np.abs(K0p).max())


def test_builder_argument_errors():
    good = dict(scenes.BASE_PARAMS)
    for bad, code in [(dict(N=4), mmpc.MMPC_ERR_SHAPE), (dict(n=17), mmpc.MMPC_ERR_SHAPE),
                      (dict(rho=0.0), mmpc.MMPC_ERR_INVALID_ARG), (dict(v_min=0.0), mmpc.MMPC_ERR_INVALID_ARG),
                      (dict(check_every=0), mmpc.MMPC_ERR_INVALID_ARG), (dict(a=-1.0), mmpc.MMPC_ERR_INVALID_ARG)]:
        kw = dict(good)
        kw.update(bad)
        with pytest.raises(mmpc.MmpcError) as ei:
            mmpc.mmpc_build(mmpc.make_params(**kw), 10)
        assert ei.value.code == code, bad
    for m in (-1, 1025):
        with pytest.raises(mmpc.MmpcError) as ei:
            mmpc.mmpc_build(mmpc.make_params(**good), m)
        assert ei.value.code == mmpc.MMPC_ERR_SHAPE
    assert mmpc.mmpc_problem_size(4, 12) == 0
    assert mmpc.mmpc_problem_size(100, 17) == 0


def test_calls_without_context_fail_cleanly():
    L = mmpc.lib()
    meta = mmpc.make_meta()
    assert L.mmpc_solve(None, None, None, 0, None, 0, None, None, None, None, None, None, None) == mmpc.MMPC_ERR_NOT_SETUP
    assert L.mmpc_score(None, ctypes.byref(meta), None, 0, None, None, None) == mmpc.MMPC_ERR_NOT_SETUP
    assert L.mmpc_last_error(None)
    L.mmpc_destroy(None)
    # batches: argument and context checks come before any CUDA call
    out = ctypes.c_void_p()
    assert L.mmpc_batch_create(None, 1, ctypes.byref(meta), ctypes.byref(out)) == mmpc.MMPC_ERR_INVALID_ARG
    desc = (mmpc.MmpcScene * 2)()
    assert L.mmpc_batch_create(desc, 0, ctypes.byref(meta), ctypes.byref(out)) == mmpc.MMPC_ERR_INVALID_ARG
    assert L.mmpc_batch_create(desc, 2, ctypes.byref(meta), ctypes.byref(out)) == mmpc.MMPC_ERR_NOT_SETUP
    assert not out.value
    bad = mmpc.make_meta(kind=9)
    assert L.mmpc_batch_create(desc, 2, ctypes.byref(bad), ctypes.byref(out)) == mmpc.MMPC_ERR_INVALID_ARG
    assert L.mmpc_batch_run(None, None) == mmpc.MMPC_ERR_NOT_SETUP
    assert L.mmpc_batch_set_schedule(None, 1) == mmpc.MMPC_ERR_NOT_SETUP
    assert L.mmpc_batch_times(None, None, None) == mmpc.MMPC_ERR_NOT_SETUP
    L.mmpc_batch_destroy(None)
    # the peak probe checks its arguments before touching the device
    pk = mmpc.MmpcPeaks()
    assert L.mmpc_measure_peaks(None, 3, None) == mmpc.MMPC_ERR_INVALID_ARG
    assert L.mmpc_measure_peaks(ctypes.byref(pk), 0, None) == mmpc.MMPC_ERR_INVALID_ARG
    # status and the failure-path hook need a context or batch
    assert L.mmpc_status(None, None) == mmpc.MMPC_ERR_NOT_SETUP
    assert L.mmpc_batch_status(None, None) == mmpc.MMPC_ERR_NOT_SETUP
    assert L.mmpc_debug_expire_wait(None, 1) == mmpc.MMPC_ERR_NOT_SETUP


def test_setup_rejects_bad_buffers():
    p = mmpc.make_params(**scenes.BASE_PARAMS)
    buf = mmpc.mmpc_build(p, 5)
    with pytest.raises(mmpc.MmpcError) as ei:
        mmpc.mmpc_setup(p, 5, buf[:-1])
    assert ei.value.code == mmpc.MMPC_ERR_INVALID_ARG
    bad = buf.copy()
    bad[7] = np.nan
    with pytest.raises(mmpc.MmpcError) as ei:
        mmpc.mmpc_setup(p, 5, bad)
    assert ei.value.code == mmpc.MMPC_ERR_INVALID_ARG


def test_warm_start_calls_check_arguments_first():
    from paper_2109_10392_gb300 import mlp
    L = mlp.lib()
    assert L.mmpc_features(None, -1, 5.6, 2.5, None) == mmpc.MMPC_ERR_INVALID_ARG
    assert L.mmpc_features(None, 0, 0.0, 2.5, None) == mmpc.MMPC_ERR_INVALID_ARG
    assert L.mmpc_warm_decode(None, 0, 3, 8.0, 9, None, None, None, None) == mmpc.MMPC_ERR_INVALID_ARG
    assert L.mmpc_warm_encode(None, 0, 12, 8.0, 37, None, None, None) == mmpc.MMPC_ERR_INVALID_ARG
    assert L.mmpc_column_stats(None, 0, 1, None, None, None) == mmpc.MMPC_ERR_INVALID_ARG
    cfg = mlp.MlpConfig()
    cfg.layers = 0
    out = ctypes.c_void_p()
    W = (ctypes.c_void_p * 1)()
    assert L.mmpc_mlp_create(ctypes.byref(cfg), W, W, ctypes.byref(out)) == mmpc.MMPC_ERR_INVALID_ARG
    cfg.layers, cfg.width[0], cfg.width[1], cfg.max_batch = 1, 4, 2000, 8   # width above the limit
    cfg.beta1, cfg.beta2, cfg.eps = 0.9, 0.999, 1e-8
    assert L.mmpc_mlp_create(ctypes.byref(cfg), W, W, ctypes.byref(out)) == mmpc.MMPC_ERR_INVALID_ARG
    assert L.mmpc_mlp_forward(None, None, 0, None, None) == mmpc.MMPC_ERR_NOT_SETUP
    assert L.mmpc_mlp_adamw(None, 1e-3, None) == mmpc.MMPC_ERR_NOT_SETUP
    assert L.mmpc_mlp_last_error()
    L.mmpc_mlp_destroy(None)
