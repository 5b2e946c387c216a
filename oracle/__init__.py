"""FP64 CPU oracle of the batch non-holonomic AM trajectory optimizer.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` import this package.  The product
path (the CUDA library behind ``include/mmpc.h`` and its Python binding in
``paper_2109_10392_gb300``) never imports it, and the two share no code.

This module is a ctypes wrapper around ``mmpc_oracle.c`` (plain C99, FP64),
which restates Algorithm 1 of the paper (Sec. III-E) step by step.  The
function-level parity status is listed in the header of ``mmpc_oracle.c``;
the exact trajectories on obstacle-dense scenes are "parity unpinned" (the
paper prints no worked example), everything else is pinned by the tests in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mmpc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libmmpc_oracle.so")
_lock = threading.Lock()
_lib = None

META_CRUISE = 0
META_HSRL = 1
META_ABS = 2

NEQ_X, NEQ_Y, NEQ_PSI = 5, 6, 4


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("T", ctypes.c_double),
        ("N", ctypes.c_int),
        ("n", ctypes.c_int),
        ("rho", ctypes.c_double),
        ("a", ctypes.c_double),
        ("b", ctypes.c_double),
        ("v_min", ctypes.c_double),
        ("v_max", ctypes.c_double),
        ("a_max", ctypes.c_double),
        ("iters", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("check_every", ctypes.c_int),
        ("psi_sign_printed", ctypes.c_int),
        ("basis_bits", ctypes.c_int),
        ("basis_split", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile mmpc_oracle.c into libmmpc_oracle.so next to it (gcc, FP64,
    no fast-math, no FMA contraction; OpenMP when the compiler has it)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        base = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
        return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        pp = ctypes.POINTER(OrcParams)
        L.orc_round_bits.argtypes = [ctypes.c_double, ctypes.c_int]
        L.orc_round_bits.restype = ctypes.c_double
        L.orc_invert.argtypes = [ctypes.c_int, dp, dp]
        L.orc_bernstein.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp]
        L.orc_boundary.argtypes = [dp, dp, dp, dp]
        L.orc_matrices.argtypes = [pp, ctypes.c_int] + [dp] * 11
        L.orc_qp_xy.argtypes = [pp, ctypes.c_int, dp, dp, dp, dp, dp]
        L.orc_qp_psi.argtypes = [pp, dp, dp, dp, dp, dp]
        L.orc_velocity.argtypes = [ctypes.c_double] * 4
        L.orc_velocity.restype = ctypes.c_double
        L.orc_project_obstacle.argtypes = [ctypes.c_double] * 4 + [dp, dp]
        L.orc_project_accel.argtypes = [ctypes.c_double] * 3 + [dp, dp]
        L.orc_solve.argtypes = [pp, dp, dp, ctypes.c_int, dp, ctypes.c_int, dp, dp, ctypes.c_int,
                                dp, dp, dp, ip, dp]
        L.orc_meta_cost.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 5 + [dp, ip]
        for f in ("orc_invert", "orc_bernstein", "orc_boundary", "orc_matrices", "orc_qp_xy",
                  "orc_qp_psi", "orc_solve", "orc_meta_cost"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def params(**kw) -> OrcParams:
    """OrcParams from keyword arguments (T, N, n, rho, a, b, v_min, v_max,
    a_max, iters, tol, check_every, psi_sign_printed); extra keys ignored."""
    p = OrcParams()
    p.T = float(kw["T"])
    p.N = int(kw["N"])
    p.n = int(kw["n"])
    p.rho = float(kw["rho"])
    p.a = float(kw["a"])
    p.b = float(kw["b"])
    p.v_min = float(kw["v_min"])
    p.v_max = float(kw["v_max"])
    p.a_max = float(kw["a_max"])
    p.iters = int(kw.get("iters", 100))
    p.tol = float(kw.get("tol", 0.0))
    p.check_every = int(kw.get("check_every", 1))
    p.basis_bits = int(kw.get("basis_bits", 0))
    p.basis_split = int(kw.get("basis_split", 0))
    p.psi_sign_printed = int(kw.get("psi_sign_printed", 0))
    return p


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def invert(A):
    A = _f64(A)
    out = np.empty_like(A)
    _check(lib().orc_invert(A.shape[0], _dp(A), _dp(out)), "invert")
    return out


def bernstein(N, n, T):
    P = np.empty((N, n)); Pd = np.empty((N, n)); Pdd = np.empty((N, n))
    _check(lib().orc_bernstein(N, n, float(T), _dp(P), _dp(Pd), _dp(Pdd)), "bernstein")
    return P, Pd, Pdd


def boundary(ego, goal):
    e = _f64(ego, (4,)); g = _f64(goal, (3,))
    bxy = np.empty(NEQ_X + NEQ_Y); bpsi = np.empty(NEQ_PSI)
    _check(lib().orc_boundary(_dp(e), _dp(g), _dp(bxy), _dp(bpsi)), "boundary")
    return bxy, bpsi


def matrices(p: OrcParams, m: int) -> dict:
    N, n = p.N, p.n
    R = (m + 2) * N
    dxy, dps = 2 * n + NEQ_X + NEQ_Y, n + NEQ_PSI
    out = dict(P=np.empty((N, n)), Pd=np.empty((N, n)), Pdd=np.empty((N, n)), Q=np.empty((n, n)),
               F=np.empty((2 * R, 2 * n)), Axy=np.empty((NEQ_X + NEQ_Y, 2 * n)), Apsi=np.empty((NEQ_PSI, n)),
               Kxy_inv=np.empty((dxy, dxy)), Kpsi_inv=np.empty((dps, dps)),
               K0xy_inv=np.empty((dxy, dxy)), K0psi_inv=np.empty((dps, dps)))
    keys = ["P", "Pd", "Pdd", "Q", "F", "Axy", "Apsi", "Kxy_inv", "Kpsi_inv", "K0xy_inv", "K0psi_inv"]
    _check(lib().orc_matrices(ctypes.byref(p), m, *[_dp(out[k]) for k in keys]), "matrices")
    return out


def qp_xy(p: OrcParams, m: int, g, lam, bxy):
    n = p.n
    g = _f64(g, (2 * (m + 2) * p.N,)); lam = _f64(lam, (2 * n,)); bxy = _f64(bxy, (NEQ_X + NEQ_Y,))
    c = np.empty(2 * n); mu = np.empty(NEQ_X + NEQ_Y)
    _check(lib().orc_qp_xy(ctypes.byref(p), m, _dp(g), _dp(lam), _dp(bxy), _dp(c), _dp(mu)), "qp_xy")
    return c, mu


def qp_psi(p: OrcParams, theta, lam_psi, bpsi):
    n = p.n
    th = _f64(theta, (p.N,)); lp = _f64(lam_psi, (n,)); bp = _f64(bpsi, (NEQ_PSI,))
    c = np.empty(n); mu = np.empty(NEQ_PSI)
    _check(lib().orc_qp_psi(ctypes.byref(p), _dp(th), _dp(lp), _dp(bp), _dp(c), _dp(mu)), "qp_psi")
    return c, mu


def velocity(xd, yd, v_min, v_max):
    return lib().orc_velocity(float(xd), float(yd), float(v_min), float(v_max))


def project_obstacle(wx, wy, a, b):
    al = ctypes.c_double(); d = ctypes.c_double()
    lib().orc_project_obstacle(float(wx), float(wy), float(a), float(b), ctypes.byref(al), ctypes.byref(d))
    return al.value, d.value


def project_accel(xdd, ydd, a_max):
    al = ctypes.c_double(); d = ctypes.c_double()
    lib().orc_project_accel(float(xdd), float(ydd), float(a_max), ctypes.byref(al), ctypes.byref(d))
    return al.value, d.value


def solve(p: OrcParams, ego, obst, goals, init=None, init_lam=None, nthreads=1, trace=False) -> dict:
    """Algorithm 1 for a batch.  Returns coef [B,3n] (c_x, c_y, c_psi), lam
    [B,3n], resid [B,4] (obstacle, acceleration, non-holonomic, heading
    components, Euclidean norms), iters [B] and optionally trace
    [B, iters+1, 4] (residuals after every iteration, index 0 = initial)."""
    n = p.n
    ego = _f64(ego, (4,))
    obst = _f64(obst).reshape(-1, 4) if obst is not None and np.size(obst) else np.zeros((0, 4))
    obst = np.ascontiguousarray(obst)
    m = obst.shape[0]
    goals = _f64(goals).reshape(-1, 3)
    B = goals.shape[0]
    init = None if init is None else _f64(init, (B, 3 * n))
    init_lam = None if init_lam is None else _f64(init_lam, (B, 3 * n))
    coef = np.empty((B, 3 * n)); lam = np.empty((B, 3 * n)); resid = np.empty((B, 4))
    iters = np.empty(B, dtype=np.int32)
    tr = np.empty((B, p.iters + 1, 4)) if trace else None
    rc = lib().orc_solve(ctypes.byref(p), _dp(ego), _dp(obst) if m else None, m, _dp(goals), B,
                         _dp(init), _dp(init_lam), int(nthreads), _dp(coef), _dp(lam), _dp(resid),
                         iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(tr))
    _check(rc, "solve")
    out = dict(coef=coef, lam=lam, resid=resid, iters=iters)
    if trace:
        out["trace"] = tr
    return out


def meta_cost(p: OrcParams, coef, kind=META_ABS, w1=1.0, w2=0.25, v_ref=20.0, y_ref=-5.25,
              psi_max=np.deg2rad(13.0)):
    coef = _f64(coef).reshape(-1, 3 * p.n)
    B = coef.shape[0]
    cost = np.empty(B)
    am = ctypes.c_int(-2)
    _check(lib().orc_meta_cost(ctypes.byref(p), _dp(coef), B, int(kind), float(w1), float(w2), float(v_ref),
                               float(y_ref), float(psi_max), _dp(cost), ctypes.byref(am)), "meta_cost")
    return cost, am.value


def positions(p: OrcParams, coef):
    """x(t), y(t), psi(t) samples [B, N] of coefficient rows (oracle basis)."""
    P, Pd, Pdd = bernstein(p.N, p.n, p.T)
    coef = _f64(coef).reshape(-1, 3 * p.n)
    n = p.n
    return coef[:, :n] @ P.T, coef[:, n:2 * n] @ P.T, coef[:, 2 * n:] @ P.T


def round_bits(x: float, k: int) -> float:
    """x rounded to k significant bits, ties to even (the oracle's operand
    rounding for the reduced-precision emulation)."""
    return float(lib().orc_round_bits(float(x), int(k)))
