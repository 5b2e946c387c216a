"""Thin Python binding of the mmpc C ABI (include/mmpc.h).

Argument marshalling only: torch CUDA tensors are passed as raw device
pointers together with the current CUDA stream; every step of the optimizer
runs inside libmmpc.so.  There is no fallback: if the library is missing or
fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import _build

MMPC_OK = 0
MMPC_PREC_FP32, MMPC_PREC_TF32, MMPC_PREC_TF32_SPLIT, MMPC_PREC_BF16, MMPC_PREC_BF16_SPLIT = 0, 1, 2, 3, 4
MMPC_ERR_INVALID_ARG = -1
MMPC_ERR_SHAPE = -2
MMPC_ERR_CUDA = -3
MMPC_ERR_TIMEOUT = -4
MMPC_ERR_NOT_SETUP = -5

MMPC_META_CRUISE = 0
MMPC_META_HSRL = 1
MMPC_META_ABS = 2

EXPORTED = ("mmpc_problem_size", "mmpc_build", "mmpc_setup", "mmpc_solve", "mmpc_score", "mmpc_destroy",
            "mmpc_last_error", "mmpc_version", "mmpc_score_static", "mmpc_take_work_count", "mmpc_batch_create",
            "mmpc_batch_set_schedule", "mmpc_batch_autotune", "mmpc_batch_run", "mmpc_batch_times",
            "mmpc_batch_destroy", "mmpc_batch_set_fallback", "mmpc_batch_set_fallback_near", "mmpc_batch_describe", "mmpc_batch_set_timing", "mmpc_batch_fallbacks", "mmpc_step_host",
            "mmpc_measure_peaks", "mmpc_status", "mmpc_batch_status", "mmpc_debug_expire_wait")
MMPC_STATIC_SCORE_MAX_B = 65536


class MmpcParams(ctypes.Structure):
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
        ("tol", ctypes.c_float),
        ("check_every", ctypes.c_int),
        ("cull", ctypes.c_int),
        ("variant", ctypes.c_int),
        ("stall_tol", ctypes.c_float),
        ("stall_ratio", ctypes.c_float),
        ("precision", ctypes.c_int),
    ]


class MmpcMeta(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("w1", ctypes.c_float),
        ("w2", ctypes.c_float),
        ("v_ref", ctypes.c_float),
        ("y_ref", ctypes.c_float),
        ("psi_max", ctypes.c_float),
    ]


class MmpcLaunchShape(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("threads", ctypes.c_int), ("grid", ctypes.c_int),
                ("smem_bytes", ctypes.c_int), ("trajectories", ctypes.c_int)]


class MmpcScene(ctypes.Structure):
    _fields_ = [
        ("ctx", ctypes.c_void_p),
        ("ego", ctypes.c_void_p),
        ("obst", ctypes.c_void_p),
        ("goals", ctypes.c_void_p),
        ("B", ctypes.c_int),
        ("coef_out", ctypes.c_void_p),
        ("lam_out", ctypes.c_void_p),
        ("resid_out", ctypes.c_void_p),
        ("iters_out", ctypes.c_void_p),
        ("cost_out", ctypes.c_void_p),
        ("argmin_out", ctypes.c_void_p),
        ("warm_coef", ctypes.c_void_p),
        ("warm_lam", ctypes.c_void_p),
    ]


class MmpcPeaks(ctypes.Structure):
    _fields_ = [("ffma", ctypes.c_double), ("ffma2", ctypes.c_double), ("rsqrt", ctypes.c_double),
                ("ms_ffma", ctypes.c_double), ("ms_ffma2", ctypes.c_double), ("ms_rsqrt", ctypes.c_double),
                ("sms", ctypes.c_int), ("clock_khz", ctypes.c_int)]


class MmpcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mmpc error {code}: {msg}")
        self.code = code


_lib = None


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libmmpc.so (building it in-tree first when it is missing or
    older than its sources)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmmpc.so not found at {path}; run paper_2109_10392_gb300._build.build()")
    L = ctypes.CDLL(path)
    vp, dp, fp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p
    L.mmpc_problem_size.argtypes = [ctypes.c_int, ctypes.c_int]
    L.mmpc_problem_size.restype = ctypes.c_size_t
    L.mmpc_build.argtypes = [ctypes.POINTER(MmpcParams), ctypes.c_int, dp, ctypes.c_size_t]
    L.mmpc_build.restype = ctypes.c_int
    L.mmpc_setup.argtypes = [ctypes.POINTER(MmpcParams), ctypes.c_int, dp, ctypes.c_size_t, ctypes.POINTER(vp)]
    L.mmpc_setup.restype = ctypes.c_int
    L.mmpc_solve.argtypes = [vp, fp, fp, ctypes.c_int, fp, ctypes.c_int, fp, fp, fp, fp, fp, ip, vp]
    L.mmpc_solve.restype = ctypes.c_int
    L.mmpc_score.argtypes = [vp, ctypes.POINTER(MmpcMeta), fp, ctypes.c_int, fp, ip, vp]
    L.mmpc_score.restype = ctypes.c_int
    L.mmpc_destroy.argtypes = [vp]
    L.mmpc_destroy.restype = None
    L.mmpc_last_error.argtypes = [vp]
    L.mmpc_last_error.restype = ctypes.c_char_p
    L.mmpc_version.argtypes = []
    L.mmpc_version.restype = ctypes.c_int
    L.mmpc_score_static.argtypes = [ctypes.POINTER(MmpcMeta), ctypes.c_int, ctypes.c_int, fp, fp, fp, ctypes.c_int,
                                    fp, ip, vp]
    L.mmpc_score_static.restype = ctypes.c_int
    L.mmpc_take_work_count.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong)]
    L.mmpc_take_work_count.restype = ctypes.c_int
    L.mmpc_batch_create.argtypes = [ctypes.POINTER(MmpcScene), ctypes.c_int, ctypes.POINTER(MmpcMeta),
                                    ctypes.POINTER(vp)]
    L.mmpc_batch_create.restype = ctypes.c_int
    L.mmpc_batch_set_schedule.argtypes = [vp, ctypes.c_int]
    L.mmpc_batch_set_schedule.restype = ctypes.c_int
    L.mmpc_batch_autotune.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int)]
    L.mmpc_batch_autotune.restype = ctypes.c_int
    L.mmpc_batch_run.argtypes = [vp, vp]
    L.mmpc_batch_run.restype = ctypes.c_int
    L.mmpc_batch_times.argtypes = [vp, fp, ctypes.POINTER(ctypes.c_float)]
    L.mmpc_batch_times.restype = ctypes.c_int
    L.mmpc_batch_destroy.argtypes = [vp]
    L.mmpc_batch_destroy.restype = None
    L.mmpc_step_host.argtypes = [vp, ctypes.POINTER(MmpcMeta), fp, fp, ctypes.c_int, fp, ctypes.c_int, fp, fp, fp, ip,
                                 vp]
    L.mmpc_step_host.restype = ctypes.c_int
    L.mmpc_batch_set_fallback.argtypes = [vp, ctypes.c_int]
    L.mmpc_batch_set_fallback.restype = ctypes.c_int
    L.mmpc_batch_set_fallback_near.argtypes = [vp, ctypes.c_float]
    L.mmpc_batch_set_fallback_near.restype = ctypes.c_int
    L.mmpc_batch_describe.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(MmpcLaunchShape), ctypes.c_int]
    L.mmpc_batch_describe.restype = ctypes.c_int
    L.mmpc_batch_set_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_void_p)]
    L.mmpc_batch_set_timing.restype = ctypes.c_int
    L.mmpc_batch_fallbacks.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.mmpc_batch_fallbacks.restype = ctypes.c_int
    L.mmpc_measure_peaks.argtypes = [ctypes.POINTER(MmpcPeaks), ctypes.c_int, vp]
    L.mmpc_measure_peaks.restype = ctypes.c_int
    L.mmpc_status.argtypes = [vp, vp]
    L.mmpc_status.restype = ctypes.c_int
    L.mmpc_batch_status.argtypes = [vp, vp]
    L.mmpc_batch_status.restype = ctypes.c_int
    L.mmpc_debug_expire_wait.argtypes = [vp, ctypes.c_int]
    L.mmpc_debug_expire_wait.restype = ctypes.c_int
    _lib = L
    return L


def make_params(T, N, n, rho, a, b, v_min, v_max, a_max, iters=100, tol=0.0, check_every=10, cull=1, variant=0,
                stall_tol=0.0, stall_ratio=0.5, precision=0, **_ignored) -> MmpcParams:
    return MmpcParams(float(T), int(N), int(n), float(rho), float(a), float(b), float(v_min), float(v_max),
                      float(a_max), int(iters), float(tol), int(check_every), int(cull), int(variant),
                      float(stall_tol), float(stall_ratio), int(precision))


def make_meta(kind=MMPC_META_ABS, w1=1.0, w2=0.25, v_ref=20.0, y_ref=-5.25, psi_max_deg=13.0, psi_max=None,
              **_ignored) -> MmpcMeta:
    pm = float(psi_max) if psi_max is not None else math.radians(float(psi_max_deg))
    return MmpcMeta(int(kind), float(w1), float(w2), float(v_ref), float(y_ref), pm)


def _err(ctx, code):
    msg = lib().mmpc_last_error(ctx)
    raise MmpcError(code, msg.decode() if msg else "")


def mmpc_problem_size(N: int, n: int) -> int:
    return int(lib().mmpc_problem_size(int(N), int(n)))


def mmpc_build(params: MmpcParams, m: int) -> np.ndarray:
    """Host FP64 builder (basis, KKT inverse blocks); returns the packed buffer."""
    size = mmpc_problem_size(params.N, params.n)
    buf = np.zeros(max(size, 1), dtype=np.float64)
    rc = lib().mmpc_build(ctypes.byref(params), int(m), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), size)
    if rc != MMPC_OK:
        _err(None, rc)
    return buf[:size]


# (N, n, m) of every context set up here, so that the calls below can refuse
# buffers too small for the batch before anything is launched (the C ABI
# takes raw pointers and trusts their sizes)
_CTX_SHAPE: dict = {}


def _ctx_shape(ctx):
    return _CTX_SHAPE.get(getattr(ctx, "value", ctx))


def _need(t, count: int, what: str) -> None:
    if t is not None and t.numel() < count:
        raise ValueError(f"{what} holds {t.numel()} elements, the call needs {count}")


def _check_batch_inputs(ego, obst, m: int, goals) -> int:
    """B of a [B, 3] goal tensor; ego holds 4 values, obst [m, 4]."""
    B = int(goals.shape[0])
    if goals.numel() != 3 * B:
        raise ValueError("goals must be [B, 3]")
    _need(ego, 4, "ego")
    if m:
        _need(obst, 4 * m, "obst")
    return B


def mmpc_setup(params: MmpcParams, m: int, buf: np.ndarray) -> ctypes.c_void_p:
    buf = np.ascontiguousarray(buf, dtype=np.float64)
    ctx = ctypes.c_void_p()
    rc = lib().mmpc_setup(ctypes.byref(params), int(m), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          buf.size, ctypes.byref(ctx))
    if rc != MMPC_OK:
        _err(None, rc)
    _CTX_SHAPE[ctx.value] = (int(params.N), int(params.n), int(m))
    return ctx


def _ptr(t, dtype_name="float32"):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def mmpc_solve(ctx, ego, obst, goals, coef_out, warm_coef=None, warm_lam=None, lam_out=None, resid_out=None,
               iters_out=None, stream=None) -> None:
    """Enqueue Algorithm 1 for the batch on `stream` (default: torch's current
    stream).  All tensors are CUDA, contiguous, float32 (iters_out int32)."""
    m = 0 if obst is None else int(obst.shape[0])
    B = _check_batch_inputs(ego, obst, m, goals)
    shp = _ctx_shape(ctx)
    if shp is not None:
        n = shp[1]
        for t, what in ((coef_out, "coef_out"), (lam_out, "lam_out"), (warm_coef, "warm_coef"),
                        (warm_lam, "warm_lam")):
            _need(t, 3 * n * B, what)
        _need(resid_out, 4 * B, "resid_out")
        _need(iters_out, B, "iters_out")
    rc = lib().mmpc_solve(ctx, _ptr(ego), _ptr(obst) if m else None, m, _ptr(goals), B, _ptr(warm_coef),
                          _ptr(warm_lam), _ptr(coef_out), _ptr(lam_out), _ptr(resid_out),
                          _ptr(iters_out, "int32"), _stream(stream))
    if rc != MMPC_OK:
        _err(ctx, rc)


def mmpc_score(ctx, meta: MmpcMeta, coef, cost_out, argmin_out, stream=None) -> None:
    B = int(coef.shape[0])
    shp = _ctx_shape(ctx)
    if shp is not None:
        _need(coef, 3 * shp[1] * B, "coef")
    _need(cost_out, B, "cost_out")
    _need(argmin_out, 1, "argmin_out")
    rc = lib().mmpc_score(ctx, ctypes.byref(meta), _ptr(coef), B, _ptr(cost_out), _ptr(argmin_out, "int32"),
                          _stream(stream))
    if rc != MMPC_OK:
        _err(ctx, rc)


def mmpc_score_static(meta: MmpcMeta, N: int, n: int, P, Pd, coef, cost_out, argmin_out, stream=None) -> None:
    """Allocation-free scoring without a context (see include/mmpc.h): P and Pd
    are device float32 [N, n]; no device memory is allocated by the call."""
    B = int(coef.shape[0])
    _need(P, int(N) * int(n), "P")
    _need(Pd, int(N) * int(n), "Pd")
    _need(coef, 3 * int(n) * B, "coef")
    _need(cost_out, B, "cost_out")
    _need(argmin_out, 1, "argmin_out")
    rc = lib().mmpc_score_static(ctypes.byref(meta), int(N), int(n), _ptr(P), _ptr(Pd), _ptr(coef), B,
                                 _ptr(cost_out), _ptr(argmin_out, "int32"), _stream(stream))
    if rc != MMPC_OK:
        _err(None, rc)


def _hptr(t, dtype_name="float32"):
    """Host pointer of a contiguous CPU tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("expected a CPU tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def mmpc_step_host(ctx, meta: MmpcMeta, ego, obst, goals, coef_out, cost_out, argmin_out, resid_out=None,
                   stream=None) -> None:
    """One MPC step through host memory (CPU tensors, ideally pinned):
    inputs copied in, solve + score, outputs copied back, stream waited."""
    m = 0 if obst is None else int(obst.shape[0])
    B = _check_batch_inputs(ego, obst, m, goals)
    shp = _ctx_shape(ctx)
    if shp is not None:
        _need(coef_out, 3 * shp[1] * B, "coef_out")
    _need(resid_out, 4 * B, "resid_out")
    _need(cost_out, B, "cost_out")
    _need(argmin_out, 1, "argmin_out")
    rc = lib().mmpc_step_host(ctx, ctypes.byref(meta), _hptr(ego), _hptr(obst) if m else None, m, _hptr(goals), B,
                              _hptr(coef_out), _hptr(resid_out), _hptr(cost_out), _hptr(argmin_out, "int32"),
                              _stream(stream))
    if rc != MMPC_OK:
        _err(ctx, rc)


def mmpc_take_work_count(ctx) -> int:
    """Obstacle-sample pairs evaluated by this context's solves since the last
    call (synchronises the device; resets the count)."""
    out = ctypes.c_ulonglong(0)
    rc = lib().mmpc_take_work_count(ctx, ctypes.byref(out))
    if rc != MMPC_OK:
        _err(ctx, rc)
    return int(out.value)


def mmpc_measure_peaks(reps: int = 3, stream=None) -> dict:
    """Measured FP32 pipe throughput of the current device (mmpc_peaks.h):
    scalar FFMA and packed FFMA2 lane operations/s, MUFU rsqrt/s."""
    pk = MmpcPeaks()
    rc = lib().mmpc_measure_peaks(ctypes.byref(pk), int(reps), _stream(stream))
    if rc != MMPC_OK:
        raise MmpcError(rc, "mmpc_measure_peaks failed")
    return {f: getattr(pk, f) for f, _ in MmpcPeaks._fields_}


def mmpc_destroy(ctx) -> None:
    if ctx:
        _CTX_SHAPE.pop(getattr(ctx, "value", ctx), None)
        lib().mmpc_destroy(ctx)


def mmpc_last_error(ctx=None) -> str:
    return lib().mmpc_last_error(ctx).decode()


@dataclass
class SolveResult:
    coef: "object"
    lam: "object"
    resid: "object"
    iters: "object"


class Solver:
    """Owns one mmpc context (one scene size: N, n and m obstacles)."""

    def __init__(self, params: dict, m: int, problem: np.ndarray | None = None):
        self.params = make_params(**params)
        self.m = int(m)
        self.n = self.params.n
        self.problem = mmpc_build(self.params, self.m) if problem is None else problem
        self.ctx = mmpc_setup(self.params, self.m, self.problem)

    def close(self):
        if self.ctx:
            mmpc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, ego, obst, goals, warm_coef=None, warm_lam=None, stream=None, want_lam=True) -> SolveResult:
        import torch
        B = int(goals.shape[0])
        dev = goals.device
        coef = torch.empty((B, 3 * self.n), dtype=torch.float32, device=dev)
        lam = torch.empty((B, 3 * self.n), dtype=torch.float32, device=dev) if want_lam else None
        resid = torch.empty((B, 4), dtype=torch.float32, device=dev)
        iters = torch.empty((B,), dtype=torch.int32, device=dev)
        mmpc_solve(self.ctx, ego, obst, goals, coef, warm_coef, warm_lam, lam, resid, iters, stream)
        return SolveResult(coef, lam, resid, iters)

    def status(self, stream=None) -> None:
        """Raises MmpcError(MMPC_ERR_TIMEOUT) if a bounded device wait of a
        solve on this context expired since the last call (mmpc_status)."""
        rc = lib().mmpc_status(self.ctx, _stream(stream))
        if rc != MMPC_OK:
            _err(self.ctx, rc)

    def expire_waits(self, on: bool) -> None:
        """Test hook of the failure path (mmpc_debug_expire_wait)."""
        rc = lib().mmpc_debug_expire_wait(self.ctx, 1 if on else 0)
        if rc != MMPC_OK:
            _err(self.ctx, rc)

    def score(self, meta: dict | MmpcMeta, coef, stream=None):
        import torch
        mt = meta if isinstance(meta, MmpcMeta) else make_meta(**meta)
        B = int(coef.shape[0])
        cost = torch.empty((B,), dtype=torch.float32, device=coef.device)
        am = torch.empty((1,), dtype=torch.int32, device=coef.device)
        mmpc_score(self.ctx, mt, coef, cost, am, stream)
        return cost, am


def ctypes_dtype(cstruct) -> np.dtype:
    """numpy structured dtype with the field offsets of a ctypes structure
    (pointer fields as uint64), for building descriptor arrays vectorised."""
    names, formats, offsets = [], [], []
    for name, typ in cstruct._fields_:
        names.append(name)
        offsets.append(getattr(cstruct, name).offset)
        formats.append(np.int32 if typ is ctypes.c_int else np.float32 if typ is ctypes.c_float else np.uint64)
    return np.dtype(dict(names=names, formats=formats, offsets=offsets, itemsize=ctypes.sizeof(cstruct)))


def _params_key(params: dict, m: int):
    return (tuple(sorted((k, float(v)) for k, v in params.items())), int(m))


class Batch:
    """Many scenes solved and scored together (mmpc_batch_*): one persistent
    solve launch over all (scene, trajectory) items, one scoring launch, a
    per-scene argmin.  `scenes` is a list of dicts with keys params (dict),
    ego, obst (CUDA float32 tensors, obst [m, 4] or None), goals ([B, 3]) and
    optionally warm_coef, warm_lam ([B, 3n]) and solver (a caller-owned
    Solver of the scene's parameters and obstacle count, used as is and not
    closed here).  Other scenes with equal parameters and obstacle counts
    share one context.  The outputs are allocated here
    once, as flat tensors over all scenes (`flat`) with per-scene views
    (`out`); `run` only enqueues kernels, so it can be captured in a CUDA
    graph.  All scenes must have n <= 12, or all n > 12."""

    def __init__(self, scenes: list, meta: dict | MmpcMeta, want_lam: bool = False, _desc=None, _solvers=None,
                 _flat=None, _offsets=None):
        import torch
        self.meta = meta if isinstance(meta, MmpcMeta) else make_meta(**meta)
        self.handle = None
        if _desc is not None:  # prepared by from_uniform
            self.solvers, self.inputs, self.out, self.flat, self.offsets = _solvers, scenes, [], _flat, _offsets
            self.S = len(_offsets)
            desc = _desc
        else:
            self.solvers, self.inputs, self.out = [], [], []
            self.S = len(scenes)
            cache = {}
            dev = scenes[0]["goals"].device if scenes else torch.device("cuda:0")
            Bs = [int(sc["goals"].shape[0]) for sc in scenes]
            ns = [int(sc["params"]["n"]) for sc in scenes]
            tot_c = sum(3 * b * n for b, n in zip(Bs, ns))
            tot_b = sum(Bs)
            z = lambda k, dt=torch.float32: torch.zeros((k,), dtype=dt, device=dev)  # noqa: E731
            self.flat = dict(coef=z(tot_c), lam=z(tot_c) if want_lam else None, resid=z(4 * tot_b),
                             iters=z(tot_b, torch.int32), cost=z(tot_b), argmin=z(max(1, self.S), torch.int32))
            self.offsets = []
            desc = (MmpcScene * max(1, self.S))()
            oc = ob = 0
            for i, sc in enumerate(scenes):
                obst = sc["obst"]
                m = 0 if obst is None else int(obst.shape[0])
                if sc.get("solver") is not None:  # a caller-owned context, shared, not closed here
                    sv = sc["solver"]
                else:
                    key = _params_key(sc["params"], m)
                    if key not in cache:
                        cache[key] = Solver(sc["params"], m)
                        self.solvers.append(cache[key])
                    sv = cache[key]
                B, n = Bs[i], ns[i]
                _check_batch_inputs(sc["ego"], obst, m, sc["goals"])
                _need(sc.get("warm_coef"), 3 * n * B, "warm_coef")
                _need(sc.get("warm_lam"), 3 * n * B, "warm_lam")
                F = self.flat
                o = dict(coef=F["coef"][oc:oc + 3 * n * B].view(B, 3 * n),
                         lam=None if F["lam"] is None else F["lam"][oc:oc + 3 * n * B].view(B, 3 * n),
                         resid=F["resid"][4 * ob:4 * (ob + B)].view(B, 4), iters=F["iters"][ob:ob + B],
                         cost=F["cost"][ob:ob + B], argmin=F["argmin"][i:i + 1])
                self.offsets.append((oc, ob))
                oc += 3 * n * B
                ob += B
                desc[i] = MmpcScene(sv.ctx, _ptr(sc["ego"]), _ptr(obst) if m else None, _ptr(sc["goals"]), B,
                                    _ptr(o["coef"]), _ptr(o["lam"]), _ptr(o["resid"]), _ptr(o["iters"], "int32"),
                                    _ptr(o["cost"]), _ptr(o["argmin"], "int32"), _ptr(sc.get("warm_coef")),
                                    _ptr(sc.get("warm_lam")))
                self.inputs.append(sc)
                self.out.append(o)
        self.handle = ctypes.c_void_p()
        rc = lib().mmpc_batch_create(desc, self.S, ctypes.byref(self.meta), ctypes.byref(self.handle))
        if rc != MMPC_OK:
            self.handle = None
            self.close()
            _err(None, rc)

    @classmethod
    def from_uniform(cls, params: dict, ego, obst, goals, meta, warm_coef=None, warm_lam=None, want_lam=False):
        """S scenes of one shape sharing one context, from stacked device
        tensors ego [S, 4], obst [S, m, 4], goals [S, B, 3] (warm [S, B, 3n]).
        Outputs in `flat` (coef [S B, 3n], resid [S B, 4], ...), scene-major."""
        import torch
        S, B = int(goals.shape[0]), int(goals.shape[1])
        m = int(obst.shape[1]) if obst is not None else 0
        sv = Solver(params, m)
        n = sv.n
        dev = goals.device
        z = lambda *shape, dt=torch.float32: torch.zeros(shape, dtype=dt, device=dev)  # noqa: E731
        flat = dict(coef=z(S * B, 3 * n), lam=z(S * B, 3 * n) if want_lam else None, resid=z(S * B, 4),
                    iters=z(S * B, dt=torch.int32), cost=z(S * B), argmin=z(max(1, S), dt=torch.int32))
        for t in (ego, obst, goals, warm_coef, warm_lam):
            if t is not None:
                _ptr(t)  # type / contiguity checks
        if goals.numel() != 3 * S * B:
            sv.close()
            raise ValueError("goals must be [S, B, 3]")
        try:  # the per-scene pointers below step through these with fixed strides
            _need(ego, 4 * S, "ego")
            if m:
                _need(obst, 4 * m * S, "obst")
            _need(warm_coef, 3 * n * B * S, "warm_coef")
            _need(warm_lam, 3 * n * B * S, "warm_lam")
        except ValueError:
            sv.close()
            raise
        arr = np.zeros(max(1, S), dtype=ctypes_dtype(MmpcScene))
        i = np.arange(S, dtype=np.uint64)
        base = lambda t: np.uint64(t.data_ptr())  # noqa: E731
        arr["ctx"][:S] = sv.ctx.value
        arr["ego"][:S] = base(ego) + i * np.uint64(16)
        if m:
            arr["obst"][:S] = base(obst) + i * np.uint64(m * 16)
        arr["goals"][:S] = base(goals) + i * np.uint64(B * 12)
        arr["B"][:S] = B
        row = np.uint64(B * 3 * n * 4)
        arr["coef_out"][:S] = base(flat["coef"]) + i * row
        if want_lam:
            arr["lam_out"][:S] = base(flat["lam"]) + i * row
        arr["resid_out"][:S] = base(flat["resid"]) + i * np.uint64(B * 16)
        arr["iters_out"][:S] = base(flat["iters"]) + i * np.uint64(B * 4)
        arr["cost_out"][:S] = base(flat["cost"]) + i * np.uint64(B * 4)
        arr["argmin_out"][:S] = base(flat["argmin"]) + i * np.uint64(4)
        if warm_coef is not None:
            arr["warm_coef"][:S] = base(warm_coef) + i * row
        if warm_lam is not None:
            arr["warm_lam"][:S] = base(warm_lam) + i * row
        desc = (MmpcScene * max(1, S)).from_buffer_copy(arr.tobytes())
        offsets = [(i * B * 3 * n, i * B) for i in range(S)]
        keep = dict(ego=ego, obst=obst, goals=goals, warm_coef=warm_coef, warm_lam=warm_lam)
        out = cls(keep, meta, want_lam, _desc=desc, _solvers=[sv], _flat=flat, _offsets=offsets)
        out.S = S
        return out

    def set_fallback(self, on, near=None) -> None:
        """False / 0: off; True / 1: every warm-started miss; 2: only the misses
        that ran the whole iteration budget (not stopped by the stall rule);
        3: of those only the near misses, residual <= near x tol (near: the
        factor, kept when None; default 5)."""
        mode = int(on) if not isinstance(on, bool) else (1 if on else 0)
        rc = lib().mmpc_batch_set_fallback(self.handle, mode)
        if rc == MMPC_OK and near is not None:
            rc = lib().mmpc_batch_set_fallback_near(self.handle, float(near))
        if rc != MMPC_OK:
            _err(None, rc)

    def set_timing(self, events) -> None:
        """Four torch.cuda.Event(enable_timing=True) recorded around the solve
        launch(es) and the fallback launch of every run, or None (off)."""
        if events is None:
            rc = lib().mmpc_batch_set_timing(self.handle, None)
        else:
            if len(events) != 4:
                raise ValueError("set_timing needs four events")
            if any(not e.cuda_event for e in events):
                raise ValueError("set_timing: record each event once before passing it (torch creates it lazily)")
            arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) for e in events])
            self._timing_events = events  # kept alive while the library holds them
            rc = lib().mmpc_batch_set_timing(self.handle, arr)
        if rc != MMPC_OK:
            _err(None, rc)

    def status(self, stream=None) -> None:
        """Raises MmpcError(MMPC_ERR_TIMEOUT) if a bounded device wait of the
        batch's solves expired since the last call (mmpc_batch_status)."""
        rc = lib().mmpc_batch_status(self.handle, _stream(stream))
        if rc != MMPC_OK:
            _err(None, rc)

    def fallbacks(self) -> int:
        c = ctypes.c_int(0)
        rc = lib().mmpc_batch_fallbacks(self.handle, ctypes.byref(c))
        if rc != MMPC_OK:
            _err(None, rc)
        return int(c.value)

    def set_schedule(self, schedule: int) -> None:
        rc = lib().mmpc_batch_set_schedule(self.handle, int(schedule))
        if rc != MMPC_OK:
            _err(None, rc)

    def autotune(self, stream=None) -> int:
        chosen = ctypes.c_int(0)
        rc = lib().mmpc_batch_autotune(self.handle, _stream(stream), ctypes.byref(chosen))
        if rc != MMPC_OK:
            _err(None, rc)
        return int(chosen.value)

    def describe(self) -> dict:
        """The current schedule and its solve launches: a list of dicts with
        kernel ("fp32 pair" or "tensor cores"), threads, grid, smem_bytes and
        trajectories (one per horizon group in schedule 4)."""
        sch, n = ctypes.c_int(0), ctypes.c_int(0)
        rc = lib().mmpc_batch_describe(self.handle, ctypes.byref(sch), ctypes.byref(n), None, 0)
        if rc == MMPC_OK and n.value > 0:
            arr = (MmpcLaunchShape * n.value)()
            rc = lib().mmpc_batch_describe(self.handle, None, None, arr, n.value)
        if rc != MMPC_OK:
            _err(None, rc)
        return dict(schedule=int(sch.value), launches=[
            dict(kernel="tensor cores" if a.kernel == 1 else "fp32 pair", threads=a.threads, grid=a.grid,
                 smem_bytes=a.smem_bytes, trajectories=a.trajectories) for a in (arr if n.value > 0 else [])])

    def run(self, stream=None) -> None:
        rc = lib().mmpc_batch_run(self.handle, _stream(stream))
        if rc != MMPC_OK:
            _err(None, rc)

    def times(self):
        """(per-scene completion times in ms since the first CTA started, makespan)."""
        ms = np.zeros(max(1, self.S), dtype=np.float32)
        mk = ctypes.c_float(0.0)
        rc = lib().mmpc_batch_times(self.handle, ctypes.c_void_p(ms.ctypes.data), ctypes.byref(mk))
        if rc != MMPC_OK:
            _err(None, rc)
        return ms[:self.S], float(mk.value)

    def take_work_count(self) -> int:
        """Obstacle-sample pairs evaluated by the batch's runs (summed over scenes)."""
        return sum(mmpc_take_work_count(s.ctx) for s in self.solvers)

    def close(self):
        if getattr(self, "handle", None):
            lib().mmpc_batch_destroy(self.handle)
            self.handle = None
        for s in getattr(self, "solvers", []):
            s.close()
        self.solvers = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _time_scene(goals: int, obstacles: int, N: int, n: int, iters: int, reps: int, seed: int, tol: float = 1e-2,
                variant: int = 0, precision: int = 0) -> dict:
    """Times solve + score of one seeded highway scene (goals, obstacles, N, n)
    with CUDA events between L2 flushes: median of `reps` steps (after three
    untimed ones)."""
    import torch

    from . import scenes
    sc = scenes.scene_custom(seed, goals, obstacles, N=N, n=n, x_range=(-50.0, 250.0))
    params = dict(sc.params, iters=iters, tol=tol, check_every=10, variant=variant, precision=precision)
    s = Solver(params, obstacles)
    meta = make_meta(**sc.meta)
    dev = torch.device("cuda:0")
    t = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev).contiguous()  # noqa: E731
    ego, obst, gl = t(sc.ego), t(sc.obst), t(sc.goals)
    coef = torch.empty((goals, 3 * s.n), device=dev)
    resid = torch.empty((goals, 4), device=dev)
    cost = torch.empty(goals, device=dev)
    am = torch.empty(1, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ms = []
    for i in range(reps + 3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        mmpc_solve(s.ctx, ego, obst if obstacles else None, gl, coef, resid_out=resid)
        mmpc_score(s.ctx, meta, coef, cost, am)
        b.record()
        torch.cuda.synchronize()
        if i >= 3:
            ms.append(a.elapsed_time(b))
    s.status()
    s.close()
    ms.sort()
    return dict(goals=goals, obstacles=obstacles, N=N, n=n, iters=iters, tol=tol, variant=variant,
                precision=precision, reps=reps, ms_median=ms[len(ms) // 2],
                trajectories_per_s=goals / (ms[len(ms) // 2] * 1e-3), best_goal=int(am.item()))


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="time solve + score of one seeded highway scene on cuda:0")
    ap.add_argument("--goals", type=int, default=11)
    ap.add_argument("--obstacles", type=int, default=10)
    ap.add_argument("--N", type=int, default=100)
    ap.add_argument("--n", type=int, default=12)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--reps", type=int, default=100)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-2)
    ap.add_argument("--variant", type=int, default=0, help="solve kernel (3: tensor cores, needs --precision)")
    ap.add_argument("--precision", type=int, default=0, help="MMPC_PREC_*: 1 TF32, 2 TF32 hi+lo, 3 BF16, 4 BF16 hi+lo")
    a = ap.parse_args()
    print(json.dumps(_time_scene(a.goals, a.obstacles, a.N, a.n, a.iters, a.reps, a.seed, a.tol, a.variant,
                                 a.precision)))
