"""Thin Python binding of the warm-start C ABI (include/mmpc_mlp.h).

Argument marshalling only: torch CUDA tensors go to libmmpc.so as raw device
pointers with the current CUDA stream; the features, the network's forward,
backward and AdamW steps, and the encoding all run in the library's kernels.
No fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import mmpc

FEATURES = 64
MAX_LAYERS = 8
EXPORTED = ("mmpc_features", "mmpc_warm_decode", "mmpc_warm_encode", "mmpc_column_stats", "mmpc_gather_rows",
            "mmpc_standardize",
            "mmpc_mlp_create", "mmpc_mlp_forward", "mmpc_mlp_loss_grad", "mmpc_mlp_adamw", "mmpc_mlp_read",
            "mmpc_mlp_write", "mmpc_mlp_destroy", "mmpc_mlp_last_error", "mmpc_mlp_set_tensor_cores",
            "mmpc_mlp_set_train_tensor_cores", "mmpc_mlp_forward_launches", "mmpc_mlp_status")
READ_W, READ_B, READ_DW, READ_DB, READ_MW, READ_VW, READ_MB, READ_VB = range(8)


class WarmScene(ctypes.Structure):
    _fields_ = [
        ("ego", ctypes.c_void_p),
        ("obst", ctypes.c_void_p),
        ("m", ctypes.c_int),
        ("goals", ctypes.c_void_p),
        ("B", ctypes.c_int),
        ("X", ctypes.c_void_p),
        ("Y", ctypes.c_void_p),
        ("coef", ctypes.c_void_p),
        ("lam", ctypes.c_void_p),
        ("Z", ctypes.c_void_p),
    ]


class MlpConfig(ctypes.Structure):
    _fields_ = [
        ("layers", ctypes.c_int),
        ("width", ctypes.c_int * (MAX_LAYERS + 1)),
        ("max_batch", ctypes.c_int),
        ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float),
        ("eps", ctypes.c_float),
        ("weight_decay", ctypes.c_float),
    ]


_bound = False


def lib():
    global _bound
    L = mmpc.lib()
    if _bound:
        return L
    vp, ip, fp = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    L.mmpc_features.argtypes = [vp, ip, fp, fp, vp]
    L.mmpc_warm_decode.argtypes = [vp, ip, ip, fp, ip, vp, vp, vp, vp]
    L.mmpc_warm_encode.argtypes = [vp, ip, ip, fp, ip, vp, vp, vp]
    L.mmpc_column_stats.argtypes = [vp, ip, ip, vp, vp, vp]
    L.mmpc_gather_rows.argtypes = [vp, ip, ip, vp, ip, vp, vp]
    L.mmpc_standardize.argtypes = [vp, ip, ip, vp, vp, vp, vp]
    L.mmpc_mlp_create.argtypes = [ctypes.POINTER(MlpConfig), ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.mmpc_mlp_forward.argtypes = [vp, vp, ip, vp, vp]
    L.mmpc_mlp_loss_grad.argtypes = [vp, vp, vp, ip, vp, vp]
    L.mmpc_mlp_adamw.argtypes = [vp, fp, vp]
    L.mmpc_mlp_read.argtypes = [vp, ip, ip, vp, ctypes.c_size_t]
    L.mmpc_mlp_write.argtypes = [vp, ip, ip, vp, ctypes.c_size_t]
    L.mmpc_mlp_set_tensor_cores.argtypes = [vp, ip]
    L.mmpc_mlp_set_train_tensor_cores.argtypes = [vp, ip]
    L.mmpc_mlp_forward_launches.argtypes = [vp, ip]
    L.mmpc_mlp_status.argtypes = [vp]
    L.mmpc_mlp_destroy.argtypes = [vp]
    L.mmpc_mlp_destroy.restype = None
    L.mmpc_mlp_last_error.argtypes = []
    L.mmpc_mlp_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("mmpc_mlp_destroy", "mmpc_mlp_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _bound = True
    return L


def _check(rc):
    if rc != mmpc.MMPC_OK:
        raise mmpc.MmpcError(rc, lib().mmpc_mlp_last_error().decode())


_ptr = mmpc._ptr
_stream = mmpc._stream
_need = mmpc._need


class SceneTable:
    """A device array of mmpc_warm_scene descriptors (kept alive with the
    tensors it points to)."""

    def __init__(self, rows: list, device):
        import torch
        self.rows = rows
        arr = (WarmScene * max(1, len(rows)))(*[WarmScene(**r) for r in rows])
        raw = np.frombuffer(bytes(arr), dtype=np.uint8)
        self.dev = torch.from_numpy(raw.copy()).to(device)
        self.S = len(rows)

    @property
    def ptr(self):
        return ctypes.c_void_p(self.dev.data_ptr())


def uniform_table(device, ego=None, obst=None, goals=None, X=None, Y=None, coef=None, lam=None, Z=None, S=None):
    """A SceneTable of S scenes of one shape from stacked tensors: ego [S, 4],
    obst [S, m, 4], goals [S, B, 3], X [S, B, 64], Y / Z [S, B, 6n],
    coef / lam [S, B, 3n] (any may be None)."""
    ts = [t for t in (goals, X, Y, coef, lam, Z) if t is not None]
    S = int(ts[0].shape[0]) if S is None else S
    B = int(ts[0].shape[1])
    m = 0 if obst is None else int(obst.shape[1])
    arr = np.zeros(max(1, S), dtype=mmpc.ctypes_dtype(WarmScene))
    i = np.arange(S, dtype=np.uint64)
    for name, t in (("ego", ego), ("obst", obst), ("goals", goals), ("X", X), ("Y", Y), ("coef", coef), ("lam", lam),
                    ("Z", Z)):
        if t is None or (name == "obst" and m == 0):
            continue
        _ptr(t)
        arr[name][:S] = np.uint64(t.data_ptr()) + i * np.uint64(t[0].numel() * 4)
    arr["m"][:S] = m
    arr["B"][:S] = B
    tab = SceneTable([], device)
    import torch
    tab.dev = torch.from_numpy(np.frombuffer(arr.tobytes(), dtype=np.uint8).copy()).to(device)
    tab.S = S
    return tab


def scene_row(ego=None, obst=None, goals=None, X=None, Y=None, coef=None, lam=None, Z=None):
    """Descriptor fields from CUDA tensors (None -> NULL)."""
    m = 0 if obst is None else int(obst.shape[0])
    B = 0 if goals is None else int(goals.shape[0])
    if goals is None:
        for t in (X, Y, coef, lam, Z):
            if t is not None:
                B = int(t.shape[0])
                break
    p = lambda t: None if t is None else _ptr(t).value  # noqa: E731
    return dict(ego=p(ego), obst=p(obst) if m else None, m=m, goals=p(goals), B=B, X=p(X), Y=p(Y), coef=p(coef),
                lam=p(lam), Z=p(Z))


def features(table: SceneTable, a: float, b: float, stream=None):
    _check(lib().mmpc_features(table.ptr, table.S, float(a), float(b), _stream(stream)))


def warm_decode(table: SceneTable, n: int, T: float, mu, sigma, Q=None, stream=None):
    """outputs = mu.numel() (3n or 6n); Q: device float32 [n, n] or None."""
    _check(lib().mmpc_warm_decode(table.ptr, table.S, int(n), float(T), int(mu.numel()), _ptr(mu), _ptr(sigma),
                                  _ptr(Q), _stream(stream)))


def warm_encode(table: SceneTable, n: int, T: float, mu, sigma, stream=None):
    """outputs = mu.numel() (3n or 6n)."""
    _check(lib().mmpc_warm_encode(table.ptr, table.S, int(n), float(T), int(mu.numel()), _ptr(mu), _ptr(sigma),
                                  _stream(stream)))


def column_stats(X, mean_out, std_out, stream=None):
    rows, cols = int(X.shape[0]), int(X.shape[1])
    _need(mean_out, cols, "mean_out")
    _need(std_out, cols, "std_out")
    _check(lib().mmpc_column_stats(_ptr(X), rows, cols, _ptr(mean_out), _ptr(std_out), _stream(stream)))


def standardize(X, mean, sd, out, stream=None):
    _need(mean, int(X.shape[1]), "mean")
    _need(sd, int(X.shape[1]), "sd")
    _need(out, X.numel(), "out")
    _check(lib().mmpc_standardize(_ptr(X), int(X.shape[0]), int(X.shape[1]), _ptr(mean), _ptr(sd), _ptr(out),
                                  _stream(stream)))


def gather_rows(src, idx, out, stream=None):
    _need(out, int(idx.shape[0]) * int(src.shape[1]), "out")
    _check(lib().mmpc_gather_rows(_ptr(src), int(src.shape[0]), int(src.shape[1]), _ptr(idx, "int32"),
                                  int(idx.shape[0]), _ptr(out), _stream(stream)))


class Mlp:
    """Owns one mmpc_mlp (weights, gradients, AdamW moments, activations)."""

    def __init__(self, widths, Ws, bs, max_batch=4096, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4):
        L = len(widths) - 1
        cfg = MlpConfig()
        cfg.layers = L
        for i, w in enumerate(widths):
            cfg.width[i] = int(w)
        cfg.max_batch = int(max_batch)
        cfg.beta1, cfg.beta2, cfg.eps, cfg.weight_decay = beta1, beta2, eps, weight_decay
        self.widths = [int(w) for w in widths]
        self._W = [np.ascontiguousarray(W, dtype=np.float32) for W in Ws]
        self._b = [np.ascontiguousarray(b, dtype=np.float32) for b in bs]
        for i, (W, b) in enumerate(zip(self._W, self._b)):
            assert W.shape == (widths[i], widths[i + 1]) and b.shape == (widths[i + 1],)
        Wp = (ctypes.c_void_p * L)(*[W.ctypes.data for W in self._W])
        bp = (ctypes.c_void_p * L)(*[b.ctypes.data for b in self._b])
        self.handle = ctypes.c_void_p()
        _check(lib().mmpc_mlp_create(ctypes.byref(cfg), Wp, bp, ctypes.byref(self.handle)))
        self.max_batch = int(max_batch)

    def forward(self, X, Y, stream=None):
        M = int(X.shape[0])
        _need(X, M * self.widths[0], "X")
        _need(Y, M * self.widths[-1], "Y")
        _check(lib().mmpc_mlp_forward(self.handle, _ptr(X), int(X.shape[0]), _ptr(Y), _stream(stream)))

    def loss_grad(self, X, Z, loss=None, stream=None):
        M = int(X.shape[0])
        _need(X, M * self.widths[0], "X")
        _need(Z, M * self.widths[-1], "Z")
        _need(loss, 1, "loss")
        _check(lib().mmpc_mlp_loss_grad(self.handle, _ptr(X), _ptr(Z), int(X.shape[0]), _ptr(loss), _stream(stream)))

    def set_tensor_cores(self, on):
        """False/0: SIMT; True/1: the TMA-fed tcgen05 pipeline; 2: the single-stage tcgen05 GEMM."""
        _check(lib().mmpc_mlp_set_tensor_cores(self.handle, int(on)))

    def set_train_tensor_cores(self, on):
        """False/0: training on the FP32 SIMT kernels; True/1: its three
        products per layer on the tcgen05 pipeline (bfloat16 operands)."""
        _check(lib().mmpc_mlp_set_train_tensor_cores(self.handle, int(on)))

    def forward_launches(self, rows):
        """Kernel launches a forward pass over `rows` rows enqueues."""
        k = lib().mmpc_mlp_forward_launches(self.handle, int(rows))
        if k < 0:
            raise RuntimeError("mmpc_mlp_forward_launches: bad arguments")
        return k

    def status(self):
        _check(lib().mmpc_mlp_status(self.handle))

    def adamw(self, lr, stream=None):
        _check(lib().mmpc_mlp_adamw(self.handle, float(lr), _stream(stream)))

    def read(self, what, layer):
        i, o = self.widths[layer], self.widths[layer + 1]
        shape = (i, o) if what in (READ_W, READ_DW, READ_MW, READ_VW) else (o,)
        out = np.zeros(shape, dtype=np.float32)
        _check(lib().mmpc_mlp_read(self.handle, int(what), int(layer), ctypes.c_void_p(out.ctypes.data), out.size))
        return out

    def write(self, what, layer, arr):
        a = np.ascontiguousarray(arr, dtype=np.float32)
        _check(lib().mmpc_mlp_write(self.handle, int(what), int(layer), ctypes.c_void_p(a.ctypes.data), a.size))

    def weights(self):
        L = len(self.widths) - 1
        return [self.read(READ_W, i) for i in range(L)], [self.read(READ_B, i) for i in range(L)]

    def close(self):
        if getattr(self, "handle", None):
            lib().mmpc_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _time_forward(rows: int, reps: int = 10, seed: int = 0) -> list:
    """Times one forward pass of the warm-start network (64 -> 256 x 3 -> 36,
    seeded random weights) over `rows` random rows: FP32 SIMT path (mode 0),
    the single-stage tcgen05 GEMM (2) and the TMA-fed pipeline (1); CUDA
    events, median of reps."""
    import torch

    from . import scenes
    widths = (64, 256, 256, 256, 36)
    Ws, bs = scenes.mlp_init(seed, widths)
    net = Mlp(widths, Ws, bs, max_batch=4096)
    flops = 2.0 * rows * sum(i * o for i, o in zip(widths[:-1], widths[1:]))
    X = torch.randn((rows, widths[0]), device="cuda:0")
    Y = torch.empty((rows, widths[-1]), device="cuda:0")
    out = []
    for on in (0, 2, 1):
        net.set_tensor_cores(on)
        net.forward(X, Y)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            net.forward(X, Y)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = float(np.median(ts))
        out.append(dict(rows=rows, tensor_cores=on, ms=ms, tflops=flops / (ms * 1e-3) / 1e12))
    net.status()
    net.close()
    return out


def _time_train(batch: int = 4096, reps: int = 50, seed: int = 0) -> list:
    """Times one training step (loss and gradients, then AdamW) of the
    warm-start network (64 -> 256 x 3 -> 72, seeded random weights) on a
    random batch: FP32 SIMT kernels, then the tensor-core products; CUDA
    events over `reps` consecutive steps.  FLOPs: the forward products, the
    weight gradients and the backward products of every layer but the first."""
    import torch

    from . import scenes
    widths = (64, 256, 256, 256, 72)
    Ws, bs = scenes.mlp_init(seed, widths)
    net = Mlp(widths, Ws, bs, max_batch=batch)
    prods = [i * o for i, o in zip(widths[:-1], widths[1:])]
    flops = 2.0 * batch * (2 * sum(prods) + sum(prods[1:]))
    g = torch.Generator("cuda:0").manual_seed(seed)
    X = torch.randn((batch, widths[0]), device="cuda:0", generator=g)
    Z = torch.randn((batch, widths[-1]), device="cuda:0", generator=g)
    loss = torch.zeros((1,), device="cuda:0")
    out = []
    for on in (0, 1):
        net.set_train_tensor_cores(on)
        for _ in range(3):
            net.loss_grad(X, Z, loss)
            net.adamw(1e-4)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            net.loss_grad(X, Z, loss)
            net.adamw(1e-4)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        out.append(dict(batch=batch, train_tensor_cores=on, ms_per_step=ms, tflops=flops / (ms * 1e-3) / 1e12))
    net.status()
    net.close()
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="time the warm-start network's forward pass and training step")
    ap.add_argument("--rows", type=int, nargs="+", default=[65536, 1 << 20])
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--train-batch", type=int, nargs="*", default=[],
                    help="also time one training step at these batch sizes")
    a = ap.parse_args()
    for r in a.rows:
        for line in _time_forward(r, a.reps):
            print(json.dumps(line), flush=True)
    for bsz in a.train_batch:
        for line in _time_train(bsz):
            print(json.dumps(line), flush=True)
