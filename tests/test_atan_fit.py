"""The kernels' own atan2 (octant reduction + fitted odd polynomial): its
coefficients are the output of csrc/fit_atan.py, and a float32 emulation of
its steps stays within the stated error of the exact arctan2 in every octant,
including the signed-zero cases of IEEE atan2."""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2109_10392_gb300", "csrc")


def _fit_module():
    spec = importlib.util.spec_from_file_location("fit_atan", os.path.join(CSRC, "fit_atan.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _kernel_coefficients():
    src = open(os.path.join(CSRC, "mmpc_solve.cu")).read()
    body = src[src.index("__device__ __forceinline__ float2 atan2_pair"):]
    body = body[:body.index("float2 r = __fmul2_rn(a, p);")]
    return [float(x) for x in re.findall(r"f2\((-?[0-9.]+e[-+][0-9]+)f\)", body)]


def test_kernel_coefficients_come_from_the_fit():
    fit = _fit_module().fit()
    kern = _kernel_coefficients()
    assert len(kern) == len(fit) == 8
    assert np.allclose(np.float32(fit), np.float32(kern), rtol=0, atol=0)


def _atan2_emulated(y, x, c):
    f = np.float32
    y = np.asarray(y, f); x = np.asarray(x, f)
    ax, ay = np.abs(x), np.abs(y)
    hi = np.maximum(np.maximum(ax, ay), f(1e-30))
    a = (np.minimum(ax, ay) / hi).astype(f)
    z = (a * a).astype(f)
    p = np.full_like(a, f(c[0]))
    for cj in c[1:]:
        p = (p.astype(np.float64) * z + f(cj)).astype(f)  # one rounding, as an FMA
    r = (a * p).astype(f)
    r = np.where(ay > ax, (f(1.5707963268) - r).astype(f), r)
    r = np.where(np.signbit(x), (f(3.1415926536) - r).astype(f), r)
    return np.copysign(r, y)


def test_error_bound_all_octants():
    c = np.float32(_fit_module().fit())
    rng = np.random.default_rng(0)
    ang = rng.uniform(-np.pi, np.pi, 200000)
    rad = 10.0 ** rng.uniform(-3, 3, ang.size)
    y, x = (rad * np.sin(ang)).astype(np.float32), (rad * np.cos(ang)).astype(np.float32)
    got = _atan2_emulated(y, x, c)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    assert np.max(np.abs(got - ref)) < 4e-7


def test_special_cases():
    c = np.float32(_fit_module().fit())
    cases = [(0.0, 1.0, 0.0), (0.0, -1.0, np.pi), (-0.0, -1.0, -np.pi), (1.0, 0.0, np.pi / 2),
             (-1.0, 0.0, -np.pi / 2), (0.0, 0.0, 0.0), (1.0, 1.0, np.pi / 4), (-2.0, -2.0, -3 * np.pi / 4)]
    for y, x, want in cases:
        got = float(_atan2_emulated(np.float32(y), np.float32(x), c))
        assert abs(got - want) < 4e-7, (y, x, got, want)
