"""Fits the polynomial used for GELU by the tensor-core GEMM epilogue.

GELU(x) = x Phi(x), Phi the standard normal distribution function, equals
x / 2 + g(x) with g(x) = x (Phi(x) - 1/2) = (x / 2) erf(x / sqrt 2): an even,
entire function of x, hence an entire function of t = x^2.  For |x| <= C,

    g ~ P(u),     u = 2 t / C^2 - 1 in [-1, 1],

P of degree DEG in u (monomials in the Chebyshev variable keep the float32
Horner scheme well conditioned), fitted by linear least squares in absolute
error on Chebyshev nodes of [0, C^2] in t and refined towards the minimax by
iterative reweighting (Lawson's algorithm).  For |x| > C the kernel takes
g = |x| / 2 (GELU = max(x, 0)), wrong by x (1 - Phi(|x|)) <= 1.5e-6 at C = 5; with DEG = 12 the whole
epilogue GELU is within 2e-6 of the exact one in float32 evaluation.
The evaluation needs only fused multiply-adds (two lanes per packed f32x2
instruction), no special-function unit.

    python paper_2109_10392_gb300/csrc/fit_gelu.py

prints the coefficients (highest power first, as Horner's scheme uses them)
and the maximum absolute errors of GELU in float64 and in float32 evaluation.
"""
import math

import numpy as np

DEG = 12
C = 5.0


def _lawson(V, f):
    w = np.ones(V.shape[0])
    for _ in range(300):
        c, *_ = np.linalg.lstsq(V * w[:, None], f * w, rcond=None)
        err = np.abs(V @ c - f)
        w = w * (err + 1e-30)
        w = np.sqrt(w / w.max())
    return c


def _g(x):
    return 0.5 * x * np.vectorize(math.erf)(x / math.sqrt(2.0))


def fit():
    """P's coefficients, highest power of u first."""
    k = np.arange(6001)
    u = -np.cos(np.pi * k / 6000)
    t = (u + 1.0) * (C * C / 2.0)
    V = np.stack([u ** j for j in range(DEG + 1)], axis=1)
    return _lawson(V, _g(np.sqrt(t)))[::-1]


def _fma32(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def gelu32(x, P):
    """float32 emulation of the epilogue's steps."""
    f = np.float32
    x = np.asarray(x, f)
    with np.errstate(over="ignore"):            # x^2 = inf clamps to C^2, as on the GPU
        t = np.minimum((x * x).astype(f), f(C * C))
    u = _fma32(t, f(2.0 / (C * C)), f(-1.0))
    p = np.full_like(x, f(P[0]))
    for a in P[1:]:
        p = _fma32(p, u, f(a))
    ax = np.abs(x)
    g = np.where(ax > f(C), (f(0.5) * ax).astype(f), p)
    return _fma32(f(0.5), x, g)


def gelu64(x):
    x = np.asarray(x, np.float64)
    return 0.5 * x + _g(x)


if __name__ == "__main__":
    P = fit()
    x = np.linspace(-8.0, 8.0, 400001)
    t = np.minimum(x * x, C * C)
    u = 2.0 * t / (C * C) - 1.0
    p64 = np.polyval(P, u)
    e64 = np.max(np.abs(0.5 * x + np.where(np.abs(x) > C, 0.5 * np.abs(x), p64) - gelu64(x)))
    x32 = x.astype(np.float32)
    e32 = np.max(np.abs(gelu32(x32, P).astype(np.float64) - gelu64(x32.astype(np.float64))))
    print("P =", ", ".join(f"{float(np.float32(c)):.9e}f" for c in P))
    print(f"max |error| float64 {e64:.3e}  float32 {e32:.3e}")
