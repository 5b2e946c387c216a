"""Fits the polynomial used for GELU by the tensor-core GEMM epilogues.

GELU(x) = x Phi(x), Phi the standard normal distribution function.  Write

    Phi(x) = 1/2 + x k(x^2),     k(t) = erf(sqrt(t / 2)) / (2 sqrt t),

k an entire function of t = x^2 (k(0) = 1 / sqrt(2 pi)).  For t <= C^2

    k ~ P(u),     u = 2 t / C^2 - 1 in [-1, 1],

P of degree DEG in u (monomials in the Chebyshev variable keep the float32
Horner scheme well conditioned), fitted by linear least squares on
Chebyshev nodes of [0, C^2] in t, weighted by t (the error of k reaches GELU
multiplied by x^2), and refined towards the weighted minimax by iterative
reweighting (Lawson's algorithm).  The kernel evaluates

    GELU(x) = x sat(1/2 + x P(u(min(x^2, C^2)))),   sat = clamp to [0, 1],

one saturating fused multiply-add per lane: beyond |x| = C the clamp gives
the limits x and 0 (wrong by |x| (1 - Phi(|x|)) <= 1.5e-6 at C = 5), and no
branch or select is needed.  With DEG = 12 the float32 evaluation is within
1.5e-6 of the exact GELU everywhere.  Only fused multiply-adds (two lanes per
packed f32x2 instruction) and two minima, no special-function unit.

    python paper_2109_10392_gb300/csrc/fit_gelu.py

prints the coefficients (highest power first, as Horner's scheme uses them)
and the maximum absolute errors of GELU in float64 and in float32 evaluation.
"""
import math

import numpy as np

DEG = 12
C = 5.0


def _lawson(V, f, wt):
    w = np.ones(V.shape[0])
    for _ in range(300):
        c, *_ = np.linalg.lstsq(V * (w * wt)[:, None], f * w * wt, rcond=None)
        err = np.abs(V @ c - f) * wt
        w = w * (err + 1e-30)
        w = np.sqrt(w / w.max())
    return c


def _k(t):
    """erf(sqrt(t / 2)) / (2 sqrt t), its limit 1 / sqrt(2 pi) at t = 0."""
    t = np.asarray(t, np.float64)
    x = np.sqrt(t)
    safe = np.maximum(x, 1e-300)
    return np.where(x > 0, np.vectorize(math.erf)(x / math.sqrt(2.0)) / (2.0 * safe), 1.0 / math.sqrt(2.0 * math.pi))


def fit():
    """P's coefficients, highest power of u first."""
    k = np.arange(6001)
    u = -np.cos(np.pi * k / 6000)
    t = (u + 1.0) * (C * C / 2.0)
    V = np.stack([u ** j for j in range(DEG + 1)], axis=1)
    return _lawson(V, _k(t), t)[::-1]


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
    with np.errstate(invalid="ignore"):
        phi = np.clip(_fma32(x, p, f(0.5)), f(0.0), f(1.0))
    return (x * phi).astype(f)


def gelu64(x):
    x = np.asarray(x, np.float64)
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


if __name__ == "__main__":
    P = fit()
    x = np.linspace(-8.0, 8.0, 400001)
    t = np.minimum(x * x, C * C)
    u = 2.0 * t / (C * C) - 1.0
    phi64 = np.clip(0.5 + x * np.polyval(P, u), 0.0, 1.0)
    e64 = np.max(np.abs(x * phi64 - gelu64(x)))
    x32 = x.astype(np.float32)
    e32 = np.max(np.abs(gelu32(x32, P).astype(np.float64) - gelu64(x32.astype(np.float64))))
    print("P =", ", ".join(f"{float(np.float32(c)):.9e}f" for c in P))
    print(f"max |error| float64 {e64:.3e}  float32 {e32:.3e}")
