"""Fits the odd polynomial used for atan on [0, 1] by the solve kernels.

Method: argument reduction to a = min(|x|, |y|) / max(|x|, |y|) in [0, 1]
(atan2 by octants, as in Hastings, "Approximations for Digital Computers",
1955), then atan(a) ~ a * p(a^2) with p of degree 7 in a^2, fitted by linear
least squares in relative error on 4001 Chebyshev nodes of [0, 1] and refined
by iterative reweighting towards the minimax (Lawson's algorithm).

    python paper_2109_10392_gb300/csrc/fit_atan.py

prints the coefficients (highest power first, as used by Horner's scheme)
and the maximum absolute error in float64 and in float32 evaluation.
"""
import numpy as np

DEG = 7  # polynomial degree in a^2


def fit():
    k = np.arange(4001)
    a = 0.5 - 0.5 * np.cos(np.pi * k / 4000)        # Chebyshev nodes on [0, 1]
    z = a * a
    V = np.stack([a * z ** j for j in range(DEG + 1)], axis=1)  # a * z^j
    f = np.arctan(a)
    w = np.ones_like(a)
    for _ in range(200):  # Lawson iterations towards the minimax fit
        c, *_ = np.linalg.lstsq(V * w[:, None], f * w, rcond=None)
        err = np.abs(V @ c - f)
        w = w * (err + 1e-30)
        w = np.sqrt(w / w.max())
    return c[::-1]  # highest power first


def eval32(coef, a):
    a = a.astype(np.float32)
    z = a * a
    p = np.float32(coef[0])
    for cj in coef[1:]:
        p = np.float32(p * z + np.float32(cj))
    return (a * p).astype(np.float64)


if __name__ == "__main__":
    c = fit()
    a = np.linspace(0.0, 1.0, 200001)
    e64 = np.max(np.abs(sum(ci * a * (a * a) ** (DEG - i) for i, ci in enumerate(c)) - np.arctan(a)))
    e32 = np.max(np.abs(eval32(c, a) - np.arctan(a)))
    print("coefficients (highest power first):")
    for ci in c:
        print(f"    {float(np.float32(ci)):.9e}f,")
    print(f"max abs error float64 {e64:.3e}, float32 evaluation {e32:.3e}")
