"""Fits the polynomials used for sin and cos of the heading by the solve kernels.

Method: Cody and Waite's argument reduction (Cody & Waite, "Software Manual
for the Elementary Functions", 1980): q = rint(psi 2/pi) and
r = psi - q pi/2 in two steps, with pi/2 split into a float32 head and a
float32 tail, so r lies in [-pi/4, pi/4] and (sin, cos) of psi follow from
(sin r, cos r) by the quadrant q mod 4.  On the reduced range

    sin r ~ r + r^3 S(r^2),        cos r ~ 1 - r^2 / 2 + r^4 C(r^2),

with S and C of degree DEG in r^2, fitted by linear least squares in
absolute error on 4001 Chebyshev nodes of [0, pi/4] and refined by
iterative reweighting towards the minimax (Lawson's algorithm).

    python paper_2109_10392_gb300/csrc/fit_sincos.py

prints the two coefficient lists (highest power first, as used by Horner's
scheme), the split of pi/2 and the maximum absolute errors in float64 and in
float32 evaluation.
"""
import numpy as np

DEG = 2                 # degree of S and C in r^2
PIO2_HI = np.float32(np.pi / 2)
PIO2_LO = np.float32(np.pi / 2 - np.float64(PIO2_HI))


def _lawson(V, f):
    w = np.ones(V.shape[0])
    for _ in range(200):
        c, *_ = np.linalg.lstsq(V * w[:, None], f * w, rcond=None)
        err = np.abs(V @ c - f)
        w = w * (err + 1e-30)
        w = np.sqrt(w / w.max())
    return c


def fit():
    """(S, C): coefficients, highest power of r^2 first."""
    k = np.arange(4001)
    r = np.pi / 8 - np.pi / 8 * np.cos(np.pi * k / 4000)   # Chebyshev nodes on [0, pi/4]
    z = r * r
    Vs = np.stack([r ** 3 * z ** j for j in range(DEG + 1)], axis=1)
    Vc = np.stack([z * z * z ** j for j in range(DEG + 1)], axis=1)
    S = _lawson(Vs, np.sin(r) - r)
    C = _lawson(Vc, np.cos(r) - 1.0 + 0.5 * z)
    return S[::-1], C[::-1]


def _fma32(a, b, c):
    """float32 fused multiply-add: one rounding of the exact a b + c."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(np.float32)


def sincos32(psi, S, C):
    """float32 emulation of the kernels' steps (every operation rounded as on
    the GPU; the FMAs with one rounding)."""
    f = np.float32
    psi = np.asarray(psi, f)
    q = np.rint((psi * f(2.0 / np.pi)).astype(f)).astype(f)
    r = _fma32(-q, PIO2_HI, psi)
    r = _fma32(-q, PIO2_LO, r)
    z = (r * r).astype(f)
    ps = np.full_like(z, f(S[0]))
    for cj in S[1:]:
        ps = _fma32(ps, z, f(cj))
    pc = np.full_like(z, f(C[0]))
    for cj in C[1:]:
        pc = _fma32(pc, z, f(cj))
    s = _fma32((z * r).astype(f), ps, r)
    c = _fma32(z, _fma32(z, pc, f(-0.5)), f(1.0))
    j = q.astype(np.int64) & 3
    sn = np.where(j == 0, s, np.where(j == 1, c, np.where(j == 2, -s, -c)))
    cs = np.where(j == 0, c, np.where(j == 1, -s, np.where(j == 2, -c, s)))
    return sn.astype(np.float64), cs.astype(np.float64)


if __name__ == "__main__":
    S, C = fit()
    r = np.linspace(0.0, np.pi / 4, 200001)
    z = r * r
    es = np.max(np.abs(r + r ** 3 * np.polyval(S, z) - np.sin(r)))
    ec = np.max(np.abs(1 - z / 2 + z * z * np.polyval(C, z) - np.cos(r)))
    psi = np.linspace(-20.0, 20.0, 400001).astype(np.float32)
    sn, cs = sincos32(psi, np.float32(S), np.float32(C))
    p64 = psi.astype(np.float64)
    e32 = max(np.max(np.abs(sn - np.sin(p64))), np.max(np.abs(cs - np.cos(p64))))
    print("sin polynomial S (highest power first):")
    for ci in S:
        print(f"    {float(np.float32(ci)):.9e}f,")
    print("cos polynomial C (highest power first):")
    for ci in C:
        print(f"    {float(np.float32(ci)):.9e}f,")
    print(f"pi/2 = {float(PIO2_HI):.9e}f + {float(PIO2_LO):.9e}f")
    print(f"max abs error float64: sin {es:.3e}, cos {ec:.3e}; float32 evaluation on [-20, 20]: {e32:.3e}")
