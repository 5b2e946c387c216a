"""The kernels' own heading sin/cos (Cody-Waite reduction by pi/2 + fitted
polynomials): the coefficients in the kernel are the output of
csrc/fit_sincos.py, and a float32 emulation of its steps stays within an ulp
of the exact sin and cos over the heading range, in every quadrant."""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2109_10392_gb300", "csrc")


def _fit_module():
    spec = importlib.util.spec_from_file_location("fit_sincos", os.path.join(CSRC, "fit_sincos.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _kernel_constants():
    src = open(os.path.join(CSRC, "mmpc_solve.cu")).read()
    body = src[src.index("__device__ __forceinline__ void sincos_pair"):]
    body = body[:body.index("const float2 s = ")]
    return [float(x) for x in re.findall(r"f2\((-?[0-9.]+e[-+][0-9]+)f\)", body)]


def test_kernel_constants_come_from_the_fit():
    mod = _fit_module()
    S, C = mod.fit()
    k = np.float32(_kernel_constants())
    # order in the kernel: 2/pi, pi/2 head, pi/2 tail, S (highest first), C (highest first)
    assert len(k) == 3 + len(S) + len(C) == 9
    assert k[0] == np.float32(2.0 / np.pi)
    assert k[1] == mod.PIO2_HI and k[2] == mod.PIO2_LO
    assert np.float64(mod.PIO2_HI) + np.float64(mod.PIO2_LO) == np.float64(np.float32(np.pi / 2)) + \
        np.float64(np.float32(np.pi / 2 - np.float64(np.float32(np.pi / 2))))
    assert np.array_equal(k[3:6], np.float32(S))
    assert np.array_equal(k[6:9], np.float32(C))


def test_error_within_an_ulp():
    mod = _fit_module()
    S, C = (np.float32(v) for v in mod.fit())
    rng = np.random.default_rng(0)
    psi = np.concatenate([rng.uniform(-20.0, 20.0, 300000), rng.uniform(-0.5, 0.5, 100000)]).astype(np.float32)
    sn, cs = mod.sincos32(psi, S, C)
    p = psi.astype(np.float64)
    assert np.max(np.abs(sn - np.sin(p))) < 1.2e-7
    assert np.max(np.abs(cs - np.cos(p))) < 1.2e-7
    # relative accuracy near zero, where sin psi ~ psi
    small = np.abs(p) < 0.1
    assert np.max(np.abs(sn[small] - np.sin(p[small])) / np.maximum(np.abs(np.sin(p[small])), 1e-30)) < 2e-7


def test_quadrants_and_special_values():
    mod = _fit_module()
    S, C = (np.float32(v) for v in mod.fit())
    pts = np.float32([0.0, -0.0, np.pi / 4, -np.pi / 4, np.pi / 2, -np.pi / 2, 3 * np.pi / 4, np.pi, -np.pi,
                      5 * np.pi / 4, 3 * np.pi / 2, -3 * np.pi / 2, 2 * np.pi, 1e-20, -7.0, 13.0])
    sn, cs = mod.sincos32(pts, S, C)
    p = pts.astype(np.float64)
    assert np.max(np.abs(sn - np.sin(p))) < 1.2e-7
    assert np.max(np.abs(cs - np.cos(p))) < 1.2e-7
    assert sn[0] == 0.0 and cs[0] == 1.0
    # sin^2 + cos^2 = 1 to float32 accuracy everywhere
    psi = np.linspace(-20, 20, 100001).astype(np.float32)
    sn, cs = mod.sincos32(psi, S, C)
    assert np.max(np.abs(sn * sn + cs * cs - 1.0)) < 3e-7
