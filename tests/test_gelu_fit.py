"""The tensor-core epilogues' GELU (x times a saturated polynomial in x^2
for Phi, no special functions): the constants in the kernel are the output
of csrc/fit_gelu.py, and a float32 emulation of its steps stays within 1.5e-6
of the exact x Phi(x) everywhere, with the exact limits (0 and x) beyond
|x| = 5."""
import importlib.util
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2109_10392_gb300", "csrc")


def _fit_module():
    spec = importlib.util.spec_from_file_location("fit_gelu", os.path.join(CSRC, "fit_gelu.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _kernel_constants():
    src = open(os.path.join(CSRC, "mmpc_mlp.cu")).read()
    body = src[src.index("__device__ __forceinline__ float2 gelu_poly2"):]
    body = body[:body.index("const float2 t = ")]
    return [float(x) for x in re.findall(r"(-?[0-9.]+e[-+][0-9]+)f", body)]


def _exact(x):
    x = np.asarray(x, np.float64)
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def test_kernel_constants_come_from_the_fit():
    mod = _fit_module()
    P = mod.fit()
    k = np.float32(_kernel_constants())
    assert len(k) == len(P) == mod.DEG + 1
    assert np.array_equal(k, np.float32(P))


def test_error_bound():
    mod = _fit_module()
    P = np.float32(mod.fit())
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-10, 10, 200000), rng.normal(0, 1.5, 200000),
                        np.float32([4.999999, 5.0, 5.000001, -5.0, -4.999999])]).astype(np.float32)
    got = mod.gelu32(x, P).astype(np.float64)
    assert np.max(np.abs(got - _exact(x))) < 1.5e-6


def test_limits_and_special_values():
    mod = _fit_module()
    P = np.float32(mod.fit())
    x = np.float32([0.0, -0.0, 6.0, 100.0, 1e30, -6.0, -100.0, -1e30])
    got = mod.gelu32(x, P)
    assert float(got[0]) == 0.0 and float(got[1]) == 0.0
    assert np.array_equal(got[2:5], x[2:5])          # GELU(x) = x beyond 5
    assert np.all(got[5:] == 0.0)                    # GELU(x) = 0 below -5
