"""Pins of the oracle's trajectory parameterisation (Eq. param, Sec. III-B).

The paper only says the basis is "e.g. polynomials"; the oracle uses Bernstein
polynomials of degree n-1 on tau = t/T.  These tests pin the basis and both
derivative matrices by facts of the mathematics, not by re-typing them:
partition of unity, endpoint interpolation, exact reproduction of
polynomials of degree <= 2 (with their exact derivatives) and central finite
differences.
"""
import numpy as np
import pytest

SIZES = [(100, 12, 8.0), (16, 7, 3.0), (200, 16, 8.0), (2, 3, 1.0)]


@pytest.mark.parametrize("N,n,T", SIZES)
def test_partition_of_unity(orc, N, n, T):
    P, Pd, Pdd = orc.bernstein(N, n, T)
    assert np.allclose(P.sum(1), 1.0, atol=1e-13)
    assert np.allclose(Pd.sum(1), 0.0, atol=1e-11)
    assert np.allclose(Pdd.sum(1), 0.0, atol=1e-9)
    assert (P >= -1e-15).all()


@pytest.mark.parametrize("N,n,T", SIZES)
def test_endpoint_interpolation(orc, N, n, T):
    P, _, _ = orc.bernstein(N, n, T)
    e0 = np.zeros(n); e0[0] = 1
    e1 = np.zeros(n); e1[-1] = 1
    assert np.allclose(P[0], e0, atol=1e-15)
    assert np.allclose(P[-1], e1, atol=1e-15)


@pytest.mark.parametrize("N,n,T", SIZES)
def test_reproduces_linear_and_quadratic(orc, N, n, T):
    """Bernstein coefficients of tau are k/p and of tau^2 are k(k-1)/(p(p-1)),
    so x = x0 + v t + w t^2 has c_k = x0 + v T k/p + w T^2 k(k-1)/(p(p-1))."""
    P, Pd, Pdd = orc.bernstein(N, n, T)
    p = n - 1
    k = np.arange(n)
    x0, v, w = 3.7, -12.5, 0.8
    c = x0 + v * T * k / p + w * T * T * k * (k - 1) / (p * (p - 1))
    t = T * np.arange(N) / (N - 1)
    assert np.allclose(P @ c, x0 + v * t + w * t * t, atol=1e-10)
    assert np.allclose(Pd @ c, v + 2 * w * t, atol=1e-9)
    assert np.allclose(Pdd @ c, 2 * w, atol=1e-8)


def test_derivatives_match_finite_differences(orc):
    N, n, T = 4001, 12, 8.0
    P, Pd, Pdd = orc.bernstein(N, n, T)
    h = T / (N - 1)
    fd1 = (P[2:] - P[:-2]) / (2 * h)
    fd2 = (P[2:] - 2 * P[1:-1] + P[:-2]) / (h * h)
    assert np.max(np.abs(fd1 - Pd[1:-1])) < 1e-4 * np.max(np.abs(Pd))
    assert np.max(np.abs(fd2 - Pdd[1:-1])) < 1e-3 * np.max(np.abs(Pdd))


def test_rejects_bad_sizes(orc):
    with pytest.raises(RuntimeError):
        orc.bernstein(1, 12, 8.0)
    with pytest.raises(RuntimeError):
        orc.bernstein(10, 2, 8.0)
