"""Pins for the oracle's Boys function F_m(T) = int_0^1 t^2m exp(-T t^2) dt
(the analytic [00|00] base case of Sec. 2.2)."""
import math

import numpy as np
import pytest
from scipy import special

import oracle


def test_zero_argument():
    # F_m(0) = 1 / (2m + 1)
    F = oracle.boys(16, 0.0)
    assert np.allclose(F, [1.0 / (2 * m + 1) for m in range(17)], rtol=0, atol=1e-16)


@pytest.mark.parametrize("T", [1e-8, 1e-3, 0.5, 3.0, 12.5, 29.99, 30.0, 45.0, 120.0])
def test_f0_closed_form(T):
    # F_0(T) = sqrt(pi/T) erf(sqrt(T)) / 2, evaluated to 40 digits (the same
    # closed form in double carries ~2 ulp of its own rounding)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    ref = float(0.5 * mpmath.sqrt(mpmath.pi / T) * mpmath.erf(mpmath.sqrt(T)))
    assert abs(oracle.boys(0, T)[0] - ref) <= 2e-16 * max(1.0, ref) + 1e-17
    # and the double closed form within its own rounding
    ref64 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(oracle.boys(0, T)[0] - ref64) <= 4e-16 * max(1.0, ref64) + 1e-16


@pytest.mark.parametrize("T", [1e-6, 0.1, 1.0, 5.0, 17.0, 29.5, 31.0, 60.0])
def test_incomplete_gamma(T):
    # F_m(T) = Gamma(m+1/2) P(m+1/2, T) / (2 T^(m+1/2)) with P scipy's regularised lower gamma
    F = oracle.boys(13, T)
    for m in range(14):
        a = m + 0.5
        ref = special.gamma(a) * special.gammainc(a, T) / (2.0 * T ** a)
        assert abs(F[m] - ref) <= 1e-13 * ref, (m, T, F[m], ref)


@pytest.mark.parametrize("T", [35.0, 80.0, 200.0])
def test_asymptote(T):
    # large T: F_m = (2m-1)!! / 2^(m+1) sqrt(pi / T^(2m+1)) up to terms of order exp(-T)
    F = oracle.boys(8, T)
    for m in range(9):
        dfact = 1.0
        for i in range(2 * m - 1, 1, -2):
            dfact *= i
        ref = dfact / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert abs(F[m] - ref) <= 1e-12 * ref + math.exp(-T)


@pytest.mark.parametrize("T", [0.01, 2.0, 9.0, 25.0, 29.9, 30.1, 50.0])
def test_downward_recursion_identity(T):
    # F_m = (2T F_{m+1} + exp(-T)) / (2m + 1)
    F = oracle.boys(12, T)
    for m in range(12):
        assert abs(F[m] - (2 * T * F[m + 1] + math.exp(-T)) / (2 * m + 1)) <= 1e-14 * F[m]


def test_monotone():
    Ts = np.linspace(0, 60, 241)
    tab = np.array([oracle.boys(10, T) for T in Ts])
    assert np.all(np.diff(tab, axis=0) <= 0)        # decreasing in T
    assert np.all(np.diff(tab, axis=1) <= 0)        # decreasing in m
