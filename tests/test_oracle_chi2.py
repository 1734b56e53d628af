"""Pins for the chi-squared approximations of Section 5.5.

A sample S of chi^2_nu has mean nu, variance 2 nu and third central moment
8 nu.  Approximation (c), A(x^2 - 1) + sqrt(2(nu - A^2)) x + nu with x ~ N(0,1),
has mean nu and variance 2 nu for any A, and third central moment
12 A nu - 4 A^3, which equals 8 nu exactly when A^3 - 3 nu A + 2 nu = 0 --
the cubic the paper gives for A.  The moments are integrated with
Gauss-Hermite quadrature, which is exact for these polynomials in x.
"""
import math

import numpy as np
import pytest

import oracle

NUS = [4.0, 16.0, 1024.0, 4096.0, 16384.0]


def _moments(kind, nu, deg=40):
    # E f(x), x ~ N(0,1): nodes of the probabilists' Hermite weight exp(-x^2/2)
    x, w = np.polynomial.hermite_e.hermegauss(deg)
    w = w / math.sqrt(2 * math.pi)
    S = np.array([oracle.chi2(kind, nu, float(xi)) for xi in x])
    m1 = float(np.sum(w * S))
    m2 = float(np.sum(w * (S - m1) ** 2))
    m3 = float(np.sum(w * (S - m1) ** 3))
    return m1, m2, m3


@pytest.mark.parametrize("nu", NUS)
def test_A_solves_cubic_and_tends_to_two_thirds(nu):
    A = oracle.chi2_A(nu)
    assert abs(A ** 3 - 3 * nu * A + 2 * nu) < 1e-12 * nu
    # A = 2/3 + O(1/nu)
    assert abs(A - 2.0 / 3.0) < 1.0 / nu


@pytest.mark.parametrize("nu", NUS)
def test_approximation_c_matches_three_moments(nu):
    m1, m2, m3 = _moments("c", nu)
    assert abs(m1 - nu) < 1e-10 * nu
    assert abs(m2 - 2 * nu) < 1e-10 * nu
    assert abs(m3 - 8 * nu) < 1e-8 * nu


@pytest.mark.parametrize("nu", NUS)
def test_approximation_a_mean_and_variance(nu):
    # S = (x + sqrt(2 nu - 1))^2 / 2: E S = nu exactly, Var S = 2 nu - 1/2
    m1, m2, _ = _moments("a", nu)
    assert abs(m1 - nu) < 1e-10 * nu
    assert abs(m2 - (2 * nu - 0.5)) < 1e-10 * nu


@pytest.mark.parametrize("nu", NUS)
def test_approximation_b_mean(nu):
    # Wilson-Hilferty: E S = nu (1 - h^3) exactly, h = 2/(9 nu)
    h = 2.0 / (9.0 * nu)
    m1, m2, _ = _moments("b", nu)
    assert abs(m1 - nu * (1 - h ** 3)) < 1e-10 * nu
    assert abs(m2 - 2 * nu) < 0.05 * nu


@pytest.mark.parametrize("nu", [4.0, 64.0, 1024.0, 16384.0])
def test_approximation_c_is_positive(nu):
    # S(x) = A x^2 + B x + (nu - A) has minimum nu - A - B^2/(4A) > 0
    A = oracle.chi2_A(nu)
    B = math.sqrt(2 * (nu - A * A))
    smin = nu - A - B * B / (4 * A)
    assert smin > 0
    xs = np.linspace(-50, 50, 20001)
    vals = np.array([oracle.chi2("c", nu, float(x)) for x in xs[::50]])
    assert vals.min() >= smin * (1 - 1e-12)
    assert abs(oracle.chi2("c", nu, -B / (2 * A)) - smin) < 1e-9 * nu


def test_correction_off_is_constant():
    assert oracle.chi2("off", 1024.0, 3.7) == 1024.0
