"""Pins of the oracle's multipliers (Eq. 3-5), rational interpolation (Sec. 2) and Psi stencils.

Each check rests on something other than the oracle's own formula: Taylor coefficients worked out
by hand from Eq. 3-5, special cases with closed forms, the paper's stated interpolation accuracy,
and the Fourier symbol of the (1,-2,1) operator.
"""
import math

import numpy as np
import pytest

import oracle as O

ALPHAS = [0.1, 0.3, 0.45, 0.5, 0.55, 0.7]


@pytest.mark.parametrize("alpha", ALPHAS)
def test_multiplier_taylor(alpha):
    # M_G = 1 + (1 - 2 a^2) s^2 / 3 + O(s^4)
    # M_U = 1 + (1 - 4 a^2) s^2 / 6 + O(s^4)
    # M_M = 1 - (1 + 2 a^2) s^2 / 3 + O(s^4)
    expect = {O.GALERKIN: (1 - 2 * alpha ** 2) / 3, O.UNIFORM: (1 - 4 * alpha ** 2) / 6,
              O.MOMENTUM: -(1 + 2 * alpha ** 2) / 3}
    for scheme, c2 in expect.items():
        for s in (1e-2, 2e-2):
            m = O.multiplier(scheme, alpha, s)
            # the remainder after the s^2 term is O(s^4): divided by s^2 it is O(s^2)
            assert abs((m - 1) / s ** 2 - c2) < 0.5 * s ** 2, (scheme, alpha, s)
        assert O.multiplier(scheme, alpha, 0.0) == 1.0


def test_magic_step_uniform_is_one():
    # Sec. 4: Uniform at v dt/dz = 1/2 is the magic time step; Eq. 4 is identically 1 there.
    for s in np.linspace(1e-3, math.pi / 2, 50):
        assert abs(O.multiplier(O.UNIFORM, 0.5, s) - 1.0) < 1e-15


def test_galerkin_half_is_asin_ratio():
    # Eq. 3 at alpha = 1/2 reduces to s / sin s = asin(sqrt(xi)) / sqrt(xi).
    for xi in np.linspace(0.01, 1.0, 40):
        s = math.asin(math.sqrt(xi))
        assert abs(O.multiplier(O.GALERKIN, 0.5, s) - math.asin(math.sqrt(xi)) / math.sqrt(xi)) < 1e-14


def test_scheme_ratios():
    # Eq. 3 / Eq. 4 = s / sin s and Eq. 5 / Eq. 4 = cos s, for every alpha.
    for a in ALPHAS:
        for s in (0.3, 0.9, 1.4):
            mu = O.multiplier(O.UNIFORM, a, s)
            assert abs(O.multiplier(O.GALERKIN, a, s) / mu - s / math.sin(s)) < 1e-14
            assert abs(O.multiplier(O.MOMENTUM, a, s) / mu - math.cos(s)) < 1e-14


def _ratio(pe, pb, xi):
    return np.polyval(pe[::-1], xi) / np.polyval(pb[::-1], xi)


@pytest.mark.parametrize("scheme", [O.GALERKIN, O.UNIFORM])
@pytest.mark.parametrize("alpha", [0.1, 0.3, 0.45, 0.55, 0.7])
def test_rational_interpolation(scheme, alpha):
    st, pe, pb = O.rational_coeffs(scheme, alpha)
    assert st == 0
    # normalisation and DC gain
    assert pb[0] == 1.0 and abs(pe[0] - 1.0) < 1e-12
    # the interpolant passes through all nine nodes xi_j = j/8
    for j in range(9):
        xi = j / 8
        m = O.multiplier(scheme, alpha, math.asin(math.sqrt(xi)))
        assert abs(_ratio(pe, pb, xi) - m) < 1e-11
    # Psi_B has no zero on [0, 1]
    xi = np.linspace(0, 1, 4001)
    assert np.polyval(pb[::-1], xi).min() > 0
    # accuracy claimed in Sec. 2: 1e-6, and better than 1e-5 at the largest k_z dz shown
    s = np.arcsin(np.sqrt(xi))
    m = np.array([O.multiplier(scheme, alpha, v) for v in s])
    err = np.abs(_ratio(pe, pb, xi) - m)
    k = 2 * s
    assert err[k <= 2.1].max() < 1e-6
    assert err[k <= 2.4].max() < 1e-5


def test_rational_matches_independent_solve():
    # an independent dense solve of the same interpolation conditions (numpy LAPACK)
    for scheme in (O.GALERKIN, O.UNIFORM):
        for alpha in (0.3, 0.7):
            xi = np.arange(9) / 8
            m = np.array([O.multiplier(scheme, alpha, math.asin(math.sqrt(x))) for x in xi])
            A = np.zeros((9, 9))
            for n in range(5):
                A[:, n] = xi ** n
            for n in range(1, 5):
                A[:, 4 + n] = -m * xi ** n
            sol = np.linalg.solve(A, m)
            _, pe, pb = O.rational_coeffs(scheme, alpha)
            np.testing.assert_allclose(pe, sol[:5], rtol=1e-7, atol=1e-9)
            np.testing.assert_allclose(pb[1:], sol[5:], rtol=1e-7, atol=1e-9)


def test_degenerate_uniform_half():
    # Uniform at alpha = 1/2: M == 1, the 9x9 system is singular; the constant interpolant is returned.
    st, pe, pb = O.rational_coeffs(O.UNIFORM, 0.5)
    assert st == 0
    assert list(pe) == [1, 0, 0, 0, 0] and list(pb) == [1, 0, 0, 0, 0]


def test_galerkin_alpha_half_coefficient_values():
    # Galerkin alpha = 0.5 coefficients (4-digit sanity values recomputed independently with numpy).
    _, pe, pb = O.rational_coeffs(O.GALERKIN, 0.5)
    np.testing.assert_allclose(pe, [1, -2.3886, 1.8991, -0.5428, 0.0336], atol=1e-4)
    np.testing.assert_allclose(pb, [1, -2.5553, 2.25, -0.7708, 0.0769], atol=1e-4)


def test_psi_taps_fourier_symbol():
    # D = -(1,-2,1)/4 has symbol sin^2(k/2); the 9-tap stencil of Psi(D) must have symbol Psi(sin^2(k/2)).
    rng = np.random.default_rng(5)
    for _ in range(5):
        a = rng.normal(size=5)
        t = O.psi_taps(a)
        assert np.allclose(t, t[::-1], atol=0)  # symmetric
        for k in rng.uniform(0, math.pi, 7):
            sym = sum(t[m + 4] * math.cos(k * m) for m in range(-4, 5))
            xi = math.sin(k / 2) ** 2
            assert abs(sym - np.polyval(a[::-1], xi)) < 1e-13
        assert abs(t.sum() - a[0]) < 1e-14  # DC gain = Psi(0)
        nyq = sum(t[m + 4] * (-1) ** m for m in range(-4, 5))
        assert abs(nyq - a.sum()) < 1e-13  # Nyquist gain = Psi(1)


def test_psi_taps_powers_of_d():
    # D^1 taps are exactly (-1/4, 1/2, -1/4); D^2 = (1, -4, 6, -4, 1)/16 (binomial)
    t1 = O.psi_taps([0, 1, 0, 0, 0])
    np.testing.assert_array_equal(t1, [0, 0, 0, -0.25, 0.5, -0.25, 0, 0, 0])
    t2 = O.psi_taps([0, 0, 1, 0, 0])
    np.testing.assert_array_equal(t2, np.array([0, 0, 1, -4, 6, -4, 1, 0, 0]) / 16)
    t4 = O.psi_taps([0, 0, 0, 0, 1])
    np.testing.assert_array_equal(t4, np.array([1, -8, 28, -56, 70, -56, 28, -8, 1]) / 256)
