"""Pins for the closed-form bounds (Theorem 2.2, eq. entropy_polyapprox_Chebyshev)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import bounds


@pytest.mark.parametrize("k", [2, 3, 5, 10])
@pytest.mark.parametrize("g", [0.0, 1e-4, 0.01, 0.3])
def test_theorem22_integral_closed_form(k, g):
    # The proof of Theorem 2.2 evaluates I_k = int_0^inf (sqrt(1+t) - sqrt(g+t))^(2k) dt
    # from an antiderivative.  Its first closed form (the limit of the
    # antiderivative) agrees with quadrature; its simplified second form carries
    # an extra factor 2 -- the reading used here is the first form, which equals
    # (1 - sqrt g)^(2k) (1 + g + 2 k sqrt g) / (2 (k^2 - 1)).
    val, _ = integrate.quad(lambda t: (math.sqrt(1 + t) - math.sqrt(g + t)) ** (2 * k), 0, np.inf,
                            limit=500, epsabs=0, epsrel=1e-11)
    sg = math.sqrt(g)
    simplified = (1 - sg) ** (2 * k) * (1 + g + 2 * sg * k) / (2 * (k * k - 1))
    assert math.isclose(val, simplified, rel_tol=1e-8)
    if g > 0:
        first = sg * (1 - sg) ** (2 * k) * ((1 - g) ** 2 / (2 * k - 2) - (1 - sg) ** 4 / (2 * k + 2)) / (
            2 * (1 - sg) * (sg - g))
        assert math.isclose(val, first, rel_tol=1e-8)


@pytest.mark.parametrize("k", [2, 3, 6, 12])
@pytest.mark.parametrize("g", [0.0, 1e-3, 0.2])
def test_theorem22_bound_dominates_integral_form(k, g):
    # E_k <= b * int_0^inf t (sqrt(kappa)+1)^2 / (2(1+t)) ((sqrt(kappa)-1)/(sqrt(kappa)+1))^(k+1) dt
    #     <= the closed-form bound of Theorem 2.2 (here b = 1).
    def integrand(t):
        kap = (1 + t) / (g + t) if g + t > 0 else np.inf
        sk = math.sqrt(kap)
        return t * (sk + 1) ** 2 / (2 * (1 + t)) * ((sk - 1) / (sk + 1)) ** (k + 1)
    val, _ = integrate.quad(integrand, 0, np.inf, limit=500, epsrel=1e-10)
    assert val <= bounds.thm22_bound(k, g, 1.0) * (1 + 1e-9)


def test_theorem22_remark_special_case_and_chebyshev_comparison():
    for k in range(2, 30):
        assert math.isclose(bounds.thm22_bound(k, 0.0, 3.0), 3.0 / (4 * (k * k - 1)), rel_tol=1e-15)
        # the remark calls the new bound better for all k >= 2; at k = 2 the two
        # coincide (4(k^2-1) = 2k(k+1) exactly when k = 2), strictly better after
        if k == 2:
            assert math.isclose(bounds.thm22_bound(k, 0.0, 1.0), bounds.chebyshev_bound(k, 1.0), rel_tol=1e-15)
        else:
            assert bounds.thm22_bound(k, 0.0, 1.0) < bounds.chebyshev_bound(k, 1.0)


def test_chebyshev_interpolant_respects_bound():
    # E_k <= error of any degree-k polynomial; the Chebyshev interpolant's error
    # must therefore be >= E_k, and E_k's bound must exceed the interpolant error
    # divided by the Lebesgue-constant factor (1 + Lambda_k).  This checks the
    # bound is not too small by orders of magnitude.
    a, b = 1e-6, 1e-2
    x = np.geomspace(a, b, 20001)
    f = x * np.log(x)
    for k in (4, 8, 16):
        nodes = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * (2 * np.arange(k + 1) + 1) / (2 * k + 2))
        coef = np.polynomial.chebyshev.chebfit((2 * nodes - a - b) / (b - a), nodes * np.log(nodes), k)
        err = np.max(np.abs(np.polynomial.chebyshev.chebval((2 * x - a - b) / (b - a), coef) - f))
        lebesgue = 1 + 2 / np.pi * math.log(k + 1)
        assert err / (1 + lebesgue) <= bounds.thm22_bound(k, a, b)


def test_probing_heuristic_recovers_model():
    # |T_{d+1} - T_d| = C q^d / d^k exactly -> the fitted model gives d*
    C, q, k = 0.5, 0.6, 2
    e = lambda d: C * q ** d / d ** k
    T1 = 1.0
    T2 = T1 + e(1)
    T3 = T2 + e(2)
    d = bounds.probing_heuristic_d(T1, T2, T3, 1e-4)
    d_want = min(dd for dd in range(1, 64) if e(dd) <= 1e-4)
    assert d >= d_want  # the max over k in {2,3} is at least the k = 2 choice


def test_gm_divided_differences_against_high_precision():
    """The stable divided differences of f(x) = -x log x used by g_m agree
    with 50-digit evaluations of the plain quotients of eq.
    error-bound--gm-definition, including points next to the node where the
    double-precision quotients cancel."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    from oracle import bounds
    for t in (1.3e-3, 0.25, 7.0):
        for rel in (0.0, 1e-13, -3e-9, 2e-5, 0.05, -0.07, 0.1, 0.5, 2.0, -0.8):
            z = t * (1.0 + rel)
            d1, d2 = bounds._dd1_dd2(np.array([z]), t)
            T, Z = mp.mpf(t), mp.mpf(z)
            if Z == T:
                r1, r2 = -mp.log(T) - 1, -1 / (2 * T)
            else:
                r1 = (-Z * mp.log(Z) + T * mp.log(T)) / (Z - T)
                r2 = (r1 + mp.log(T) + 1) / (Z - T)
            assert abs(d1[0] - float(r1)) <= 1e-14 * abs(float(r1)) + 1e-300
            assert abs(d2[0] - float(r2)) <= 1e-13 * abs(float(r2))
