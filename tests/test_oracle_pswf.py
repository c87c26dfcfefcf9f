"""Pins for the oracle's prolate spheroidal function (oracle/pswf.py)."""
import numpy as np
import pytest
from scipy.special import roots_legendre

from oracle.pswf import PSWF0, taper_bandwidth


@pytest.mark.parametrize("c", [1.0, taper_bandwidth(7), taper_bandwidth(15), taper_bandwidth(31)])
def test_integral_eigen_relation(c):
    """int_{-1}^{1} exp(i c x t) psi_0(t) dt = lambda_0 psi_0(x), with an
    independent high-order quadrature (the solver uses no quadrature)."""
    p = PSWF0(c)
    t, w = roots_legendre(600)
    x = np.linspace(-0.9, 0.9, 19)
    lhs = np.array([np.sum(w * np.exp(1j * c * xx * t) * p(t)) for xx in x])
    rhs = p.lambda0 * p(x)
    assert np.max(np.abs(lhs - rhs)) <= 1e-11 * np.max(np.abs(rhs))
    assert np.max(np.abs(lhs.imag)) <= 1e-12 * np.max(np.abs(rhs))


@pytest.mark.parametrize("c", [0.5, 5.0, taper_bandwidth(7), 40.0])
def test_ode_residual(c):
    """(1 - x^2) psi'' - 2 x psi' + (chi_0 - c^2 x^2) psi = 0."""
    p = PSWF0(c)
    x = np.linspace(-0.99, 0.99, 41)
    r = (1 - x * x) * p.derivative(x, 2) - 2 * x * p.derivative(x, 1) + (p.chi0 - c * c * x * x) * p(x)
    scale = np.max(np.abs(p.chi0 * p(x))) + np.max(np.abs((1 - x * x) * p.derivative(x, 2)))
    assert np.max(np.abs(r)) <= 1e-9 * scale


def test_small_c_expansion():
    """Perturbation theory about c = 0: chi_0 = c^2/3 - 2 c^4/135 + O(c^6)."""
    for c in (0.05, 0.1):
        p = PSWF0(c)
        assert abs(p.chi0 - (c * c / 3 - 2 * c ** 4 / 135)) <= 5 * c ** 6


def test_normalisation_and_sign():
    p = PSWF0(taper_bandwidth(7))
    t, w = roots_legendre(400)
    assert abs(np.sum(w * p(t) ** 2) - 1.0) <= 1e-12
    assert p(0.0) > 0
    # even function, decreasing away from the centre
    x = np.linspace(0, 1, 11)
    assert np.allclose(p(x), p(-x), rtol=0, atol=1e-14)
    assert np.all(np.diff(p(x)) < 0)
