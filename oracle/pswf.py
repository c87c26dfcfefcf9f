"""Zeroth-order prolate spheroidal wave function psi_0(c, x) on [-1, 1].

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The thesis takes a prolate spheroidal function as its gridding taper
(Section 2.3.4, "The form of the GCF"; Section 3.5.4, "The GCF") and says it
is generated as in CASA, without giving parameters.  Reading used here: the
standard psi_0 (no weighting, alpha = 0) with bandwidth c = pi * S / 2 for a
uv support of S pixels, computed from its definition rather than from CASA's
rational approximation.

Definition.  psi_0 is the eigenfunction with the smallest eigenvalue chi_0 of
the prolate differential operator

    L psi = -d/dx[(1 - x^2) dpsi/dx] + c^2 x^2 psi = chi psi .

Expanded in orthonormal Legendre functions Pn_n = sqrt((2n+1)/2) P_n, the
operator is a symmetric matrix (Bouwkamp's method).  With
x Pn_n = a_{n+1} Pn_{n+1} + a_n Pn_{n-1}, a_n = n / sqrt(4 n^2 - 1):

    <Pn_n | L | Pn_n>     = n (n + 1) + c^2 (a_{n+1}^2 + a_n^2)
    <Pn_{n+2} | L | Pn_n> = c^2 a_{n+1} a_{n+2}

psi_0 is even, so only even n enter.  The eigenvector is found with a dense
symmetric eigensolver (a library primitive).

Pins (tests/test_oracle_pswf.py): the integral eigen-relation
int_{-1}^{1} exp(i c x t) psi_0(t) dt = lambda_0 psi_0(x), checked by an
independent quadrature; the ODE residual through the Legendre derivative;
the small-c expansion chi_0 = c^2/3 - 2 c^4/135 + O(c^6).
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg


def _n_terms(c: float) -> int:
    return int(math.ceil(0.5 * c)) + 40


def pswf0_expansion(c: float, n_terms: int | None = None):
    """Return (chi_0, d) where psi_0(x) = sum_k d[k] Pn_{2k}(x).

    The eigenvector is normalised to unit L2 norm on [-1, 1] and signed so
    that psi_0(0) > 0.
    """
    K = _n_terms(c) if n_terms is None else int(n_terms)
    n = 2 * np.arange(K, dtype=np.float64)

    def a(m):
        m = np.asarray(m, dtype=np.float64)
        return m / np.sqrt(4.0 * m * m - 1.0)

    diag = n * (n + 1.0) + c * c * (a(n + 1.0) ** 2 + np.where(n > 0, a(np.maximum(n, 1.0)) ** 2, 0.0))
    off = c * c * a(n[:-1] + 1.0) * a(n[:-1] + 2.0)
    M = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    evals, evecs = np.linalg.eigh(M)
    chi0 = float(evals[0])
    d = evecs[:, 0].copy()
    # sign: psi_0(0) > 0
    if _eval(d, np.array([0.0]))[0] < 0:
        d = -d
    return chi0, d


def _legendre_coeffs(d: np.ndarray) -> np.ndarray:
    """Coefficients on the plain Legendre polynomials P_n."""
    K = d.shape[0]
    coef = np.zeros(2 * K - 1)
    k = np.arange(K)
    coef[2 * k] = d * np.sqrt((4.0 * k + 1.0) / 2.0)
    return coef


def _eval(d: np.ndarray, x: np.ndarray) -> np.ndarray:
    return npleg.legval(np.asarray(x, dtype=np.float64), _legendre_coeffs(d))


class PSWF0:
    """psi_0(c, x) for one bandwidth c."""

    def __init__(self, c: float, n_terms: int | None = None):
        self.c = float(c)
        self.chi0, self.d = pswf0_expansion(self.c, n_terms)
        self._coef = _legendre_coeffs(self.d)

    def __call__(self, x) -> np.ndarray:
        return npleg.legval(np.asarray(x, dtype=np.float64), self._coef)

    def derivative(self, x, order: int = 1) -> np.ndarray:
        return npleg.legval(np.asarray(x, dtype=np.float64), npleg.legder(self._coef, order))

    @property
    def lambda0(self) -> float:
        """Eigenvalue of int_{-1}^{1} exp(i c x t) psi_0(t) dt = lambda_0 psi_0(x).

        At x = 0 only the constant Legendre term integrates to non-zero:
        int Pn_0 = sqrt(2), so lambda_0 = sqrt(2) d_0 / psi_0(0).
        """
        return math.sqrt(2.0) * float(self.d[0]) / float(self(0.0))


def taper_bandwidth(support: int) -> float:
    """c = pi * S / 2 for a uv support of S pixels."""
    return math.pi * float(support) / 2.0
