"""The moment form of the Gaussian splat (forward and adjoint kernels) replaces
phi(m + c), |c| <= 1/2, by its Taylor polynomial of degree 5 about the
integer bin offset m. Its truncation error, relative to the kernel's peak,
underlies the splat's parity bar. This test computes that error
independently, taking the Gaussian's derivatives from numpy's probabilists'
Hermite polynomials. It checks the bounds the kernels state: 1.3e-6 at
sigma = 2.5 bins (the smallest sigma the moment form is used for), falling
to 3.1e-7 at the workloads' sigma of 3.185. It also checks that five terms
would not be enough."""
import math

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermeval


def _truncation(sigma: float, terms: int = 6) -> float:
    """max over bin offsets m and c in [-1/2, 1/2] of
    |sum_{n < terms} phi^(n)(m) c^n / n! - phi(m + c)|, over phi(0)."""
    def phi(x):
        return np.exp(-x * x / (2 * sigma * sigma)) / (sigma * math.sqrt(2 * math.pi))

    c = np.linspace(-0.5, 0.5, 201)
    reach = math.ceil(6 * sigma) + 1
    worst = 0.0
    for m in range(-reach, reach + 1):
        approx = np.zeros_like(c)
        for n in range(terms):
            he = np.zeros(n + 1)
            he[n] = 1.0
            # phi^(n)(x) = (-1)^n He_n(x / sigma) phi(x) / sigma^n
            d = (-1) ** n * hermeval(m / sigma, he) * phi(m) / sigma ** n
            approx += d * c ** n / math.factorial(n)
        worst = max(worst, float(np.abs(approx - phi(m + c)).max()))
    return worst / phi(0.0)


def test_stated_bounds():
    assert _truncation(2.5) <= 1.35e-6
    assert _truncation(3.18496) <= 3.2e-7


def test_error_falls_with_sigma_so_the_threshold_is_the_worst_case():
    errs = [_truncation(s) for s in (2.5, 2.75, 3.18496, 4.0, 6.0, 9.5)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert _truncation(2.4) > _truncation(2.5)


@pytest.mark.parametrize("sigma", [2.5, 3.18496])
def test_five_terms_would_not_do(sigma):
    assert _truncation(sigma, terms=5) > 5 * _truncation(sigma, terms=6)
    assert _truncation(2.5, terms=5) > 1e-5
