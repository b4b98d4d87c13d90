"""Pins of the Wendland C2 kernel (oracle.kernel) against quadrature and finite differences."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kernel


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("h", [0.013, 1.0])
def test_unit_integral(dim, h):
    # int W dV = 1 over the support (radial quadrature, independent of alpha's derivation)
    if dim == 2:
        f = lambda r: float(kernel.W(r, h, 2)) * 2.0 * math.pi * r
    else:
        f = lambda r: float(kernel.W(r, h, 3)) * 4.0 * math.pi * r * r
    val, _ = integrate.quad(f, 0.0, 2.0 * h, epsabs=1e-14, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_derivative_matches_finite_difference(dim):
    h = 0.37
    r = np.linspace(0.01, 1.99, 57) * h
    eps = 1e-6 * h
    fd = (kernel.W(r + eps, h, dim) - kernel.W(r - eps, h, dim)) / (2 * eps)
    assert np.allclose(kernel.dW(r, h, dim), fd, rtol=1e-6, atol=1e-9 / h ** (dim + 1))


@pytest.mark.parametrize("dim", [2, 3])
def test_compact_support(dim):
    h = 0.5
    r = np.array([2.0 * h, 2.5 * h, 10 * h])
    assert np.all(kernel.W(r, h, dim) == 0.0)
    assert np.all(kernel.dW(r, h, dim) == 0.0)
    assert kernel.W(0.0, h, dim) == pytest.approx(kernel.alpha(dim, h))
    assert kernel.dW(0.0, h, dim) == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_partition_of_unity(dim):
    # sum_j W_ij dp^d ~ 1 on a full lattice (SPH zeroth-order consistency at h = 1.3 dp)
    dp = 0.01
    s = kernel.lattice_sum_w0(dim, dp, 1.3 * dp)
    assert abs(s * dp ** dim - 1.0) < 0.02
