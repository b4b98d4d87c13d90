"""Pins of the closed forms (oracle.analytic): Eq. (27), Eq. (28), Eq. (29)."""
import numpy as np
import pytest

from oracle import analytic


def test_poiseuille_plane_properties():
    d, dP, eta, L = 1e-3, 0.1, 2.5e-4, 4e-3
    y = np.linspace(-d / 2, d / 2, 101)
    v = analytic.poiseuille_plane(y, dP, eta, L, d)
    assert v[0] == pytest.approx(0.0, abs=1e-18) and v[-1] == pytest.approx(0.0, abs=1e-18)
    # centre-line speed dP d^2 / (8 eta L); the paper's VIPO numbers give 12.5 mm/s
    assert v[50] == pytest.approx(dP * d * d / (8 * eta * L), rel=1e-12)
    assert v[50] == pytest.approx(0.0125, rel=1e-12)
    # eta v'' = -dP / L
    h = y[1] - y[0]
    vpp = (v[2:] - 2 * v[1:-1] + v[:-2]) / h ** 2
    assert np.allclose(eta * vpp, -dP / L, rtol=1e-6)


def test_viscosity_of_the_vipo_case():
    # Sec. 5.1: eta = sqrt(rho d^3 dP / (8 L Re)) with rho 1000, d 1 mm, dP 0.1 Pa, L 4 mm, Re 50
    eta = np.sqrt(1000.0 * 1e-3 ** 3 * 0.1 / (8 * 4e-3 * 50))
    assert eta == pytest.approx(2.5e-4, rel=1e-12)


def test_rmsep():
    assert analytic.rmsep([1.0, 2.0], [1.0, 2.0]) == 0.0
    assert analytic.rmsep([1.0, 2.0], [1.1, 1.8]) == pytest.approx(np.sqrt((0.01 + 0.01) / 2))


def test_womersley_reduces_to_quasi_steady_poiseuille_at_small_alpha():
    R, rho, omega = 0.5e-3, 1000.0, 1.0
    eta = 10.0  # alpha = R sqrt(omega rho / eta) = 0.005
    G = 25.0
    assert analytic.womersley_number(R, omega, rho, eta) < 0.01
    r = np.linspace(0, R, 11)
    for t in (0.0, 0.7, 2.0):
        v = analytic.womersley(r, t, R, rho, eta, omega, [G])
        steady = G * np.cos(omega * t) / (4 * eta) * (R * R - r * r)
        assert np.allclose(v, steady, rtol=1e-4, atol=1e-12 * G * R * R / eta)


def test_womersley_wall_and_phase_lag():
    R, rho, eta, omega = 0.5e-3, 1000.0, 3.536e-4, 1.0
    # the paper's pulsatile case: alpha = 0.8409
    assert analytic.womersley_number(R, omega, rho, eta) == pytest.approx(0.8409, abs=2e-4)
    t = np.linspace(0, 2 * np.pi, 400)
    assert np.allclose(analytic.womersley(R, t, R, rho, eta, omega, [25.0]), 0.0, atol=1e-15)
    vc = analytic.womersley(0.0, t, R, rho, eta, omega, [25.0])
    # inertia makes the centre-line speed lag the driving gradient cos(t) (0 < lag < pi/2)
    lag = t[np.argmax(vc)]
    assert 0.0 < lag < np.pi / 2
