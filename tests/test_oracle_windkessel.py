"""Pins of the RCR Windkessel outlet (Eq. (31), Sec. 6.2; oracle/buffer.py windkessel_step).

The oracle integrates Eq. (31) split as P = P_d + R_p Q, C dP_d/dt = Q - P_d / R_d.  Pins,
independent of that split: the exact solution of the explicit recurrence for a constant flux
and its steady state Q (R_p + R_d), which is Eq. (31) with d/dt = 0; and, for a sinusoidal
flux, the amplitude and phase of P against the impedance of Eq. (31) in the frequency domain,
Z(w) = (1 + R_p/R_d + i w C R_p) / (1/R_d + i w C), to the O(w dt) error of the scheme.
Parameters: the right common carotid of the paper's table, converted to SI
(1 dyn s / cm^5 = 1e5 Pa s / m^3, 1 cm^5 / dyn = 1e-5 m^3 / Pa)."""
import cmath
import math

import numpy as np
import pytest

from oracle import buffer as OB
from paper_2406_16786_gb300 import workloads as wl

RP, C, RD = 1180 * 1e5, 7.70e-5 * 1e-5, 18400 * 1e5


def _buffer(pd0=0.0):
    spec = wl.BufferSpec(origin=np.zeros(3), rotation=np.eye(3), extent=np.array([0.01, 0.02, 0.02]),
                         bc=wl.PRESSURE_OUTLET, wk_rp=RP, wk_c=C, wk_rd=RD, wk_pd0=pd0)
    return OB.Buffer(0, spec, 3)


def test_constant_flux_closed_form_and_steady_state():
    q, dt, pd0 = 2.0e-6, 1e-3, 500.0
    b = _buffer(pd0)
    n = 3000
    out = []
    for i in range(n):
        b.windkessel_step(q, dt, i == 0)
        out.append(b.p_b(0.0))
    k = np.arange(n)
    pd_exact = q * RD + (pd0 - q * RD) * (1.0 - dt / (RD * C)) ** k
    assert np.allclose(np.array(out), pd_exact + RP * q, rtol=1e-12, atol=1e-9)
    # long run: Eq. (31) at rest, (1 + R_p/R_d) Q = P / R_d
    for _ in range(40000):
        b.windkessel_step(q, dt, False)
    assert abs(b.p_b(0.0) - q * (RP + RD)) < 1e-6 * q * (RP + RD)


@pytest.mark.parametrize("omega", [2.0, 8.302])
def test_sinusoidal_flux_matches_eq31_impedance(omega):
    dt = 1e-5
    q0 = 1.0e-6
    b = _buffer()
    period = 2 * math.pi / omega
    n = int(round(12 * RD * C / dt)) + int(round(2 * period / dt))
    t = np.arange(n) * dt
    qs = q0 * np.sin(omega * (t - dt))  # the step at t_n sees the flux of the step before
    p = np.empty(n)
    for i in range(n):
        b.windkessel_step(float(qs[i]) if i > 0 else 0.0, dt, i == 0)
        p[i] = b.p_b(0.0)
    # fit P = A sin(w t) + B cos(w t) + P0 over the last two periods
    m = t > t[-1] - 2 * period
    X = np.stack([np.sin(omega * t[m]), np.cos(omega * t[m]), np.ones(m.sum())], axis=1)
    A, B, _ = np.linalg.lstsq(X, p[m], rcond=None)[0]
    Z = (1 + RP / RD + 1j * omega * C * RP) / (1 / RD + 1j * omega * C)
    got = complex(A, B) / q0  # P = Im(Z q0 e^{iwt}) -> A = Re Z q0, B = Im Z q0
    assert abs(got - Z) < 20 * omega * dt * abs(Z) + 1e-9 * abs(Z)
    assert abs(cmath.phase(got) - cmath.phase(Z)) < 20 * omega * dt
