"""Closed-form flows and the error measure of the validation cases (Sec. 5.1, Sec. 6.1)."""
import numpy as np
from scipy import special


def poiseuille_plane(y, dP: float, eta: float, L: float, d: float):
    """Eq. (27): v_x'(y') = dP / (2 eta L) (d/2 - y')(d/2 + y'), y' in [-d/2, d/2]."""
    y = np.asarray(y, dtype=np.float64)
    return dP / (2.0 * eta * L) * (0.5 * d - y) * (0.5 * d + y)


def rmsep(v_exact, v_num) -> float:
    """Eq. (28): sqrt( mean( ((v - v~) / v)^2 ) ) over the measuring points."""
    v_exact = np.asarray(v_exact, dtype=np.float64)
    v_num = np.asarray(v_num, dtype=np.float64)
    return float(np.sqrt(np.mean(((v_exact - v_num) / v_exact) ** 2)))


def womersley(r, t, R: float, rho: float, eta: float, omega: float, P_n):
    """Eq. (29): pipe velocity for a driving pressure drop per length sum_n P'_n e^{i n omega t}.

    v(r, t) = Re{ sum_n -i P'_n / (rho n omega) [1 - J0(alpha n^1/2 i^3/2 r/R) / J0(alpha n^1/2 i^3/2)]
    e^{i n omega t} },  alpha = R sqrt(omega rho / eta).  ``P_n`` lists P'_1, P'_2, ... (complex
    allowed).

    Reading: Sec. 6.1 defines P' = dP / L = 25 cos(t) as the pressure drop per length, which
    drives flow along +X'; Eq. (29) as printed (factor +i) is written for P' = dp/dx, and at
    small alpha gives v = -P' (R^2 - r^2) / (4 eta).  The factor -i used here gives the
    quasi-steady Poiseuille flow v = +P' (R^2 - r^2) / (4 eta) for the text's P'.
    """
    r = np.asarray(r, dtype=np.float64)
    alpha = R * np.sqrt(omega * rho / eta)
    i32 = np.exp(1j * 3.0 * np.pi / 4.0)  # i^(3/2)
    out = np.zeros(np.broadcast(r, t).shape, dtype=np.complex128)
    for n, Pn in enumerate(P_n, start=1):
        z = alpha * np.sqrt(n) * i32
        shape = 1.0 - special.jv(0, z * r / R) / special.jv(0, z)
        out = out - 1j * Pn / (rho * n * omega) * shape * np.exp(1j * n * omega * np.asarray(t))
    return np.real(out)


def womersley_number(R: float, omega: float, rho: float, eta: float) -> float:
    return float(R * np.sqrt(omega * rho / eta))
