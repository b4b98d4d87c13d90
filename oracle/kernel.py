"""Wendland C2 smoothing kernel (Sec. 3: compact support 2h, h = 1.3 dp).

W(r, h) = alpha_d (1 - q/2)^4 (2q + 1) for q = r/h < 2, zero beyond.
alpha_2 = 7 / (4 pi h^2), alpha_3 = 21 / (16 pi h^3) normalise W to unit integral.
dW/dr = -(5 alpha_d / h) q (1 - q/2)^3.
"""
import math

import numpy as np


def alpha(dim: int, h: float) -> float:
    if dim == 2:
        return 7.0 / (4.0 * math.pi * h * h)
    if dim == 3:
        return 21.0 / (16.0 * math.pi * h ** 3)
    raise ValueError("dim must be 2 or 3")


def W(r, h: float, dim: int):
    q = np.asarray(r, dtype=np.float64) / h
    t = np.clip(1.0 - 0.5 * q, 0.0, None)
    return alpha(dim, h) * t ** 4 * (2.0 * q + 1.0)


def dW(r, h: float, dim: int):
    q = np.asarray(r, dtype=np.float64) / h
    t = np.clip(1.0 - 0.5 * q, 0.0, None)
    return -5.0 * alpha(dim, h) / h * q * t ** 3


def lattice_sum_w0(dim: int, dp: float, h: float) -> float:
    """Sum of W over a full-support Cartesian lattice of spacing dp, self included.

    This is the reference denominator of the density summation, Eq. (9), taken as one
    global constant of the initial (unperturbed lattice) configuration.
    """
    m = int(math.ceil(2.0 * h / dp)) + 1
    ax = np.arange(-m, m + 1) * dp
    grids = np.meshgrid(*([ax] * dim), indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    w = W(r, h, dim)
    return float(np.sum(w[r < 2.0 * h]))
