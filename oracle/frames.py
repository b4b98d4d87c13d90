"""Local in-/outlet frames (Sec. 3.1).

2-D, Eq. (11):  X' = [[cos t, sin t], [-sin t, cos t]] (X - O'), t > 0 anticlockwise.
3-D, Eqs. (12)-(15): rotation axis n = (OX x O'X') / |OX x O'X'|, its cross-product matrix S,
Rodrigues' matrix, then X' = R (X - O').
Inverse maps Eqs. (16)-(17): X = R^T X' + O'.   Boundary normal Eqs. (20)-(21): u = R^T e_x.

Reading of Eq. (14) (3-D sign).  With n = e_x x d and theta = angle(e_x, d) in [0, pi], the
printed R = I + S sin(theta) + S^2 (1 - cos(theta)) turns e_x onto d.  The local map
X' = R (X - O') and u = R^T e_x need the opposite: R d = e_x.  The 2-D matrix of Eq. (11)
is likewise the transpose of the planar rotation by theta.  This module therefore uses
R = I - S sin(theta) + S^2 (1 - cos(theta)), which equals Eq. (11) for d in the xy-plane.
Degenerate axis (d parallel to e_x, where Eq. (12) divides by zero): R = I for d = +e_x and
R = diag(-1, -1, 1) (half turn about z) for d = -e_x.
"""
import math

import numpy as np


def rotation_2d(theta: float) -> np.ndarray:
    """Eq. (11) coefficient matrix."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, s], [-s, c]])


def rotation_axis(d) -> np.ndarray:
    """Eq. (12): unit vector of OX x O'X' (OX = e_x, O'X' = d)."""
    ex = np.array([1.0, 0.0, 0.0])
    c = np.cross(ex, np.asarray(d, dtype=np.float64))
    return c / np.linalg.norm(c)


def skew(n) -> np.ndarray:
    """Eq. (13): antisymmetric matrix with S v = n x v."""
    nx, ny, nz = n
    return np.array([[0.0, -nz, ny], [nz, 0.0, -nx], [-ny, nx, 0.0]])


def rotation_3d(d) -> np.ndarray:
    """Eq. (14) under the sign reading above: R with R d = e_x."""
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    ex = np.array([1.0, 0.0, 0.0])
    if np.linalg.norm(np.cross(ex, d)) < 1e-12:
        return np.eye(3) if d[0] > 0 else np.diag([-1.0, -1.0, 1.0])
    n = rotation_axis(d)
    S = skew(n)
    theta = math.acos(max(-1.0, min(1.0, float(np.dot(ex, d)))))
    return np.eye(3) - S * math.sin(theta) + S @ S * (1.0 - math.cos(theta))


def roll_about_x(R: np.ndarray, psi: float) -> np.ndarray:
    """Compose a roll psi about the local X' axis: R <- Rx(psi) R (X' is unchanged)."""
    c, s = math.cos(psi), math.sin(psi)
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, c, s], [0.0, -s, c]])
    return Rx @ R


def normal(R: np.ndarray) -> np.ndarray:
    """Eqs. (20)-(21): u = R^T e_x."""
    e = np.zeros(R.shape[0])
    e[0] = 1.0
    return R.T @ e


def to_local(R: np.ndarray, origin, X) -> np.ndarray:
    """Eqs. (11)/(15) for an array of points X (n, d): rows of R (X - O')."""
    d = R.shape[0]
    X = np.asarray(X, dtype=np.float64)
    return (X - np.asarray(origin, dtype=np.float64)[None, :d]) @ R.T


def to_global(R: np.ndarray, origin, Xp) -> np.ndarray:
    """Eqs. (16)/(17): X = R^T X' + O'."""
    d = R.shape[0]
    return np.asarray(Xp, dtype=np.float64) @ R + np.asarray(origin, dtype=np.float64)[None, :d]


def in_box(Xp: np.ndarray, extent, dim: int) -> np.ndarray:
    """Algorithm 1-3 identification test: |X'| < a/2, |Y'| < b/2 (and |Z'| < c/2 in 3-D)."""
    m = (np.abs(Xp[:, 0]) < 0.5 * extent[0]) & (np.abs(Xp[:, 1]) < 0.5 * extent[1])
    if dim == 3:
        m &= np.abs(Xp[:, 2]) < 0.5 * extent[2]
    return m
