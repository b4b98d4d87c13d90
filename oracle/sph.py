"""Riemann-based weakly-compressible SPH step in FP64 (Sec. 2, Sec. 4).

All sums run over the neighbours j of fluid particle i within the kernel support 2h: other
fluid particles and the fixed wall particles.  Pairs are found with a k-d tree radius
query (scipy ``cKDTree``), which returns exactly the set {j : |r_i - r_j| <= 2h}; W and dW/dr
vanish at 2h, so the boundary of that set contributes nothing.

Particle mass m = rho0 dp^d for fluid and wall.  Dynamic viscosity eta = rho0 nu.

Readings (the paper cites these parts without restating them):
* Wall neighbours (Sec. 5: one-sided Riemann solver and no-slip walls, both cited): a wall
  particle j takes the mirrored state of i, rho_j = rho_i, p_j = p_i, v_j = -v_i, in every
  Riemann, viscous and continuity term.  For a wall at rest this gives U_R = -U_L in
  Eqs. (6)-(8) and v_ij = 2 v_i in the viscous term (no-slip at the wall surface).
* Intermediate velocity of the continuity equation, Eq. (4): the Riemann problem of
  Eqs. (6)-(7) is posed along -e_ij (U_L = -v_i.e_ij), so U* and U-bar are components along
  -e_ij and v* = v-bar + (U-bar - U*) e_ij.  (Printed with the opposite sign on the e_ij
  components, which would make the pressure term anti-diffusive.)
* Eq. (9) with one global reference sum: rho_i = rho0 sum_j W_ij / sum W0, sum W0 over the
  unperturbed lattice (``kernel.lattice_sum_w0``).  It is applied to every non-buffer fluid
  particle each step; buffer particles instead integrate Eq. (4) (Sec. 4: no
  re-initialisation near the boundary).
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.spatial import cKDTree

from . import kernel


@dataclasses.dataclass
class Params:
    dim: int
    dp: float
    h: float
    rho0: float
    c0: float
    nu: float
    dt: float
    p_bg: float = 0.0  # background pressure of the EoS (reading A22; 0 = Eq. (3) as printed)
    tvf_lambda: float = 0.0  # transport velocity, Eq. (10): p_max = lambda rho0 v_max^2 (0 = off)

    @property
    def eta(self) -> float:
        return self.rho0 * self.nu

    @property
    def mass(self) -> float:
        return self.rho0 * self.dp ** self.dim

    @property
    def sum_w0(self) -> float:
        return kernel.lattice_sum_w0(self.dim, self.dp, self.h)


def make_params(dim, dp, h_over_dp, rho0, c0, nu, dt, p_bg=0.0, tvf_lambda=0.0) -> Params:
    return Params(dim=int(dim), dp=float(dp), h=float(h_over_dp) * float(dp), rho0=float(rho0),
                  c0=float(c0), nu=float(nu), dt=float(dt), p_bg=float(p_bg), tvf_lambda=float(tvf_lambda))


def eos(rho, P: Params):
    """Eq. (3): p = c0^2 (rho - rho0), plus the constant background pressure p_bg (reading
    A22: keeps the pressure positive where the flow would put it below zero; only pressure
    differences and the open-boundary term of Eq. (18), which carries p_bg in p_b, act)."""
    return P.c0 * P.c0 * (np.asarray(rho) - P.rho0) + P.p_bg


@dataclasses.dataclass
class Pairs:
    """Ordered neighbour pairs (i fluid; j fluid or wall) with r_ij = r_i - r_j."""

    i: np.ndarray
    j: np.ndarray
    rij: np.ndarray  # (npairs, d)
    r: np.ndarray  # (npairs,)


def neighbor_pairs(fpos: np.ndarray, wpos: np.ndarray, h: float):
    """Fluid-fluid pairs (both orders, i != j) and fluid-wall pairs within 2h."""
    radius = 2.0 * h
    n = fpos.shape[0]
    if n == 0:
        e = np.zeros(0, dtype=np.int64)
        z = np.zeros((0, fpos.shape[1]))
        return Pairs(e, e, z, np.zeros(0)), Pairs(e, e, z, np.zeros(0))
    tf = cKDTree(fpos)
    ij = tf.query_pairs(radius, output_type="ndarray")
    i = np.concatenate([ij[:, 0], ij[:, 1]]).astype(np.int64)
    j = np.concatenate([ij[:, 1], ij[:, 0]]).astype(np.int64)
    rij = fpos[i] - fpos[j]
    r = np.sqrt(np.sum(rij * rij, axis=1))
    keep = r > 0.0
    ff = Pairs(i[keep], j[keep], rij[keep], r[keep])
    if wpos.shape[0]:
        tw = cKDTree(wpos)
        sdm = tf.sparse_distance_matrix(tw, radius, output_type="ndarray")
        iw = sdm["i"].astype(np.int64)
        jw = sdm["j"].astype(np.int64)
        rw = fpos[iw] - wpos[jw]
        dw = np.sqrt(np.sum(rw * rw, axis=1))
        keep = dw > 0.0
        fw = Pairs(iw[keep], jw[keep], rw[keep], dw[keep])
    else:
        e = np.zeros(0, dtype=np.int64)
        fw = Pairs(e, e, np.zeros((0, fpos.shape[1])), np.zeros(0))
    return ff, fw


def _scatter(idx, vals, n):
    if vals.ndim == 1:
        return np.bincount(idx, weights=vals, minlength=n)
    return np.stack([np.bincount(idx, weights=vals[:, a], minlength=n) for a in range(vals.shape[1])], axis=1)


def density_summation(P: Params, n: int, ff: Pairs, fw: Pairs) -> np.ndarray:
    """Eq. (9): rho_i = rho0 (W(0) + sum_j W_ij) / sum W0 for every fluid particle."""
    w0 = float(kernel.W(0.0, P.h, P.dim))
    s = np.full(n, w0)
    s += _scatter(ff.i, kernel.W(ff.r, P.h, P.dim), n)
    s += _scatter(fw.i, kernel.W(fw.r, P.h, P.dim), n)
    return P.rho0 * s / P.sum_w0


def _riemann_v_star_term(vi, vj, rho_i, rho_j, p_i, p_j, e, c0):
    """(v_i - v*_ij) . e_ij from Eqs. (4), (6), (7) under the reading in the module header."""
    UL = -np.sum(vi * e, axis=1)
    UR = -np.sum(vj * e, axis=1)
    Ubar = 0.5 * (UL + UR)
    rho_bar = 0.5 * (rho_i + rho_j)
    Ustar = Ubar + (p_i - p_j) / (2.0 * rho_bar * c0)
    vbar = 0.5 * (vi + vj)
    vstar = vbar + (Ubar - Ustar)[:, None] * e
    return np.sum((vi - vstar) * e, axis=1)


def continuity_rate(P: Params, vel, rho, ff: Pairs, fw: Pairs) -> np.ndarray:
    """Eq. (4): drho_i/dt = 2 rho_i sum_j m_j / rho_j (v_i - v*_ij) . grad W_ij."""
    n = rho.shape[0]
    p = eos(rho, P)
    m = P.mass
    # fluid neighbours
    e = ff.rij / ff.r[:, None]
    dw = kernel.dW(ff.r, P.h, P.dim)
    t = _riemann_v_star_term(vel[ff.i], vel[ff.j], rho[ff.i], rho[ff.j], p[ff.i], p[ff.j], e, P.c0)
    s = _scatter(ff.i, m / rho[ff.j] * t * dw, n)
    # wall neighbours: mirrored state rho_j = rho_i, p_j = p_i, v_j = -v_i
    ew = fw.rij / fw.r[:, None]
    dww = kernel.dW(fw.r, P.h, P.dim)
    tw = _riemann_v_star_term(vel[fw.i], -vel[fw.i], rho[fw.i], rho[fw.i], p[fw.i], p[fw.i], ew, P.c0)
    s += _scatter(fw.i, m / rho[fw.i] * tw * dww, n)
    return 2.0 * rho * s


def _riemann_p_star(vi, vj, rho_i, rho_j, p_i, p_j, e, c0):
    """Eqs. (7)-(8): P* = P-bar + 1/2 beta rho-bar (U_L - U_R), beta = min(3 max(U_L - U_R, 0), c0)."""
    UL = -np.sum(vi * e, axis=1)
    UR = -np.sum(vj * e, axis=1)
    beta = np.minimum(3.0 * np.maximum(UL - UR, 0.0), c0)
    return 0.5 * (p_i + p_j) + 0.5 * beta * 0.5 * (rho_i + rho_j) * (UL - UR)


def transport_sum(P: Params, rho, ff: Pairs, fw: Pairs) -> np.ndarray:
    """The sum of Eq. (10): sum_j 2 m_j / (rho_i rho_j) dW_ij/dr_ij e_ij (fluid and wall
    neighbours; a wall neighbour takes rho_j = rho_i as in the force)."""
    n = rho.shape[0]
    d = ff.rij.shape[1] if ff.i.size else fw.rij.shape[1]
    out = np.zeros((n, d))
    for pairs, wall in ((ff, False), (fw, True)):
        if pairs.i.size == 0:
            continue
        i = pairs.i
        e = pairs.rij / pairs.r[:, None]
        rho_j = rho[i] if wall else rho[pairs.j]
        coef = 2.0 * P.mass / (rho[i] * rho_j) * kernel.dW(pairs.r, P.h, P.dim)
        out += _scatter(i, coef[:, None] * e, n)
    return out


# Boundary particles of the transport velocity (Sec. 2.2: the TVF serves the inner fluid; the
# paper identifies about three layers of boundary particles with a cited spatio-temporal
# method that it does not restate).  Reading A27:
#   spatial   psi_i = -sum_j V_j r_ij . grad_i W_ij over fluid and wall neighbours (V_j = dp^d),
#             the SPH estimate of div r = d; a particle is a candidate when psi_i < 0.75 d
#             (its kernel support is cut by a free or open boundary);
#   temporal  a candidate is a core boundary particle when it was a candidate in the previous
#             step too (a particle without a previous step counts the current one);
#   layers    a particle is a boundary particle when it is core or a fluid neighbour within 2h
#             is core (2h = 2.6 dp: the core layer and about two more).
PSI_CANDIDATE = 0.75


def position_divergence(P: Params, n: int, ff: Pairs, fw: Pairs) -> np.ndarray:
    """psi_i = -sum_j V_j r_ij . grad_i W_ij = sum_j V_j r_ij (-dW/dr) (fluid and wall j)."""
    V = P.dp ** P.dim
    s = _scatter(ff.i, -V * ff.r * kernel.dW(ff.r, P.h, P.dim), n)
    s += _scatter(fw.i, -V * fw.r * kernel.dW(fw.r, P.h, P.dim), n)
    return s


def boundary_layers(P: Params, psi: np.ndarray, prev, ff: Pairs):
    """(candidate, core, boundary) flags of the reading above; prev: the previous step's
    candidate flags (None, or -1 entries, where a particle has no previous step)."""
    cand = psi < PSI_CANDIDATE * P.dim
    if prev is None:
        before = cand
    else:
        prev = np.asarray(prev)
        before = np.where(prev < 0, cand, prev > 0)
    core = cand & before
    near = np.zeros(psi.shape[0], dtype=bool)
    if ff.i.size:
        np.logical_or.at(near, ff.i, core[ff.j])
    return cand, core, core | near


def moved(pairs: Pairs, fpos, other) -> Pairs:
    """The same pairs with r_ij recomputed from new positions (fixed configuration)."""
    rij = fpos[pairs.i] - other[pairs.j]
    return Pairs(pairs.i, pairs.j, rij, np.sqrt(np.sum(rij * rij, axis=1)))


def acceleration(P: Params, vel, rho, p_bc, ff: Pairs, fw: Pairs, pressure=True, viscous=True) -> np.ndarray:
    """Eq. (5), and Eq. (18) for particles with a finite boundary pressure ``p_bc[i]``.

    dv_i/dt = -2 sum_j m P*_ij/(rho_i rho_j) grad W_ij + 2 sum_j m eta v_ij/(rho_i rho_j r_ij) dW_ij
              [+ 2 p_b sum_j m/(rho_i rho_j) grad W_ij   for buffer particles]
    ``p_bc`` is NaN for particles without the boundary term.  ``pressure`` / ``viscous``
    select the terms (the pressure part includes Eq. (18)).
    """
    n = rho.shape[0]
    d = vel.shape[1]
    p = eos(rho, P)
    m = P.mass
    acc = np.zeros((n, d))
    has_bc = ~np.isnan(p_bc)
    pb = np.where(has_bc, p_bc, 0.0)
    for pairs, wall in ((ff, False), (fw, True)):
        if pairs.i.size == 0:
            continue
        i = pairs.i
        e = pairs.rij / pairs.r[:, None]
        dw = kernel.dW(pairs.r, P.h, P.dim)
        gradW = dw[:, None] * e
        vi = vel[i]
        if wall:
            vj = -vi
            rho_j = rho[i]
            p_j = p[i]
        else:
            vj = vel[pairs.j]
            rho_j = rho[pairs.j]
            p_j = p[pairs.j]
        rho_i = rho[i]
        inv = m / (rho_i * rho_j)
        term = np.zeros_like(gradW)
        if pressure:
            pstar = _riemann_p_star(vi, vj, rho_i, rho_j, p[i], p_j, e, P.c0)
            term += -2.0 * (inv * pstar)[:, None] * gradW
            term += 2.0 * (pb[i] * inv)[:, None] * gradW * has_bc[i][:, None]
        if viscous:
            term += 2.0 * (inv * P.eta * dw / pairs.r)[:, None] * (vi - vj)
        acc += _scatter(i, term, n)
    return acc
