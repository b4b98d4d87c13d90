"""Pins of the oracle's WCSPH arithmetic (oracle.sph) against closed forms and invariants."""
import itertools

import numpy as np
import pytest

from oracle import kernel, sph


def _lattice(dim, n, dp):
    ax = (np.arange(n) + 0.5) * dp
    g = np.meshgrid(*([ax] * dim), indexing="ij")
    return np.stack([x.ravel() for x in g], axis=1)


def _params(dim, dp=0.01, c0=10.0, nu=1e-3):
    return sph.make_params(dim, dp, 1.3, 1000.0, c0, nu, 1e-4)


def _lattice_moment(dim, dp, h):
    """-sum_j V_j x_ji dW/dx_i on a full lattice: the discrete version of 1 (about 0.97-0.98)."""
    ax = np.arange(-4, 5) * dp
    g = np.meshgrid(*([ax] * dim), indexing="ij")
    X = np.stack([x.ravel() for x in g], axis=1)
    r = np.linalg.norm(X, axis=1)
    k = (r > 0) & (r < 2 * h)
    return float(np.sum(dp ** dim * X[k, 0] ** 2 / r[k] * -kernel.dW(r[k], h, dim)))


def _interior(pos, lo, hi, margin):
    return np.all((pos > lo + margin) & (pos < hi - margin), axis=1)


@pytest.mark.parametrize("dim", [2, 3])
def test_pairs_match_brute_force(dim):
    rng = np.random.default_rng(dim)
    h = 0.013
    f = rng.uniform(0, 0.08, (60, dim))
    w = rng.uniform(0, 0.08, (30, dim))
    ff, fw = sph.neighbor_pairs(f, w, h)
    got = set(zip(ff.i.tolist(), ff.j.tolist()))
    want = {(i, j) for i, j in itertools.permutations(range(60), 2) if 0 < np.linalg.norm(f[i] - f[j]) <= 2 * h}
    assert got == want
    gw = set(zip(fw.i.tolist(), fw.j.tolist()))
    ww = {(i, j) for i in range(60) for j in range(30) if 0 < np.linalg.norm(f[i] - w[j]) <= 2 * h}
    assert gw == ww
    assert np.allclose(ff.rij, f[ff.i] - f[ff.j])
    assert np.allclose(fw.r, np.linalg.norm(f[fw.i] - w[fw.j], axis=1))


@pytest.mark.parametrize("dim", [2, 3])
def test_summation_density_of_an_unperturbed_lattice_is_rho0(dim):
    P = _params(dim)
    n = 16 if dim == 2 else 9
    pos = _lattice(dim, n, P.dp)
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, dim)), P.h)
    rho = sph.density_summation(P, pos.shape[0], ff, fw)
    inner = _interior(pos, 0, n * P.dp, 2 * P.h)
    assert inner.sum() > 0
    assert np.allclose(rho[inner], P.rho0, rtol=1e-12)
    assert np.all(rho[~inner] <= P.rho0 * (1 + 1e-12))  # truncated support near the free edges
    assert rho[0] < 0.7 * P.rho0  # corner particle


def test_pair_forces_conserve_momentum():
    dim = 2
    P = _params(dim)
    rng = np.random.default_rng(7)
    pos = _lattice(dim, 14, P.dp) + rng.uniform(-0.2, 0.2, (196, 2)) * P.dp
    vel = rng.standard_normal((196, 2)) * 0.5
    rho = P.rho0 * (1 + 0.01 * rng.standard_normal(196))
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, dim)), P.h)
    acc = sph.acceleration(P, vel, rho, np.full(196, np.nan), ff, fw)
    # equal masses: sum_i a_i = 0 (pairwise antisymmetry of Eq. (5) incl. the Riemann P*)
    assert np.linalg.norm(acc.sum(axis=0)) < 1e-11 * np.abs(acc).sum()
    assert np.abs(acc).sum() > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_pressure_field_gives_minus_grad_p_over_rho(dim):
    P = _params(dim, c0=10.0)
    n = 16 if dim == 2 else 9
    pos = _lattice(dim, n, P.dp)
    G = 500.0  # Pa/m along x
    rho = P.rho0 + G * pos[:, 0] / P.c0 ** 2
    vel = np.zeros_like(pos)
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, dim)), P.h)
    acc = sph.acceleration(P, vel, rho, np.full(pos.shape[0], np.nan), ff, fw)
    inner = _interior(pos, 0, n * P.dp, 2 * P.h)
    ax = acc[inner, 0] * rho[inner] / (-G)
    assert np.allclose(ax, 1.0, atol=0.04)
    assert np.allclose(ax, _lattice_moment(dim, P.dp, P.h), atol=0.005)
    assert np.allclose(acc[inner, 1:], 0.0, atol=0.02 * G / P.rho0)


@pytest.mark.parametrize("dim", [2, 3])
def test_viscous_term_is_nu_laplacian(dim):
    P = _params(dim, nu=2e-3)
    n = 20 if dim == 2 else 10
    pos = _lattice(dim, n, P.dp)
    A = 0.5  # v_x = A (y^2 [+ z^2])  =>  nu lap v_x = 2 (d - 1) A nu
    vel = np.zeros_like(pos)
    vel[:, 0] = A * np.sum(pos[:, 1:] ** 2, axis=1)
    rho = np.full(pos.shape[0], P.rho0)
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, dim)), P.h)
    acc = sph.acceleration(P, vel, rho, np.full(pos.shape[0], np.nan), ff, fw)
    inner = _interior(pos, 0, n * P.dp, 2 * P.h)
    want = 2 * (dim - 1) * A * P.nu
    assert np.allclose(acc[inner, 0] / want, 1.0, atol=0.04)


@pytest.mark.parametrize("dim", [2, 3])
def test_continuity_of_uniform_expansion(dim):
    P = _params(dim)
    n = 16 if dim == 2 else 9
    pos = _lattice(dim, n, P.dp)
    E = 0.3
    vel = np.zeros_like(pos)
    vel[:, 0] = E * pos[:, 0]  # div v = E
    rho = np.full(pos.shape[0], P.rho0)
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, dim)), P.h)
    drho = sph.continuity_rate(P, vel, rho, ff, fw)
    inner = _interior(pos, 0, n * P.dp, 2 * P.h)
    assert np.allclose(drho[inner] / (-P.rho0 * E), 1.0, atol=0.04)
    assert np.allclose(drho[inner] / (-P.rho0 * E), _lattice_moment(dim, P.dp, P.h), atol=0.005)


def test_continuity_pressure_term_diffuses():
    dim = 2
    P = _params(dim)
    pos = _lattice(dim, 16, P.dp)
    x = pos[:, 0] - 8 * P.dp
    rho = P.rho0 + 1e-3 * (x / P.dp) ** 2  # pressure minimum in the middle column
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, dim)), P.h)
    drho = sph.continuity_rate(P, np.zeros_like(pos), rho, ff, fw)
    inner = _interior(pos, 0, 16 * P.dp, 2 * P.h)
    # at rest only the Riemann pressure term acts: density rises where pressure is lowest
    assert np.all(drho[inner & (np.abs(x) < 0.6 * P.dp)] > 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_continuity_pressure_term_magnitude(dim):
    # Eq. (4) at rest with the Riemann state of Eqs. (6)-(7): U_L = U_R = 0, so
    # (v_i - v*_ij) . e_ij = (p_i - p_j) / (2 rho-bar c0) and
    # drho_i/dt = (rho_i / rho-bar) / c0 sum_j V_j (p_i - p_j) dW/dr.
    # For p = k x^2 the odd part of p_i - p_j cancels inside a full neighbourhood, leaving
    # k sum_j V_j x_ji^2 |dW/dr|.  Its continuum limit is (d + 1) / d E_W[r] (integrate
    # x^2 |W'| by parts over the support), and for the Wendland C2 kernel E_W[r] is a pair of
    # Beta integrals: 2h/3 in 2-D, 5h/6 in 3-D, so the moment is h and 10h/9.  A lost factor
    # 2 or c0, or the opposite sign of the pressure jump, fails the first check below
    # (whether rho_i or rho-bar divides is second order here: |drho| / rho0 < 1e-6).
    P = _params(dim)
    n = 18 if dim == 2 else 10
    pos = _lattice(dim, n, P.dp)
    x = pos[:, 0] - 0.5 * n * P.dp
    k = 2.0
    rho = P.rho0 + k * x ** 2 / P.c0 ** 2  # p = k x^2 by Eq. (3); |drho| / rho0 < 1e-6
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, dim)), P.h)
    drho = sph.continuity_rate(P, np.zeros_like(pos), rho, ff, fw)
    inner = _interior(pos, 0, n * P.dp, 2 * P.h)
    # the same moment summed over an unbounded lattice
    ax = np.arange(-4, 5) * P.dp
    g = np.meshgrid(*([ax] * dim), indexing="ij")
    X = np.stack([c.ravel() for c in g], axis=1)
    r = np.linalg.norm(X, axis=1)
    s = (r > 0) & (r < 2 * P.h)
    m2_lattice = float(np.sum(P.dp ** dim * X[s, 0] ** 2 * -kernel.dW(r[s], P.h, dim)))
    m2_continuum = P.h if dim == 2 else 10.0 * P.h / 9.0
    assert np.allclose(drho[inner] / (k * m2_lattice / P.c0), 1.0, atol=2e-6)
    assert abs(m2_lattice / m2_continuum - 1.0) < 0.025


def _pair(P, r, vi, vj):
    pos = np.array([[0.0, 0.0], [r, 0.0]])
    vel = np.array([[vi, 0.0], [vj, 0.0]])
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, 2)), P.h)
    return pos, vel, ff, fw


def test_riemann_velocity_at_rest_is_the_linear_acoustic_solution():
    # Eq. (6) at rest: U* = (P_L - P_R) / (2 rho-bar c0) = (P_L - P_R) / (Z_L + Z_R) with the
    # acoustic impedances Z = rho c0, the linear acoustic Riemann solution, at any density
    # contrast.  Two particles at rest with a 20 % density jump; Eq. (4) carries U* as
    # (v_i - v*_ij) . e_ij.  (Half the jump over rho_i alone would be off by 10 % here.)
    P = _params(2, c0=10.0)
    r = 1.1 * P.dp
    _, vel, ff, fw = _pair(P, r, 0.0, 0.0)
    rho = np.array([1000.0, 1200.0])
    p = P.c0 ** 2 * (rho - P.rho0)
    drho = sph.continuity_rate(P, vel, rho, ff, fw)
    dw = float(kernel.dW(r, P.h, 2))
    for i, j in ((0, 1), (1, 0)):
        u_star = (p[i] - p[j]) / (rho[i] * P.c0 + rho[j] * P.c0)
        assert np.isclose(drho[i], 2 * rho[i] * P.mass / rho[j] * u_star * dw, rtol=1e-12)


@pytest.mark.parametrize("w", [0.05, 0.2, 1.0, 3.0, -0.5])
def test_riemann_pressure_limiter(w):
    # Two equal particles closing at 2w (w < 0: separating), U_L - U_R = 2w.  Eqs. (7)-(8):
    # in expansion P* = P-bar (no dissipation); in weak compression the low-dissipation value
    # P-bar + 3/2 rho (U_L - U_R)^2; once 3 (U_L - U_R) >= c0 the limiter gives the linear
    # acoustic Riemann pressure P-bar + rho c0 (U_L - U_R) / 2.  Eq. (5) turns P* into
    # a_i = -2 m P* / rho^2 grad W_ij (no viscosity here).
    P = sph.make_params(2, 0.01, 1.3, 1000.0, 10.0, 0.0, 1e-4)
    r = 1.1 * P.dp
    _, vel, ff, fw = _pair(P, r, w, -w)
    rho = np.full(2, 1001.0)
    pbar = P.c0 ** 2 * 1.0
    du = 2 * w
    if du <= 0:
        pstar = pbar
    elif 3 * du < P.c0:
        pstar = pbar + 1.5 * rho[0] * du ** 2
    else:
        pstar = pbar + 0.5 * rho[0] * P.c0 * du
    acc = sph.acceleration(P, vel, rho, np.full(2, np.nan), ff, fw)
    dw = float(kernel.dW(r, P.h, 2))
    # e_01 = (r_0 - r_1) / r = -e_x, so a_0 = +2 m P* dW/dr / rho^2 e_x (dW/dr < 0: pushed back)
    assert np.isclose(acc[0, 0], 2 * P.mass * pstar * dw / rho[0] ** 2, rtol=1e-12)
    assert np.isclose(acc[1, 0], -acc[0, 0], rtol=1e-12) and acc[0, 1] == 0.0


def test_boundary_pressure_term_cancels_truncation():
    # a lattice block at uniform pressure p_b: with Eq. (18) the edge particles feel no force
    dim = 2
    P = _params(dim)
    pos = _lattice(dim, 12, P.dp)
    pb = 37.0
    rho = np.full(pos.shape[0], P.rho0 + pb / P.c0 ** 2)
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, dim)), P.h)
    vel = np.zeros_like(pos)
    with_bc = sph.acceleration(P, vel, rho, np.full(pos.shape[0], pb), ff, fw)
    without = sph.acceleration(P, vel, rho, np.full(pos.shape[0], np.nan), ff, fw)
    assert np.abs(with_bc).max() < 1e-12 * np.abs(without).max()
    edge = ~_interior(pos, 0, 12 * P.dp, 2 * P.h)
    assert np.abs(without[edge]).max() > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_pressure_is_in_equilibrium_inside_walls(dim):
    # A fluid block at rest at uniform density, wrapped in a wall layer 2h thick that
    # continues the fluid lattice.  The wall neighbours take p_j = p_i, rho_j = rho_i
    # (reading A11), so every pair of Eq. (5) carries the same coefficient and the sum of
    # grad W over a full lattice neighbourhood is zero by symmetry: no particle moves and
    # Eq. (4) gives no density change.  Without the walls the edge particles are pushed
    # out, so a wall term with the wrong sign, factor or state fails here.
    P = _params(dim)
    n = 10 if dim == 2 else 6
    t = int(np.ceil(2 * P.h / P.dp))
    grid = _lattice(dim, n + 2 * t, P.dp) - t * P.dp
    inside = np.all((grid > 0) & (grid < n * P.dp), axis=1)
    pos, wall = grid[inside], grid[~inside]
    rho = np.full(pos.shape[0], P.rho0 + 50.0 / P.c0 ** 2)  # p = 50 Pa
    vel = np.zeros_like(pos)
    nan = np.full(pos.shape[0], np.nan)
    ff, fw = sph.neighbor_pairs(pos, wall, P.h)
    acc = sph.acceleration(P, vel, rho, nan, ff, fw)
    scale = 50.0 / P.rho0 / P.dp
    assert np.abs(acc).max() < 1e-10 * scale
    assert np.abs(sph.continuity_rate(P, vel, rho, ff, fw)).max() < 1e-12 * P.rho0
    ff0, fw0 = sph.neighbor_pairs(pos, np.zeros((0, dim)), P.h)
    assert np.abs(sph.acceleration(P, vel, rho, nan, ff0, fw0)).max() > 0.1 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_wall_continuity_accumulates_the_stopped_mass_flux(dim):
    # A fluid block at uniform density moving at -u e_x onto a flat wall slab (2h thick,
    # 2h wider than the block on every side).  Between fluid particles v_i = v_j and
    # p_i = p_j, so v* = v and Eq. (4) has no fluid term; the mirrored wall state of reading
    # A11 gives v* = 0, so each wall pair adds 2 rho V (v_i . e_ij) dW/dr.  Summed over the
    # block, the pairs straddling the wall plane give sum_i V drho_i/dt = rho0 u A times the
    # lattice moment (1 in the continuum): the density rises at the rate of the mass flux
    # the wall stops.  A wall at rest (v_j = 0) would give half of it; dropping the wall
    # term, none.
    P = _params(dim)
    n = 8 if dim == 2 else 6
    t = int(np.ceil(2 * P.h / P.dp))
    pos = _lattice(dim, n, P.dp)
    slab = _lattice(dim, n + 2 * t, P.dp) - t * P.dp
    slab = slab[(slab[:, 0] < 0) & np.all(slab[:, 1:] > -t * P.dp, axis=1)]
    u = 0.2
    vel = np.zeros_like(pos)
    vel[:, 0] = -u
    rho = np.full(pos.shape[0], P.rho0)
    ff, fw = sph.neighbor_pairs(pos, slab, P.h)
    drho = sph.continuity_rate(P, vel, rho, ff, fw)
    area = (n * P.dp) ** (dim - 1)
    got = float(np.sum(P.dp ** dim * drho))
    assert np.isclose(got, P.rho0 * u * area * _lattice_moment(dim, P.dp, P.h), rtol=1e-10)
    reach = pos[:, 0] + 0.5 * P.dp < 2 * P.h  # the nearest wall layer sits at -dp/2
    assert np.all(drho[reach] > 0.0)
    assert np.all(drho[~reach] == 0.0)


def test_wall_neighbours_stop_an_approaching_particle():
    dim = 2
    P = _params(dim)
    wall = _lattice(dim, 8, P.dp) - np.array([0.0, 8 * P.dp])  # block below y = 0
    pos = np.array([[4 * P.dp, 0.5 * P.dp]])
    rho = np.array([P.rho0])
    ff, fw = sph.neighbor_pairs(pos, wall, P.h)
    down = sph.acceleration(P, np.array([[0.0, -0.5]]), rho, np.array([np.nan]), ff, fw)
    rest = sph.acceleration(P, np.array([[0.0, 0.0]]), rho, np.array([np.nan]), ff, fw)
    assert abs(rest[0, 1]) < 1e-12
    assert down[0, 1] > 0  # pushed back up, away from the wall
    assert kernel.W(0.0, P.h, 2) > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_background_pressure_leaves_interior_forces_and_is_carried_by_the_boundary_term(dim):
    # reading A22: p = c0^2 (rho - rho0) + p_bg.  At uniform density the constant adds no force
    # inside a lattice (sum_j grad W_ij = 0 by symmetry); with a density gradient it adds the
    # known discretisation error of the symmetric pressure term, of order p_bg |grad rho| / rho^2;
    # on an open edge it is cancelled by Eq. (18) when p_b carries it too
    P0 = _params(dim, c0=10.0)
    Pb = sph.make_params(dim, P0.dp, 1.3, P0.rho0, P0.c0, P0.nu, P0.dt, p_bg=2000.0)
    n = 16 if dim == 2 else 9
    pos = _lattice(dim, n, P0.dp)
    vel = np.zeros_like(pos)
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, dim)), P0.h)
    nan = np.full(pos.shape[0], np.nan)
    inner = _interior(pos, 0, n * P0.dp, 2 * P0.h)
    rho_u = np.full(pos.shape[0], P0.rho0)
    au = sph.acceleration(Pb, vel, rho_u, nan, ff, fw)
    assert np.abs(au[inner]).max() < 1e-9 * Pb.p_bg / P0.rho0 / P0.dp
    assert np.abs(au[~inner]).max() > 1.0  # an open edge feels the background...
    # ... unless it is an open boundary whose p_b includes it (Eq. (18))
    with_bc = sph.acceleration(Pb, vel, rho_u, np.full(pos.shape[0], Pb.p_bg), ff, fw)
    assert np.abs(with_bc).max() < 1e-9 * Pb.p_bg / P0.rho0 / P0.dp
    grad_rho = 500.0 / P0.c0 ** 2
    rho = P0.rho0 + grad_rho * pos[:, 0]
    a0 = sph.acceleration(P0, vel, rho, nan, ff, fw)
    ab = sph.acceleration(Pb, vel, rho, nan, ff, fw)
    assert np.abs(ab[inner] - a0[inner]).max() < 2.0 * Pb.p_bg * grad_rho / P0.rho0 ** 2
    assert np.allclose(sph.eos(np.array([P0.rho0]), Pb), Pb.p_bg)


@pytest.mark.parametrize("dim", [2, 3])
def test_transport_sum_vanishes_inside_and_pushes_into_voids(dim):
    # Eq. (10): the shift -dt p_max sum_j 2 m/(rho_i rho_j) dW/dr e_ij is zero inside a regular
    # lattice (sum_j grad W_ij = 0 by symmetry) and moves an edge particle away from its
    # neighbours (into the void); it equals -2 (m / rho^2) times the lattice's grad of sum W
    P = _params(dim)
    n = 12 if dim == 2 else 8
    pos = _lattice(dim, n, P.dp)
    rho = np.full(pos.shape[0], P.rho0)
    ff, fw = sph.neighbor_pairs(pos, np.zeros((0, dim)), P.h)
    B = sph.transport_sum(P, rho, ff, fw)
    inner = _interior(pos, 0, n * P.dp, 2 * P.h)
    assert np.abs(B[inner]).max() < 1e-9 * np.abs(B).max()
    # the particle at the lower-left corner: its neighbours lie at +x, +y (, +z); B points
    # toward them, so the shift -B points out of the block
    k = int(np.argmin(pos.sum(axis=1)))
    assert np.all(B[k] > 0)
    # brute force for that particle
    r = pos[k] - pos
    d = np.linalg.norm(r, axis=1)
    m = (d > 0) & (d < 2 * P.h)
    from oracle import kernel
    ref = (2 * P.mass / P.rho0 ** 2 * kernel.dW(d[m], P.h, dim))[:, None] * r[m] / d[m][:, None]
    assert np.allclose(B[k], ref.sum(axis=0), rtol=1e-12)
