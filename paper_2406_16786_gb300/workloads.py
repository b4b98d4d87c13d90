"""Seeded synthetic inputs: channel and pipe geometries, particle lattices, velocity fields.

This module only *describes problems*: where fluid and wall particles start, what each
in-/outlet buffer box is (origin, frame, extent, boundary type) and the physical
constants.  It performs no step of the open-boundary method and no SPH arithmetic, so both
the CUDA library's tests/bench and the CPU oracle's tests can take their inputs from it.

Conventions shared with the library header ``include/sphbuf.h``:

* positions are global coordinates in metres; ``dim`` is 2 or 3 (2-D cases keep z = 0);
* a buffer frame is a row-major 3x3 matrix ``R`` with ``X' = R (X - O')``; its first row is
  the unit normal of the in-/outlet, pointing in the *inflow* direction for inflow and
  bidirectional buffers and in the *outflow* direction for outflow buffers (Sec. 3.1, 3.2);
* the cell-relative encoding of a position is the storage format of the library: integer
  cell coordinates on a dense grid of cell size ``cs = 2 h`` anchored at ``lo`` plus an FP32
  offset inside the cell (``encode_positions``).

Lattices follow the paper's set-up: particles on a Cartesian lattice of spacing ``dp`` with
three wall layers (Sec. 3, 5.1); a seeded uniform jitter of +-0.01 dp is added to fluid
particles so that threshold ties are rare.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Boundary-type codes; identical numbering in include/sphbuf.h (sphbuf_bc_type).
VELOCITY_INLET = 0
PRESSURE_OUTLET = 1
PRESSURE_INLET = 2
VELOCITY_OUTLET = 3
BIDIR_PRESSURE = 4
BIDIR_VELOCITY = 5
BC_NAMES = {
    VELOCITY_INLET: "velocity_inlet",
    PRESSURE_OUTLET: "pressure_outlet",
    PRESSURE_INLET: "pressure_inlet",
    VELOCITY_OUTLET: "velocity_outlet",
    BIDIR_PRESSURE: "bidir_pressure",
    BIDIR_VELOCITY: "bidir_velocity",
}

BASE_SEED = 20240616


@dataclasses.dataclass
class BufferSpec:
    """One in-/outlet buffer box as the user states it (Sec. 3.1, Fig. of the buffer)."""

    origin: np.ndarray  # (3,) box centre O'
    rotation: np.ndarray  # (3, 3) row-major, X' = R (X - O')
    extent: np.ndarray  # (3,) a (along X'), b (along Y'), c (along Z'; ignored in 2-D)
    bc: int
    umax: float = 0.0  # velocity BC: peak speed of the profile
    half_width: float = 0.0  # velocity BC: R of the profile 1-(Y'/R)^2; 0 => plug
    p_b: float = 0.0  # pressure BC: p_b(t) = p_b + p_amp sin(p_omega t + p_phase)
    p_amp: float = 0.0
    p_omega: float = 0.0
    p_phase: float = 0.0
    # time-varying frame of an inflow buffer (Sec. 5.3): turned by omega per second about the
    # pivot (about z in 2-D, about ``axis`` in 3-D); None = fixed frame
    pivot: Optional[np.ndarray] = None
    axis: Optional[np.ndarray] = None
    omega: float = 0.0
    # RCR Windkessel outlet (Eq. (31)) of a pressure buffer: R_p, C, R_d (SI), initial P_d;
    # wk_c None = p_b(t) as above
    wk_rp: float = 0.0
    wk_c: Optional[float] = None
    wk_rd: float = 0.0
    wk_pd0: float = 0.0


@dataclasses.dataclass
class Case:
    """A complete synthetic problem: grid box, constants, particles, buffers."""

    name: str
    dim: int
    lo: np.ndarray  # (3,)
    hi: np.ndarray  # (3,)
    dp: float
    h_over_dp: float
    rho0: float
    c0: float
    nu: float
    dt: float
    fluid_pos: np.ndarray  # (n, dim) float64
    fluid_vel: np.ndarray  # (n, dim) float64
    fluid_rho: np.ndarray  # (n,) float64
    wall_pos: np.ndarray  # (nw, dim) float64
    buffers: List[BufferSpec]
    capacity: int
    steps: int = 1
    p_bg: float = 0.0  # background pressure of the EoS (Pa); buffer p_b values include it
    tvf_lambda: float = 0.0  # transport velocity (Eq. (10)) coefficient, 5-10 in the paper; 0 = off
    dual_substeps: int = 0  # dual-criteria time stepping: acoustic steps per dt (0 = single-rate)

    @property
    def n(self) -> int:
        return int(self.fluid_pos.shape[0])

    @property
    def cs(self) -> float:
        # grid cell size = kernel support 2h, with h = h_over_dp * dp
        return 2.0 * (self.h_over_dp * self.dp)

    def grid_dims(self):
        return grid_dims(self.lo, self.hi, self.cs, self.dim)


def grid_dims(lo, hi, cs, dim):
    n = [int(math.ceil((float(hi[a]) - float(lo[a])) / cs)) for a in range(3)]
    if dim == 2:
        n[2] = 1
    return n


def encode_positions(pos: np.ndarray, lo, cs: float, dims: Sequence[int]):
    """Global FP64 positions -> (linear cell index int32, FP32 in-cell offset).

    cell_a = floor((x_a - lo_a) / cs); frac_a = fl32((x_a - lo_a) - cell_a * cs), then folded
    back into [0, cs32) with at most one FP32 add/sub of cs32.  Linear index
    (cz * ny + cy) * nx + cx.  Positions outside the grid raise ValueError.
    """
    pos = np.asarray(pos, dtype=np.float64)
    n, d = pos.shape
    cs32 = np.float32(cs)
    cells = np.zeros((n, 3), dtype=np.int64)
    frac = np.zeros((n, d), dtype=np.float32)
    for a in range(d):
        t = pos[:, a] - float(lo[a])
        c = np.floor(t / cs).astype(np.int64)
        f = (t - c.astype(np.float64) * cs).astype(np.float32)
        hi_m = f >= cs32
        f[hi_m] = f[hi_m] - cs32
        c[hi_m] += 1
        lo_m = f < np.float32(0)
        f[lo_m] = f[lo_m] + cs32
        c[lo_m] -= 1
        # a value that rounds up to cs32 after the add above is folded once more
        hi_m = f >= cs32
        f[hi_m] = np.float32(0)
        c[hi_m] += 1
        cells[:, a] = c
        frac[:, a] = f
    nx, ny, nz = dims
    bad = (cells[:, 0] < 0) | (cells[:, 0] >= nx) | (cells[:, 1] < 0) | (cells[:, 1] >= ny)
    if d == 3:
        bad |= (cells[:, 2] < 0) | (cells[:, 2] >= nz)
    if np.any(bad):
        raise ValueError("%d positions lie outside the grid box" % int(bad.sum()))
    lin = (cells[:, 2] * ny + cells[:, 1]) * nx + cells[:, 0]
    return lin.astype(np.int32), frac


def decode_positions(cell: np.ndarray, frac: np.ndarray, lo, cs: float, dims: Sequence[int]):
    """Inverse of ``encode_positions`` in FP64: x_a = lo_a + cell_a * cs + frac_a."""
    nx, ny, _ = dims
    cell = np.asarray(cell, dtype=np.int64)
    d = frac.shape[1]
    cc = [cell % nx, (cell // nx) % ny, cell // (nx * ny)]
    out = np.zeros((cell.shape[0], d), dtype=np.float64)
    for a in range(d):
        out[:, a] = float(lo[a]) + cc[a].astype(np.float64) * cs + frac[:, a].astype(np.float64)
    return out


# ----------------------------------------------------------------------------- frames
def frame_2d(angle_rad: float) -> np.ndarray:
    """Frame whose first row is the unit vector at ``angle_rad`` in the xy-plane."""
    c, s = math.cos(angle_rad), math.sin(angle_rad)
    return np.array([[c, s, 0.0], [-s, c, 0.0], [0.0, 0.0, 1.0]])


def frame_3d(normal, roll: float = 0.0) -> np.ndarray:
    """An orthonormal right-handed frame with first row ``normal`` (Gram-Schmidt).

    The second row is the component of the coordinate axis least aligned with the normal,
    orthogonalised against it and turned by ``roll`` about the normal; the third row is
    normal x second.  Any roll is a valid local frame: the buffer box only needs its X'
    axis on the normal.
    """
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    k = int(np.argmin(np.abs(n)))
    helper = np.zeros(3)
    helper[k] = 1.0
    e2 = helper - np.dot(helper, n) * n
    e2 /= np.linalg.norm(e2)
    e3 = np.cross(n, e2)
    c, s = math.cos(roll), math.sin(roll)
    e2r = c * e2 + s * e3
    e3r = np.cross(n, e2r)
    return np.stack([n, e2r, e3r])


# --------------------------------------------------------------------------- lattices
def _jitter(rng, shape, dp, amount=0.01):
    return rng.uniform(-amount * dp, amount * dp, size=shape)


def _grid_box(points_list, margin):
    allp = np.concatenate([p for p in points_list if p.size], axis=0)
    lo = np.zeros(3)
    hi = np.zeros(3)
    d = allp.shape[1]
    lo[:d] = allp.min(axis=0) - margin
    hi[:d] = allp.max(axis=0) + margin
    if d == 2:
        lo[2], hi[2] = 0.0, 1.0
    return lo, hi


def channel_2d_local(length, width, dp, wall_layers=3, wall_extend=3):
    """Fluid and wall lattice points of a straight 2-D channel in its own frame (s, t)."""
    ns = int(round(length / dp))
    nt = int(round(width / dp))
    s = (np.arange(ns) + 0.5) * dp
    t = -0.5 * width + (np.arange(nt) + 0.5) * dp
    S, T = np.meshgrid(s, t, indexing="ij")
    fluid = np.stack([S.ravel(), T.ravel()], axis=1)
    sw = (np.arange(-wall_extend, ns + wall_extend) + 0.5) * dp
    tw = np.concatenate([0.5 * width + (np.arange(wall_layers) + 0.5) * dp,
                         -0.5 * width - (np.arange(wall_layers) + 0.5) * dp])
    SW, TW = np.meshgrid(sw, tw, indexing="ij")
    wall = np.stack([SW.ravel(), TW.ravel()], axis=1)
    return fluid, wall


def pipe_3d_local(length, radius, dp, wall_layers=3, wall_extend=3):
    """Fluid and wall lattice points of a straight circular pipe in its frame (s, y, z)."""
    ns = int(round(length / dp))
    m = int(math.ceil((radius + wall_layers * dp) / dp))
    yz = (np.arange(-m, m) + 0.5) * dp
    Y, Z = np.meshgrid(yz, yz, indexing="ij")
    r = np.sqrt(Y * Y + Z * Z).ravel()
    Y, Z = Y.ravel(), Z.ravel()
    inner = r < radius
    ring = (r >= radius) & (r < radius + wall_layers * dp)
    s = (np.arange(ns) + 0.5) * dp
    sw = (np.arange(-wall_extend, ns + wall_extend) + 0.5) * dp
    fluid = np.stack([np.repeat(s, inner.sum()), np.tile(Y[inner], ns), np.tile(Z[inner], ns)], axis=1)
    nsw = sw.shape[0]
    wall = np.stack([np.repeat(sw, ring.sum()), np.tile(Y[ring], nsw), np.tile(Z[ring], nsw)], axis=1)
    return fluid, wall


def _to_global(local, frame, origin):
    d = local.shape[1]
    M = frame[:d, :d]
    return origin[:d][None, :] + local @ M


def straight_channel_case(
    *,
    name="channel2d",
    length=10.0,
    width=1.0,
    dp=0.025,
    angle_deg=0.0,
    inlet_bc=VELOCITY_INLET,
    outlet_bc=PRESSURE_OUTLET,
    umax=1.0,
    profile="plug",
    p_in=0.0,
    p_out=0.0,
    p_amp=0.0,
    p_omega=0.0,
    rho0=1000.0,
    c0=10.0,
    nu=1e-2,
    dt=None,
    h_over_dp=1.3,
    buffer_layers=4,
    seed=BASE_SEED + 1,
    init_velocity="bc",
    capacity_factor=1.5,
    steps=200,
) -> Case:
    """2-D straight channel of ``length`` x ``width`` along ``angle_deg`` (Sec. 5.1 set-up)."""
    rng = np.random.default_rng(seed)
    theta = math.radians(angle_deg)
    fluid_l, wall_l = channel_2d_local(length, width, dp)
    fluid_l = fluid_l + _jitter(rng, fluid_l.shape, dp)
    frame = frame_2d(theta)
    origin = np.zeros(3)
    fluid = _to_global(fluid_l, frame, origin)
    wall = _to_global(wall_l, frame, origin)
    h = h_over_dp * dp
    lo, hi = _grid_box([fluid, wall], margin=2.0 * (2.0 * h))
    a = buffer_layers * dp
    e_s = frame[0]
    half = 0.5 * width
    bufs = []
    inlet_is_bidir = inlet_bc in (BIDIR_PRESSURE, BIDIR_VELOCITY)
    outlet_is_bidir = outlet_bc in (BIDIR_PRESSURE, BIDIR_VELOCITY)
    prof_hw = half if profile == "parabolic" else 0.0
    # inlet box: centred a/2 inside the channel start, X' along +e_s (into the channel)
    bufs.append(BufferSpec(origin=origin + 0.5 * a * e_s, rotation=frame.copy(),
                           extent=np.array([a, width, 0.0]), bc=inlet_bc, umax=umax,
                           half_width=prof_hw, p_b=p_in, p_amp=p_amp, p_omega=p_omega))
    # outlet box: X' along +e_s for an outflow buffer, along -e_s (inflow direction) if bidirectional
    out_frame = frame_2d(theta + math.pi) if outlet_is_bidir else frame.copy()
    bufs.append(BufferSpec(origin=origin + (length - 0.5 * a) * e_s, rotation=out_frame,
                           extent=np.array([a, width, 0.0]), bc=outlet_bc, umax=umax,
                           half_width=prof_hw, p_b=p_out))
    del inlet_is_bidir
    vel = np.zeros_like(fluid)
    if init_velocity == "bc":
        # every particle starts at the inlet profile value along the channel axis
        t_loc = fluid_l[:, 1]
        if profile == "parabolic":
            u = umax * np.clip(1.0 - (t_loc / half) ** 2, 0.0, None)
        else:
            u = np.full(fluid.shape[0], umax)
        vel = u[:, None] * e_s[None, :2]
    elif init_velocity == "inlet_only":
        t_loc = fluid_l[:, 1]
        in_box = fluid_l[:, 0] < a
        if profile == "parabolic":
            u = umax * np.clip(1.0 - (t_loc / half) ** 2, 0.0, None)
        else:
            u = np.full(fluid.shape[0], umax)
        vel[in_box] = u[in_box, None] * e_s[None, :2]
    if dt is None:
        dt = min(0.25 * h / (c0 + umax), 0.125 * h * h / nu if nu > 0 else 1e30)
    n = fluid.shape[0]
    return Case(name=name, dim=2, lo=lo, hi=hi, dp=dp, h_over_dp=h_over_dp, rho0=rho0, c0=c0,
                nu=nu, dt=dt, fluid_pos=fluid, fluid_vel=vel, fluid_rho=np.full(n, rho0),
                wall_pos=wall, buffers=bufs, capacity=int(capacity_factor * n) + 1024, steps=steps)


def pipe_case(
    *,
    name="pipe3d",
    length=5.09,
    radius=0.5,
    dp=0.01,
    axis=(1.0, 1.0, 1.0),
    roll=None,
    inlet_bc=BIDIR_PRESSURE,
    outlet_bc=BIDIR_PRESSURE,
    p_in=0.0,
    p_amp=50.0,
    p_omega=math.pi,
    p_out=0.0,
    umax=0.0,
    rho0=1000.0,
    c0=3.0,
    nu=1e-2,
    dt=None,
    umax_est=0.03,
    h_over_dp=1.3,
    buffer_layers=4,
    seed=BASE_SEED + 3,
    init_velocity="rest",
    capacity_factor=1.25,
    steps=1000,
) -> Case:
    """3-D circular pipe along ``axis`` with a buffer box at each end (Sec. 6.1 set-up)."""
    rng = np.random.default_rng(seed)
    if roll is None:
        roll = float(rng.uniform(0.0, 2.0 * math.pi))
    frame = frame_3d(axis, roll)
    fluid_l, wall_l = pipe_3d_local(length, radius, dp)
    fluid_l = fluid_l + _jitter(rng, fluid_l.shape, dp)
    origin = np.zeros(3)
    fluid = _to_global(fluid_l, frame, origin)
    wall = _to_global(wall_l, frame, origin)
    h = h_over_dp * dp
    lo, hi = _grid_box([fluid, wall], margin=2.0 * (2.0 * h))
    a = buffer_layers * dp
    e_s = frame[0]
    flip = np.diag([-1.0, -1.0, 1.0]) @ frame  # first row -e_s, still right-handed
    inlet_bidir = inlet_bc in (BIDIR_PRESSURE, BIDIR_VELOCITY)
    outlet_bidir = outlet_bc in (BIDIR_PRESSURE, BIDIR_VELOCITY)
    del inlet_bidir
    bufs = [
        BufferSpec(origin=origin + 0.5 * a * e_s, rotation=frame.copy(),
                   extent=np.array([a, 2 * radius, 2 * radius]), bc=inlet_bc, umax=umax,
                   half_width=radius, p_b=p_in, p_amp=p_amp, p_omega=p_omega),
        BufferSpec(origin=origin + (length - 0.5 * a) * e_s,
                   rotation=flip if outlet_bidir else frame.copy(),
                   extent=np.array([a, 2 * radius, 2 * radius]), bc=outlet_bc, umax=umax,
                   half_width=radius, p_b=p_out),
    ]
    vel = np.zeros_like(fluid)
    if init_velocity == "profile" and umax > 0:
        r2 = fluid_l[:, 1] ** 2 + fluid_l[:, 2] ** 2
        u = umax * np.clip(1.0 - r2 / radius ** 2, 0.0, None)
        vel = u[:, None] * e_s[None, :]
    if dt is None:
        dt = min(0.25 * h / (c0 + umax_est), 0.125 * h * h / nu if nu > 0 else 1e30)
    n = fluid.shape[0]
    return Case(name=name, dim=3, lo=lo, hi=hi, dp=dp, h_over_dp=h_over_dp, rho0=rho0, c0=c0,
                nu=nu, dt=dt, fluid_pos=fluid, fluid_vel=vel, fluid_rho=np.full(n, rho0),
                wall_pos=wall, buffers=bufs, capacity=int(capacity_factor * n) + 4096, steps=steps)


def shear_velocity(case: Case, u0: float, lateral: float = 0.1, seed: int = 7) -> np.ndarray:
    """A velocity field that crosses every buffer face in both directions.

    Along each buffer's first frame row the speed is ``u0 * sin(2 pi Y'/b + phase)`` (half the
    cross-section moves in, half out), plus seeded lateral noise of relative size ``lateral``.
    Used by the kinematic (drift-only) lockstep tests.
    """
    rng = np.random.default_rng(seed)
    d = case.dim
    pos = case.fluid_pos
    e = case.buffers[0].rotation
    y = (pos - case.buffers[0].origin[None, :d]) @ e[1, :d]
    b = case.buffers[0].extent[1]
    u = u0 * np.sin(2.0 * math.pi * y / b + 0.3)
    v = u[:, None] * e[0, :d][None, :]
    v += lateral * u0 * rng.standard_normal(v.shape)
    return v


def perturbed_state(case: Case, dv: float, drho: float, seed: int = 11):
    """Seeded small perturbations of velocity (absolute, m/s) and density (relative)."""
    rng = np.random.default_rng(seed)
    vel = case.fluid_vel + dv * rng.standard_normal(case.fluid_vel.shape)
    rho = case.fluid_rho * (1.0 + drho * rng.standard_normal(case.fluid_rho.shape))
    return vel, rho


def random_rotation(rng) -> np.ndarray:
    """A seeded proper rotation (QR of a Gaussian matrix, sign-fixed)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def tjunction_case(*, dp=0.006, R=0.5, L=4.0, Rb=0.3, Lb=1.2, branch_deg=60.0, umax=1.0, c0=10.0, nu=1e-2,
                   rho0=1000.0, h_over_dp=1.3, buffer_layers=4, seed=BASE_SEED + 4, developed=True,
                   capacity_factor=1.15, name="cfg4_tjunction") -> Case:
    """3-D T-junction: main pipe (R, L) with a branch (Rb, Lb from the main axis) leaving its
    middle at ``branch_deg`` to the main axis; the assembly is given a seeded arbitrary rotation.
    Velocity inlet (pipe profile, ``umax``) at the main pipe's start, pressure outlets (p = 0) at
    the main pipe's end and the branch end.  With ``developed`` the main pipe starts on the
    Poiseuille profile so that particles cross both main-pipe buffers from the first step.
    """
    rng = np.random.default_rng(seed)
    wl_ = 3 * dp
    ph = math.radians(branch_deg)
    eb = np.array([math.cos(ph), math.sin(ph), 0.0])  # branch axis in the main pipe's frame
    sb0 = 0.5 * L
    m = int(math.ceil((R + wl_) / dp)) + 1
    xs = (np.arange(-4, int(math.ceil(L / dp)) + 4) + 0.5) * dp
    ys_max = sb0 * 0 + Lb * eb[1] + Rb + wl_
    ys = (np.arange(-m, int(math.ceil(ys_max / dp)) + 1) + 0.5) * dp
    zs = (np.arange(-m, m) + 0.5) * dp
    fluid_l, wall_l = [], []
    for x in xs:  # slab by slab keeps memory bounded
        Y, Z = np.meshgrid(ys, zs, indexing="ij")
        Y, Z = Y.ravel(), Z.ravel()
        X = np.full_like(Y, x)
        r_main = np.sqrt(Y * Y + Z * Z)
        in_main = (X >= 0) & (X < L) & (r_main < R)
        rel = np.stack([X - sb0, Y, Z], axis=1)
        sb = rel @ eb
        rb = np.linalg.norm(rel - sb[:, None] * eb[None, :], axis=1)
        in_br = (sb >= 0) & (sb < Lb) & (rb < Rb)
        fl = in_main | in_br
        near_main = (X >= -wl_) & (X < L + wl_) & (r_main < R + wl_)
        near_br = (sb >= 0) & (sb < Lb + wl_) & (rb < Rb + wl_)
        wa = (near_main | near_br) & ~fl
        # open ends: no wall in front of the three cross-sections
        wa &= ~((X < 0) & (r_main < R))
        wa &= ~((X >= L) & (r_main < R))
        wa &= ~((sb >= Lb) & (rb < Rb))
        pts = np.stack([X, Y, Z], axis=1)
        fluid_l.append(pts[fl])
        wall_l.append(pts[wa])
    fluid_l = np.concatenate(fluid_l)
    wall_l = np.concatenate(wall_l)
    fluid_l = fluid_l + rng.uniform(-0.01 * dp, 0.01 * dp, fluid_l.shape)
    Q = random_rotation(rng)  # local -> global: x_g = Q x_l
    fluid = fluid_l @ Q.T
    wall = wall_l @ Q.T
    h = h_over_dp * dp
    lo, hi = _grid_box([fluid, wall], margin=2.0 * (2.0 * h))
    a = buffer_layers * dp
    e_main = Q[:, 0]
    e_br = Q @ eb
    bufs = [
        BufferSpec(origin=Q @ np.array([0.5 * a, 0.0, 0.0]), rotation=frame_3d(e_main, rng.uniform(0, 6.28)),
                   extent=np.array([a, 2 * R, 2 * R]), bc=VELOCITY_INLET, umax=umax, half_width=R),
        BufferSpec(origin=Q @ np.array([L - 0.5 * a, 0.0, 0.0]), rotation=frame_3d(e_main, rng.uniform(0, 6.28)),
                   extent=np.array([a, 2 * R, 2 * R]), bc=PRESSURE_OUTLET, p_b=0.0),
        BufferSpec(origin=Q @ (np.array([sb0, 0.0, 0.0]) + (Lb - 0.5 * a) * eb),
                   rotation=frame_3d(e_br, rng.uniform(0, 6.28)), extent=np.array([a, 2 * Rb, 2 * Rb]),
                   bc=PRESSURE_OUTLET, p_b=0.0),
    ]
    vel = np.zeros_like(fluid)
    r2 = fluid_l[:, 1] ** 2 + fluid_l[:, 2] ** 2
    in_main = (fluid_l[:, 0] >= 0) & (fluid_l[:, 0] < L) & (r2 < R * R)
    if developed:
        u = umax * np.clip(1.0 - r2 / (R * R), 0.0, None) * in_main
    else:
        u = umax * np.clip(1.0 - r2 / (R * R), 0.0, None) * (in_main & (fluid_l[:, 0] < a))
    vel = u[:, None] * e_main[None, :]
    dt = min(0.25 * h / (c0 + umax), 0.125 * h * h / nu)
    n = fluid.shape[0]
    return Case(name="%s_dp%g_n%d" % (name, dp, n), dim=3, lo=lo, hi=hi, dp=dp, h_over_dp=h_over_dp, rho0=rho0,
                c0=c0, nu=nu, dt=dt, fluid_pos=fluid, fluid_vel=vel, fluid_rho=np.full(n, rho0), wall_pos=wall,
                buffers=bufs, capacity=int(capacity_factor * n) + 8192, steps=500)


def config4(dp=0.006) -> Case:
    """3-D T-junction, main pipe R 0.5 x 4 m, branch R 0.3 x 1.2 m at 60 deg, arbitrary rotation,
    one velocity inlet (Umax 1) and two pressure outlets; about 16 M fluid particles at dp 0.006."""
    return tjunction_case(dp=dp)


def star_case(*, seed, n_target, arms, width, name="star", umax=1.0, c0=10.0, nu=1e-2, rho0=1000.0,
              h_over_dp=1.3, buffer_layers=4, p_amp=500.0, p_freq=2.0, capacity_factor=1.6) -> Case:
    """2-D "star" channel: ``arms`` straight arms of width ``width`` leaving a central junction.

    Arm directions are seeded uniform angles at least 40 deg apart; arm length = 4 x width; the
    spacing dp is chosen so that about ``n_target`` fluid particles fill the star.  Fluid = a
    global lattice (jittered) inside any arm rectangle or the junction disc; walls = three
    lattice layers around it, left open at the arm ends.  With two or more arms, arm 0 ends in
    a plug velocity inlet (U = ``umax``) and the others in pressure outlets (p = 0); a single
    arm is a dead end whose open end carries a bidirectional pressure buffer with
    p_b(t) = ``p_amp`` sin(2 pi ``p_freq`` t).
    """
    rng = np.random.default_rng(seed)
    for _ in range(1000):
        ang = np.sort(rng.uniform(0.0, 2.0 * math.pi, arms))
        gaps = np.diff(np.concatenate([ang, ang[:1] + 2.0 * math.pi]))
        if arms == 1 or gaps.min() >= math.radians(40.0):
            break
    L = 4.0 * width
    half = 0.5 * width
    area = arms * L * width + math.pi * half * half
    dp = math.sqrt(area / n_target)
    ext = L + 4 * dp
    ax = (np.arange(-int(ext / dp) - 1, int(ext / dp) + 2) + 0.5) * dp
    X, Y = np.meshgrid(ax, ax, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel()], axis=1)
    E = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    N = np.stack([-np.sin(ang), np.cos(ang)], axis=1)
    s = P @ E.T  # (npts, arms)
    t = P @ N.T
    r = np.linalg.norm(P, axis=1)
    fluid_m = (r < half) | np.any((s >= 0.0) & (s < L) & (np.abs(t) < half), axis=1)
    wall_band = 3 * dp
    near = (r < half + wall_band) | np.any((s >= -half) & (s < L + wall_band) & (np.abs(t) < half + wall_band),
                                           axis=1)
    wall_m = near & ~fluid_m
    # keep the arm ends open: no wall beyond s = L in front of an arm's cross-section
    for k in range(arms):
        wall_m &= ~((s[:, k] >= L) & (np.abs(t[:, k]) < half))
    fluid = P[fluid_m] + rng.uniform(-0.01 * dp, 0.01 * dp, size=(int(fluid_m.sum()), 2))
    wall = P[wall_m]
    h = h_over_dp * dp
    lo, hi = _grid_box([fluid, wall], margin=2.0 * (2.0 * h))
    a = buffer_layers * dp
    bufs = []
    for k in range(arms):
        e = E[k]
        theta = math.atan2(e[1], e[0])
        centre = np.array([e[0] * (L - 0.5 * a), e[1] * (L - 0.5 * a), 0.0])
        if arms == 1:
            bufs.append(BufferSpec(origin=centre, rotation=frame_2d(theta + math.pi), extent=np.array([a, width, 0.0]),
                                   bc=BIDIR_PRESSURE, p_b=0.0, p_amp=p_amp, p_omega=2.0 * math.pi * p_freq))
        elif k == 0:
            bufs.append(BufferSpec(origin=centre, rotation=frame_2d(theta + math.pi), extent=np.array([a, width, 0.0]),
                                   bc=VELOCITY_INLET, umax=umax, half_width=0.0))
        else:
            bufs.append(BufferSpec(origin=centre, rotation=frame_2d(theta), extent=np.array([a, width, 0.0]),
                                   bc=PRESSURE_OUTLET, p_b=0.0))
    vel = np.zeros_like(fluid)
    if arms >= 2:
        loc = fluid @ E[0]
        tt = fluid @ N[0]
        inb = (loc > L - a) & (np.abs(tt) < half)
        vel[inb] = -umax * E[0][None, :]
    dt = min(0.25 * h / (c0 + umax), 0.125 * h * h / nu)
    n = fluid.shape[0]
    return Case(name="%s_k%d_w%.2f_n%d" % (name, arms, width, n), dim=2, lo=lo, hi=hi, dp=dp, h_over_dp=h_over_dp,
                rho0=rho0, c0=c0, nu=nu, dt=dt, fluid_pos=fluid, fluid_vel=vel, fluid_rho=np.full(n, rho0),
                wall_pos=wall, buffers=bufs, capacity=int(capacity_factor * n) + 1024, steps=500)


def bent_channel_case(*, dp=0.005, width=1.0, leg_in=5.0, leg_out=3.0, bend_radius=2.0, angle_in_deg=30.0,
                      angle_out_deg=-15.0, umax=1.5, c0=15.0, nu=1e-2, rho0=1000.0, h_over_dp=1.3,
                      buffer_layers=4, init_velocity="inlet_profile", speed=0.0, seed=BASE_SEED + 2,
                      name="bent", capacity_factor=1.4, steps=2000) -> Case:
    """2-D non-orthogonal bent channel: an inlet leg at ``angle_in_deg``, a circular bend of
    centre-line radius ``bend_radius``, an outlet leg at ``angle_out_deg``.

    The centre line starts at the origin.  Fluid = a global lattice (jittered) within
    ``width``/2 of the centre line between its two ends; walls = three lattice layers on both
    sides, open at the ends.  Inlet: a velocity buffer with the parabolic profile
    ``umax`` (1 - (Y'/R)^2), R = width/2, normal along the inlet leg; outlet: a pressure buffer
    (p = 0) with its normal along the outlet leg.  ``init_velocity``: "inlet_profile" (rest,
    the inlet buffer's particles on their profile), "rest", or "tangent" (every fluid particle
    moves at ``speed`` along the local centre-line direction).
    """
    rng = np.random.default_rng(seed)
    half = 0.5 * width
    t1, t2 = math.radians(angle_in_deg), math.radians(angle_out_deg)
    if not t2 < t1:
        raise ValueError("the bend turns clockwise: angle_out_deg must be below angle_in_deg")
    e1, n1 = np.array([math.cos(t1), math.sin(t1)]), np.array([-math.sin(t1), math.cos(t1)])
    e2, n2 = np.array([math.cos(t2), math.sin(t2)]), np.array([-math.sin(t2), math.cos(t2)])
    p0 = np.zeros(2)
    p1 = p0 + leg_in * e1
    centre = p1 - bend_radius * n1  # clockwise turn: centre on the right of the inlet leg
    p2 = centre + bend_radius * n2
    p3 = p2 + leg_out * e2
    wall_band = 3 * dp
    pts = np.stack([p0, p1, p2, p3, centre])
    span_lo = pts.min(axis=0) - half - wall_band - 2 * dp
    span_hi = pts.max(axis=0) + half + wall_band + 2 * dp
    ax = np.arange(math.floor(span_lo[0] / dp), math.ceil(span_hi[0] / dp) + 1) * dp + 0.5 * dp
    ay = np.arange(math.floor(span_lo[1] / dp), math.ceil(span_hi[1] / dp) + 1) * dp + 0.5 * dp
    X, Y = np.meshgrid(ax, ay, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel()], axis=1)
    # (along, across) coordinates of every lattice point against each piece of the centre line
    s_a = (P - p0) @ e1
    n_a = (P - p0) @ n1
    v = P - centre
    r = np.linalg.norm(v, axis=1)
    heading = np.arctan2(-v[:, 0], v[:, 1])  # tangent angle whose left normal points at P
    n_b = r - bend_radius
    s_c = (P - p2) @ e2
    n_c = (P - p2) @ n2
    on_a = (s_a >= 0.0) & (s_a < leg_in)
    on_b = (heading <= t1) & (heading >= t2) & (r > 0.0)
    on_c = (s_c >= 0.0) & (s_c <= leg_out)
    fluid_m = (on_a & (np.abs(n_a) < half)) | (on_b & (np.abs(n_b) < half)) | (on_c & (np.abs(n_c) < half))
    band = lambda nn: (np.abs(nn) >= half) & (np.abs(nn) < half + wall_band)  # noqa: E731
    wall_m = (((s_a >= -wall_band) & (s_a < leg_in) & band(n_a)) | (on_b & band(n_b))
              | ((s_c >= 0.0) & (s_c <= leg_out + wall_band) & band(n_c))) & ~fluid_m
    fluid = P[fluid_m] + rng.uniform(-0.01 * dp, 0.01 * dp, size=(int(fluid_m.sum()), 2))
    wall = P[wall_m]
    h = h_over_dp * dp
    lo, hi = _grid_box([fluid, wall], margin=2.0 * (2.0 * h))
    a = buffer_layers * dp
    bufs = [BufferSpec(origin=np.array([*(p0 + 0.5 * a * e1), 0.0]), rotation=frame_2d(t1),
                       extent=np.array([a, width, 0.0]), bc=VELOCITY_INLET, umax=umax, half_width=half),
            BufferSpec(origin=np.array([*(p3 - 0.5 * a * e2), 0.0]), rotation=frame_2d(t2),
                       extent=np.array([a, width, 0.0]), bc=PRESSURE_OUTLET, p_b=0.0)]
    vel = np.zeros_like(fluid)
    if init_velocity == "inlet_profile":
        sa = (fluid - p0) @ e1
        na = (fluid - p0) @ n1
        inb = (sa < a) & (np.abs(na) < half)
        vel[inb] = (umax * np.clip(1.0 - (na[inb] / half) ** 2, 0.0, None))[:, None] * e1[None, :]
    elif init_velocity == "tangent":
        fv = fluid - centre
        hd = np.arctan2(-fv[:, 0], fv[:, 1])
        tang = np.stack([np.cos(hd), np.sin(hd)], axis=1)
        tang[(fluid - p0) @ e1 < leg_in] = e1
        tang[(fluid - p2) @ e2 >= 0.0] = e2
        vel = speed * tang
    elif init_velocity != "rest":
        raise ValueError("init_velocity must be inlet_profile, rest or tangent")
    dt = min(0.25 * h / (c0 + umax), 0.125 * h * h / nu)
    n = fluid.shape[0]
    return Case(name="%s_dp%g_n%d" % (name, dp, n), dim=2, lo=lo, hi=hi, dp=dp, h_over_dp=h_over_dp, rho0=rho0,
                c0=c0, nu=nu, dt=dt, fluid_pos=fluid, fluid_vel=vel, fluid_rho=np.full(n, rho0), wall_pos=wall,
                buffers=bufs, capacity=int(capacity_factor * n) + 1024, steps=steps)


def config2(dp=0.005, **kw) -> Case:
    """2-D channel 1 m wide: inlet leg 5 m at +30 deg, bend of centre-line radius 2 m, outlet leg
    3 m at -15 deg; parabolic velocity inlet Umax = 1.5 (R = 0.5), pressure outlet p = 0, c0 = 15,
    nu = 1e-2; dp = 0.005 gives about 0.38 M fluid particles."""
    return bent_channel_case(dp=dp, name="cfg2_bent", **kw)


def sprinkler_case(*, dim=2, dp=0.002, r_nozzle=0.1, width=0.04, umax=1.0, omega=2.0, theta0=0.0,
                   axis=(0.0, 0.0, 1.0), domain_radius=0.3, ambient=False, c0=10.0, nu=1e-2, rho0=1000.0,
                   h_over_dp=1.3, buffer_layers=4, seed=BASE_SEED + 53, name="sprinkler") -> Case:
    """Rotating sprinkler (Sec. 5.3): a velocity-inlet nozzle that turns about a pivot.

    The pivot is the origin; the nozzle box (``buffer_layers`` dp along its normal, ``width``
    across) sits at distance ``r_nozzle`` along its own normal, a radial jet (the paper does
    not fix the nozzle's orientation; reading), at the angle ``theta0`` (2-D) or perpendicular
    to ``axis`` (3-D, square cross-section).  Its profile is U (1 - (Y'/R)^2), R = width/2 (the
    paper's 2500 (0.02^2 - y'^2) is U = 1, R = 0.02); it turns at ``omega`` rad/s about the
    z axis (2-D) or ``axis`` (3-D).  Fluid: the nozzle's lattice (its buffer particles, on the
    profile) and, with ``ambient``, fluid at rest on a lattice outside the disc (ball) the
    nozzle sweeps.  No walls; the grid covers ``domain_radius`` around the pivot.
    """
    rng = np.random.default_rng(seed)
    a = buffer_layers * dp
    half = 0.5 * width
    if dim == 2:
        e = np.array([math.cos(theta0), math.sin(theta0), 0.0])
        R = frame_2d(theta0)
    else:
        ax = np.asarray(axis, dtype=np.float64)
        ax = ax / np.linalg.norm(ax)
        k = int(np.argmin(np.abs(ax)))
        helper = np.zeros(3)
        helper[k] = 1.0
        e = helper - np.dot(helper, ax) * ax
        e /= np.linalg.norm(e)
        R = frame_3d(e, roll=float(rng.uniform(0.0, 2.0 * math.pi)))
    origin = r_nozzle * e
    # the nozzle's lattice in its own frame, rotated into place
    nx = int(round(a / dp))
    ny = int(round(width / dp))
    lx = (np.arange(nx) + 0.5) * dp - 0.5 * a
    ly = (np.arange(ny) + 0.5) * dp - half
    if dim == 2:
        X, Y = np.meshgrid(lx, ly, indexing="ij")
        loc = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    else:
        X, Y, Z = np.meshgrid(lx, ly, ly, indexing="ij")
        loc = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    glob = loc @ R + origin
    rr = loc[:, 1] ** 2 + (loc[:, 2] ** 2 if dim == 3 else 0.0)
    prof = umax * np.clip(1.0 - rr / half ** 2, 0.0, None)
    fluid = glob[:, :dim]
    vel = (prof[:, None] * e[None, :])[:, :dim]
    if ambient:
        reach = r_nozzle + 0.5 * a + 4 * dp
        ext = domain_radius - 4 * dp
        g1 = (np.arange(-int(ext / dp), int(ext / dp) + 1) + 0.5) * dp
        grids = np.meshgrid(*([g1] * dim), indexing="ij")
        P = np.stack([q.ravel() for q in grids], axis=1)
        r = np.linalg.norm(P, axis=1)
        P = P[(r > reach) & (r < ext)]
        fluid = np.concatenate([fluid, P])
        vel = np.concatenate([vel, np.zeros_like(P)])
    fluid = fluid + rng.uniform(-0.01 * dp, 0.01 * dp, size=fluid.shape)
    lo = np.zeros(3)
    hi = np.zeros(3)
    lo[:dim] = -domain_radius
    hi[:dim] = domain_radius
    if dim == 2:
        lo[2], hi[2] = 0.0, 1.0
    h = h_over_dp * dp
    dt = min(0.25 * h / (c0 + umax), 0.125 * h * h / nu)
    ext3 = np.array([a, width, width if dim == 3 else 0.0])
    buf = BufferSpec(origin=origin, rotation=R, extent=ext3, bc=VELOCITY_INLET, umax=umax, half_width=half,
                     pivot=np.zeros(3), axis=np.array([0.0, 0.0, 1.0]) if dim == 2 else np.asarray(axis, float),
                     omega=omega)
    n = fluid.shape[0]
    return Case(name="%s%dd_dp%g_n%d" % (name, dim, dp, n), dim=dim, lo=lo, hi=hi, dp=dp, h_over_dp=h_over_dp,
                rho0=rho0, c0=c0, nu=nu, dt=dt, fluid_pos=fluid, fluid_vel=vel, fluid_rho=np.full(n, rho0),
                wall_pos=np.zeros((0, dim)), buffers=[buf], capacity=4 * n + 4096, steps=500)


def config5(ndomains=64, n_lo=10_000, n_hi=500_000, seed=BASE_SEED + 5) -> List[Case]:
    """64 independent 2-D star channels: log-uniform sizes in [10 k, 500 k] particles, 1-6 arms,
    widths 0.2-1 m, seeded angles (the batched workload)."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(ndomains):
        n_t = int(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))
        arms = int(rng.integers(1, 7))
        width = float(rng.uniform(0.2, 1.0))
        out.append(star_case(seed=seed * 1000 + q, n_target=n_t, arms=arms, width=width, name="star%02d" % q))
    return out


def config1() -> Case:
    """10 x 1 m straight channel along x, dp 0.025: plug velocity inlet U = 1, pressure outlet p = 0."""
    return straight_channel_case(name="cfg1_channel_10x1_dp0.025", length=10.0, width=1.0, dp=0.025,
                                 angle_deg=0.0, inlet_bc=VELOCITY_INLET, outlet_bc=PRESSURE_OUTLET,
                                 umax=1.0, profile="plug", c0=10.0, nu=1e-2,
                                 seed=BASE_SEED + 1, init_velocity="inlet_only", steps=200)


def config3(length=5.09, dp=0.01, developed=True) -> Case:
    """3-D pipe R 0.5 along (1,1,1)/sqrt3, random roll, two bidirectional pressure buffers.

    Inlet pressure 50 sin(pi t) Pa (period 2 s), outlet 0 Pa, c0 = 3 m/s, nu = 1e-2.
    ``length`` 5.09 m gives about 4.0 M fluid particles at dp = 0.01.  With ``developed`` the
    fluid starts on the parabolic profile of the peak driving pressure (50 Pa over 5.09 m at
    eta = 10 Pa s: U = dP R^2 / (4 eta L) ~ 0.06 m/s on the axis), so particles cross both
    buffer faces from the first step; otherwise it starts at rest.
    """
    return pipe_case(name="cfg3_pipe_R0.5_L%.2f_dp%g" % (length, dp), length=length, radius=0.5,
                     dp=dp, axis=(1.0, 1.0, 1.0), inlet_bc=BIDIR_PRESSURE, outlet_bc=BIDIR_PRESSURE,
                     p_in=0.0, p_amp=50.0, p_omega=math.pi, p_out=0.0, c0=3.0, nu=1e-2,
                     umax=0.06 if developed else 0.0, init_velocity="profile" if developed else "rest",
                     umax_est=0.06, seed=BASE_SEED + 3, steps=1000)
