"""Pins of the time-varying buffer frames (Sec. 5.3, oracle/moving.py): the FP64 recurrence
against closed-form rotations, particles that turn with the buffer keep their local
coordinates, the FP32 contract against FP64, and generation along the turning normal."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import buffer as OB
from oracle import fp32 as OF
from oracle import moving as MV
from paper_2406_16786_gb300 import workloads as wl


def _closed(dim, axis, angle):
    if dim == 2:
        axis = (0.0, 0.0, 1.0)
    ax = np.asarray(axis, dtype=np.float64)
    return Rotation.from_rotvec(angle * ax / np.linalg.norm(ax)).as_matrix()


@pytest.mark.parametrize("dim,axis", [(2, None), (3, (0.2, 0.3, 1.0)), (3, (1.0, -2.0, 0.5))])
def test_recurrence_matches_closed_form_rotation(dim, axis):
    omega, dt, n = 2.7, 1e-3, 500
    rng = np.random.default_rng(1)
    R0 = wl.frame_3d(rng.normal(size=3), roll=0.4) if dim == 3 else wl.frame_2d(0.7)
    O0 = np.array([0.3, -0.2, 0.1 if dim == 3 else 0.0])
    C = np.array([0.05, 0.1, -0.02 if dim == 3 else 0.0])
    mf = MV.MovingFrame(dim, R0, O0, C, axis, omega, dt)
    M = np.array(mf.M)
    assert np.allclose(M @ M.T, np.eye(3), atol=1e-15) and abs(np.linalg.det(M) - 1.0) < 1e-14
    for _ in range(n):
        mf.advance()
    Q = _closed(dim, axis, omega * dt * n)
    assert np.abs(np.array(mf.Q) - Q).max() < 1e-12
    R, O = mf.frame()
    assert np.abs(R - R0 @ Q.T).max() < 1e-12
    assert np.abs(O - (C + Q @ (O0 - C))).max() < 1e-12
    # a point carried by the buffer keeps its local coordinates; the normal turns with it
    X0 = rng.normal(size=3) * 0.1
    if dim == 2:
        X0[2] = 0.0
    Xn = C + Q @ (X0 - C)
    assert np.abs(R @ (Xn - O) - R0 @ (X0 - O0)).max() < 1e-12
    assert np.abs(R[0] - Q @ R0[0]).max() < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_buffer_particles_turn_about_the_pivot(dim):
    # particles at rest: the buffer's particles only turn; after n steps they sit at
    # C + Rot(n omega dt)(r0 - C) and keep their local coordinates
    c = wl.sprinkler_case(dim=dim, dp=0.004 if dim == 3 else 0.002, umax=0.0, omega=40.0, axis=(0.2, 0.3, 1.0))
    sim = OB.OracleSim(c)
    sim.commit()
    b0 = sim.buffers[0]
    m0 = sim.label == b0.label
    assert m0.sum() == c.n
    ids0, p0 = sim.id[m0].copy(), sim.pos[m0].copy()
    loc0 = b0.local(p0)
    n = 60
    sim.step(n, physics=False)
    assert sim.injected.sum() == 0 and sim.n == c.n
    Q = _closed(dim, (0.2, 0.3, 1.0), 40.0 * c.dt * n)[:dim, :dim]
    order = np.argsort(sim.id)
    pos = sim.pos[order][np.searchsorted(sim.id[order], ids0)]
    assert np.abs(pos - p0 @ Q.T).max() < 1e-12
    assert np.abs(sim.buffers[0].local(pos) - loc0).max() < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_generation_follows_the_turning_normal(dim):
    # the buffer's particles move along its normal and turn with it: the same particles
    # cross the face, at the same steps, as with a fixed buffer (relative motion unchanged)
    kw = dict(dim=dim, dp=0.004 if dim == 3 else 0.002, umax=1.0, axis=(0.2, 0.3, 1.0))
    fixed = wl.sprinkler_case(omega=0.0, **kw)
    turning = wl.sprinkler_case(omega=25.0, **kw)
    for cc in (fixed, turning):
        cc.fluid_vel = cc.fluid_vel * 20.0
    a, b = OB.OracleSim(fixed), OB.OracleSim(turning)
    a.commit()
    b.commit()
    total = 0
    for _ in range(12):
        a.step(1, physics=False)
        b.step(1, physics=False)
        assert [(k, p) for k, p, _ in a.last_inj] == [(k, p) for k, p, _ in b.last_inj]
        total += len(b.last_inj)
    assert total > 0
    # the duplicates left the turning box through its current X' = a/2 face
    ids = np.array([new for _, _, new in b.last_inj])
    sel = np.isin(b.id, ids)
    Xp = b.buffers[0].local(b.pos[sel])
    assert np.all(Xp[:, 0] > 0.5 * b.buffers[0].extent[0] - 1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_fp32_rotation_tracks_fp64(dim):
    c = wl.sprinkler_case(dim=dim, dp=0.004 if dim == 3 else 0.002, umax=1.0, omega=30.0, axis=(0.2, 0.3, 1.0))
    c.fluid_vel = c.fluid_vel * 20.0
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    s32 = OF.Fp32Sim(c, cell, frac, c.fluid_vel.astype(np.float32), c.fluid_rho.astype(np.float32))
    pos = wl.decode_positions(cell, frac, c.lo, c.cs, c.grid_dims())
    s64 = OB.OracleSim(c, pos=pos, vel=c.fluid_vel.astype(np.float32).astype(np.float64))
    s32.commit()
    s64.commit()
    total = 0
    nsteps = 15
    for _ in range(nsteps):
        s32.step(1)
        s64.step(1, physics=False)
        assert s32.last_inj == s64.last_inj
        total += len(s32.last_inj)
    assert total > 0
    p32 = wl.decode_positions(s32.cell, np.pad(s32.f, ((0, 0), (0, 3 - dim))), c.lo, c.cs, c.grid_dims())
    order = np.argsort(s64.id)
    p64 = s64.pos[order][np.searchsorted(s64.id[order], s32.id)]
    # the FP32 rotation rounds the pivot offset D (|D| <= r_max) and uses fl32(M): a few
    # units of 6e-8 |D| per step
    r_max = np.linalg.norm(p64, axis=1).max()
    assert np.abs(p32[:, :dim] - p64).max() < nsteps * 4 * 6e-8 * r_max
