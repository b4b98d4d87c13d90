"""Strict inequalities on the GPU (reading A3): a buffer particle exactly at X' = a/2, in the
FP32 decision contract, is neither injected (inlet, Algorithm 1) nor deleted (outlet,
Algorithm 2); one FP32 ulp further it is.  The positions are found with the FP32-mode oracle's
local coordinates; the GPU's decisions must equal the oracle's."""
import numpy as np
import pytest

from oracle import buffer as OB
from oracle import fp32 as OF
from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
KIN = _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER
F32 = np.float32


def _at(g32, b32, y_cell, y_f, target):
    """(cell coords, offsets) of a point of the lane (y_cell, y_f) whose FP32 X' is target."""
    t = float(b32.cO[0]) * g32.cs + float(b32.fO[0]) + float(target)  # near the wanted x
    cx = int(np.floor(t / g32.cs))
    f = F32(t - cx * g32.cs)
    for _ in range(64):
        c = np.array([[cx, y_cell, 0]])
        X = OF.local32(g32, b32, c, np.array([[f, y_f]], dtype=F32))[0, 0]
        if X == target:
            return cx, f
        f = np.nextafter(f, F32(np.inf) if X < target else F32(-np.inf), dtype=F32)
    raise AssertionError("no FP32 offset reaches X' = %r" % target)


def test_ties_are_not_crossings():
    from paper_2406_16786_gb300.domain import Domain

    c = wl.straight_channel_case(length=0.6, width=0.2, dp=0.01, angle_deg=0.0, inlet_bc=wl.VELOCITY_INLET,
                                 outlet_bc=wl.PRESSURE_OUTLET, umax=1.0, c0=10.0, nu=1e-2, seed=81,
                                 init_velocity="rest")
    g32 = OF.Grid32(c.dim, c.lo, c.hi, c.dp, c.h_over_dp)
    bufs = [OF.Buffer32(OB.Buffer(k, s, c.dim), g32) for k, s in enumerate(c.buffers)]
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    cc = g32.coords(cell)
    labels = np.zeros(c.n, np.int64)
    labels[OF.in_box32(OF.local32(g32, bufs[0], cc, frac), bufs[0], 2)] = 1
    # four extra particles on the lane at mid-channel: inlet tie / tie + 1 ulp, outlet the same
    y = 0.0017 - c.lo[1]  # 1.7 mm off the channel axis
    y_cell = int(np.floor(y / g32.cs))
    y_f = F32(y - y_cell * g32.cs)
    extra_c, extra_f, extra_l = [], [], []
    for k, lab in ((0, 1), (1, 0)):
        b = bufs[k]
        for target in (b.ha, np.nextafter(b.ha, F32(np.inf), dtype=F32)):
            cx, f = _at(g32, b, y_cell, y_f, target)
            extra_c.append((0 * 0 + y_cell) * g32.dims[0] + cx)
            extra_f.append((f, y_f))
            extra_l.append(lab)
    cell = np.concatenate([cell, np.array(extra_c, np.int32)])
    frac = np.concatenate([frac, np.array(extra_f, dtype=F32)])
    labels = np.concatenate([labels, np.array(extra_l)])
    n = cell.shape[0]
    vel = np.zeros((n, 2), F32)
    rho = np.full(n, c.rho0, F32)
    ids = np.arange(n, dtype=np.uint32)
    dom = Domain(c.dim, c.lo, c.hi, c.dp, c.h_over_dp, c.rho0, c.c0, c.nu, c.dt, c.capacity)
    dom.set_walls(c.wall_pos)
    for s in c.buffers:
        dom.add_buffer(s)
    dom.write_particles(cell, frac, vel, rho, ids=ids, labels=labels.astype(np.uint8), next_id=n)
    sim = OF.Fp32Sim(c, cell, frac, vel, rho, ids=ids, labels=labels, next_id=n)
    sim.commit()
    dom.step(1, KIN)
    sim.step(1)
    inj, dels = dom.last_decisions()
    assert inj == sim.last_inj
    assert sorted(dels) == sorted(sim.last_del)
    tie_in, plus_in, tie_out, plus_out = (c.n + q for q in range(4))
    assert [p for _, p, _ in inj] == [plus_in]
    assert [p for _, p in dels] == [plus_out]
    assert tie_in not in [p for _, p, _ in inj] and tie_out not in [p for _, p in dels]
    dom.close()


def test_bidirectional_ties_at_both_faces():
    """Algorithm 3: a buffer particle that moves to X' = a/2 exactly is not injected, one that
    moves to X' = -a/2 exactly is not deleted; one FP32 ulp beyond either face they are.  The
    particles start inside the box (so the relabelling after the set-up rebuild keeps them in
    the buffer) and reach the faces in one kinematic step with an exact FP32 move."""
    from paper_2406_16786_gb300.domain import Domain

    c = wl.straight_channel_case(length=0.6, width=0.2, dp=0.01, angle_deg=0.0, inlet_bc=wl.BIDIR_PRESSURE,
                                 outlet_bc=wl.PRESSURE_OUTLET, umax=0.0, p_in=1.0, c0=10.0, nu=1e-2, seed=82,
                                 init_velocity="rest")
    g32 = OF.Grid32(c.dim, c.lo, c.hi, c.dp, c.h_over_dp)
    b = OF.Buffer32(OB.Buffer(0, c.buffers[0], c.dim), g32)
    dt32 = F32(c.dt)
    delta = F32(2.0 ** -14)  # the move, 0.006 dp, exact in FP32
    v = F32(delta / dt32)
    for _ in range(64):  # a speed whose FP32 product with dt32 is exactly delta
        m = F32(v * dt32)
        if m == delta:
            break
        v = np.nextafter(v, F32(np.inf) if m < delta else F32(-np.inf), dtype=F32)
    assert F32(v * dt32) == delta
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    y = -0.0023 - c.lo[1]
    y_cell = int(np.floor(y / g32.cs))
    y_f = F32(y - y_cell * g32.cs)
    targets = (b.ha, np.nextafter(b.ha, F32(np.inf), dtype=F32), -b.ha, np.nextafter(-b.ha, F32(-np.inf), dtype=F32))
    ec, ef, ev = [], [], []
    for target in targets:
        cx, f = _at(g32, b, y_cell, y_f, F32(target))
        sgn = F32(1.0) if target > 0 else F32(-1.0)
        f0 = F32(f - sgn * delta)  # one move before the face
        assert F32(f0 + sgn * delta) == f and F32(0.0) <= f0 < g32.cs32
        ec.append(y_cell * g32.dims[0] + cx)
        ef.append((f0, y_f))
        ev.append((sgn * v, F32(0.0)))
    cell = np.concatenate([cell, np.array(ec, np.int32)])
    frac = np.concatenate([frac, np.array(ef, dtype=F32)])
    n = cell.shape[0]
    vel = np.zeros((n, 2), F32)
    vel[c.n:] = np.array(ev, dtype=F32)
    rho = np.full(n, c.rho0, F32)
    dom = Domain(c.dim, c.lo, c.hi, c.dp, c.h_over_dp, c.rho0, c.c0, c.nu, c.dt, c.capacity)
    dom.set_walls(c.wall_pos)
    for s in c.buffers:
        dom.add_buffer(s)
    dom.write_particles(cell, frac, vel, rho)
    sim = OF.Fp32Sim(c, cell, frac, vel, rho)
    sim.commit()
    assert (sim.label[np.isin(sim.id, np.arange(c.n, n))] == 1).all()  # in the buffer
    dom.step(1, KIN)
    sim.step(1)
    inj, dels = dom.last_decisions()
    assert inj == sim.last_inj
    assert sorted(dels) == sorted(sim.last_del)
    assert [p for _, p, _ in inj] == [c.n + 1]
    assert [p for _, p in dels] == [c.n + 3]
    dom.close()
