"""Pins of the oracle's buffer method (Algorithms 1-3) in FP64 and FP32 decision mode."""
import math

import numpy as np
import pytest

from oracle import buffer as OB
from oracle import fp32 as OF
from paper_2406_16786_gb300 import workloads as wl


def _spec(bc, normal, roll=0.3, origin=(0.5, 0.6, 0.7), extent=(0.04, 0.3, 0.2), **kw):
    R = wl.frame_3d(normal, roll)
    return wl.BufferSpec(origin=np.array(origin, float), rotation=R, extent=np.array(extent, float), bc=bc, **kw)


def _expected(bc, Xp, label, ext, cs):
    """Algorithms 1-3 on known local coordinates (the particles were placed at Xp)."""
    ha = 0.5 * ext[0]
    inj, dels = set(), set()
    for i, (x, y, z) in enumerate(Xp):
        mine = label[i] == 1
        if bc in OB.INFLOW and mine and x > ha:
            inj.add(i)
        if bc in OB.OUTFLOW and abs(x) < ha + cs and abs(y) < 0.5 * ext[1] + cs and abs(z) < 0.5 * ext[2] + cs and x > ha:
            dels.add(i)
        if bc in OB.BIDIR and mine and x > ha:
            inj.add(i)
        if bc in OB.BIDIR and mine and x < -ha:
            dels.add(i)
    return inj, dels


@pytest.mark.parametrize("bc", range(6))
def test_decisions_on_particles_placed_in_the_local_frame(bc):
    rng = np.random.default_rng(100 + bc)
    normal = rng.standard_normal(3)
    spec = _spec(bc, normal, roll=rng.uniform(0, 6.28))
    ext = spec.extent
    cs = 0.026
    eps = 1e-4
    ha, hb, hc = 0.5 * ext
    xs = [-(ha + cs) - eps, -ha - eps, -ha + eps, 0.0, ha - eps, ha + eps, ha + cs - eps, ha + cs + eps]
    ys = [0.0, hb - eps, hb + eps, hb + cs - eps, -(hb + cs) - eps]
    zs = [0.0, -(hc + cs) + eps, hc + cs + eps]
    Xp = np.array([[x, y, z] for x in xs for y in ys for z in zs])
    label = rng.integers(0, 2, Xp.shape[0])
    pos = spec.origin[None, :] + Xp @ spec.rotation  # X = O' + R^T X'
    b = OB.Buffer(0, spec, 3)
    inj, dels = OB.decide([b], pos, label, cs)
    e_inj, e_del = _expected(bc, Xp, label, ext, cs)
    assert {i for _, i in inj} == e_inj
    assert {i for _, i in dels} == e_del
    assert len(e_inj) + len(e_del) > 0


def _channel(angle=0.0, inlet=wl.VELOCITY_INLET, outlet=wl.PRESSURE_OUTLET, length=1.0, width=0.2,
             dp=0.02, seed=5):
    return wl.straight_channel_case(length=length, width=width, dp=dp, angle_deg=angle, inlet_bc=inlet,
                                    outlet_bc=outlet, umax=1.0, c0=10.0, nu=1e-2, seed=seed,
                                    init_velocity="bc", profile="plug")


def test_inlet_injection_schedule_and_count_invariant():
    case = _channel()
    sim = OB.OracleSim(case)
    sim.commit()
    lanes = int(round(case.buffers[0].extent[1] / case.dp))
    assert int(np.sum(sim.label == 1)) == 4 * lanes  # a = 4 dp, one particle per layer per lane
    T = 37
    sim.step(T, physics=False)
    # buffer particles move exactly at U: each lane crosses X' = a/2 once per dp/U
    crossings = 1.0 * T * case.dt / case.dp
    assert lanes * (math.floor(crossings) - 1) <= sim.injected[0] <= lanes * (math.ceil(crossings) + 1)
    assert sim.n == sim.n0 + sim.injected.sum() - sim.deleted.sum() - sim.escaped
    assert sim.escaped == 0
    assert sim.deleted[1] > 0  # the outlet deleted the particles that crossed it
    # inflow buffer particles never leave their box (recycled each time they cross)
    b0 = sim.buffers[0]
    Xp = b0.local(sim.pos[sim.label == 1])
    assert np.all(np.abs(Xp[:, 0]) < 0.5 * b0.extent[0])


def test_recycled_parent_moves_by_minus_a_u_and_duplicate_keeps_state():
    case = _channel(angle=33.0, inlet=wl.PRESSURE_INLET)
    case.buffers[0].p_b = 7.0
    sim = OB.OracleSim(case)
    sim.commit()
    before = {int(i): (p.copy(), v.copy()) for i, p, v in zip(sim.id, sim.pos, sim.vel)}
    for _ in range(40):
        sim.step(1, physics=False)
        if sim.last_inj:
            break
    assert sim.last_inj
    ids = list(sim.id)
    b = sim.buffers[0]
    for k, pid, nid in sim.last_inj:
        p = sim.pos[ids.index(pid)]
        d = sim.pos[ids.index(nid)]
        assert np.allclose(d - p, b.extent[0] * b.u, atol=1e-12)
        assert sim.label[ids.index(nid)] == 0
        assert sim.rho[ids.index(pid)] == pytest.approx(case.rho0 + 7.0 / case.c0 ** 2, rel=1e-15)
        assert np.array_equal(sim.vel[ids.index(nid)], before[pid][1])
    new_ids = [nid for _, _, nid in sim.last_inj]
    assert new_ids == list(range(new_ids[0], new_ids[0] + len(new_ids)))


def test_rotated_channel_gives_identical_decision_counts():
    a = OB.OracleSim(_channel(angle=0.0, outlet=wl.BIDIR_PRESSURE))
    b = OB.OracleSim(_channel(angle=30.0, outlet=wl.BIDIR_PRESSURE))
    a.commit()
    b.commit()
    # bidirectional outlet: reverse half of the flow so both deletion and injection happen
    for sim in (a, b):
        e = sim.buffers[0].R[0]
        y = (sim.pos - sim.buffers[0].origin[None, :2]) @ sim.buffers[0].R[1]
        sim.vel = np.where((y > 0)[:, None], 1.0, -1.0) * e[None, :]
    for _ in range(25):
        a.step(1, physics=False)
        b.step(1, physics=False)
        assert (len(a.last_inj), len(a.last_del)) == (len(b.last_inj), len(b.last_del))
    assert a.injected.sum() > 0 and a.deleted.sum() > 0


def test_relabel_marks_exactly_the_in_box_particles():
    case = wl.pipe_case(length=0.5, radius=0.1, dp=0.02, seed=3)
    sim = OB.OracleSim(case)
    sim.commit()
    sim.vel = wl.shear_velocity(case, u0=2.0)[sim.id]
    sim.step(3, physics=False)
    for b in sim.buffers:
        inside = (np.abs(b.local(sim.pos)) < 0.5 * b.extent[None, :]).all(axis=1)
        assert np.array_equal(sim.label == b.label, inside)


def _encoded(case):
    g = OF.Grid32(case.dim, case.lo, case.hi, case.dp, case.h_over_dp)
    cell, frac = wl.encode_positions(case.fluid_pos, case.lo, case.cs, g.dims)
    return g, cell, frac


@pytest.mark.parametrize("dim", [2, 3])
def test_fp32_local_coordinates_match_fp64(dim):
    case = _channel(angle=21.0) if dim == 2 else wl.pipe_case(length=0.4, radius=0.1, dp=0.02)
    g, cell, frac = _encoded(case)
    c = g.coords(cell)
    for spec in case.buffers:
        b = OB.Buffer(0, spec, dim)
        X32 = OF.local32(g, OF.Buffer32(b, g), c, frac)
        X64 = b.local(wl.decode_positions(cell, frac, case.lo, case.cs, g.dims))
        assert np.max(np.abs(X32 - X64)) < 4e-7 * (np.max(np.abs(X64)) + g.cs)


def test_fp32_move_keeps_the_position_and_normalises():
    case = _channel(angle=10.0)
    g, cell, frac = _encoded(case)
    c = g.coords(cell)
    rng = np.random.default_rng(4)
    delta = rng.uniform(-2.4 * g.cs, 2.4 * g.cs, frac.shape).astype(np.float32)
    before = wl.decode_positions(cell, frac, case.lo, case.cs, g.dims)
    f = frac.copy()
    OF.move32(g, c, f, delta)
    after = wl.decode_positions(g.linear(c), f, case.lo, case.cs, g.dims)
    assert np.all((f >= 0) & (f < g.cs32))
    assert np.max(np.abs(after - before - delta.astype(np.float64))) < 1e-6 * g.cs


@pytest.mark.parametrize("outlet", [wl.PRESSURE_OUTLET, wl.BIDIR_VELOCITY])
def test_fp32_mode_agrees_with_fp64_mode(outlet):
    case = _channel(angle=-15.0, inlet=wl.BIDIR_PRESSURE, outlet=outlet)
    case.fluid_vel = wl.shear_velocity(case, u0=15.0)  # about 0.5 dp per step
    g, cell, frac = _encoded(case)
    s32 = OF.Fp32Sim(case, cell, frac, case.fluid_vel, case.fluid_rho)
    s64 = OB.OracleSim(case, pos=wl.decode_positions(cell, frac, case.lo, case.cs, g.dims),
                       vel=case.fluid_vel.astype(np.float32).astype(np.float64))
    s32.commit()
    s64.commit()
    assert np.array_equal(s32.id, s64.id) and np.array_equal(s32.label, s64.label)
    total = 0
    for _ in range(12):
        s32.step(1)
        s64.step(1, physics=False)
        assert sorted(s32.last_inj) == sorted(s64.last_inj)
        assert sorted(s32.last_del) == sorted(s64.last_del)
        total += len(s32.last_inj) + len(s32.last_del)
    assert total > 0
    assert s32.n == s32.n0 + s32.injected.sum() - s32.deleted.sum() - s32.escaped
    assert np.array_equal(s32.id, s64.id)


def test_fp32_threshold_tie_is_not_a_crossing():
    case = _channel(angle=0.0)
    g = OF.Grid32(case.dim, case.lo, case.hi, case.dp, case.h_over_dp)
    b = OF.Buffer32(OB.Buffer(0, case.buffers[0], 2), g)
    m = int(math.floor((float(b.fO[0]) + float(b.ha)) / float(g.cs32)))
    c = np.array([[b.cO[0] + m, b.cO[1], 0]])
    # search an in-cell offset f whose local X' is exactly a/2 in FP32
    f0 = np.float32(float(b.fO[0]) + float(b.ha) - m * float(g.cs32))
    hit = None
    for k in range(-64, 65):
        f = np.array([[np.float32(f0 + np.float32(k) * np.spacing(f0)), b.fO[1]]], dtype=np.float32)
        if 0 <= f[0, 0] < g.cs32 and OF.local32(g, b, c, f)[0, 0] == b.ha:
            hit = f
            break
    assert hit is not None
    lab = np.array([1])
    assert OF.decide32(g, [b], c, hit, lab) == ([], [])
    up = hit.copy()
    crossed = False
    for _ in range(64):
        up[0, 0] = np.nextafter(up[0, 0], np.float32(1))
        X = OF.local32(g, b, c, up)[0, 0]
        inj, _ = OF.decide32(g, [b], c, up, lab)
        assert (inj == [(0, 0)]) == bool(X > b.ha)
        if X > b.ha:
            crossed = True
            break
    assert crossed


def test_boundary_velocity_states_after_a_step():
    # After a full FP64 step of a small 3-D pipe along an oblique axis d:
    #  - velocity-inlet particles carry the pipe profile of Eqs. (23)-(26) with reading A15,
    #    v = U (1 - rho^2 / R^2) d, rho their distance from the pipe's axis (a closed form from
    #    the geometry; the drift and the recycling move them along d, which keeps rho);
    #  - pressure-outlet particles carry the projection of Eq. (19), v parallel to u = d.
    axis = np.array([1.0, -2.0, 0.5])
    d = axis / np.linalg.norm(axis)
    U, R = 0.5, 0.08
    case = wl.pipe_case(length=0.3, radius=R, dp=0.02, axis=tuple(axis), inlet_bc=wl.VELOCITY_INLET,
                        outlet_bc=wl.PRESSURE_OUTLET, umax=U, init_velocity="profile", c0=5.0, nu=1e-3,
                        umax_est=U, seed=9)
    sim = OB.OracleSim(case)
    sim.commit()
    b_in, b_out = sim.buffers
    was_in = set(sim.id[sim.label == b_in.label].tolist())
    was_out = set(sim.id[sim.label == b_out.label].tolist())
    assert was_in and was_out
    sim.step(1)
    ids = sim.id.tolist()
    rows_in = [ids.index(i) for i in was_in]
    x = sim.pos[rows_in]
    rho2 = np.sum(x * x, axis=1) - (x @ d) ** 2  # the pipe's axis passes through the origin
    want = U * np.clip(1.0 - rho2 / R ** 2, 0.0, None)[:, None] * d[None, :]
    assert np.allclose(sim.vel[rows_in], want, atol=1e-12)
    assert np.allclose(b_in.u, d) and np.allclose(b_out.u, d)
    rows_out = [ids.index(i) for i in was_out if i in set(ids)]
    v = sim.vel[rows_out]
    assert np.abs(np.cross(v, d)).max() < 1e-12 * max(1.0, np.abs(v).max())
    assert np.abs(v @ d).max() > 0  # the outlet particles do move


def test_plug_inlet_flux_is_u_times_width():
    # The volume flux through a buffer (the Q that drives the Windkessel outlet of Eq. (31)) is
    # sum over its particles of (v . u) dp^d / a.  A plug velocity inlet holds one particle per
    # layer per lane and imposes v = U u, so Q = U x (lanes dp) = U x width exactly.
    case = _channel(angle=21.0)
    sim = OB.OracleSim(case)
    sim.commit()
    sim.step(1)
    assert sim.flux[0] == pytest.approx(1.0 * 0.2, rel=1e-12)
