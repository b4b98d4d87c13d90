"""RCR Windkessel outlet (Eq. (31)) on the GPU against the FP64 oracle: a 25 deg channel with
a plug velocity inlet and a Windkessel pressure outlet, the whole fluid moving from the first
step so that the outlet's flux is nonzero at once.  Over 40 physics steps the boundary
pressure p_b(t_n) and the flux it was computed from follow the oracle's (each side integrates
Eq. (31) from its own flux; FP32 fields vs FP64: agreement to 1e-4 of the pressure scale)."""
import dataclasses

import numpy as np
import pytest

from oracle import buffer as OB
from paper_2406_16786_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _case():
    c = wl.straight_channel_case(length=0.6, width=0.2, dp=0.01, angle_deg=25.0, inlet_bc=wl.VELOCITY_INLET,
                                 outlet_bc=wl.PRESSURE_OUTLET, umax=1.0, c0=10.0, nu=1e-2, seed=41,
                                 init_velocity="bc", profile="plug")
    # Q ~ U w = 0.2 m^2/s; R_d C = 0.02 s (~70 steps), P_d -> Q R_d = 400 Pa, R_p Q = 40 Pa
    c.buffers[1] = dataclasses.replace(c.buffers[1], wk_rp=200.0, wk_c=1e-5, wk_rd=2000.0, wk_pd0=5.0)
    return c


def test_windkessel_pressure_follows_oracle():
    from paper_2406_16786_gb300.domain import Domain

    c = _case()
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    vel32 = c.fluid_vel.astype(np.float32)
    rho32 = c.fluid_rho.astype(np.float32)
    dom = Domain(c.dim, c.lo, c.hi, c.dp, c.h_over_dp, c.rho0, c.c0, c.nu, c.dt, c.capacity)
    dom.set_walls(c.wall_pos)
    for b in c.buffers:
        dom.add_buffer(b)
    dom.write_particles(cell, frac, vel32, rho32)
    pos = wl.decode_positions(cell, frac, c.lo, c.cs, c.grid_dims())
    sim = OB.OracleSim(c, pos=pos, vel=vel32.astype(np.float64), rho=rho32.astype(np.float64))
    sim.commit()
    pg, qg, po, qo = [], [], [], []
    for _ in range(40):
        q_prev_oracle = float(sim.flux[1])
        dom.step(1)
        sim.step(1)
        pb, pd, q = dom.boundary_pressure(1)
        pg.append(pb)
        qg.append(q)
        po.append(sim.buffers[1].pb_now)
        qo.append(q_prev_oracle)
    pg, qg, po, qo = map(np.array, (pg, qg, po, qo))
    assert pg[0] == pytest.approx(5.0)  # P_d(0) + R_p * 0
    assert np.all(np.diff(pg[5:]) > 0)  # filling: P_d rises toward Q R_d
    scale = np.abs(po).max()
    assert np.abs(pg - po).max() < 1e-4 * scale
    assert np.abs(qg - qo).max() < 1e-4 * np.abs(qo).max()
    # the inlet keeps its prescribed velocity BC: its pressure is p_i (no Windkessel)
    assert dom.boundary_pressure(0)[1] == 0.0
    dom.close()
