"""Transport velocity (Eq. (10)) on the GPU against the FP64 oracle: three full steps of a
small 2-D channel and a 3-D pipe from a perturbed state, lambda = 7.5; v_max and p_max carry
over from step to step.  Positions, densities and velocities of every particle present on both
sides agree to the multi-step tolerances; the transport shift itself is checked to be active
(its size against lambda = 0)."""
import numpy as np
import pytest

from oracle import buffer as OB
from paper_2406_16786_gb300 import workloads as wl
from tests import cases

pytestmark = pytest.mark.gpu


def _run(c, nsteps):
    from paper_2406_16786_gb300.domain import Domain

    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    vel32 = c.fluid_vel.astype(np.float32)
    rho32 = c.fluid_rho.astype(np.float32)
    dom = Domain.from_case(c)
    dom.write_particles(cell, frac, vel32, rho32)
    pos = wl.decode_positions(cell, frac, c.lo, c.cs, c.grid_dims())
    sim = OB.OracleSim(c, pos=pos, vel=vel32.astype(np.float64), rho=rho32.astype(np.float64))
    sim.commit()
    dom.step(nsteps)
    sim.step(nsteps)
    g = dom.read()
    gpos = dom.positions()
    dom.close()
    return g, gpos, sim


def _compare(g, gpos, sim, c, pos_tol):
    gid = g["id"].astype(np.int64)
    common = np.intersect1d(gid, sim.id)
    assert common.size > 0.95 * sim.n
    gi = np.searchsorted(gid, common, sorter=np.argsort(gid))
    gi = np.argsort(gid)[gi]
    oi = np.argsort(sim.id)[np.searchsorted(sim.id, common, sorter=np.argsort(sim.id))]
    dpos = np.linalg.norm(gpos[gi] - sim.pos[oi], axis=1)
    assert np.quantile(dpos, 0.99) < pos_tol
    rg, ro = g["rho"][gi].astype(np.float64), sim.rho[oi]
    assert np.linalg.norm(rg - ro) / np.linalg.norm(ro) < 3e-5
    vg, vo = g["vel"][gi].astype(np.float64), sim.vel[oi]
    assert np.linalg.norm(vg - vo) / np.linalg.norm(vo) < 3e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_transport_velocity_three_steps_match_oracle(dim):
    c = cases.physics_case(dim)
    c.fluid_vel, c.fluid_rho = wl.perturbed_state(c, dv=0.3, drho=2e-3, seed=5)
    c.tvf_lambda = 7.5
    g, gpos, sim = _run(c, 3)
    _compare(g, gpos, sim, c, 1e-5 * c.cs)
    # the shift is active: against the same steps without it the positions move measurably
    c0 = cases.physics_case(dim)
    c0.fluid_vel, c0.fluid_rho = c.fluid_vel, c.fluid_rho
    sim0 = OB.OracleSim(c0)
    sim0.commit()
    sim0.step(3)
    common = np.intersect1d(sim.id, sim0.id)
    a = sim.pos[np.argsort(sim.id)][np.searchsorted(np.sort(sim.id), common)]
    b = sim0.pos[np.argsort(sim0.id)][np.searchsorted(np.sort(sim0.id), common)]
    assert np.abs(a - b).max() > 30 * 1e-5 * c.cs
