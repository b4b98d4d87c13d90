"""Dual-criteria time stepping (reading A26) on the GPU against the FP64 oracle: two advection
steps of four acoustic steps each on the 2-D and 3-D physics cases (every particle present on
both sides; multi-step tolerances), and a batch of dual-stepped domains equal, bit for bit, to
the same domains stepped alone."""
import numpy as np
import pytest

from oracle import buffer as OB
from paper_2406_16786_gb300 import workloads as wl
from tests import cases

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim", [2, 3])
def test_dual_time_stepping_matches_oracle(dim):
    from paper_2406_16786_gb300.domain import Domain

    c = cases.physics_case(dim)
    c.dt = 3.0 * c.dt
    c.dual_substeps = 4
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    vel32 = c.fluid_vel.astype(np.float32)
    rho32 = c.fluid_rho.astype(np.float32)
    dom = Domain.from_case(c)
    dom.write_particles(cell, frac, vel32, rho32)
    pos = wl.decode_positions(cell, frac, c.lo, c.cs, c.grid_dims())
    sim = OB.OracleSim(c, pos=pos, vel=vel32.astype(np.float64), rho=rho32.astype(np.float64))
    sim.commit()
    dom.step(2)
    sim.step(2, dual=4)
    g = dom.read()
    gpos = dom.positions()
    dom.close()
    gid = g["id"].astype(np.int64)
    common = np.intersect1d(gid, sim.id)
    assert common.size > 0.95 * sim.n
    gi = np.argsort(gid)[np.searchsorted(gid, common, sorter=np.argsort(gid))]
    oi = np.argsort(sim.id)[np.searchsorted(sim.id, common, sorter=np.argsort(sim.id))]
    dpos = np.linalg.norm(gpos[gi] - sim.pos[oi], axis=1)
    assert np.quantile(dpos, 0.99) < 1e-5 * c.cs
    rg, ro = g["rho"][gi].astype(np.float64), sim.rho[oi]
    assert np.linalg.norm(rg - ro) / np.linalg.norm(ro) < 3e-5
    vg, vo = g["vel"][gi].astype(np.float64), sim.vel[oi]
    assert np.linalg.norm(vg - vo) / np.linalg.norm(vo) < 3e-4


def test_dual_batch_equals_individual():
    from paper_2406_16786_gb300.domain import Batch, Domain

    cs = [wl.star_case(seed=900 + q, n_target=nt, arms=k, width=w, name="t%d" % q)
          for q, (nt, k, w) in enumerate([(4000, 1, 0.3), (12000, 3, 0.5), (2500, 2, 0.25)])]
    for c in cs:
        c.dt = 2.0 * c.dt
        c.dual_substeps = 3
    alone = [Domain.from_case(c) for c in cs]
    for d in alone:
        d.step(4)
    together = [Domain.from_case(c) for c in cs]
    b = Batch(together)
    b.use_graph(True)
    b.step(4)
    b.sync()
    for a, t in zip(alone, together):
        ra, rt = a.read(), t.read()
        for key in ra:
            assert np.array_equal(ra[key], rt[key]), key
    b.close()
