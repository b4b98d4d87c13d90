"""One full GPU step (density, force, BC, drift, buffer update, rebuild) vs the FP64 oracle.

Both sides start from the same seeded FP32 state (the oracle reads it in FP64).  Particles are
matched by id.  Tolerances (relative L2 over all particles unless stated):
  density 1e-5;  pressure |dp| / (rho0 c0^2) <= 1e-6 per particle;  velocity 1e-5;
  position 1e-6 cs per particle;  acceleration (from the velocity change) 2e-4.
The id sets (the injections and deletions of the step) must be identical.
"""
import numpy as np
import pytest

from oracle import buffer as OB
from paper_2406_16786_gb300 import workloads as wl
from tests import cases

pytestmark = pytest.mark.gpu


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("dim", [2, 3])
def test_one_step_matches_fp64_oracle(dim):
    from paper_2406_16786_gb300.domain import Domain

    case = cases.physics_case(dim)
    cell, frac = cases.encode(case)
    vel32 = case.fluid_vel.astype(np.float32)
    rho32 = case.fluid_rho.astype(np.float32)
    dom = Domain.from_case(case)
    pos0 = wl.decode_positions(cell, frac, case.lo, case.cs, case.grid_dims())
    ora = OB.OracleSim(case, pos=pos0, vel=vel32.astype(np.float64), rho=rho32.astype(np.float64))
    ora.commit()
    g0 = dom.read()
    assert np.array_equal(g0["id"].astype(np.int64), ora.id)
    assert np.array_equal(g0["label"].astype(np.int64), ora.label)
    v_before = {int(i): v for i, v in zip(ora.id, ora.vel)}
    dom.step(1)
    ora.step(1)
    g = dom.read()
    gp = dom.positions()
    assert sorted(g["id"].tolist()) == sorted(ora.id.tolist())
    o = np.argsort(g["id"])
    q = np.argsort(ora.id)
    rho_g, rho_o = g["rho"][o].astype(np.float64), ora.rho[q]
    assert _rel_l2(rho_g, rho_o) < 1e-5
    P = ora.P
    assert np.max(np.abs(rho_g - rho_o)) * P.c0 ** 2 / (P.rho0 * P.c0 ** 2) < 1e-6
    v_g, v_o = g["vel"][o].astype(np.float64), ora.vel[q]
    assert _rel_l2(v_g, v_o) < 1e-5
    assert np.max(np.abs(gp[o] - ora.pos[q])) < 1e-6 * case.cs
    # acceleration of the particles that existed before the step and carry no boundary velocity
    ids = ora.id[q]
    keep = np.array([(int(i) in v_before) for i in ids]) & (ora.label[q] == 0)
    dv_o = np.stack([v_o[m] - v_before[int(i)] for m, i in enumerate(ids) if keep[m]])
    dv_g = np.stack([v_g[m] - v_before[int(i)] for m, i in enumerate(ids) if keep[m]])
    assert _rel_l2(dv_g, dv_o) < 2e-4
    inj, dels = dom.last_decisions()
    assert [(k, p) for k, p, _ in inj] == [(k, p) for k, p, _ in ora.last_inj]
    assert sorted(dels) == sorted(ora.last_del)
    dom.close()
