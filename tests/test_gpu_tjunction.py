"""T-junction (velocity inlet + two pressure outlets, arbitrary rotation): bit-exact buffer
update against the FP32-mode oracle, and the full-domain decision variant equal to the
restricted one, on a coarse (dp 0.02, ~0.42 M particles) version of the 16 M workload."""
import numpy as np
import pytest

from oracle import fp32 as OF
from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
KIN = _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.int32)


def test_tjunction_kinematic_bit_exact_and_full_check():
    from paper_2406_16786_gb300.domain import Domain

    c = wl.tjunction_case(dp=0.02)
    c.fluid_vel = c.fluid_vel * 20.0  # 0.6 dp per step on the axis: crossings at every buffer
    cell, frac = wl.encode_positions(c.fluid_pos, c.lo, c.cs, c.grid_dims())
    vel = c.fluid_vel.astype(np.float32)
    rho = c.fluid_rho.astype(np.float32)
    a = Domain.from_case(c)
    b = Domain.from_case(c)
    a.use_graph(True)
    sim = OF.Fp32Sim(c, cell, frac, vel, rho)
    sim.commit()
    total = 0
    for _ in range(4):
        a.step(1, KIN)
        b.step(1, KIN | _ffi.PHASE_FULL_CHECK)
        sim.step(1)
        ia, da = a.last_decisions()
        ib, db = b.last_decisions()
        assert ia == sim.last_inj and ib == sim.last_inj
        assert sorted(da) == sorted(sim.last_del) == sorted(db)
        total += len(ia) + len(da)
        g = a.read()
        assert np.array_equal(g["id"].astype(np.int64), sim.id)
        assert np.array_equal(g["cell"].astype(np.int64), sim.cell)
        assert np.array_equal(_bits(g["frac"]), _bits(sim.f))
        assert np.array_equal(g["label"].astype(np.int64), sim.label)
    assert total > 0
    for k in range(3):
        assert a.counters(k)["injected"] == sim.injected[k]
        assert a.counters(k)["deleted"] == sim.deleted[k]
    a.close()
    b.close()
