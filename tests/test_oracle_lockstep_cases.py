"""The lockstep cases are meaningful: the FP32 oracle sees injections and deletions in each."""
import numpy as np
import pytest

from oracle import fp32 as OF
from tests import cases


@pytest.mark.parametrize("name,case", cases.lockstep_cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_lockstep_case_has_decisions(name, case):
    cell, frac = cases.encode(case)
    sim = OF.Fp32Sim(case, cell, frac, case.fluid_vel, case.fluid_rho)
    sim.commit()
    n_inj = n_del = 0
    for _ in range(6):
        sim.step(1)
        n_inj += len(sim.last_inj)
        n_del += len(sim.last_del)
    kinds = [b.bc for b in case.buffers]
    assert n_inj + n_del > 0
    if any(k in (0, 2, 4, 5) for k in kinds):
        assert n_inj > 0
    if any(k in (1, 3, 4, 5) for k in kinds):
        assert n_del > 0
    assert sim.n == sim.n0 + sim.injected.sum() - sim.deleted.sum() - sim.escaped
    assert np.all(np.diff(sim.cell) >= 0)
