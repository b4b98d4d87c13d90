"""The CPU local-cell restriction of the buffer decisions (oracle/local_cell.py, the paper's
CPU method timed as a baseline) gives the plain definition's decisions: every particle
against every buffer (oracle/buffer.py), over several steps of the lockstep cases."""
import numpy as np
import pytest

from oracle import buffer as OB
from oracle import local_cell as LC
from tests import cases


@pytest.mark.parametrize("name,case", cases.lockstep_cases(), ids=[n for n, _ in cases.lockstep_cases()])
def test_local_cell_decisions_equal_all_particle_decisions(name, case):
    sim = OB.OracleSim(case)
    sim.commit()
    cand = [LC.candidate_cells(b, sim.lo, sim.cs, sim.dims, sim.dim) for b in sim.buffers]
    total = 0
    for _ in range(6):
        start = sim.cell_start.copy()
        sim.kinematic()
        n_before = sim.n
        sim.drop_escaped()
        assert sim.n == n_before
        inj, dels = OB.decide(sim.buffers, sim.pos, sim.label, sim.cs)
        li, ld = LC.decide_local(sim.buffers, sim.pos, sim.label, sim.cs, start, cand)
        assert sorted(inj) == li
        assert sorted(dels) == ld
        total += len(inj) + len(dels)
        sim.buffer_update()
        sim.rebuild()
        OB.relabel(sim.buffers, sim.pos, sim.label)
        sim.step_index += 1
    assert total > 0
    # the restriction visits a small part of the particles
    visited = sum(LC.candidates(sim.cell_start, c).size for c in cand)
    assert visited < sim.n
