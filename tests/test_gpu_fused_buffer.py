"""The buffer decisions fused into the drift epilogue equal the separate buffer kernel.

By default a step takes the Algorithm 1-3 decisions of every particle sorted into a candidate
cell of some buffer right after its drift (decide.cuh).  SPHBUF_PHASE_BUFFER_KERNEL runs the
same decisions in a kernel of their own after the drift, visiting the candidate cells.  Both
read the same post-drift state with the same FP32 arithmetic, so the states after every step
(sorted particle arrays, cell lists), the decision lists and the counters must be bit-for-bit
equal: over physics steps (single-rate and dual-criteria) and kinematic steps of the lockstep
cases, in plain launches and graph replay, and in a batch.  (The FP32-mode oracle itself is
checked against the fused form by the lockstep tests.)
"""
import copy

import numpy as np
import pytest

from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl
from tests import cases

pytestmark = pytest.mark.gpu

SEP = _ffi.PHASE_BUFFER_KERNEL


def _same(a, b):
    ra, rb = a.read(), b.read()
    for key in ra:
        assert np.array_equal(ra[key], rb[key]), key
    assert np.array_equal(a.cell_start(), b.cell_start())
    assert a.global_counters() == b.global_counters()
    (ia, da), (ib, db) = a.last_decisions(), b.last_decisions()
    assert ia == ib and sorted(da) == sorted(db)
    return len(ia) + len(da)


@pytest.mark.parametrize("name,case", cases.lockstep_cases(), ids=lambda x: x if isinstance(x, str) else "")
@pytest.mark.parametrize("phases,graph", [(_ffi.STEP_DEFAULT, False), (_ffi.STEP_DEFAULT, True),
                                          (_ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER, False)])
def test_fused_equals_buffer_kernel(name, case, phases, graph):
    from paper_2406_16786_gb300.domain import Domain

    case = copy.deepcopy(case)
    if phases & _ffi.PHASE_PHYSICS:
        # physics from the lockstep velocities would be violent; start from the BC state
        case.fluid_vel = case.fluid_vel * 0.05
    fused, sep = Domain.from_case(case), Domain.from_case(case)
    fused.use_graph(graph)
    sep.use_graph(graph)
    decided = 0
    for _ in range(6):
        fused.step(1, phases)
        sep.step(1, phases | SEP)
        decided += _same(fused, sep)
        nb = len(case.buffers)
        for k in range(nb):
            assert fused.counters(k) == sep.counters(k)
    assert decided > 0 or phases & _ffi.PHASE_PHYSICS
    fused.close()
    sep.close()


def test_fused_equals_buffer_kernel_dual_stepping():
    from paper_2406_16786_gb300.domain import Domain

    case = cases.physics_case(3)
    case.dual_substeps = 3
    fused, sep = Domain.from_case(case), Domain.from_case(case)
    for _ in range(4):
        fused.step(1)
        sep.step(1, _ffi.STEP_DEFAULT | SEP)
        _same(fused, sep)
    fused.close()
    sep.close()


def test_fused_equals_buffer_kernel_in_a_batch():
    from paper_2406_16786_gb300.domain import Batch, Domain

    cs = [wl.star_case(seed=700 + q, n_target=nt, arms=k, width=w, name="f%d" % q)
          for q, (nt, k, w) in enumerate([(6000, 1, 0.3), (15000, 4, 0.5), (9000, 6, 0.7)])]
    for c in cs:
        c.fluid_vel = wl.shear_velocity(c, u0=6.0) + 4.0 * c.buffers[0].rotation[0, :2]
    kin = _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER
    a = [Domain.from_case(c) for c in cs]
    b = [Domain.from_case(c) for c in cs]
    ba, bb = Batch(a), Batch(b)
    ba.use_graph(True)
    decided = 0
    for _ in range(5):
        ba.step(1, kin)
        bb.step(1, kin | SEP)
        ba.sync()
        bb.sync()
        decided += sum(_same(x, y) for x, y in zip(a, b))
    assert decided > 0
    ba.close()
    bb.close()
    for d in a + b:
        d.close()
