"""Batched multi-domain steps: every domain ends exactly where it would have stepping alone.

Five 2-D domains of different sizes and buffer sets (star channels with 1-6 arms, and a
bidirectional channel) are stepped together by the multi-domain kernels and, separately,
one by one with the single-domain kernels; the sorted states, decisions and counters must be
bit-for-bit equal (same arithmetic, deterministic order).
"""
import numpy as np
import pytest

from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl
from tests import cases

pytestmark = pytest.mark.gpu


def _cases():
    out = [wl.star_case(seed=900 + q, n_target=nt, arms=k, width=w, name="t%d" % q)
           for q, (nt, k, w) in enumerate([(4000, 1, 0.3), (12000, 3, 0.5), (2500, 2, 0.25), (20000, 6, 0.8)])]
    out.append(cases.lockstep_cases()[2][1])
    return out


@pytest.mark.parametrize("phases,graph", [(_ffi.STEP_DEFAULT, False), (_ffi.STEP_DEFAULT, True),
                                          (_ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER, True)])
def test_batched_equals_individual(phases, graph):
    from paper_2406_16786_gb300.domain import Batch, Domain

    cs = _cases()
    if phases & _ffi.PHASE_KINEMATIC:
        for c in cs:
            c.fluid_vel = wl.shear_velocity(c, u0=8.0) if len(c.buffers) > 1 else c.fluid_vel + 3.0
    alone = [Domain.from_case(c) for c in cs]
    for d in alone:
        d.step(6, phases)
    together = [Domain.from_case(c) for c in cs]
    b = Batch(together)
    b.use_graph(graph)
    decided = 0
    for _ in range(6):
        b.step(1, phases)
        decided += sum(len(x) for d in together for x in d.last_decisions())
    b.sync()
    for a, t in zip(alone, together):
        ra, rt = a.read(), t.read()
        for key in ra:
            assert np.array_equal(ra[key], rt[key]), key
        assert a.global_counters() == t.global_counters()
        (ia, da), (it, dt) = a.last_decisions(), t.last_decisions()
        assert ia == it  # injections are ordered by (buffer, parent id)
        assert sorted(da) == sorted(dt)  # deletions are a set
    assert decided > 0
    b.close()


def test_batch_autotune_keeps_results_valid():
    from paper_2406_16786_gb300.domain import Batch, Domain

    cs = _cases()
    doms = [Domain.from_case(c) for c in cs]
    b = Batch(doms)
    m, ms = b.autotune(trial_steps=2)
    assert m in (1, 2, 4, 8, 16)
    assert ms["force"] > 0
    b.use_graph(True)
    b.step(3)
    b.sync()
    for d, c in zip(doms, cs):
        g = d.global_counters()
        # 4 block sizes x 5 grids of trial steps, then the chosen configuration's timed steps
        assert g["steps"] == (4 * 5 + 1) * 2 + 3
        inj = sum(d.counters(k)["injected"] for k in range(len(c.buffers)))
        dele = sum(d.counters(k)["deleted"] for k in range(len(c.buffers)))
        assert d.count() == c.n + inj - dele - g["escaped"]
    b.close()


def test_batched_rotating_and_transport_velocity_equal_individual():
    """The batch's variants: domains with a rotating nozzle (the buffer kernel with the turn)
    and a domain with the transport velocity (the force kernel's TVF variant), stepped
    together, end bit for bit where each ends alone."""
    from paper_2406_16786_gb300.domain import Batch, Domain

    def _cases():
        a = wl.sprinkler_case(dim=2, dp=0.004, umax=1.0, omega=30.0, ambient=True, domain_radius=0.2)
        b = wl.sprinkler_case(dim=2, dp=0.005, umax=1.0, omega=-20.0, theta0=1.0, ambient=True, domain_radius=0.2)
        t = cases.physics_case(2)
        t.tvf_lambda = 7.5
        return [a, b, t]

    alone = [Domain.from_case(c) for c in _cases()]
    for d in alone:
        d.step(40)
    together = [Domain.from_case(c) for c in _cases()]
    b = Batch(together)
    b.use_graph(True)
    b.step(40)
    b.sync()
    for a_, t_ in zip(alone, together):
        ra, rt = a_.read(), t_.read()
        for key in ra:
            assert np.array_equal(ra[key], rt[key]), key
        assert a_.global_counters() == t_.global_counters()
    assert together[0].counters(0)["injected"] > 0
    b.close()
