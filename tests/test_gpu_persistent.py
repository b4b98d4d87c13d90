"""The persistent batched step: one cooperative launch per default step, grid barriers
between the phases.

* It gives, bit for bit, the states of the domains stepped alone (plain launches and graph
  replay), with the fused buffer decisions and the transport-velocity variant, with lists
  rebuilt every step and with kept lists (over several reuse cycles).
* Its barrier waits are bounded: with a spin limit of zero every block that has to wait gives
  up at once, the step latches SPHBUF_ERR_TIMEOUT in every domain (reported by the next
  synchronising call) and the launch ends; the GPU context stays usable.
* Batches it cannot serve (rotating buffers, dual-criteria stepping) are refused.
"""
import numpy as np
import pytest

from paper_2406_16786_gb300 import workloads as wl
from tests import cases

pytestmark = pytest.mark.gpu


def _cases():
    out = [wl.star_case(seed=950 + q, n_target=nt, arms=k, width=w, name="p%d" % q)
           for q, (nt, k, w) in enumerate([(4000, 1, 0.3), (16000, 4, 0.6), (9000, 6, 0.8)])]
    out.append(cases.lockstep_cases()[2][1])  # bidirectional channel
    t = cases.physics_case(2)
    t.tvf_lambda = 7.5
    out.append(t)
    return out


@pytest.mark.parametrize("graph,skin", [(False, 0.0), (True, 0.0), (True, 0.2)])
def test_persistent_equals_individual(graph, skin):
    from paper_2406_16786_gb300.domain import Batch, Domain

    steps = 25 if skin else 12
    alone = [Domain.from_case(c) for c in _cases()]
    for d in alone:
        if skin:
            d.set_list_reuse(skin)
        d.step(steps)
    together = [Domain.from_case(c) for c in _cases()]
    for d in together:
        if skin:
            d.set_list_reuse(skin)
    b = Batch(together)
    b.set_persistent(True)
    b.use_graph(graph)
    b.step(steps)
    b.sync()
    kept = 0
    for a, t in zip(alone, together):
        ra, rt = a.read(), t.read()
        for key in ra:
            assert np.array_equal(ra[key], rt[key]), key
        assert a.global_counters() == t.global_counters()
        (ia, da), (it, dt) = a.last_decisions(), t.last_decisions()
        assert ia == it and sorted(da) == sorted(dt)
        if skin:
            assert a.list_builds() == t.list_builds()
            kept += a.list_builds() < steps
    # (the fast shear flow of the lockstep channel outruns the skin every step)
    assert not skin or kept >= 3
    b.close()
    for d in alone + together:
        d.close()


def test_barrier_spin_limit_zero_returns_timeout():
    from paper_2406_16786_gb300.domain import Batch, Domain, SphbufError

    doms = [Domain.from_case(c) for c in _cases()[:3]]
    b = Batch(doms)
    b.set_persistent(True, spin_limit=0)
    b.step(1)
    with pytest.raises(SphbufError) as e:
        b.sync()
    assert e.value.status == 5
    for d in doms:
        with pytest.raises(SphbufError) as e:
            d.sync()
        assert e.value.status == 5
    b.close()
    # the context is still usable: a fresh domain steps normally
    d2 = Domain.from_case(_cases()[0])
    d2.step(2)
    d2.sync()
    assert d2.global_counters()["steps"] == 2
    d2.close()
    for d in doms:
        d.close()


def test_persistent_refuses_rotating_and_dual_batches():
    from paper_2406_16786_gb300.domain import Batch, Domain, SphbufError

    rot = wl.sprinkler_case(dim=2, dp=0.005, umax=1.0, omega=10.0, ambient=True, domain_radius=0.2)
    dual = cases.physics_case(2)
    dual.dual_substeps = 2
    for c in (rot, dual):
        d = Domain.from_case(c)
        b = Batch([d])
        with pytest.raises(SphbufError) as e:
            b.set_persistent(True)
        assert e.value.status == 1
        b.close()
        d.close()
