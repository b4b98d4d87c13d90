"""Kept neighbour lists (sphbuf_set_list_reuse): lists with a skin, kept over steps, with the
particles' slots kept between full rebuilds.

* Forty full steps with kept lists track the FP64 oracle with the tolerances of lists rebuilt
  every step (same ids and counters, fields within the accumulated FP32 rounding), 2-D and
  3-D, over several reuse cycles (full rebuilds counted), reading the state in between.
* Kept lists and lists rebuilt every step give the same particles and counters over sixty
  steps, with fields that differ only by the order of FP32 sums.
* Reads in a step whose rebuild kept the slots give the live particles sorted by (cell, id),
  consistent with the cell list and the count.
* A batch of domains with kept lists ends bit for bit where each ends alone.
* Steps with the separate buffer kernel, dual-criteria stepping and rotating buffers refuse
  kept lists.
"""
import numpy as np
import pytest

from oracle import buffer as OB
from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl
from tests import cases

pytestmark = pytest.mark.gpu

SKIN = 0.2  # skin / h


def _sorted_ok(dom, g):
    """The read state is sorted by (cell, id) and matches the cell list and the count."""
    assert g["id"].shape[0] == dom.count()
    key = g["cell"].astype(np.int64) * (1 << 32) + g["id"].astype(np.int64)
    assert np.all(np.diff(key) > 0)
    cs = dom.cell_start().astype(np.int64)
    assert cs[-1] == g["id"].shape[0]
    assert np.array_equal(np.diff(cs), np.bincount(g["cell"], minlength=cs.shape[0] - 1))


@pytest.mark.parametrize("dim", [2, 3])
def test_forty_steps_with_kept_lists_track_the_fp64_oracle(dim):
    from paper_2406_16786_gb300.domain import Domain

    case = cases.physics_case(dim)
    cell, frac = cases.encode(case)
    vel32 = case.fluid_vel.astype(np.float32)
    rho32 = case.fluid_rho.astype(np.float32)
    dom = Domain.from_case(case)
    dom.set_list_reuse(SKIN)
    dom.use_graph(True)
    pos0 = wl.decode_positions(cell, frac, case.lo, case.cs, case.grid_dims())
    ora = OB.OracleSim(case, pos=pos0, vel=vel32.astype(np.float64), rho=rho32.astype(np.float64))
    ora.commit()
    for q in range(40):
        dom.step(1)
        ora.step(1)
        if q % 10 == 9:
            _sorted_ok(dom, dom.read())
    builds = dom.list_builds()
    print("dim %d: %d full list builds in 40 steps (commit included)" % (dim, builds))
    assert 3 <= builds <= 25
    g = dom.read()
    gp = dom.positions()
    assert sorted(g["id"].tolist()) == sorted(ora.id.tolist())
    for k in range(len(case.buffers)):
        c = dom.counters(k)
        assert (c["injected"], c["deleted"]) == (int(ora.injected[k]), int(ora.deleted[k]))
    assert sum(int(x) for x in ora.injected) + sum(int(x) for x in ora.deleted) > 0
    o, q = np.argsort(g["id"]), np.argsort(ora.id)
    rho_g, rho_o = g["rho"][o].astype(np.float64), ora.rho[q]
    v_g, v_o = g["vel"][o].astype(np.float64), ora.vel[q]
    assert np.linalg.norm(rho_g - rho_o) / np.linalg.norm(rho_o) < 1e-6
    assert np.linalg.norm(v_g - v_o) / np.linalg.norm(v_o) < 2e-5
    assert np.max(np.linalg.norm(gp[o] - ora.pos[q], axis=1)) < 1e-5 * case.cs
    dom.close()


@pytest.mark.parametrize("name,case", cases.lockstep_cases()[2:4], ids=lambda x: x if isinstance(x, str) else "")
def test_kept_lists_equal_lists_rebuilt_every_step(name, case):
    from paper_2406_16786_gb300.domain import Domain

    case.fluid_vel = case.fluid_vel * 0.05
    kept, every = Domain.from_case(case), Domain.from_case(case)
    kept.set_list_reuse(SKIN)
    for d in (kept, every):
        d.use_graph(True)
        d.step(60)
    gk, ge = kept.read(), every.read()
    assert np.array_equal(gk["id"], ge["id"])
    assert np.array_equal(gk["cell"], ge["cell"])
    assert np.array_equal(gk["label"], ge["label"])
    for key, tol in (("frac", 1e-6 * case.cs), ("vel", 1e-5), ("rho", 1e-3)):
        assert np.max(np.abs(gk[key].astype(np.float64) - ge[key])) < tol, key
    for k in range(len(case.buffers)):
        assert kept.counters(k)["injected"] == every.counters(k)["injected"]
        assert kept.counters(k)["deleted"] == every.counters(k)["deleted"]
    assert kept.list_builds() < every.list_builds()
    kept.close()
    every.close()


def test_reads_between_full_rebuilds_are_sorted():
    from paper_2406_16786_gb300.domain import Domain

    case = cases.physics_case(3)
    dom = Domain.from_case(case)
    dom.set_list_reuse(SKIN)
    seen_kept = False
    for _ in range(12):
        b0 = dom.list_builds()
        dom.step(1)
        g = dom.read()
        _sorted_ok(dom, g)
        p = dom.positions()
        assert p.shape[0] == g["id"].shape[0]
        seen_kept |= dom.list_builds() == b0
    assert seen_kept
    dom.close()


def test_batch_with_kept_lists_equals_individual():
    from paper_2406_16786_gb300.domain import Batch, Domain

    def _cases():
        out = [wl.star_case(seed=970 + q, n_target=nt, arms=k, width=w, name="r%d" % q)
               for q, (nt, k, w) in enumerate([(6000, 1, 0.3), (15000, 4, 0.6)])]
        out.append(cases.physics_case(2))
        return out

    alone = [Domain.from_case(c) for c in _cases()]
    for d in alone:
        d.set_list_reuse(SKIN)
        d.step(25)
    together = [Domain.from_case(c) for c in _cases()]
    for d in together:
        d.set_list_reuse(SKIN)
    b = Batch(together)
    b.use_graph(True)
    b.step(25)
    b.sync()
    for a, t in zip(alone, together):
        ra, rt = a.read(), t.read()
        for key in ra:
            assert np.array_equal(ra[key], rt[key]), key
        assert a.global_counters() == t.global_counters()
        assert a.list_builds() == t.list_builds()
    b.close()
    for d in alone + together:
        d.close()


def test_kept_lists_refuse_what_they_cannot_serve():
    from paper_2406_16786_gb300.domain import Domain, SphbufError

    case = cases.physics_case(2)
    d = Domain.from_case(case)
    d.set_list_reuse(SKIN)
    for ph in (_ffi.STEP_DEFAULT | _ffi.PHASE_BUFFER_KERNEL, _ffi.STEP_DEFAULT | _ffi.PHASE_FULL_CHECK):
        with pytest.raises(SphbufError) as e:
            d.step(1, ph)
        assert e.value.status == 1
    # a kinematic step after kept-list steps ends sorted
    d.step(3)
    d.step(1, _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER)
    _sorted_ok(d, d.read())
    d.close()
    dual = cases.physics_case(2)
    dual.dual_substeps = 2
    d = Domain.from_case(dual)
    with pytest.raises(SphbufError) as e:
        d.set_list_reuse(SKIN)
    assert e.value.status == 1
    d.close()
    rot = wl.sprinkler_case(dim=2, dp=0.005, umax=1.0, omega=10.0, ambient=True, domain_radius=0.2)
    d = Domain.from_case(rot)
    with pytest.raises(SphbufError):
        d.set_list_reuse(SKIN)
    d.close()
