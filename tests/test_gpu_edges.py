"""Edge cases and error paths of the GPU library."""
import numpy as np
import pytest

from paper_2406_16786_gb300 import _ffi
from paper_2406_16786_gb300 import workloads as wl
from tests import cases

pytestmark = pytest.mark.gpu


def _dom(case, **kw):
    from paper_2406_16786_gb300.domain import Domain

    return Domain.from_case(case, **kw)


def test_empty_domain_steps():
    from paper_2406_16786_gb300.domain import Domain

    case = cases.lockstep_cases()[0][1]
    d = Domain(2, case.lo, case.hi, case.dp, 1.3, 1000.0, 10.0, 1e-2, case.dt, 100)
    d.set_walls(case.wall_pos)
    d.add_buffer(case.buffers[0])
    d.write_particles(np.zeros(0, np.int32), np.zeros((0, 2), np.float32), np.zeros((0, 2), np.float32),
                      np.zeros(0, np.float32))
    d.step(3)
    assert d.count() == 0
    assert d.last_decisions() == ([], [])
    d.close()


@pytest.mark.parametrize("what", ["cell", "frac", "label", "next_id"])
def test_write_particles_rejects_bad_arrays(what):
    from paper_2406_16786_gb300.domain import SphbufError

    case = cases.lockstep_cases()[0][1]
    d = _dom(case)
    s = d.read()
    n = s["id"].shape[0]
    nid = int(s["id"].max()) + 1
    k = n // 2
    if what == "cell":
        s["cell"][k] = d.ncell
    elif what == "frac":
        s["frac"][k, 1] = -1e-7
    elif what == "label":
        s["label"][k] = len(case.buffers) + 1
    else:
        nid = int(s["id"].max())
    with pytest.raises(SphbufError) as e:
        d.write_particles(s["cell"], s["frac"], s["vel"], s["rho"], ids=s["id"], labels=s["label"], next_id=nid)
    assert e.value.status == 1
    assert d.count() == 0
    # a correct write afterwards restores the state exactly
    s2 = _dom(case).read()
    d.write_particles(s2["cell"], s2["frac"], s2["vel"], s2["rho"], ids=s2["id"], labels=s2["label"],
                      next_id=int(s2["id"].max()) + 1)
    back = d.read()
    for key in s2:
        assert np.array_equal(back[key], s2[key]), key
    d.close()


def test_read_into_preallocated_arrays():
    case = cases.lockstep_cases()[0][1]
    d = _dom(case)
    d.step(3)
    ref = d.read()
    n = ref["id"].shape[0]
    out = dict(cell=np.full(n + 7, -5, np.int32), frac=np.zeros((n + 7, 2), np.float32),
               vel=np.zeros((n + 7, 2), np.float32), rho=np.zeros(n + 7, np.float32), id=np.zeros(n + 7, np.uint32),
               label=np.zeros(n + 7, np.uint8))
    got = d.read(out=out)
    for key in ref:
        assert np.array_equal(got[key], ref[key]), key
        assert np.shares_memory(got[key], out[key])
    assert (out["cell"][n:] == -5).all()
    with pytest.raises(ValueError):
        d.read(out=dict(out, frac=np.zeros((n, 3), np.float32)))
    d.close()


def test_capacity_overflow_is_latched_not_faulted():
    from paper_2406_16786_gb300.domain import SphbufError

    case = cases.lockstep_cases()[0][1]
    d = _dom(case, capacity=case.n)  # no room for a single injected particle
    with pytest.raises(SphbufError) as e:
        for _ in range(20):
            d.step(1, _ffi.PHASE_KINEMATIC | _ffi.PHASE_BUFFER)
        d.sync()
    assert e.value.status == 2
    d.close()


def test_overlapping_buffers_rejected():
    from paper_2406_16786_gb300.domain import Domain, SphbufError

    case = cases.lockstep_cases()[0][1]
    d = Domain(2, case.lo, case.hi, case.dp, 1.3, 1000.0, 10.0, 1e-2, case.dt, case.capacity)
    d.add_buffer(case.buffers[0])
    b = case.buffers[0]
    moved = wl.BufferSpec(origin=b.origin + 0.02 * b.rotation[0], rotation=b.rotation, extent=b.extent, bc=b.bc)
    with pytest.raises(SphbufError) as e:
        d.add_buffer(moved)
    assert e.value.status == 3
    bad = wl.BufferSpec(origin=b.origin + 0.5, rotation=2.0 * b.rotation, extent=b.extent, bc=b.bc)
    with pytest.raises(SphbufError) as e:
        d.add_buffer(bad)
    assert e.value.status == 1
    d.close()


def test_particle_count_invariant_and_mass_balance():
    case = cases.lockstep_cases()[3][1]
    d = _dom(case)
    n0 = d.count()
    d.step(25)
    inj = sum(d.counters(k)["injected"] for k in range(2))
    dele = sum(d.counters(k)["deleted"] for k in range(2))
    g = d.global_counters()
    assert d.count() == n0 + inj - dele - g["escaped"]
    m = case.rho0 * case.dp ** 3
    mi = sum(d.counters(k)["mass_in"] for k in range(2))
    mo = sum(d.counters(k)["mass_out"] for k in range(2))
    assert mi - mo == pytest.approx((d.count() - n0 + g["escaped"]) * m, rel=1e-12, abs=1e-15)
    d.close()


def test_physics_steps_are_deterministic():
    """Two identical domains stepped 30 times end bit for bit equal (the atomics of the step
    only assign arrival slots, list positions and fixed-point sums, never an order that
    reaches the state)."""
    case = cases.physics_case(3)
    a, b = _dom(case), _dom(case)
    for d in (a, b):
        d.use_graph(True)
        d.step(30)
    ra, rb = a.read(), b.read()
    for key in ra:
        assert np.array_equal(ra[key], rb[key]), key
    assert a.global_counters() == b.global_counters()
    for k in range(len(case.buffers)):
        assert a.counters(k) == b.counters(k)
    a.close()
    b.close()


def test_nan_velocity_written_by_the_host_latches_the_nan_status():
    """A NaN velocity written through sphbuf_write_particles (the transfer checks cells,
    offsets, labels and ids, not velocities) makes the step's drift non-finite: the step
    stops with SPHBUF_ERR_NAN at the next synchronising call, without a device fault, and a
    clean write afterwards steps normally."""
    from paper_2406_16786_gb300.domain import SphbufError

    case = cases.physics_case(2)
    d = _dom(case)
    clean = d.read()
    s = {k: v.copy() for k, v in clean.items()}
    s["vel"][s["id"].shape[0] // 3, 0] = np.nan
    nid = int(s["id"].max()) + 1
    d.write_particles(s["cell"], s["frac"], s["vel"], s["rho"], ids=s["id"], labels=s["label"], next_id=nid)
    d.step(1)
    with pytest.raises(SphbufError) as e:
        d.sync()
    assert e.value.status == 6
    d.write_particles(clean["cell"], clean["frac"], clean["vel"], clean["rho"], ids=clean["id"],
                      labels=clean["label"], next_id=nid)
    d.step(2)
    d.sync()
    assert d.global_counters()["escaped"] >= 0 and d.count() > 0
    d.close()
